// clot_model.cuh -- device-side model functions shared by the species-step
// kernels: hindered transport W (App. A), van Leer face value (App. D), binding
// affinity g (App. A), the reaction right-hand side (App. A platelet sources,
// App. B mass action and injury-wall exchange) and its RK4 integration
// (Sec. 3.2 step 2).
#pragma once

#include "clot_internal.cuh"

namespace clot {

// ---------------------------------------------------------------- model

// W(theta_T) = tanh(pi (1 - theta_T)), theta_T clamped to [0, 1] (App. A),
// from the identity tanh(a) = 1 - 2 / (exp(2a) + 1) with a in [0, pi]
// (exp(2a) <= e^{2 pi} ~ 535, no overflow); absolute error ~1e-7.
__device__ __forceinline__ float hindrance(float theta) {
  theta = fminf(fmaxf(theta, 0.0f), 1.0f);
  const float e = __expf(6.28318530717959f * (1.0f - theta));
  return 1.0f - __fdividef(2.0f, e + 1.0f);
}

// van Leer limited face value (App. D): with a = cU - cUU, b = cD - cU the
// limiter psi(r) = (r + |r|)/(1 + |r|), r = a/b, gives cU + a b/(a + b) when a
// and b have the same sign and cU otherwise.  Written as a * (b / (a + b)) so
// the product cannot underflow for tiny concentrations.
__device__ __forceinline__ float vanleer(float cUU, float cU, float cD, int limiter) {
  if (!limiter) return cU;
  const float a = cU - cUU, b = cD - cU;
  // same sign: a b > 0 (one multiply and one compare; it underflows only for
  // |a b| < 1.4e-45, where the limited correction is below 1e-22 and the
  // upwind value is kept)
  return (a * b > 0.0f) ? fmaf(a, __fdividef(b, a + b), cU) : cU;
}

// g(eta) of App. A: zero at and below eta_t, g0 chosen so that g(1) = 1.
__device__ __forceinline__ float affinity(const RxnConst& k, float eta) {
  float u = eta - k.eta_t;
  if (!(u > 0.0f)) return 0.0f;
  float u3 = u * u * u;
  return k.g0 * u3 / (k.eta_star3 + u3);
}

// Reaction right-hand side for one cell (App. A platelet terms, App. B mass
// action).  ADP has no reaction term (its source enters in transport), so
// f[CLOT_ADP] is left untouched and never used.  adhH = k_adh H_adh,
// A1 = k_adp [ADP]/([ADP]* + [ADP]) (constant over the reaction solve since
// ADP does not react), coh = k_coh g(eta) Pmax.  WALL adds the injury-face
// exchange: J = kC0+ S1_w E0 - kC0- C0 with the Robin wall value
// S1_w = (Dd S1 + kC0- C0)/(Dd + kC0+ E0); S1 loses (A/V) J, E1 gains
// (A/V) kC0cat C0; E0' = -J + kC0cat C0, C0' = J - kC0cat C0.  T is float
// on the species-step path; the surrogate's training pairs use double.
// y and f hold at least the CLOT_NS species (the inhibitor extension's two
// rows may follow; they are not touched here).
template <bool WALL, typename T = float>
__device__ __forceinline__ void rxn_rhs(const RxnConst& k, const T* y, T adhH, T A1, T coh, T e0, T c0, T* f,
                                        T& fe0, T& fc0) {
  const T Pmu = y[CLOT_PMU], Pma = y[CLOT_PMA], Pba = y[CLOT_PBA], Pbse = y[CLOT_PBSE];
  const T s1 = y[CLOT_S1], s2 = y[CLOT_S2], e1 = y[CLOT_E1], e2 = y[CLOT_E2];
  const T s1b = y[CLOT_S1B], s2b = y[CLOT_S2B], e1b = y[CLOT_E1B], e2b = y[CLOT_E2B];
  const T c1 = y[CLOT_C1], c2 = y[CLOT_C2];

  const T adh = adhH * (k.Pmax - Pbse);
  const T A = A1 + k.k_e2 * e2 / (k.e2_star + e2);
  f[CLOT_PMU] = -adh * Pmu - A * Pmu;
  f[CLOT_PMA] = -adh * Pma + A * Pmu - coh * Pma;
  f[CLOT_PBA] = -adh * Pba + coh * Pma;
  f[CLOT_PBSE] = adh * (Pmu + Pma + Pba);

  const T sites = Pba + Pbse;
  const T free1 = k.n1 * sites - (s1b + e1b + c1 + c2);
  const T free2 = k.n2 * sites - (s2b + e2b + c1 + c2);
  const T bS1 = k.kS1p * free1 * s1 - k.kS1m * s1b;  // net binding S1 -> S1b
  const T bE1 = k.kE1p * free1 * e1 - k.kE1m * e1b;
  const T bS2 = k.kS2p * free2 * s2 - k.kS2m * s2b;
  const T bE2 = k.kE2p * free2 * e2 - k.kE2m * e2b;
  const T a1 = k.kC1p * s2b * e1b - k.kC1m * c1;     // net association into C1
  const T a2 = k.kC2p * s1b * e2b - k.kC2m * c2;     // net association into C2
  const T cat1 = k.kC1cat * c1, cat2 = k.kC2cat * c2;
  f[CLOT_S1] = -bS1;
  f[CLOT_S2] = -bS2;
  f[CLOT_E1] = -bE1;
  f[CLOT_E2] = -bE2;
  f[CLOT_S1B] = bS1 - a2;
  f[CLOT_S2B] = bS2 - a1;
  f[CLOT_E1B] = bE1 - a1 + cat1 + cat2;
  f[CLOT_E2B] = bE2 - a2 + cat2 + cat1;
  f[CLOT_C1] = a1 - cat1;
  f[CLOT_C2] = a2 - cat2;
  if (WALL) {
    const T s1w = (k.Dd * s1 + k.kC0m * c0) / (k.Dd + k.kC0p * e0);
    const T J = k.kC0p * s1w * e0 - k.kC0m * c0;
    const T cat0 = k.kC0cat * c0;
    f[CLOT_S1] -= k.aV * J;
    f[CLOT_E1] += k.aV * cat0;
    fe0 = cat0 - J;
    fc0 = J - cat0;
  }
}

// rxn_rhs with the injury-wall exchange switched at run time (fe0, fc0 are
// left untouched when !wall).
__device__ __forceinline__ void rxn_rhs_rt(const RxnConst& k, const float* y, float adhH, float A1, float coh,
                                           bool wall, float e0, float c0, float* f, float& fe0, float& fc0) {
  rxn_rhs<false>(k, y, adhH, A1, coh, e0, c0, f, fe0, fc0);
  if (wall) {
    const float s1w = (k.Dd * y[CLOT_S1] + k.kC0m * c0) / (k.Dd + k.kC0p * e0);
    const float J = k.kC0p * s1w * e0 - k.kC0m * c0;
    const float cat0 = k.kC0cat * c0;
    f[CLOT_S1] -= k.aV * J;
    f[CLOT_E1] += k.aV * cat0;
    fe0 = cat0 - J;
    fc0 = J - cat0;
  }
}

// Row indices of the inhibitor extension's species after the CLOT_NS cell
// species in a reaction state of CLOT_NX entries.
constexpr int CLOT_NX = CLOT_NS + 2, XINH = CLOT_NS, XE2I = CLOT_NS + 1;

// The inhibitor extension's term (the paper's example of adding a species,
// I + E2 -> E2,inh at rate kI I E2): fluid-phase thrombin and I each lose
// kI I E2, E2,inh gains it.
__device__ __forceinline__ void inhibit_rhs(const RxnConst& k, const float* y, float* f) {
  const float r = k.kI * y[XINH] * y[CLOT_E2];
  f[CLOT_E2] -= r;
  f[XINH] = -r;
  f[XE2I] = r;
}

// M classic RK4 steps of size h on the cell state y (and, when wall, its
// injury face E0, C0; the wall terms are a runtime switch so one copy of the
// integrator serves every cell).  N = CLOT_NX carries the inhibitor
// extension's two rows in the same stages.  The increments of the M steps are summed in
// D apart from the state and added to it once at the end: a large state that
// changes by a little each step (bound platelets in a clot) is then rounded
// to FP32 once per reaction solve, not once per substep, where the roundings
// of slowly varying increments add up in one direction.  Each step's stages
// start from y + D.  Returns the total increment of Pba + Pbse (newly bound
// platelets); dwall, when given, receives the increments of E0 and C0, and
// dsub those of S1 and S2.
template <int N = CLOT_NS>
__device__ __forceinline__ float rxn_rk4(const RxnConst& k, float (&y)[N], float adhH, float A1,
                                         float coh, bool wall, float& e0, float& c0, float h, int M,
                                         float* dwall = nullptr, float* dsub = nullptr) {
  const float h2 = 0.5f * h, h6 = h * (1.0f / 6.0f);
  float D[N], De0 = 0.0f, Dc0 = 0.0f;
#pragma unroll
  for (int q = 0; q < N; ++q) D[q] = 0.0f;
  auto rhs = [&](const float* yt, float e, float c, float* f, float& fe, float& fc) {
    rxn_rhs_rt(k, yt, adhH, A1, coh, wall, e, c, f, fe, fc);
    if (N == CLOT_NX) inhibit_rhs(k, yt, f);
  };
  for (int m = 0; m < M; ++m) {
    float yt[N], acc[N], f[N];
    float fe0 = 0.0f, fc0 = 0.0f, ae0 = 0.0f, ac0 = 0.0f;
    const float be0 = e0 + De0, bc0 = c0 + Dc0;
#pragma unroll
    for (int q = 0; q < N; ++q) {
      f[q] = 0.0f;
      yt[q] = y[q] + D[q];
    }
    // stage 1
    rhs(yt, be0, bc0, f, fe0, fc0);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      acc[q] = f[q];
      yt[q] = (q == CLOT_ADP) ? y[q] : (y[q] + D[q]) + h2 * f[q];
    }
    ae0 = fe0; ac0 = fc0;
    // stage 2
    rhs(yt, be0 + h2 * fe0, bc0 + h2 * fc0, f, fe0, fc0);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      acc[q] += 2.0f * f[q];
      yt[q] = (q == CLOT_ADP) ? y[q] : (y[q] + D[q]) + h2 * f[q];
    }
    ae0 += 2.0f * fe0; ac0 += 2.0f * fc0;
    // stage 3
    rhs(yt, be0 + h2 * fe0, bc0 + h2 * fc0, f, fe0, fc0);
#pragma unroll
    for (int q = 0; q < N; ++q) {
      acc[q] += 2.0f * f[q];
      yt[q] = (q == CLOT_ADP) ? y[q] : (y[q] + D[q]) + h * f[q];
    }
    ae0 += 2.0f * fe0; ac0 += 2.0f * fc0;
    // stage 4
    rhs(yt, be0 + h * fe0, bc0 + h * fc0, f, fe0, fc0);
#pragma unroll
    for (int q = 0; q < N; ++q)
      if (q != CLOT_ADP) D[q] += h6 * (acc[q] + f[q]);
    De0 += h6 * (ae0 + fe0);
    Dc0 += h6 * (ac0 + fc0);
  }
#pragma unroll
  for (int q = 0; q < N; ++q)
    if (q != CLOT_ADP) y[q] += D[q];
  if (wall) {
    e0 += De0;
    c0 += Dc0;
  }
  if (dwall) {
    dwall[0] = De0;
    dwall[1] = Dc0;
  }
  if (dsub) {
    dsub[0] = D[CLOT_S1];
    dsub[1] = D[CLOT_S2];
  }
  return D[CLOT_PBA] + D[CLOT_PBSE];
}


// rxn_rk4 on a state whose S1, S2 rows may hold deviations from k.s1_ref,
// k.s2_ref (the deviation form; both zero otherwise): the rates are evaluated
// at the full values, and the increments of S1, S2 are added to the
// deviations, so the result keeps their resolution.
template <int N = CLOT_NS>
__device__ __forceinline__ float rxn_rk4_dev(const RxnConst& k, float (&y)[N], float adhH, float A1, float coh,
                                             bool wall, float& e0, float& c0, float h, int M, float* dwall) {
  const float s1d = y[CLOT_S1], s2d = y[CLOT_S2];
  y[CLOT_S1] = s1d + k.s1_ref;  // unchanged without the deviation form
  y[CLOT_S2] = s2d + k.s2_ref;
  float ds[2];
  const float bound = rxn_rk4<N>(k, y, adhH, A1, coh, wall, e0, c0, h, M, dwall, ds);
  if (k.s1_ref != 0.0f || k.s2_ref != 0.0f) {
    y[CLOT_S1] = s1d + ds[0];
    y[CLOT_S2] = s2d + ds[1];
  }
  return bound;
}

// Exact RK4 map of the reaction system for a cell where it reduces to linear
// activation: no adhesion (H_adh = 0), no cohesion (g = 0), no wall face, no
// bound platelets and no bound coagulation species.  Then every coagulation
// derivative is exactly zero (no binding sites, nothing bound), ADP and E2 are
// constant, and the platelets obey P^{m,u}' = -A P^{m,u}, P^{m,a}' = A P^{m,u}
// with A = A1 + A2(E2) constant: each RK4 step multiplies P^{m,u} by
// R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, z = -A h, and conserves the sum.
// The amount moved per step, P^{m,u} (1 - R), is formed from
// 1 - R = -z (1 + z/2 + z^2/6 + z^3/24) directly: A h is often far below
// FP32's resolution of 1 (1e-7 and less), where 1 - R taken from a rounded R
// would keep one or two significant bits of it.
// Returns false (state untouched) when the cell is not in that case.
template <int N = CLOT_NS>
__device__ __forceinline__ bool rxn_linear_rest(const RxnConst& k, float (&y)[N], float adhH, float A1,
                                                float coh, bool wall, float h, int M) {
  if (wall || adhH != 0.0f || coh != 0.0f) return false;
  if (!(y[CLOT_PBA] == 0.0f && y[CLOT_PBSE] == 0.0f && y[CLOT_S1B] == 0.0f && y[CLOT_S2B] == 0.0f &&
        y[CLOT_E1B] == 0.0f && y[CLOT_E2B] == 0.0f && y[CLOT_C1] == 0.0f && y[CLOT_C2] == 0.0f))
    return false;
  // with the inhibitor extension, E2 stays constant only while kI I E2 = 0
  if (N == CLOT_NX && k.kI * y[N == CLOT_NX ? XINH : 0] * y[CLOT_E2] != 0.0f) return false;
  const float e2 = y[CLOT_E2];
  const float A = A1 + ((e2 != 0.0f) ? k.k_e2 * e2 / (k.e2_star + e2) : e2);  // the A2 term is e2 when e2 = +-0
  if (A == 0.0f) return true;
  const float z = -A * h;
  const float q = -z * (1.0f + z * (0.5f + z * ((1.0f / 6.0f) + z * (1.0f / 24.0f))));  // 1 - R(z)
  float pmu = y[CLOT_PMU], pma = y[CLOT_PMA];
  for (int m = 0; m < M; ++m) {
    const float d = pmu * q;
    pma += d;
    pmu -= d;
  }
  y[CLOT_PMU] = pmu;
  y[CLOT_PMA] = pma;
  return true;
}

}  // namespace clot

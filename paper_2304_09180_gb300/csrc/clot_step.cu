// clot_step.cu -- the fused species step (K1): explicit finite-volume transport
// of the seven mobile species followed, in registers, by M_rxn RK4 reaction
// substeps and the injury-wall exchange, so each cell's state is read and
// written once per step.
//
// Model (clotFoam paper): fractional step of Sec. 3.2 (transport over dt, then
// M_rxn RK4 solves of h = dt/M_rxn); hindered platelet fluxes with W(theta_T)
// of the downwind cell for advection and of the larger theta_T of the face's
// two cells for diffusion (Sec. 3.2, App. D interpolation schemes); van Leer
// face values (App. D); Gauss-linear diffusion (App. D); boundary table of
// App. C (inlet Dirichlet for P^{m,u}, S1, S2, zero gradient elsewhere, walls
// impermeable); platelet sources (App. A); coagulation mass action and the
// injury-wall reactive fluxes (App. B).
#include "clot_internal.cuh"

namespace clot {

// ---------------------------------------------------------------- model

// W(theta_T) = tanh(pi (1 - theta_T)), theta_T clamped to [0, 1] (App. A).
__device__ __forceinline__ float hindrance(float theta) {
  theta = fminf(fmaxf(theta, 0.0f), 1.0f);
  return tanhf(3.14159265358979f * (1.0f - theta));
}

// van Leer limited face value (App. D): with a = cU - cUU, b = cD - cU the
// limiter psi(r) = (r + |r|)/(1 + |r|), r = a/b, gives cU + a b/(a + b) when a
// and b have the same sign and cU otherwise.  Written as a * (b / (a + b)) so
// the product cannot underflow for tiny concentrations.
__device__ __forceinline__ float vanleer(float cUU, float cU, float cD, int limiter) {
  if (!limiter) return cU;
  float a = cU - cUU, b = cD - cU;
  bool same = (a > 0.0f && b > 0.0f) || (a < 0.0f && b < 0.0f);
  return same ? cU + a * (b / (a + b)) : cU;
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
// (A/V) kC0cat C0; E0' = -J + kC0cat C0, C0' = J - kC0cat C0.
template <bool WALL>
__device__ __forceinline__ void rxn_rhs(const RxnConst& k, const float (&y)[CLOT_NS], float adhH,
                                        float A1, float coh, float e0, float c0,
                                        float (&f)[CLOT_NS], float& fe0, float& fc0) {
  const float Pmu = y[CLOT_PMU], Pma = y[CLOT_PMA], Pba = y[CLOT_PBA], Pbse = y[CLOT_PBSE];
  const float s1 = y[CLOT_S1], s2 = y[CLOT_S2], e1 = y[CLOT_E1], e2 = y[CLOT_E2];
  const float s1b = y[CLOT_S1B], s2b = y[CLOT_S2B], e1b = y[CLOT_E1B], e2b = y[CLOT_E2B];
  const float c1 = y[CLOT_C1], c2 = y[CLOT_C2];

  const float adh = adhH * (k.Pmax - Pbse);
  const float A = A1 + k.k_e2 * e2 / (k.e2_star + e2);
  f[CLOT_PMU] = -adh * Pmu - A * Pmu;
  f[CLOT_PMA] = -adh * Pma + A * Pmu - coh * Pma;
  f[CLOT_PBA] = -adh * Pba + coh * Pma;
  f[CLOT_PBSE] = adh * (Pmu + Pma + Pba);

  const float sites = Pba + Pbse;
  const float free1 = k.n1 * sites - (s1b + e1b + c1 + c2);
  const float free2 = k.n2 * sites - (s2b + e2b + c1 + c2);
  const float bS1 = k.kS1p * free1 * s1 - k.kS1m * s1b;  // net binding S1 -> S1b
  const float bE1 = k.kE1p * free1 * e1 - k.kE1m * e1b;
  const float bS2 = k.kS2p * free2 * s2 - k.kS2m * s2b;
  const float bE2 = k.kE2p * free2 * e2 - k.kE2m * e2b;
  const float a1 = k.kC1p * s2b * e1b - k.kC1m * c1;     // net association into C1
  const float a2 = k.kC2p * s1b * e2b - k.kC2m * c2;     // net association into C2
  const float cat1 = k.kC1cat * c1, cat2 = k.kC2cat * c2;
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
    const float s1w = (k.Dd * s1 + k.kC0m * c0) / (k.Dd + k.kC0p * e0);
    const float J = k.kC0p * s1w * e0 - k.kC0m * c0;
    const float cat0 = k.kC0cat * c0;
    f[CLOT_S1] -= k.aV * J;
    f[CLOT_E1] += k.aV * cat0;
    fe0 = cat0 - J;
    fc0 = J - cat0;
  }
}

// M classic RK4 steps of size h on the cell state y (and its injury face).
template <bool WALL>
__device__ __forceinline__ void rxn_rk4(const RxnConst& k, float (&y)[CLOT_NS], float adhH, float A1,
                                        float coh, float& e0, float& c0, float h, int M) {
  const float h2 = 0.5f * h, h6 = h * (1.0f / 6.0f);
  for (int m = 0; m < M; ++m) {
    float yt[CLOT_NS], acc[CLOT_NS], f[CLOT_NS];
    float fe0 = 0.0f, fc0 = 0.0f, te0 = e0, tc0 = c0, ae0 = 0.0f, ac0 = 0.0f;
#pragma unroll
    for (int q = 0; q < CLOT_NS; ++q) f[q] = 0.0f;
    // stage 1
    rxn_rhs<WALL>(k, y, adhH, A1, coh, e0, c0, f, fe0, fc0);
#pragma unroll
    for (int q = 0; q < CLOT_NS; ++q) {
      acc[q] = f[q];
      yt[q] = (q == CLOT_ADP) ? y[q] : y[q] + h2 * f[q];
    }
    if (WALL) { ae0 = fe0; ac0 = fc0; te0 = e0 + h2 * fe0; tc0 = c0 + h2 * fc0; }
    // stage 2
    rxn_rhs<WALL>(k, yt, adhH, A1, coh, te0, tc0, f, fe0, fc0);
#pragma unroll
    for (int q = 0; q < CLOT_NS; ++q) {
      acc[q] += 2.0f * f[q];
      yt[q] = (q == CLOT_ADP) ? y[q] : y[q] + h2 * f[q];
    }
    if (WALL) { ae0 += 2.0f * fe0; ac0 += 2.0f * fc0; te0 = e0 + h2 * fe0; tc0 = c0 + h2 * fc0; }
    // stage 3
    rxn_rhs<WALL>(k, yt, adhH, A1, coh, te0, tc0, f, fe0, fc0);
#pragma unroll
    for (int q = 0; q < CLOT_NS; ++q) {
      acc[q] += 2.0f * f[q];
      yt[q] = (q == CLOT_ADP) ? y[q] : y[q] + h * f[q];
    }
    if (WALL) { ae0 += 2.0f * fe0; ac0 += 2.0f * fc0; te0 = e0 + h * fe0; tc0 = c0 + h * fc0; }
    // stage 4
    rxn_rhs<WALL>(k, yt, adhH, A1, coh, te0, tc0, f, fe0, fc0);
#pragma unroll
    for (int q = 0; q < CLOT_NS; ++q)
      if (q != CLOT_ADP) y[q] += h6 * (acc[q] + f[q]);
    if (WALL) { e0 += h6 * (ae0 + fe0); c0 += h6 * (ac0 + fc0); }
  }
}

// ------------------------------------------------------------ transport

__device__ __forceinline__ float theta_at(const float* __restrict__ c, long long pitch, long long q,
                                          float invPmax) {
  return (__ldg(c + q) + __ldg(c + pitch + q) + __ldg(c + 2 * pitch + q) + __ldg(c + 3 * pitch + q)) *
         invPmax;
}

// Net outflow of the seven mobile species through the two faces of cell P
// normal to axis AX (pos = P's index along the axis, n = cells along it,
// st = index stride).  Flo / Fhi are the fluxes through the low / high face.
// Wm, WP, Wp: hindrance at P - st, P, P + st.
template <int AX>
__device__ __forceinline__ void axis_outflow(const StepArgs& A, long long P, int pos, int n, long long st,
                                             float Flo, float Fhi, float Wm, float WP, float Wp,
                                             int bidx, float Wb_in, float (&div)[NT]) {
  const StepConst& K = A.K;
  const long long pitch = K.g.pitch;
  const bool has_lo = pos > 0, has_hi = pos < n - 1;
  const bool has_lo2 = pos > 1, has_hi2 = pos < n - 2;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const float* __restrict__ r = A.cin + (long long)trow(t) * pitch;
    const bool hind = t < 2;
    const float D = K.dcoef[t][AX];
    const float cP = __ldg(r + P);
    const float cm1 = has_lo ? __ldg(r + P - st) : cP;
    const float cm2 = has_lo2 ? __ldg(r + P - 2 * st) : cm1;
    const float cp1 = has_hi ? __ldg(r + P + st) : cP;
    const float cp2 = has_hi2 ? __ldg(r + P + 2 * st) : cp1;
    float d = 0.0f;
    if (has_lo) {  // face between P - st (low) and P (high), flux counted low -> high
      const float cf = Flo >= 0.0f ? vanleer(cm2, cm1, cP, K.limiter) : vanleer(cp1, cP, cm1, K.limiter);
      const float Wa = hind ? (Flo >= 0.0f ? WP : Wm) : 1.0f;
      const float Wd = hind ? fminf(Wm, WP) : 1.0f;
      d -= Wa * Flo * cf - Wd * D * (cP - cm1);
    } else if (AX == 0 && !K.closed_ends) {  // inlet face, outward flux = -Flo
      const bool dirich = (t == 0 || t == 3 || t == 4);
      const float cb = !dirich ? cP : (t == 0 ? __ldg(A.pmu_in + bidx) : t == 3 ? __ldg(A.s1_in + bidx)
                                                                               : __ldg(A.s2_in + bidx));
      const float Fout = -Flo;
      const float Wa = hind ? (Fout > 0.0f ? Wb_in : WP) : 1.0f;
      const float Wd = hind ? fminf(WP, Wb_in) : 1.0f;
      d += Wa * Fout * cb;
      if (dirich) d -= Wd * 2.0f * D * (cb - cP);
    }
    if (has_hi) {  // face between P (low) and P + st (high)
      const float cf = Fhi >= 0.0f ? vanleer(cm1, cP, cp1, K.limiter) : vanleer(cp2, cp1, cP, K.limiter);
      const float Wa = hind ? (Fhi >= 0.0f ? Wp : WP) : 1.0f;
      const float Wd = hind ? fminf(WP, Wp) : 1.0f;
      d += Wa * Fhi * cf - Wd * D * (cp1 - cP);
    } else if (AX == 0 && !K.closed_ends) {  // outlet face: zero gradient, outward flux = Fhi
      const float Wa = hind ? WP : 1.0f;
      d += Wa * Fhi * cP;
    }
    div[t] += d;
  }
}

template <int DIM, bool TRANSPORT>
__global__ void __launch_bounds__(256) species_step_kernel(StepArgs A) {
  const StepConst& K = A.K;
  const long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= K.g.ncell) return;
  const int nx = K.g.nx, ny = K.g.ny, nz = K.g.nz;
  const long long pitch = K.g.pitch;
  const int i = (int)(P % nx);
  const int j = (int)((P / nx) % ny);
  const int k = (int)(P / ((long long)nx * ny));
  const long long sy = nx, sz = (long long)nx * ny;

  float y[CLOT_NS];
#pragma unroll
  for (int q = 0; q < CLOT_NS; ++q) y[q] = __ldg(A.cin + q * pitch + P);

  if (TRANSPORT) {
    float div[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) div[t] = 0.0f;
    const float ip = K.invPmax;
    const float WP = hindrance((y[0] + y[1] + y[2] + y[3]) * ip);
    {  // x faces: index i' + (nx + 1)(j + ny k)
      const long long f = (long long)i + (long long)(nx + 1) * (j + (long long)ny * k);
      const float Wm = i > 0 ? hindrance(theta_at(A.cin, pitch, P - 1, ip)) : WP;
      const float Wp = i < nx - 1 ? hindrance(theta_at(A.cin, pitch, P + 1, ip)) : WP;
      const int bidx = j + ny * k;
      float Wb = WP;
      if (i == 0) Wb = hindrance((__ldg(A.pmu_in + bidx) + y[1] + y[2] + y[3]) * ip);
      axis_outflow<0>(A, P, i, nx, 1, __ldg(A.fx + f), __ldg(A.fx + f + 1), Wm, WP, Wp, bidx, Wb, div);
    }
    {  // y faces: index i + nx (j' + (ny + 1) k)
      const long long f = (long long)i + (long long)nx * (j + (long long)(ny + 1) * k);
      const float Wm = j > 0 ? hindrance(theta_at(A.cin, pitch, P - sy, ip)) : WP;
      const float Wp = j < ny - 1 ? hindrance(theta_at(A.cin, pitch, P + sy, ip)) : WP;
      axis_outflow<1>(A, P, j, ny, sy, __ldg(A.fy + f), __ldg(A.fy + f + nx), Wm, WP, Wp, 0, WP, div);
    }
    if (DIM == 3) {  // z faces: index i + nx (j + ny k')
      const long long f = P;
      const float Wm = k > 0 ? hindrance(theta_at(A.cin, pitch, P - sz, ip)) : WP;
      const float Wp = k < nz - 1 ? hindrance(theta_at(A.cin, pitch, P + sz, ip)) : WP;
      axis_outflow<2>(A, P, k, nz, sz, __ldg(A.fz + f), __ldg(A.fz + f + sz), Wm, WP, Wp, 0, WP, div);
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) y[trow(t)] -= K.dtV * div[t];
    if (K.has_sigma) y[CLOT_ADP] += K.dt * __ldg(A.sigma + P);
  }

  if (K.do_reaction) {
    const RxnConst& R = K.r;
    const bool over = i >= K.g.i0 && i <= K.g.i1 && k >= K.g.k0 && k <= K.g.k1;
    const float adhH = (over && j <= K.g.hadh_jmax) ? R.kadh : 0.0f;
    const float adp = y[CLOT_ADP];
    const float A1 = R.k_adp * adp / (R.adp_star + adp);
    const float coh = R.kcohPmax * affinity(R, __ldg(A.eta + P));
    if (over && j == 0) {
      const int fidx = (i - K.g.i0) + (K.g.i1 - K.g.i0 + 1) * (k - K.g.k0);
      float e0 = A.e0[fidx], c0 = A.c0[fidx];
      rxn_rk4<true>(R, y, adhH, A1, coh, e0, c0, K.h, K.M);
      A.e0[fidx] = e0;
      A.c0[fidx] = c0;
    } else {
      float e0 = 0.0f, c0 = 0.0f;
      rxn_rk4<false>(R, y, adhH, A1, coh, e0, c0, K.h, K.M);
    }
  }
#pragma unroll
  for (int q = 0; q < CLOT_NS; ++q) A.cout[q * pitch + P] = y[q];
}

cudaError_t launch_species_step(const StepArgs& a, cudaStream_t s) {
  const int block = 256;
  const long long grid = (a.K.g.ncell + block - 1) / block;
  if (a.K.do_transport) {
    if (a.K.g.dim == 3) species_step_kernel<3, true><<<(unsigned)grid, block, 0, s>>>(a);
    else species_step_kernel<2, true><<<(unsigned)grid, block, 0, s>>>(a);
  } else {
    species_step_kernel<2, false><<<(unsigned)grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_reaction_only(const StepArgs& a, cudaStream_t s) {
  StepArgs b = a;
  b.K.do_transport = 0;
  b.K.has_sigma = 0;
  return launch_species_step(b, s);
}

}  // namespace clot

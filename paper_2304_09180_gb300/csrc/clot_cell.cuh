// clot_cell.cuh -- pieces of the fused species step shared by the tiled
// kernels (2D plane tiles, the 3D z march, the ensemble launch): the flux of
// one face, and the per-cell epilogue that turns a cell's staged state and its
// transport divergence into the end-of-step state.
//
//   face flux        App. D (van Leer face values, Gauss-linear diffusion),
//                    Sec. 3.2 (platelet fluxes hindered by W of the downwind
//                    cell for advection and of the larger theta_T for diffusion)
//   epilogue         Sec. 3.2 step 1 (explicit transport update, + dt sigma for
//                    ADP), the optional Heun average of a two-stage transport
//                    (the second-order option), the optional lagged placement
//                    of the injury-wall exchange (App. B wall fluxes and E0/C0
//                    ODEs, App. C boundary table), then Sec. 3.2 step 2: M_rxn
//                    RK4 substeps of the App. A/B reaction, coupled with E0, C0
//                    on injury faces unless the wall exchange is lagged.
#pragma once

#include "clot_model.cuh"

namespace clot {

// Net +axis flux of one species through an interior face between L and H,
// with LL / HH the cells beyond them (used only if they exist).  adv = false
// when every lane of the warp has F = 0 on this face: the advective term is
// then exactly zero and the reconstruction is skipped.
__device__ __forceinline__ float face_flux(float cLL, float cL, float cH, float cHH, bool hasLL, bool hasHH,
                                           float F, float WL, float WH, bool hind, float D, int limiter,
                                           bool adv) {
  const float Wd = hind ? fminf(WL, WH) : 1.0f;
  float f = -Wd * D * (cH - cL);
  if (adv) {
    const bool pos = F >= 0.0f;
    const float cU = pos ? cL : cH, cD = pos ? cH : cL;
    const float cUU = pos ? (hasLL ? cLL : cL) : (hasHH ? cHH : cH);
    const float cf = vanleer(cUU, cU, cD, limiter);
    const float Wa = hind ? (pos ? WH : WL) : 1.0f;
    f = fmaf(Wa * F, cf, f);
  }
  return f;
}

// M classic RK4 steps of size h of the subendothelial E0, C0 (App. B) with the
// floor cell's S1 held at s1 (its full value): J = kC0+ S1_w E0 - kC0- C0 with
// the Robin wall value S1_w = (Dd s1 + kC0- C0) / (Dd + kC0+ E0);
// E0' = -J + kC0cat C0, C0' = J - kC0cat C0.  The increments are summed apart
// from E0, C0 (as in rxn_rk4) and returned in d[0], d[1]; e0, c0 leave with
// the FP32 sums.
__device__ __forceinline__ void wall_ode_rk4(const RxnConst& R, float s1, float& e0, float& c0, float h, int M,
                                             float (&d)[2]) {
  float De = 0.0f, Dc = 0.0f;
  for (int m = 0; m < M; ++m) {
    const float eb = e0 + De, cb = c0 + Dc;
    float ke[4], kc[4];
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      const float a = st == 0 ? 0.0f : st == 3 ? h : 0.5f * h;
      const float e = st ? fmaf(a, ke[st - 1], eb) : eb;
      const float c = st ? fmaf(a, kc[st - 1], cb) : cb;
      const float w = (R.Dd * s1 + R.kC0m * c) / (R.Dd + R.kC0p * e);
      const float J = R.kC0p * w * e - R.kC0m * c;
      ke[st] = R.kC0cat * c - J;
      kc[st] = J - R.kC0cat * c;
    }
    const float h6 = h * (1.0f / 6.0f);
    De += h6 * (ke[0] + 2.0f * ke[1] + 2.0f * ke[2] + ke[3]);
    Dc += h6 * (kc[0] + 2.0f * kc[1] + 2.0f * kc[2] + kc[3]);
  }
  e0 += De;
  c0 += Dc;
  d[0] = De;
  d[1] = Dc;
}

// E0, C0 of injury face fidx after a step that moved them by d[0], d[1] from
// the stored values e0s, c0s (e0n, c0n: the FP32 sums).  With the low words
// of the deviation form the increments are added in FP64 to the (value, low
// word) pairs, which are rounded back to two floats each.
__device__ __forceinline__ void wall_store(const StepArgs& A, int fidx, float e0s, float c0s, float e0n, float c0n,
                                           const float (&d)[2]) {
  if (A.e0lo) {
    const double e = ((double)e0s + (double)A.e0lo[fidx]) + (double)d[0];
    const double c = ((double)c0s + (double)A.c0lo[fidx]) + (double)d[1];
    const float eh = (float)e, ch = (float)c;
    A.e0[fidx] = eh;
    A.e0lo[fidx] = (float)(e - (double)eh);
    A.c0[fidx] = ch;
    A.c0lo[fidx] = (float)(c - (double)ch);
  } else {
    A.e0[fidx] = e0n;
    A.c0[fidx] = c0n;
  }
}

// The rest of a cell's step once its transport divergence is known.  y holds
// the cell's 15 staged species (the state the transport stage starts from) and
// leaves with the end-of-step state, which is stored to A.cout.  dv[t] is the
// net outflow of mobile species t summed over the cell's faces (only read when
// the step transports).  sig: the cell's sigma_release; etaP: its eta.
//   - transport update c -= dt/V dv (+ dt sigma for ADP);
//   - A.cavg (two-stage Heun transport, second stage): the mobile species
//     become the mean of this stage's result and the state of A.cavg, the
//     start of the transport;
//   - K.wall_lagged on an injury floor cell: the wall fluxes of S1 and E1 over
//     dt from the start-of-transport S1, E0, C0, then the E0/C0 ODEs with S1
//     held at its post-transport value (M_rxn RK4 steps of dt / M_rxn);
//   - the reaction: K.M RK4 steps of K.h (or their exact closed form where
//     the system reduces to linear activation), the wall exchange coupled in
//     the stages unless lagged.
// IDX: the index type of the state arrays (unsigned where the caller has
// checked that CLOT_NS * pitch < 2^31, for cheaper addressing).  EXT: the
// inhibitor extension's rows ride along (A.xin after their transport, the
// result to A.xout), reacted in the same RK4 stages.
template <typename IDX = long long, bool EXT = false>
__device__ __forceinline__ void cell_epilogue(const StepArgs& A, float (&y)[CLOT_NS], const float (&dv)[NT],
                                              float sig, float etaP, int gx, int gy, int k, IDX P) {
  const StepConst& K = A.K;
  const IDX pitch = (IDX)K.g.pitch;
  float x[2] = {0.0f, 0.0f};
  if (EXT) {
    x[0] = A.xin[P];
    x[1] = A.xin[pitch + P];
  }
  auto store = [&]() {
#pragma unroll
    for (int q = 0; q < CLOT_NS; ++q) A.cout[(IDX)q * pitch + P] = y[q];
    if (EXT) {
      A.xout[P] = x[0];
      A.xout[pitch + P] = x[1];
    }
  };
  const bool over = gx >= K.g.i0 && gx <= K.g.i1 && k >= K.g.k0 && k <= K.g.k1;
  const bool wall = over && gy == 0;
  float s1_start = y[CLOT_S1];
  if (K.do_transport) {
#pragma unroll
    for (int t = 0; t < NT; ++t) y[trow(t)] -= K.dtV * dv[t];
    if (K.has_sigma) y[CLOT_ADP] += K.dt * sig;
    if (A.cavg) {
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const float ca = __ldg(A.cavg + (IDX)trow(t) * pitch + P);
        if (trow(t) == CLOT_S1) s1_start = ca;
        y[trow(t)] = 0.5f * (ca + y[trow(t)]);
      }
    }
  }
  const RxnConst& R = K.r;
  int fidx = 0;
  if (wall) fidx = (gx - K.g.i0) + (K.g.i1 - K.g.i0 + 1) * (k - K.g.k0);
  if (K.wall_lagged && wall && K.do_transport) {
    const float e0s = A.e0[fidx], c0s = A.c0[fidx];
    float e0 = e0s, c0 = c0s, d[2];
    const float s1w = (R.Dd * (s1_start + R.s1_ref) + R.kC0m * c0) / (R.Dd + R.kC0p * e0);
    const float J = R.kC0p * s1w * e0 - R.kC0m * c0;
    y[CLOT_S1] -= K.dt * R.aV * J;
    y[CLOT_E1] += K.dt * R.aV * (R.kC0cat * c0);
    wall_ode_rk4(R, y[CLOT_S1] + R.s1_ref, e0, c0, K.dt / (float)K.M, K.M, d);
    wall_store(A, fidx, e0s, c0s, e0, c0, d);
  }
  if (K.do_reaction) {
    const float adhH = (over && gy <= K.g.hadh_jmax) ? R.kadh : 0.0f;
    const float adp = y[CLOT_ADP];
    // k_adp [ADP] / ([ADP]* + [ADP]) is [ADP] itself (+-0) when [ADP] = +-0: skip the division
    const float A1 = (adp != 0.0f) ? R.k_adp * adp / (R.adp_star + adp) : adp;
    const float coh = R.kcohPmax * affinity(R, etaP);
    const bool wcpl = wall && !K.wall_lagged;
    if (EXT) {  // the reaction state with the extension's two rows
      float yx[CLOT_NX];
#pragma unroll
      for (int q = 0; q < CLOT_NS; ++q) yx[q] = y[q];
      yx[XINH] = x[0];
      yx[XE2I] = x[1];
      if (!rxn_linear_rest<CLOT_NX>(R, yx, adhH, A1, coh, wcpl, K.h, K.M)) {
        const float e0s = wcpl ? A.e0[fidx] : 0.0f, c0s = wcpl ? A.c0[fidx] : 0.0f;
        float e0 = e0s, c0 = c0s, d[2];
        const float bound = rxn_rk4_dev<CLOT_NX>(R, yx, adhH, A1, coh, wcpl, e0, c0, K.h, K.M, d);
        if (wcpl) wall_store(A, fidx, e0s, c0s, e0, c0, d);
        if (bound != 0.0f) A.bound_acc[P] += bound;
      }
#pragma unroll
      for (int q = 0; q < CLOT_NS; ++q) y[q] = yx[q];
      x[0] = yx[XINH];
      x[1] = yx[XE2I];
      store();
      return;
    }
    if (!rxn_linear_rest(R, y, adhH, A1, coh, wcpl, K.h, K.M)) {
      const float e0s = wcpl ? A.e0[fidx] : 0.0f, c0s = wcpl ? A.c0[fidx] : 0.0f;
      float e0 = e0s, c0 = c0s, d[2];
      const float bound = rxn_rk4_dev(R, y, adhH, A1, coh, wcpl, e0, c0, K.h, K.M, d);
      if (wcpl) wall_store(A, fidx, e0s, c0s, e0, c0, d);
      if (bound != 0.0f) A.bound_acc[P] += bound;
      // the full integration stores its own result: no join with the fast
      // path below while all 15 species are live
      store();
      return;
    }
  }
  store();
}

}  // namespace clot

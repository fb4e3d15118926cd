// clot_step_zmarch.cu -- K1 on 3D meshes: the fused species step (Sec. 3.2)
// marching in z through planes staged by the tensor memory accelerator.
//
// A block owns a 32 x 8 tile column of the mesh and a run of RUN planes; its
// 256 threads hold one cell each per plane.  Data movement per plane:
//   - the nine species that neighbours read (P^{m,u}, P^{m,a}, P^{b,a},
//     P^{b,se}, ADP, S1, S2, E1, E2), with a halo of 4 cells in x (so that the
//     box starts on a 16-byte boundary) and 2 in y, arrive by one 4D TMA tile
//     load (40 x 12 x 1 x 9 floats; cells outside the mesh read as zero), eta
//     and eta of the previous step by 3D loads, into a ring of four
//     shared-memory planes completing on mbarriers (waits bounded by
//     %globaltimer).  The load of plane k + 3 is issued while plane k
//     computes, so planes k, k + 1, k + 2 are resident;
//   - the six species only the cell itself reads, sigma and the face fluxes
//     are per-thread loads issued before the wait for the plane's tile, their
//     latency hidden behind that wait and the hindrance pass;
//   - results go out as coalesced stores (a warp writes 128 contiguous bytes
//     per species row).  Staging them in the ring slot of the plane just
//     computed and writing them by bulk tensor stores was measured slower
//     (the slot's refill must then wait for the store to read it).
// Compute per plane, with two block barriers (plane landed; faces published):
//   - the x and y face fluxes of every cell's low faces (and the high faces of
//     the tile's last column and row), exchanged through shared memory; the z
//     face above each cell from the own column (the face below is carried
//     from the plane underneath), so every face is computed once;
//   - W(theta_T) of the staged tile of plane k + 1 (two cells per thread, no
//     bounds tests: cells outside the mesh are never read through W) for the
//     next plane, and whether plane k + 2 holds any of the four species plain
//     plasma lacks (P^{m,a}, ADP, E1, E2), OR-ing their bit patterns; both
//     ride on the barrier that publishes the faces;
//   - a plane transports those four species only if one of them is present in
//     planes k - 1 .. k + 1 (the fluxes of an absent species are then exactly
//     zero: van Leer returns the upwind value when the two cells of a face are
//     equal).  The species set is a template parameter, so the face code runs
//     without per-species branches;
//   - the shared epilogue (clot_cell.cuh: transport update, optional Heun
//     average and lagged wall, M_rxn RK4 reaction with the injury-wall
//     exchange) and the eta prediction for the next step.
// Model: fractional step of Sec. 3.2; hindered platelet fluxes (Sec. 3.2),
// van Leer face values and Gauss-linear diffusion (App. D); boundary table of
// App. C; reaction terms of App. A and App. B.
#include "clot_cell.cuh"
#include "clot_tma.cuh"

namespace clot {
namespace {

constexpr int TX = 32, TY = 8, TNT = TX * TY;
constexpr int HXT = 4, HYT = 2;
constexpr int SXT = TX + 2 * HXT;  // 40
constexpr int SYT = TY + 2 * HYT;  // 12
constexpr int SPT = SXT * SYT;     // 480 staged cells
constexpr int NSTG = 9;            // staged species rows 0 .. 8
constexpr int RING = 4;
constexpr int RUN = 12;            // planes per block

struct alignas(128) ZPlane {
  float c[NSTG][SPT];  // 17280 B
  float eta[SPT];
  float etp[SPT];
};
struct ZSm {
  ZPlane buf[RING];
  float W[2][SPT];  // hindrance of the staged tile of plane k and of plane k + 1
  float xf[NT][TY][TX + 1];
  float yf[NT][TY + 1][TX];
  float red[2][TNT / 32];
  unsigned long long bar[RING];
};
static_assert(sizeof(ZPlane) % 128 == 0, "ring planes must stay 128-byte aligned");
static_assert(SPT % 2 == 0 && SPT / 2 <= TNT, "the hindrance pass gives each thread at most one pair");

// Species sets of the face code: the three that plain plasma carries
// (P^{m,u}, S1, S2), or all seven mobile species.
constexpr int SET_PLASMA = 0, SET_ALL = 1;
__host__ __device__ constexpr bool in_set(int S, int t) { return S == SET_ALL || t == 0 || t == 3 || t == 4; }

struct ZGeo {
  int tx, ty, tid, x0, y0, gx, gy, lastx, lasty, sc;
  bool act;
};

// Bit patterns of the non-plasma species of staged pair `tid` of a plane
// (zero exactly when all of them are +0 there).
__device__ __forceinline__ unsigned nonplasma_bits(const ZPlane& B, int tid) {
  const int q = 2 * tid;
  const uint2 a = *reinterpret_cast<const uint2*>(&B.c[CLOT_PMA][q]);
  const uint2 b = *reinterpret_cast<const uint2*>(&B.c[CLOT_ADP][q]);
  const uint2 c = *reinterpret_cast<const uint2*>(&B.c[CLOT_E1][q]);
  const uint2 d = *reinterpret_cast<const uint2*>(&B.c[CLOT_E2][q]);
  return (a.x | a.y | b.x | b.y) | (c.x | c.y | d.x | d.y);
}

// x and y face fluxes of plane k for the species of set S, before the block
// barrier that publishes them: each thread's low x and y faces (kept in xlo,
// ylo and written to xf, yf), the high x face of every row's last cell (lanes
// 0 .. TY-1 of warp 0) and the high y face of the last row.  c0 receives the
// cell's mobile species (zero for species outside S, which are absent around
// this plane).  W: hindrance of the staged cells of plane k.
template <int S>
__device__ __forceinline__ void zm_xy_faces(const StepArgs& A, ZSm& Sm, const float* W, const ZPlane& B0,
                                            const ZGeo& G, int k, float WP, float fxlo, float fylo, float fyhi,
                                            float fxhi, float (&c0)[NT], float (&xlo)[NT], float (&ylo)[NT]) {
  const StepConst& K = A.K;
  const int nx = K.g.nx, ny = K.g.ny;
  const int tx = G.tx, ty = G.ty, sc = G.sc, gx = G.gx, gy = G.gy;
  const float* pl = &B0.c[0][0];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    c0[t] = in_set(S, t) ? B0.c[trow(t)][sc] : 0.0f;
    xlo[t] = ylo[t] = 0.0f;
  }
  if (!K.do_transport) return;
  // x high face of the last cell of every tile row: lanes 0 .. TY-1 of warp 0
  if (ty == 0 && tx < TY && G.y0 + tx < ny) {
    const int row = tx, gxl = G.x0 + G.lastx;
    const int scl = (row + HYT) * SXT + (G.lastx + HXT);
    const float WPl = W[scl];
    if (gxl < nx - 1) {
      const float WH = W[scl + 1];
      const bool adv = __any_sync(__activemask(), fxhi != 0.0f);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (!in_set(S, t)) continue;
        const float* r = pl + trow(t) * SPT;
        Sm.xf[t][row][G.lastx + 1] = face_flux(r[scl - 1], r[scl], r[scl + 1], r[scl + 2], gxl >= 1, gxl + 2 < nx,
                                               fxhi, WPl, WH, t < 2, K.dcoef[t][0], K.limiter, adv);
      }
    } else {
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (in_set(S, t))
          Sm.xf[t][row][G.lastx + 1] = K.closed_ends ? 0.0f : (t < 2 ? WPl : 1.0f) * fxhi * pl[trow(t) * SPT + scl];
    }
  }
  if (!G.act) return;
  // x low face (the inlet at gx = 0)
  if (gx > 0) {
    const float WL = W[sc - 1];
    const bool adv = __any_sync(__activemask(), fxlo != 0.0f);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if (!in_set(S, t)) continue;
      const float* r = pl + trow(t) * SPT;
      xlo[t] = face_flux(r[sc - 2], r[sc - 1], c0[t], r[sc + 1], gx >= 2, gx + 1 < nx, fxlo, WL, WP, t < 2,
                         K.dcoef[t][0], K.limiter, adv);
    }
  } else if (!K.closed_ends) {
    const int b = gy + ny * k;
    const float pin = __ldg(A.pmu_in + b);
    const float Wb =
        hindrance((pin + pl[CLOT_PMA * SPT + sc] + pl[CLOT_PBA * SPT + sc] + pl[CLOT_PBSE * SPT + sc]) * K.invPmax);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if (!in_set(S, t)) continue;
      const bool hind = t < 2, dir = (t == 0 || t == 3 || t == 4);
      const float cP = c0[t];
      const float cb = !dir ? cP : (t == 0 ? pin : t == 3 ? __ldg(A.s1_in + b) : __ldg(A.s2_in + b));
      const float Fout = -fxlo;
      const float Wa = hind ? (Fout > 0.0f ? Wb : WP) : 1.0f;
      const float Wd = hind ? fminf(WP, Wb) : 1.0f;
      float out = Wa * Fout * cb;
      if (dir) out -= Wd * 2.0f * K.dcoef[t][0] * (cb - cP);
      xlo[t] = -out;
    }
  }
#pragma unroll
  for (int t = 0; t < NT; ++t)
    if (in_set(S, t)) Sm.xf[t][ty][tx] = xlo[t];
  // y low face (the floor is a wall)
  if (gy > 0) {
    const float WL = W[sc - SXT];
    const bool adv = __any_sync(__activemask(), fylo != 0.0f);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if (!in_set(S, t)) continue;
      const float* r = pl + trow(t) * SPT;
      ylo[t] = face_flux(r[sc - 2 * SXT], r[sc - SXT], c0[t], r[sc + SXT], gy >= 2, gy + 1 < ny, fylo, WL, WP, t < 2,
                         K.dcoef[t][1], K.limiter, adv);
    }
  }
#pragma unroll
  for (int t = 0; t < NT; ++t)
    if (in_set(S, t)) Sm.yf[t][ty][tx] = ylo[t];
  // y high face of the last tile row (the top wall at y = ny)
  if (ty == G.lasty) {
    if (gy < ny - 1) {
      const float WH = W[sc + SXT];
      const bool adv = __any_sync(__activemask(), fyhi != 0.0f);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (!in_set(S, t)) continue;
        const float* r = pl + trow(t) * SPT;
        Sm.yf[t][ty + 1][tx] = face_flux(r[sc - SXT], c0[t], r[sc + SXT], r[sc + 2 * SXT], gy >= 1, gy + 2 < ny, fyhi,
                                         WP, WH, t < 2, K.dcoef[t][1], K.limiter, adv);
      }
    } else {
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (in_set(S, t)) Sm.yf[t][ty + 1][tx] = 0.0f;
    }
  }
}

// After the block barrier: the z face above the cell (the one below is
// carried in fzlo from the plane underneath) and each cell's net outflow dv.
// Wp: W of the own column at k + 1.
template <int S>
__device__ __forceinline__ void zm_z_faces(const StepArgs& A, const ZSm& Sm, const ZPlane& B1, const ZPlane& B2,
                                           const ZGeo& G, int k, float WP, float Wp, float Fhi,
                                           const float (&cm1)[NT], const float (&c0)[NT], const float (&xlo)[NT],
                                           const float (&ylo)[NT], float (&fzlo)[NT], float (&dv)[NT]) {
  const StepConst& K = A.K;
  const int nz = K.g.nz, tx = G.tx, ty = G.ty, sc = G.sc;
  const bool hm1 = k >= 1, hp1 = k + 1 < nz, hp2 = k + 2 < nz;
  const bool advhi = __any_sync(__activemask(), Fhi != 0.0f);
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    if (!in_set(S, t)) {
      fzlo[t] = 0.0f;
      continue;
    }
    const float cp1 = hp1 ? B1.c[trow(t)][sc] : c0[t];
    const float cp2 = hp2 ? B2.c[trow(t)][sc] : cp1;
    const float lo = hm1 ? fzlo[t] : 0.0f;
    const float hi = hp1 ? face_flux(hm1 ? cm1[t] : c0[t], c0[t], cp1, cp2, hm1, hp2, Fhi, WP, Wp, t < 2,
                                     K.dcoef[t][2], K.limiter, advhi)
                         : 0.0f;
    dv[t] = (hi - lo) + (Sm.xf[t][ty][tx + 1] - xlo[t]) + (Sm.yf[t][ty + 1][tx] - ylo[t]);
    fzlo[t] = hi;
  }
}

// W of the staged cells of a plane, two per thread (threads 0 .. SPT/2 - 1).
__device__ __forceinline__ void zm_w_pass(const ZPlane& B, float* W, int tid, float ip) {
  if (tid >= SPT / 2) return;
  const int q = 2 * tid;
  const float2 a = *reinterpret_cast<const float2*>(&B.c[CLOT_PMU][q]);
  const float2 b = *reinterpret_cast<const float2*>(&B.c[CLOT_PMA][q]);
  const float2 c = *reinterpret_cast<const float2*>(&B.c[CLOT_PBA][q]);
  const float2 d = *reinterpret_cast<const float2*>(&B.c[CLOT_PBSE][q]);
  float2 w;
  w.x = hindrance((a.x + b.x + c.x + d.x) * ip);
  w.y = hindrance((a.y + b.y + c.y + d.y) * ip);
  *reinterpret_cast<float2*>(&W[q]) = w;
}

// Block maxima of |r| and theta_B into eta_max (float bit patterns; both >= 0).
__device__ __forceinline__ void block_max2(float rmax, float bmax, float (*red)[TNT / 32], unsigned* out, int tid) {
  for (int o = 16; o > 0; o >>= 1) {
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = rmax;
    red[1][tid >> 5] = bmax;
  }
  __syncthreads();
  if (tid == 0) {
    for (int q = 1; q < TNT / 32; ++q) {
      rmax = fmaxf(rmax, red[0][q]);
      bmax = fmaxf(bmax, red[1][q]);
    }
    if (rmax > 0.0f) atomicMax(out, __float_as_uint(rmax));
    if (bmax > 0.0f) atomicMax(out + 1, __float_as_uint(bmax));
  }
}

template <bool EXT>
__global__ void __launch_bounds__(TNT, 2)
    zmarch_step_kernel(const StepArgs A, const __grid_constant__ CUtensorMap tm_c,
                       const __grid_constant__ CUtensorMap tm_eta, const __grid_constant__ CUtensorMap tm_etp) {
  extern __shared__ unsigned char smraw[];
  ZSm& Sm = *reinterpret_cast<ZSm*>(smraw + ((128u - (smem_u32(smraw) & 127u)) & 127u));
  const StepConst& K = A.K;
  const int nx = K.g.nx, ny = K.g.ny, nz = K.g.nz;
  ZGeo G;
  G.tx = threadIdx.x;
  G.ty = threadIdx.y;
  G.tid = G.ty * TX + G.tx;
  G.x0 = blockIdx.x * TX;
  G.y0 = blockIdx.y * TY;
  G.gx = G.x0 + G.tx;
  G.gy = G.y0 + G.ty;
  G.act = G.gx < nx && G.gy < ny;
  G.lastx = min(TX - 1, nx - 1 - G.x0);
  G.lasty = min(TY - 1, ny - 1 - G.y0);
  G.sc = (G.ty + HYT) * SXT + (G.tx + HXT);
  const int tid = G.tid, sc = G.sc;
  const long long pitch = K.g.pitch, sxy = (long long)nx * ny;
  const float ip = K.invPmax;
  const int kb = blockIdx.z * RUN, ke = min(kb + RUN, nz);
  const bool need_eta = K.do_reaction || A.predict;
  const long long P0 = (long long)G.gx + (long long)nx * G.gy;
  const unsigned bytes = (unsigned)(sizeof(float) * SPT * (NSTG + (need_eta ? 1 : 0) + (A.predict ? 1 : 0)));

  if (tid == 0) {
    for (int b = 0; b < RING; ++b) mbar_init(&Sm.bar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  auto planned = [&](int k) { return k < nz && k <= ke + 1; };
  auto issue = [&](int k) {  // thread 0: arm the plane's ring slot and start its tile loads
    if (tid != 0 || !planned(k)) return;
    const int b = (k - kb) % RING;
    ZPlane& B = Sm.buf[b];
    fence_proxy_async_smem();  // earlier reads of the slot before its refill
    mbar_expect_tx(&Sm.bar[b], bytes);
    const int x = G.x0 - HXT, y = G.y0 - HYT;
    tma_load_4d(&B.c[0][0], &tm_c, x, y, k, 0, &Sm.bar[b]);
    if (need_eta) tma_load_3d(B.eta, &tm_eta, x, y, k, &Sm.bar[b]);
    if (A.predict) tma_load_3d(B.etp, &tm_etp, x, y, k, &Sm.bar[b]);
  };
  // all threads wait for plane k's loads; the block leaves together on a timeout
  auto landed = [&](int k) -> bool {
    bool ok = true;
    if (planned(k)) ok = mbar_wait_bounded(&Sm.bar[(k - kb) % RING], (unsigned)(((k - kb) / RING) & 1));
    const bool all = __syncthreads_and(ok) != 0;
    if (!all && tid == 0 && A.status) atomicOr(A.status, ST_TIMEOUT);
    return all;
  };
  // after a timeout: thread 0 waits (bounded) for the loads still in flight
  // into the ring, so that none lands after the block has left
  auto drain = [&](int from, int to) {
    if (tid != 0) return;
    for (int q = from; q <= to; ++q)
      if (planned(q)) mbar_wait_bounded(&Sm.bar[(q - kb) % RING], (unsigned)(((q - kb) / RING) & 1));
  };
  issue(kb);
  issue(kb + 1);
  issue(kb + 2);
  int issued = kb + 2;

  // own column below the run: mobile species at kb - 1 (and kb - 2 for the
  // face below the first plane), W and the eta guess at kb - 1
  float cm1[NT], fzlo[NT];
  float Wm1 = 0.0f, gm1 = 0.0f;
  unsigned pre = 0u;
  float cm2[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) cm1[t] = cm2[t] = fzlo[t] = 0.0f;
  float Flo = 0.0f;
  if (G.act && kb >= 1) {
    const long long Q = P0 + (long long)(kb - 1) * sxy;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      cm1[t] = __ldg(A.cin + (long long)trow(t) * pitch + Q);
      if (kb >= 2) cm2[t] = __ldg(A.cin + (long long)trow(t) * pitch + Q - sxy);
      if (!in_set(SET_PLASMA, t)) pre |= __float_as_uint(cm1[t]);
    }
    Wm1 = hindrance((cm1[0] + cm1[1] + __ldg(A.cin + CLOT_PBA * pitch + Q) + __ldg(A.cin + CLOT_PBSE * pitch + Q)) *
                    ip);
    if (A.predict) gm1 = 2.0f * __ldg(A.eta + Q) - __ldg(A.eta_prev + Q);
    if (K.do_transport) Flo = __ldg(A.fz + Q + sxy);
  }
  // lastp: the highest plane (up to k + 1 at plane k) known to hold a
  // non-plasma species; plane k transports only the plasma species when
  // none of planes k - 1, k, k + 1 holds one (the fluxes of an absent species
  // through the faces of plane k are exactly zero when it is absent from the
  // staged tile and from the own column one plane down and up)
  int lastp = -(1 << 29);
  if (__syncthreads_or(pre != 0u)) lastp = kb - 1;
  if (!landed(kb)) { drain(kb, issued); return; }
  if (!landed(kb + 1)) { drain(kb + 1, issued); return; }
  zm_w_pass(Sm.buf[0], Sm.W[0], tid, ip);
  if (__syncthreads_or(tid < SPT / 2 && nonplasma_bits(Sm.buf[0], tid) != 0u)) lastp = kb;
  if (planned(kb + 1) && __syncthreads_or(tid < SPT / 2 && nonplasma_bits(Sm.buf[1], tid) != 0u)) lastp = kb + 1;
  // flux through the face below the first plane, for every mobile species
  if (G.act && K.do_transport && kb >= 1) {
    const ZPlane& B0 = Sm.buf[0];
    const ZPlane& B1 = Sm.buf[1];
    const bool hm2 = kb >= 2, hp1 = kb + 1 < nz;
    const bool advlo = __any_sync(__activemask(), Flo != 0.0f);
    const float WP0 = Sm.W[0][sc];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const float c0 = B0.c[trow(t)][sc];
      const float cp1 = hp1 ? B1.c[trow(t)][sc] : c0;
      fzlo[t] = face_flux(hm2 ? cm2[t] : cm1[t], cm1[t], c0, cp1, hm2, hp1, Flo, Wm1, WP0, t < 2, K.dcoef[t][2],
                          K.limiter, advlo);
    }
  }
  float rmax = 0.0f, bmax = 0.0f;
  int wsel = 0;

  for (int k = kb; k < ke; ++k) {
    const long long P = P0 + (long long)k * sxy;
    const bool hm1 = k >= 1, hp1 = k + 1 < nz;
    // per-thread values of plane k, issued before the wait for the plane's
    // tile and in flight through it and the hindrance pass
    float yb[CLOT_NS - NSTG];
    float sig = 0.0f, fxlo = 0.0f, fylo = 0.0f, fyhi = 0.0f, fxhi = 0.0f, Fhi = 0.0f;
    if (G.act) {
#pragma unroll
      for (int q = NSTG; q < CLOT_NS; ++q) yb[q - NSTG] = __ldg(A.cin + q * pitch + P);
      if (K.do_transport) {
        if (K.has_sigma) sig = __ldg(A.sigma + P);
        const long long fxo = (long long)G.gx + (long long)(nx + 1) * (G.gy + (long long)ny * k);
        fxlo = __ldg(A.fx + fxo);
        const long long fyo = (long long)G.gx + (long long)nx * (G.gy + (long long)(ny + 1) * k);
        if (G.gy > 0) fylo = __ldg(A.fy + fyo);
        if (G.ty == G.lasty && G.gy < ny - 1) fyhi = __ldg(A.fy + fyo + nx);
        if (hp1) Fhi = __ldg(A.fz + P + sxy);
      }
    }
    if (K.do_transport && G.ty == 0 && G.tx < TY && G.y0 + G.tx < ny)
      fxhi = __ldg(A.fx + (long long)(G.x0 + G.lastx) + 1 + (long long)(nx + 1) * (G.y0 + G.tx + (long long)ny * k));

    if (!landed(k + 2)) { drain(k + 2, issued); return; }
    // every thread is past plane k - 1: its ring slot takes plane k + 3
    issue(k + 3);
    if (planned(k + 3)) issued = k + 3;
    const ZPlane& B0 = Sm.buf[(k - kb) % RING];
    const ZPlane& B1 = Sm.buf[(k + 1 - kb) % RING];
    const ZPlane& B2 = Sm.buf[(k + 2 - kb) % RING];
    const float* Wk = Sm.W[wsel];
    float* Wn = Sm.W[wsel ^ 1];

    // W of plane k + 1 for the next plane, and whether plane k + 2 holds a
    // non-plasma species; both published by the barrier after the faces
    if (hp1) zm_w_pass(B1, Wn, tid, ip);
    const unsigned np = (planned(k + 2) && tid < SPT / 2) ? nonplasma_bits(B2, tid) : 0u;

    const bool plasma = lastp < k - 1;
    const float WP = Wk[sc];
    float c0[NT], xlo[NT], ylo[NT], dv[NT];
    if (plasma)
      zm_xy_faces<SET_PLASMA>(A, Sm, Wk, B0, G, k, WP, fxlo, fylo, fyhi, fxhi, c0, xlo, ylo);
    else
      zm_xy_faces<SET_ALL>(A, Sm, Wk, B0, G, k, WP, fxlo, fylo, fyhi, fxhi, c0, xlo, ylo);
    const float yPba = B0.c[CLOT_PBA][sc], yPbse = B0.c[CLOT_PBSE][sc];
    if (__syncthreads_or(np != 0u)) lastp = k + 2;

#pragma unroll
    for (int t = 0; t < NT; ++t) dv[t] = 0.0f;
    if (G.act && K.do_transport) {
      const float Wp = hp1 ? Wn[sc] : WP;
      if (plasma)
        zm_z_faces<SET_PLASMA>(A, Sm, B1, B2, G, k, WP, Wp, Fhi, cm1, c0, xlo, ylo, fzlo, dv);
      else
        zm_z_faces<SET_ALL>(A, Sm, B1, B2, G, k, WP, Wp, Fhi, cm1, c0, xlo, ylo, fzlo, dv);
    }

    if (G.act) {
      float y[CLOT_NS];
#pragma unroll
      for (int t = 0; t < NT; ++t) y[trow(t)] = c0[t];
      y[CLOT_PBA] = yPba;
      y[CLOT_PBSE] = yPbse;
#pragma unroll
      for (int q = NSTG; q < CLOT_NS; ++q) y[q] = yb[q - NSTG];
      cell_epilogue<long long, EXT>(A, y, dv, sig, need_eta ? B0.eta[sc] : 0.0f, G.gx, G.gy, k, P);
      if (A.predict) {
        // eta for the next step: 2 eta - eta_prev, and the exact residual of
        // that guess against the new theta_B (App. A, Eq. eta)
        const float thB = (y[CLOT_PBA] + y[CLOT_PBSE]) * ip;
        auto guess = [&](int q) { return 2.0f * B0.eta[q] - B0.etp[q]; };
        const float gP = guess(sc);
        float lx = 0.0f, ly = 0.0f, lz = 0.0f;
        if (G.gx > 0) lx += guess(sc - 1) - gP;
        if (G.gx < nx - 1) lx += guess(sc + 1) - gP;
        if (G.gy > 0) ly += guess(sc - SXT) - gP;
        if (G.gy < ny - 1) ly += guess(sc + SXT) - gP;
        if (hm1) lz += gm1 - gP;
        if (hp1) lz += (2.0f * B1.eta[sc] - B1.etp[sc]) - gP;
        const float r = thB - (gP - (A.ecx * lx + A.ecy * ly + A.ecz * lz));
        A.eta_next[P] = gP;
        A.eta_res[P] = r;
        rmax = fmaxf(rmax, fabsf(r));
        bmax = fmaxf(bmax, fmaxf(thB, 0.0f));
        gm1 = gP;
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) cm1[t] = c0[t];
    }
    wsel ^= 1;
  }
  if (A.predict) block_max2(rmax, bmax, Sm.red, A.eta_max, tid);
}

}  // namespace

cudaError_t launch_zmarch_tma(const StepArgs& a, cudaStream_t s, bool* used) {
  *used = false;
  const Geom& g = a.K.g;
  auto al16 = [](const void* p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; };
  if (g.dim != 3 || g.nx % 4 != 0 || g.pitch % 4 != 0 || !al16(a.cin) || !al16(a.eta) || !al16(a.eta_prev) ||
      tensor_map_encoder() == nullptr)
    return cudaSuccess;
  const bool need_eta = a.K.do_reaction || a.predict;
  CUtensorMap tc, te, tp;
  memset(&te, 0, sizeof(te));
  memset(&tp, 0, sizeof(tp));
  if (!encode_field(&tc, a.cin, g, g.pitch, CLOT_NS, SXT, SYT, NSTG)) return cudaSuccess;
  if (need_eta && !encode_field(&te, a.eta, g, 0, 0, SXT, SYT, 0)) return cudaSuccess;
  if (a.predict && !encode_field(&tp, a.eta_prev, g, 0, 0, SXT, SYT, 0)) return cudaSuccess;
  const size_t smem = sizeof(ZSm) + 128;
  static bool attr_set[2] = {false, false};
  const bool ext = a.xin != nullptr;
  if (!attr_set[ext]) {
    cudaError_t e = cudaFuncSetAttribute(ext ? zmarch_step_kernel<true> : zmarch_step_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set[ext] = true;
  }
  dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + RUN - 1) / RUN);
  if (ext)
    zmarch_step_kernel<true><<<grid, dim3(TX, TY, 1), smem, s>>>(a, tc, te, tp);
  else
    zmarch_step_kernel<false><<<grid, dim3(TX, TY, 1), smem, s>>>(a, tc, te, tp);
  *used = true;
  return cudaGetLastError();
}

}  // namespace clot

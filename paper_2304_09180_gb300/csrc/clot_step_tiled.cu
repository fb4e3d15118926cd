// clot_step_tiled.cu -- K1, the fused species step, for the meshes the TMA z
// march of clot_step_zmarch.cu does not take, and for the ensemble launch:
//   - species_step_plane_kernel: 2D meshes (and 3D when used plane by plane).
//     A block owns a 32 x 8 tile of one plane; the nine species neighbours
//     read (P^{m,u}, P^{m,a}, P^{b,a}, P^{b,se}, ADP, S1, S2, E1, E2), eta and
//     eta of the previous step are staged by cp.async with a two-cell halo;
//     W(theta_T) is computed once per staged cell; each x / y face flux once,
//     exchanged through shared memory; z neighbours of a 3D plane from L2;
//   - species_step_zmarch_kernel: 3D meshes whose rows are not 16-byte
//     multiples (nx % 4 != 0).  A block marches a 32 x 8 tile column through
//     runs of 12 planes, staging them by cp.async into a four-plane ring,
//     three ahead; the own column's z neighbours and the flux of the z face
//     below are carried in registers;
//   - ensemble_step_kernel: the plane kernel over a work list of (channel,
//     tile, plane) items of many 3D meshes in one persistent launch;
//   - ensemble_step2d_kernel: the same for 2D channels, software-pipelined:
//     a block stages its next item (tile, eta, own-cell species, sigma and
//     face fluxes) into the second of two buffers while computing the current.
// A block skips the faces of mobile species absent from its staged data (one
// block-wide mask of OR-ed bit patterns; the 2D ensemble kernel turns the mask
// into one of two compile-time species sets, plain plasma or all seven).
// Then the shared epilogue of
// clot_cell.cuh (transport update, optional Heun average and lagged wall,
// M_rxn RK4 reaction or its closed form, injury-wall exchange) and the eta
// prediction.  Each cell's state is read from and written to HBM once per step.
//
// Model: fractional step of Sec. 3.2; hindered platelet fluxes with W of the
// downwind cell (advection) and of the larger theta_T (diffusion, localMax),
// Sec. 3.2 / App. D; van Leer face values, Gauss-linear diffusion (App. D);
// boundary table of App. C; reaction terms of App. A and App. B.
#include <type_traits>

#include "clot_cell.cuh"

namespace clot {
namespace {

constexpr int BX = 32, BY = 8, NTH = BX * BY;
// Resident blocks per SM the plane and ensemble kernels are compiled for
// (their register cap: 65536 / (NTH * PLANE_MINB)).  Three (85 registers)
// spilled the RK4 arrays: the 256-channel ensemble took 0.874 ms per step
// against 0.735 with two (128 registers, no spills).
constexpr int PLANE_MINB = 2;
constexpr int HX = 2, HY = 2;
constexpr int SX = BX + 2 * HX;  // 36
constexpr int SY = BY + 2 * HY;  // 12
constexpr int SPL = SX * SY;     // 432 cells per staged plane
constexpr int NST = 9;           // staged species rows 0 .. 8

// Staged tile layout with an x halo of HXT cells (y halo HY): 2 for the
// cp.async loaders, 4 for the TMA loads (whose x start must be a multiple of
// 4 floats, 16 bytes).
template <int HXT>
struct Lay {
  static constexpr int HX = HXT, SX = BX + 2 * HXT, SPL = SX * SY;
};
using LA = Lay<HX>;
using LT = Lay<4>;

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

// Each block is independent (no plane-to-plane dependency).  Everything a
// block reads from its neighbourhood is staged in one asynchronous batch at
// the start: the plane tile with its halo (nine species), the own-column
// values of the seven mobile species at k-2, k-1, k+1, k+2 and of P^{b,a},
// P^{b,se} at k-1, k+1 (for W there), and eta / eta of the previous step on
// the tile and at k-1, k+1.  The rest of the kernel reads shared memory only.
struct PlaneSmem {
  float plane[NST][SPL];        // rows 0..8 of plane k, halo 2 in x and y
  float zc[NT][4][NTH];         // mobile species at k-2, k-1, k+1, k+2 (own column)
  float zb[2][2][NTH];          // P^{b,a}, P^{b,se} at k-1, k+1
  float eta[SPL];               // eta on the tile (halo)
  float etp[SPL];               // eta of the previous step on the tile
  float ez[2][2][NTH];          // [eta, eta_prev][k-1, k+1] (own column)
  float W[SPL];
  float xf[NT][BY][BX + 1];
  float yf[NT][BY + 1][BX];
  float red[2][NTH / 32];
  unsigned mask;                // bit t: mobile species t is nonzero somewhere in the staged data
};

template <int VEC>
struct TileLoader {
  static constexpr int CPR = SX / VEC;
  static constexpr int NCH = SY * CPR;
  static constexpr int PER = (NCH + NTH - 1) / NTH;
  // Copies `nrow` rows (stride `rstride` floats) of the tile of plane k from
  // `src` into dst[row][SPL].
  __device__ static void load(const StepArgs& A, const float* src, long long rstride, int nrow, float* dst,
                              int k, int x0, int y0, int tid) {
    const int nx = A.K.g.nx, ny = A.K.g.ny;
    const float* base = src + (long long)k * nx * ny;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int q = tid + u * NTH;
      if (q >= NCH) continue;
      const int cx = q % CPR, sy = q / CPR;
      const int gx = x0 - HX + cx * VEC, gy = y0 - HY + sy;
      if (gy < 0 || gy >= ny || gx < 0 || gx + VEC > nx) continue;
      const int so = sy * SX + cx * VEC;
      const long long go = (long long)gy * nx + gx;
      for (int sp = 0; sp < nrow; ++sp) cp_async<VEC * 4>(dst + sp * SPL + so, base + sp * rstride + go);
    }
  }
};

// Per-thread view of one 32 x 8 tile of a plane.
struct TileGeo {
  int tx, ty, tid, x0, y0, nx, ny, nz, gx, gy, lastx, lasty, sc;
  bool act;
  long long pitch, sxy;
};

template <class L>
__device__ __forceinline__ TileGeo tile_geo(const StepConst& K, int bx, int by) {
  TileGeo G;
  G.tx = threadIdx.x;
  G.ty = threadIdx.y;
  G.tid = G.ty * BX + G.tx;
  G.x0 = bx * BX;
  G.y0 = by * BY;
  G.nx = K.g.nx;
  G.ny = K.g.ny;
  G.nz = K.g.nz;
  G.pitch = K.g.pitch;
  G.sxy = (long long)G.nx * G.ny;
  G.gx = G.x0 + G.tx;
  G.gy = G.y0 + G.ty;
  G.act = G.gx < G.nx && G.gy < G.ny;
  G.lastx = min(BX - 1, G.nx - 1 - G.x0);
  G.lasty = min(BY - 1, G.ny - 1 - G.y0);
  G.sc = (G.ty + HY) * L::SX + (G.tx + L::HX);
  return G;
}

// W per staged cell of the plane tile pl, and this thread's bits of the mobile
// species present in the staged data.  A species absent from a block's whole
// staged neighbourhood has exactly zero face fluxes there, so its transport is
// skipped (block-uniform).  Presence is the OR of the values' bit patterns
// (one logic op per value): -0.0 counts as present, which only keeps a
// species whose fluxes are zero anyway.  Blocks on the inlet keep every
// species: the inlet Dirichlet values enter there.
template <class L>
__device__ __forceinline__ unsigned w_pass(const StepConst& K, const float* pl, float* W, const TileGeo& G) {
  unsigned bits = (G.x0 == 0 && !K.closed_ends) ? ((1u << NT) - 1u) : 0u;
  unsigned ob[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) ob[t] = 0u;
  for (int q = G.tid; q < L::SPL; q += NTH) {
    const int ax = G.x0 - L::HX + q % L::SX, ay = G.y0 - HY + q / L::SX;
    float w = 0.0f;
    if (ax >= 0 && ax < G.nx && ay >= 0 && ay < G.ny) {
      w = hindrance((pl[CLOT_PMU * L::SPL + q] + pl[CLOT_PMA * L::SPL + q] + pl[CLOT_PBA * L::SPL + q] +
                     pl[CLOT_PBSE * L::SPL + q]) * K.invPmax);
#pragma unroll
      for (int t = 0; t < NT; ++t) ob[t] |= __float_as_uint(pl[trow(t) * L::SPL + q]);
    }
    W[q] = w;
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) bits |= ob[t] ? (1u << t) : 0u;
  return bits;
}

// OR of `bits` over the block into *mask (one shared atomic per warp).
__device__ __forceinline__ void mask_or(unsigned bits, unsigned* mask, int tid) {
  bits = __reduce_or_sync(0xffffffffu, bits);
  if ((tid & 31) == 0 && bits) atomicOr(mask, bits);
}

// The prescribed face fluxes a thread's faces need on plane k: its cell's x and
// y low faces, the y high face for the last tile row, and (lanes 0..BY-1 of
// warp 0) the x high face of each row's last cell.  Loaded at the top of a
// plane so that their latency overlaps the staging wait and the W pass.
struct FaceF {
  float xlo, ylo, yhi, xhi;
};
__device__ __forceinline__ FaceF load_face_fluxes(const StepArgs& A, const TileGeo& G, int k) {
  FaceF f = {0.0f, 0.0f, 0.0f, 0.0f};
  const int nx = G.nx, ny = G.ny;
  if (G.ty == 0 && G.tx < BY && G.y0 + G.tx < ny)
    f.xhi = __ldg(A.fx + (long long)(G.x0 + G.lastx) + 1 + (long long)(nx + 1) * (G.y0 + G.tx + (long long)ny * k));
  if (G.act) {
    f.xlo = __ldg(A.fx + (long long)G.gx + (long long)(nx + 1) * (G.gy + (long long)ny * k));
    const long long fyl = (long long)G.gx + (long long)nx * (G.gy + (long long)(ny + 1) * k);
    if (G.gy > 0) f.ylo = __ldg(A.fy + fyl);
    if (G.ty == G.lasty && G.gy < ny - 1) f.yhi = __ldg(A.fy + fyl + nx);
  }
  return f;
}

// Which mobile species a tile transports.  SS < 0: those whose bit is set in
// the block's presence mask (a run-time test per species); SS = SET_PLASMA or
// SET_ALL: a compile-time set, the three species of plain plasma (P^{m,u},
// S1, S2) or all seven, with no per-species branches.  The flux of a species
// absent from a tile's staged data is exactly zero (and its state +0 stays
// +0), so a set that adds absent species gives bitwise the same results.
constexpr int SET_PLASMA = 0, SET_ALL = 1;
constexpr unsigned PLASMA_BITS = (1u << 0) | (1u << 3) | (1u << 4);
template <int SS>
__device__ __forceinline__ bool species_on(unsigned mask, int t) {
  return SS < 0 ? ((mask >> t) & 1u) != 0u : (SS == SET_ALL || t == 0 || t == 3 || t == 4);
}

// x and y face fluxes of the tile into xf, yf (each face once; the low faces
// by their own cell, the high faces of the last column / row by extra lanes),
// from the fluxes FF of load_face_fluxes.
template <class L, int SS = -1>
__device__ __forceinline__ void xy_faces(const StepArgs& A, const float* pl, const float* Wk,
                                         float (*xf)[BY][BX + 1], float (*yf)[BY + 1][BX], unsigned mask,
                                         const TileGeo& G, int k, const FaceF& FF) {
  const StepConst& K = A.K;
  const int nx = G.nx, ny = G.ny, tx = G.tx, ty = G.ty, sc = G.sc, gx = G.gx, gy = G.gy;
  const float ip = K.invPmax;
  // x high faces of the last cell of every tile row: lanes 0..BY-1 of warp 0
  if (ty == 0 && tx < BY && G.y0 + tx < ny) {
    const int row = tx, gxl = G.x0 + G.lastx;
    const int scl = (row + HY) * L::SX + (G.lastx + L::HX);
    const float F = FF.xhi;
    const float WPl = Wk[scl];
    if (gxl < nx - 1) {
      const float WH = Wk[scl + 1];
      const bool adv = __any_sync(__activemask(), F != 0.0f);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (!species_on<SS>(mask, t)) continue;
        const float* r = pl + trow(t) * L::SPL;
        xf[t][row][G.lastx + 1] = face_flux(r[scl - 1], r[scl], r[scl + 1], r[scl + 2], gxl - 1 >= 0,
                                            gxl + 2 < nx, F, WPl, WH, t < 2, K.dcoef[t][0], K.limiter, adv);
      }
    } else {
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (species_on<SS>(mask, t))
          xf[t][row][G.lastx + 1] = K.closed_ends ? 0.0f : (t < 2 ? WPl : 1.0f) * F * pl[trow(t) * L::SPL + scl];
    }
  }
  if (!G.act) return;
  const float WP = Wk[sc];
  {  // x low face (inlet at gx = 0)
    const float F = FF.xlo;
    if (gx > 0) {
      const float WL = Wk[sc - 1];
      const bool adv = __any_sync(__activemask(), F != 0.0f);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (!species_on<SS>(mask, t)) continue;
        const float* r = pl + trow(t) * L::SPL;
        xf[t][ty][tx] = face_flux(r[sc - 2], r[sc - 1], r[sc], r[sc + 1], gx - 2 >= 0, gx + 1 < nx, F, WL, WP,
                                  t < 2, K.dcoef[t][0], K.limiter, adv);
      }
    } else {
      const int b = gy + ny * k;
      float Wb = WP;
      if (!K.closed_ends)
        Wb = hindrance((__ldg(A.pmu_in + b) + pl[CLOT_PMA * L::SPL + sc] + pl[CLOT_PBA * L::SPL + sc] +
                         pl[CLOT_PBSE * L::SPL + sc]) * ip);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        float out = 0.0f;
        if (!K.closed_ends) {
          const bool hind = t < 2, dir = (t == 0 || t == 3 || t == 4);
          const float cP = pl[trow(t) * L::SPL + sc];
          const float cb = !dir ? cP : (t == 0 ? __ldg(A.pmu_in + b) : t == 3 ? __ldg(A.s1_in + b)
                                                                             : __ldg(A.s2_in + b));
          const float Fout = -F;
          const float Wa = hind ? (Fout > 0.0f ? Wb : WP) : 1.0f;
          const float Wd = hind ? fminf(WP, Wb) : 1.0f;
          out = Wa * Fout * cb;
          if (dir) out -= Wd * 2.0f * K.dcoef[t][0] * (cb - cP);
        }
        xf[t][ty][tx] = -out;
      }
    }
  }
  if (gy > 0) {  // y low face (floor is a wall)
    const float F = FF.ylo;
    const float WL = Wk[sc - L::SX];
    const bool adv = __any_sync(__activemask(), F != 0.0f);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if (!species_on<SS>(mask, t)) continue;
      const float* r = pl + trow(t) * L::SPL;
      yf[t][ty][tx] = face_flux(r[sc - 2 * L::SX], r[sc - L::SX], r[sc], r[sc + L::SX], gy - 2 >= 0, gy + 1 < ny, F, WL,
                                WP, t < 2, K.dcoef[t][1], K.limiter, adv);
    }
  } else {
#pragma unroll
    for (int t = 0; t < NT; ++t) yf[t][ty][tx] = 0.0f;
  }
  if (ty == G.lasty) {  // y high face (top wall at y = ny)
    if (gy < ny - 1) {
      const float F = FF.yhi;
      const float WH = Wk[sc + L::SX];
      const bool adv = __any_sync(__activemask(), F != 0.0f);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (!species_on<SS>(mask, t)) continue;
        const float* r = pl + trow(t) * L::SPL;
        yf[t][ty + 1][tx] = face_flux(r[sc - L::SX], r[sc], r[sc + L::SX], r[sc + 2 * L::SX], gy - 1 >= 0, gy + 2 < ny,
                                      F, WP, WH, t < 2, K.dcoef[t][1], K.limiter, adv);
      }
    } else {
#pragma unroll
      for (int t = 0; t < NT; ++t) yf[t][ty + 1][tx] = 0.0f;
    }
  }
}

// The rest of a cell's step once all its face fluxes are known: the net
// outflow of each mobile species present in the block (the others have exactly
// zero fluxes), then the shared epilogue (transport update, ADP release, the
// optional Heun average and lagged wall, reaction, store).
template <bool EXT = false, int SS = -1>
__device__ __forceinline__ void finish_cell(const StepArgs& A, float (&y)[CLOT_NS], const float (&div)[NT],
                                            const float (*xf)[BY][BX + 1], const float (*yf)[BY + 1][BX],
                                            unsigned mask, float sig, float etaP, const TileGeo& G, int k,
                                            long long P) {
  const int tx = G.tx, ty = G.ty;
  float dv[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    dv[t] = 0.0f;
    if (A.K.do_transport && species_on<SS>(mask, t))
      dv[t] = div[t] + (xf[t][ty][tx + 1] - xf[t][ty][tx]) + (yf[t][ty + 1][tx] - yf[t][ty][tx]);
  }
  cell_epilogue<long long, EXT>(A, y, dv, sig, etaP, G.gx, G.gy, k, P);
}

// eta for the next step: linear extrapolation in time, 2 eta - eta_prev, and
// the exact residual of that guess against the new theta_B (App. A Eq. eta);
// em/ep are the guesses at k - 1 / k + 1 (used when hm / hp).
template <class L>
__device__ __forceinline__ float predict_cell(const StepArgs& A, const float* eta, const float* etp, float thB,
                                              bool hm, float gm, bool hp, float gp, const TileGeo& G,
                                              long long P) {
  const int sc = G.sc;
  auto guess = [&](int q) { return 2.0f * eta[q] - etp[q]; };
  const float gP = guess(sc);
  float lx = 0.0f, ly = 0.0f, lz = 0.0f;
  if (G.gx > 0) lx += guess(sc - 1) - gP;
  if (G.gx < G.nx - 1) lx += guess(sc + 1) - gP;
  if (G.gy > 0) ly += guess(sc - L::SX) - gP;
  if (G.gy < G.ny - 1) ly += guess(sc + L::SX) - gP;
  if (hm) lz += gm - gP;
  if (hp) lz += gp - gP;
  const float r = thB - (gP - (A.ecx * lx + A.ecy * ly + A.ecz * lz));
  A.eta_next[P] = gP;
  A.eta_res[P] = r;
  return r;
}

// Block maxima of |r| and theta_B into eta_max (float bit patterns; both >= 0).
__device__ __forceinline__ void block_max2(float rmax, float bmax, float (*red)[NTH / 32], unsigned* out, int tid) {
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
    for (int q = 1; q < NTH / 32; ++q) {
      rmax = fmaxf(rmax, red[0][q]);
      bmax = fmaxf(bmax, red[1][q]);
    }
    if (rmax > 0.0f) atomicMax(out, __float_as_uint(rmax));
    if (bmax > 0.0f) atomicMax(out + 1, __float_as_uint(bmax));
  }
}

// One 32 x 8 tile (tile column bx, tile row by) of plane k of the mesh A
// describes.  Called by every thread of the block (it synchronises).
template <int DIM, int VEC, bool EXT = false>
__device__ __forceinline__ void tile_step(const StepArgs& A, PlaneSmem& S, int bx, int by, int k) {
  const StepConst& K = A.K;
  const TileGeo G = tile_geo<LA>(K, bx, by);
  const int tid = G.tid, sc = G.sc, nz = G.nz;
  const long long pitch = G.pitch, sxy = G.sxy;
  const bool act = G.act;
  const float ip = K.invPmax;
  const long long P = (long long)G.gx + (long long)G.nx * (G.gy + (long long)G.ny * k);
  const bool hm1 = DIM == 3 && k >= 1, hm2 = DIM == 3 && k >= 2;
  const bool hp1 = DIM == 3 && k + 1 < nz, hp2 = DIM == 3 && k + 2 < nz;
  const bool need_eta = K.do_reaction || A.predict;

  // ---- one asynchronous staging batch
  if (tid == 0) S.mask = 0u;
  TileLoader<VEC>::load(A, A.cin, pitch, NST, &S.plane[0][0], k, G.x0, G.y0, tid);
  if (need_eta) TileLoader<VEC>::load(A, A.eta, 0, 1, S.eta, k, G.x0, G.y0, tid);
  if (A.predict) TileLoader<VEC>::load(A, A.eta_prev, 0, 1, S.etp, k, G.x0, G.y0, tid);
  if (act && DIM == 3) {
    if (K.do_transport) {
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const float* r = A.cin + (long long)trow(t) * pitch + P;
        if (hm2) cp_async<4>(&S.zc[t][0][tid], r - 2 * sxy);
        if (hm1) cp_async<4>(&S.zc[t][1][tid], r - sxy);
        if (hp1) cp_async<4>(&S.zc[t][2][tid], r + sxy);
        if (hp2) cp_async<4>(&S.zc[t][3][tid], r + 2 * sxy);
      }
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        const float* r = A.cin + (long long)(CLOT_PBA + b) * pitch + P;
        if (hm1) cp_async<4>(&S.zb[b][0][tid], r - sxy);
        if (hp1) cp_async<4>(&S.zb[b][1][tid], r + sxy);
      }
    }
    if (A.predict) {
      if (hm1) {
        cp_async<4>(&S.ez[0][0][tid], A.eta + P - sxy);
        cp_async<4>(&S.ez[1][0][tid], A.eta_prev + P - sxy);
      }
      if (hp1) {
        cp_async<4>(&S.ez[0][1][tid], A.eta + P + sxy);
        cp_async<4>(&S.ez[1][1][tid], A.eta_prev + P + sxy);
      }
    }
  }
  cp_async_commit();
  // own-cell values that only this thread needs, in registers meanwhile
  float yb[CLOT_NS - NST];
  float sig = 0.0f;
  if (act) {
#pragma unroll
    for (int q = NST; q < CLOT_NS; ++q) yb[q - NST] = __ldg(A.cin + q * pitch + P);
    if (K.do_transport && K.has_sigma) sig = __ldg(A.sigma + P);
  }
  const FaceF FF = K.do_transport ? load_face_fluxes(A, G, k) : FaceF{0.0f, 0.0f, 0.0f, 0.0f};
  cp_async_wait_all();
  __syncthreads();

  unsigned bits = w_pass<LA>(K, &S.plane[0][0], S.W, G);
  if (DIM == 3 && act && K.do_transport) {
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const bool nzv = (hm2 && S.zc[t][0][tid] != 0.0f) || (hm1 && S.zc[t][1][tid] != 0.0f) ||
                       (hp1 && S.zc[t][2][tid] != 0.0f) || (hp2 && S.zc[t][3][tid] != 0.0f);
      bits |= nzv ? (1u << t) : 0u;
    }
  }
  mask_or(bits, &S.mask, tid);
  __syncthreads();
  const unsigned mask = S.mask;

  // faces for the tile's species set (plain plasma or all seven, compile
  // time), then each cell's net outflow dv
  float dv[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) dv[t] = 0.0f;
  auto transport = [&](auto set) {
    constexpr int SS = decltype(set)::value;
    float div[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) div[t] = 0.0f;
    if (K.do_transport) {
      xy_faces<LA, SS>(A, &S.plane[0][0], S.W, S.xf, S.yf, mask, G, k, FF);
      if (DIM == 3 && act) {  // both z faces from the staged own column (floor / ceiling walls at k = 0, nz)
        const float WP = S.W[sc];
        const float Wm = hm1 ? hindrance((S.zc[0][1][tid] + S.zc[1][1][tid] + S.zb[0][0][tid] +
                                          S.zb[1][0][tid]) * ip)
                              : WP;
        const float Wp = hp1 ? hindrance((S.zc[0][2][tid] + S.zc[1][2][tid] + S.zb[0][1][tid] +
                                          S.zb[1][1][tid]) * ip)
                              : WP;
        const float Flo = hm1 ? __ldg(A.fz + P) : 0.0f;
        const float Fhi = hp1 ? __ldg(A.fz + P + sxy) : 0.0f;
        const bool advlo = __any_sync(__activemask(), Flo != 0.0f);
        const bool advhi = __any_sync(__activemask(), Fhi != 0.0f);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          if (!species_on<SS>(mask, t)) continue;
          const float c0 = S.plane[trow(t)][sc];
          const float cm1 = hm1 ? S.zc[t][1][tid] : c0;
          const float cm2 = hm2 ? S.zc[t][0][tid] : cm1;
          const float cp1 = hp1 ? S.zc[t][2][tid] : c0;
          const float cp2 = hp2 ? S.zc[t][3][tid] : cp1;
          float d = 0.0f;
          if (hm1) d -= face_flux(cm2, cm1, c0, cp1, hm2, hp1, Flo, Wm, WP, t < 2, K.dcoef[t][2], K.limiter, advlo);
          if (hp1) d += face_flux(cm1, c0, cp1, cp2, hm1, hp2, Fhi, WP, Wp, t < 2, K.dcoef[t][2], K.limiter, advhi);
          div[t] = d;
        }
      }
    }
    __syncthreads();
    if (act && K.do_transport) {  // as finish_cell
      const int tx = G.tx, ty = G.ty;
#pragma unroll
      for (int t = 0; t < NT; ++t)
        if (species_on<SS>(mask, t))
          dv[t] = div[t] + (S.xf[t][ty][tx + 1] - S.xf[t][ty][tx]) + (S.yf[t][ty + 1][tx] - S.yf[t][ty][tx]);
    }
  };
  if constexpr (DIM == 3) {  // the run-time mask: two set instances spilled at the register cap here
    transport(std::integral_constant<int, -1>{});
  } else {
    if ((mask & ~PLASMA_BITS) == 0u)
      transport(std::integral_constant<int, SET_PLASMA>{});
    else
      transport(std::integral_constant<int, SET_ALL>{});
  }

  float rmax = 0.0f, bmax = 0.0f;
  if (act) {
    float y[CLOT_NS];
#pragma unroll
    for (int q = 0; q < NST; ++q) y[q] = S.plane[q][sc];
#pragma unroll
    for (int q = NST; q < CLOT_NS; ++q) y[q] = yb[q - NST];
    cell_epilogue<long long, EXT>(A, y, dv, sig, need_eta ? S.eta[sc] : 0.0f, G.gx, G.gy, k, P);
    if (A.predict) {
      const float thB = (y[CLOT_PBA] + y[CLOT_PBSE]) * ip;
      const float gm = hm1 ? 2.0f * S.ez[0][0][tid] - S.ez[1][0][tid] : 0.0f;
      const float gp = hp1 ? 2.0f * S.ez[0][1][tid] - S.ez[1][1][tid] : 0.0f;
      rmax = fabsf(predict_cell<LA>(A, S.eta, S.etp, thB, hm1, gm, hp1, gp, G, P));
      bmax = fmaxf(thB, 0.0f);
    }
  }
  if (A.predict) block_max2(rmax, bmax, S.red, A.eta_max, tid);
}

// ---------------------------------------------------------------------------
// 3D fused step marching in z.  A block owns a 32 x 8 tile column and a run
// of KZ planes.  The planes' tiles (nine species with the halo, eta, eta of
// the previous step) stream through a ring of four shared-memory buffers by
// cp.async, three planes ahead of the one being computed, so the loads of
// plane k + 3 are in flight while plane k computes.  The own-column values of
// the two planes below stay in registers, and the flux of the z face below a
// cell is the one computed for the cell underneath one plane earlier: no z
// neighbour is loaded twice and each z face is computed once.
constexpr int ZNB = 4;
struct ZBuf {
  float c[NST][SPL];
  float eta[SPL];
  float etp[SPL];
};
struct ZSmem {
  ZBuf buf[ZNB];
  float W[SPL];
  float xf[NT][BY][BX + 1];
  float yf[NT][BY + 1][BX];
  float red[2][NTH / 32];
  unsigned mask;
};

__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }

template <int VEC>
__global__ void __launch_bounds__(NTH, 2) species_step_zmarch_kernel(StepArgs A, int KZ) {
  extern __shared__ __align__(16) unsigned char smraw[];
  ZSmem& S = *reinterpret_cast<ZSmem*>(smraw);
  const StepConst& K = A.K;
  const TileGeo G = tile_geo<LA>(K, blockIdx.x, blockIdx.y);
  const int tid = G.tid, sc = G.sc, nz = G.nz;
  const long long pitch = G.pitch, sxy = G.sxy;
  const bool act = G.act;
  const float ip = K.invPmax;
  const int kb = blockIdx.z * KZ, ke = min(kb + KZ, nz);
  const bool need_eta = K.do_reaction || A.predict;
  const long long P0 = (long long)G.gx + (long long)G.nx * G.gy;  // own cell in plane 0

  auto issue = [&](int k) {  // stage plane k (if it exists and is needed) into its ring buffer
    if (k < nz && k <= ke + 1) {
      ZBuf& B = S.buf[k % ZNB];
      TileLoader<VEC>::load(A, A.cin, pitch, NST, &B.c[0][0], k, G.x0, G.y0, tid);
      if (need_eta) TileLoader<VEC>::load(A, A.eta, 0, 1, B.eta, k, G.x0, G.y0, tid);
      if (A.predict) TileLoader<VEC>::load(A, A.eta_prev, 0, 1, B.etp, k, G.x0, G.y0, tid);
    }
    cp_async_commit();  // one group per plane, empty or not
  };
  issue(kb);
  issue(kb + 1);
  issue(kb + 2);

  // own column below the run: mobile species at kb - 1, kb - 2, W and the eta guess at kb - 1
  float cm1[NT], cm2[NT], fzlo[NT];
  float Wm1 = 0.0f, gm1 = 0.0f;
#pragma unroll
  for (int t = 0; t < NT; ++t) cm1[t] = cm2[t] = fzlo[t] = 0.0f;
  if (act && kb >= 1) {
    const long long Q = P0 + (long long)(kb - 1) * sxy;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      cm1[t] = __ldg(A.cin + (long long)trow(t) * pitch + Q);
      if (kb >= 2) cm2[t] = __ldg(A.cin + (long long)trow(t) * pitch + Q - sxy);
    }
    Wm1 = hindrance((cm1[0] + cm1[1] + __ldg(A.cin + CLOT_PBA * pitch + Q) + __ldg(A.cin + CLOT_PBSE * pitch + Q)) *
                    ip);
    if (A.predict) gm1 = 2.0f * __ldg(A.eta + Q) - __ldg(A.eta_prev + Q);
  }
  float rmax = 0.0f, bmax = 0.0f;

  for (int k = kb; k < ke; ++k) {
    const long long P = P0 + (long long)k * sxy;
    const bool hm1 = k >= 1, hm2 = k >= 2, hp1 = k + 1 < nz, hp2 = k + 2 < nz;
    issue(k + 3);
    // own-cell values that only this thread needs, meanwhile
    float yb[CLOT_NS - NST];
    float sig = 0.0f, Fhi = 0.0f, Flo = 0.0f;
    if (act) {
#pragma unroll
      for (int q = NST; q < CLOT_NS; ++q) yb[q - NST] = __ldg(A.cin + q * pitch + P);
      if (K.do_transport && K.has_sigma) sig = __ldg(A.sigma + P);
      if (K.do_transport) {
        if (hp1) Fhi = __ldg(A.fz + P + sxy);
        if (k == kb && hm1) Flo = __ldg(A.fz + P);
      }
    }
    const FaceF FF = K.do_transport ? load_face_fluxes(A, G, k) : FaceF{0.0f, 0.0f, 0.0f, 0.0f};
    if (tid == 0) S.mask = 0u;
    cp_async_wait_1();  // planes k, k + 1, k + 2 have landed
    __syncthreads();
    const ZBuf& B0 = S.buf[k % ZNB];
    const ZBuf& B1 = S.buf[(k + 1) % ZNB];
    const ZBuf& B2 = S.buf[(k + 2) % ZNB];

    float c0[NT], cp1[NT], cp2[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      c0[t] = B0.c[trow(t)][sc];
      cp1[t] = hp1 ? B1.c[trow(t)][sc] : c0[t];
      cp2[t] = hp2 ? B2.c[trow(t)][sc] : cp1[t];
    }
    unsigned bits = w_pass<LA>(K, &B0.c[0][0], S.W, G);
    if (act && K.do_transport) {
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const unsigned zb = __float_as_uint(cm2[t]) | __float_as_uint(cm1[t]) | __float_as_uint(cp1[t]) |
                            __float_as_uint(cp2[t]);
        bits |= zb ? (1u << t) : 0u;
      }
    }
    mask_or(bits, &S.mask, tid);
    __syncthreads();
    const unsigned mask = S.mask;

    float div[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) div[t] = 0.0f;
    const float WP = S.W[sc];
    const float Wp = (act && hp1) ? hindrance((cp1[0] + cp1[1] + B1.c[CLOT_PBA][sc] + B1.c[CLOT_PBSE][sc]) * ip) : WP;
    if (K.do_transport) {
      xy_faces<LA>(A, &B0.c[0][0], S.W, S.xf, S.yf, mask, G, k, FF);
      if (act) {
        const bool advlo = __any_sync(__activemask(), Flo != 0.0f);
        const bool advhi = __any_sync(__activemask(), Fhi != 0.0f);
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          float lo = 0.0f, hi = 0.0f;
          if ((mask >> t) & 1u) {
            if (hm1) {
              lo = (k == kb) ? face_flux(hm2 ? cm2[t] : cm1[t], cm1[t], c0[t], cp1[t], hm2, hp1, Flo, Wm1, WP, t < 2,
                                         K.dcoef[t][2], K.limiter, advlo)
                             : fzlo[t];
            }
            if (hp1)
              hi = face_flux(hm1 ? cm1[t] : c0[t], c0[t], cp1[t], cp2[t], hm1, hp2, Fhi, WP, Wp, t < 2,
                             K.dcoef[t][2], K.limiter, advhi);
          }
          div[t] = hi - lo;
          fzlo[t] = hi;  // the low face of the cell above
        }
      }
    }
    __syncthreads();

    if (act) {
      float y[CLOT_NS];
#pragma unroll
      for (int q = 0; q < NST; ++q) y[q] = B0.c[q][sc];
#pragma unroll
      for (int q = NST; q < CLOT_NS; ++q) y[q] = yb[q - NST];
      finish_cell(A, y, div, S.xf, S.yf, mask, sig, need_eta ? B0.eta[sc] : 0.0f, G, k, P);
      if (A.predict) {
        const float thB = (y[CLOT_PBA] + y[CLOT_PBSE]) * ip;
        const float gp = hp1 ? 2.0f * B1.eta[sc] - B1.etp[sc] : 0.0f;
        rmax = fmaxf(rmax, fabsf(predict_cell<LA>(A, B0.eta, B0.etp, thB, hm1, gm1, hp1, gp, G, P)));
        bmax = fmaxf(bmax, fmaxf(thB, 0.0f));
        gm1 = 2.0f * B0.eta[sc] - B0.etp[sc];
      }
      // own column shifts down by one plane (old values of plane k)
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        cm2[t] = cm1[t];
        cm1[t] = c0[t];
      }
      Wm1 = WP;
    }
    __syncthreads();  // plane k's buffer is refilled by the next iteration's issue
  }
  cp_async_wait_all();
  if (A.predict) block_max2(rmax, bmax, S.red, A.eta_max, tid);
}

template <int DIM, int VEC, bool EXT>
__global__ void __launch_bounds__(NTH, PLANE_MINB) species_step_plane_kernel(StepArgs A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  PlaneSmem& S = *reinterpret_cast<PlaneSmem*>(smraw);
  tile_step<DIM, VEC, EXT>(A, S, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Ensemble of independent meshes (channels) in one persistent launch: block b
// takes work items b, b + gridDim.x, ...; an item is (channel, tile column,
// tile row, plane).  The channel's step arguments are copied to shared memory
// once per item.
template <int DIM, int VEC>
__global__ void __launch_bounds__(NTH, PLANE_MINB) ensemble_step_kernel(const StepArgs* __restrict__ chans,
                                                               const int4* __restrict__ work, int nwork) {
  extern __shared__ __align__(16) unsigned char smraw[];
  PlaneSmem& S = *reinterpret_cast<PlaneSmem*>(smraw);
  __shared__ __align__(16) StepArgs sA;
  const int tid = threadIdx.y * BX + threadIdx.x;
  for (int item = blockIdx.x; item < nwork; item += gridDim.x) {
    const int4 w = work[item];
    __syncthreads();  // previous item done with sA
    {
      const int* src = reinterpret_cast<const int*>(chans + w.x);
      int* dst = reinterpret_cast<int*>(&sA);
      for (int q = tid; q < (int)(sizeof(StepArgs) / sizeof(int)); q += NTH) dst[q] = src[q];
    }
    __syncthreads();
    tile_step<DIM, VEC>(sA, S, w.y, w.z, w.w);
  }
}

// The ensemble of 2D channels, pipelined: while a block computes its work
// item, the asynchronous copies of its next item are in flight into the other
// of two staging buffers.  Everything an item reads is staged: the plane tile
// with its halo (nine species), eta and eta of the previous step on the tile,
// the six own-cell species, sigma and the face fluxes the tile's faces need.
// The copies of item i + 1 are issued before item i computes, so their
// latency hides behind a whole tile's arithmetic instead of stalling the
// block.  The addresses of those copies come from shared memory only: the
// block's work items are copied there at the start, and each channel's
// arguments two items ahead (a ring of three).  Same cell and face code as
// tile_step: the results are bitwise equal.
constexpr int EQ = 512;  // work items of a block held in shared memory (later ones are read from global memory)
struct EBuf {
  float plane[NST][SPL];
  float eta[SPL];
  float etp[SPL];
  float yb[CLOT_NS - NST][NTH];  // own-cell species NST .. CLOT_NS - 1
  float sig[NTH];
  float ff[4][NTH];              // face fluxes: x low, y low, y high, x high (the FaceF fields)
};
struct EnsSmem2 {
  EBuf buf[2];
  int4 witem[EQ];
  StepArgs args[3];
  float W[SPL];
  float xf[NT][BY][BX + 1];
  float yf[NT][BY + 1][BX];
  float red[2][NTH / 32];
  unsigned mask;
};
static_assert(sizeof(EBuf) % 16 == 0, "the work items follow the staging buffers 16-byte aligned");
static_assert(sizeof(StepArgs) % 8 == 0, "channel arguments are copied in 8-byte pieces");

// Asynchronous copy of one channel's arguments from global to shared memory.
__device__ __forceinline__ void args_async(const StepArgs* Ag, StepArgs& As, int tid) {
  constexpr int N8 = (int)(sizeof(StepArgs) / 8);
  const char* src = reinterpret_cast<const char*>(Ag);
  char* dst = reinterpret_cast<char*>(&As);
  for (int q = tid; q < N8; q += NTH) cp_async<8>(dst + 8 * q, src + 8 * q);
}

// Issues the copies of one item (tile bx, by of the 2D channel whose
// arguments A are in shared memory) into B; no wait.
template <int VEC>
__device__ __forceinline__ void stage_2d(const StepArgs& A, EBuf& B, int bx, int by) {
  const TileGeo G = tile_geo<LA>(A.K, bx, by);
  const int tid = G.tid;
  const long long pitch = G.pitch;
  TileLoader<VEC>::load(A, A.cin, pitch, NST, &B.plane[0][0], 0, G.x0, G.y0, tid);
  if (A.K.do_reaction || A.predict) TileLoader<VEC>::load(A, A.eta, 0, 1, B.eta, 0, G.x0, G.y0, tid);
  if (A.predict) TileLoader<VEC>::load(A, A.eta_prev, 0, 1, B.etp, 0, G.x0, G.y0, tid);
  const int nx = G.nx, ny = G.ny;
  if (A.K.do_transport && G.ty == 0 && G.tx < BY && G.y0 + G.tx < ny)
    cp_async<4>(&B.ff[3][tid], A.fx + (long long)(G.x0 + G.lastx) + 1 + (long long)(nx + 1) * (G.y0 + G.tx));
  if (G.act) {
    const long long P = (long long)G.gx + (long long)nx * G.gy;
#pragma unroll
    for (int q = NST; q < CLOT_NS; ++q) cp_async<4>(&B.yb[q - NST][tid], A.cin + q * pitch + P);
    if (A.K.do_transport) {
      if (A.K.has_sigma) cp_async<4>(&B.sig[tid], A.sigma + P);
      cp_async<4>(&B.ff[0][tid], A.fx + (long long)G.gx + (long long)(nx + 1) * G.gy);
      if (G.gy > 0) cp_async<4>(&B.ff[1][tid], A.fy + P);
      if (G.ty == G.lasty && G.gy < ny - 1) cp_async<4>(&B.ff[2][tid], A.fy + P + nx);
    }
  }
}

// Computes one staged item: tile_step's work from the W pass on, 2D.
__device__ __forceinline__ void compute_2d(const StepArgs& A, const EBuf& B, EnsSmem2& S, int bx, int by) {
  const StepConst& K = A.K;
  const TileGeo G = tile_geo<LA>(K, bx, by);
  const int tid = G.tid, sc = G.sc;
  const bool act = G.act;
  const bool need_eta = K.do_reaction || A.predict;
  const long long P = (long long)G.gx + (long long)G.nx * G.gy;

  mask_or(w_pass<LA>(K, &B.plane[0][0], S.W, G), &S.mask, tid);
  __syncthreads();
  const unsigned mask = S.mask;
  // the species set of the tile: plain plasma, or all seven mobile species
  const bool plasma = (mask & ~PLASMA_BITS) == 0u;

  if (K.do_transport) {
    FaceF FF = {0.0f, 0.0f, 0.0f, 0.0f};  // read under the predicates the copies were issued under
    if (G.ty == 0 && G.tx < BY && G.y0 + G.tx < G.ny) FF.xhi = B.ff[3][tid];
    if (act) {
      FF.xlo = B.ff[0][tid];
      if (G.gy > 0) FF.ylo = B.ff[1][tid];
      if (G.ty == G.lasty && G.gy < G.ny - 1) FF.yhi = B.ff[2][tid];
    }
    if (plasma)
      xy_faces<LA, SET_PLASMA>(A, &B.plane[0][0], S.W, S.xf, S.yf, mask, G, 0, FF);
    else
      xy_faces<LA, SET_ALL>(A, &B.plane[0][0], S.W, S.xf, S.yf, mask, G, 0, FF);
  }
  __syncthreads();

  float rmax = 0.0f, bmax = 0.0f;
  if (act) {
    float y[CLOT_NS];
#pragma unroll
    for (int q = 0; q < NST; ++q) y[q] = B.plane[q][sc];
#pragma unroll
    for (int q = NST; q < CLOT_NS; ++q) y[q] = B.yb[q - NST][tid];
    const float sig = (K.do_transport && K.has_sigma) ? B.sig[tid] : 0.0f;
    // net outflow of each transported species (as finish_cell, no z faces)
    float dv[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      dv[t] = 0.0f;
      const bool on = plasma ? species_on<SET_PLASMA>(0u, t) : species_on<SET_ALL>(0u, t);
      if (K.do_transport && on)
        dv[t] = 0.0f + (S.xf[t][G.ty][G.tx + 1] - S.xf[t][G.ty][G.tx]) + (S.yf[t][G.ty + 1][G.tx] - S.yf[t][G.ty][G.tx]);
    }
    cell_epilogue<long long, false>(A, y, dv, sig, need_eta ? B.eta[sc] : 0.0f, G.gx, G.gy, 0, P);
    if (A.predict) {
      const float thB = (y[CLOT_PBA] + y[CLOT_PBSE]) * K.invPmax;
      rmax = fabsf(predict_cell<LA>(A, B.eta, B.etp, thB, false, 0.0f, false, 0.0f, G, P));
      bmax = fmaxf(thB, 0.0f);
    }
  }
  if (A.predict) block_max2(rmax, bmax, S.red, A.eta_max, tid);
}

// Five block barriers per item: staged data landed (and the mask cleared),
// mask published, faces published, the eta maxima (when predicting), and the
// end of the item (its buffer and arguments free for later items).
// Block b takes items b, b + grid, b + 2 grid, ...  (Items claimed from an
// atomic counter instead, so that blocks starting late take fewer, measured
// slower: 0.652 against 0.638 ms per ensemble step.)
template <int VEC>
__global__ void __launch_bounds__(NTH, PLANE_MINB) ensemble_step2d_kernel(const StepArgs* __restrict__ chans,
                                                                  const int4* __restrict__ work, int nwork) {
  extern __shared__ __align__(16) unsigned char smraw[];
  EnsSmem2& S = *reinterpret_cast<EnsSmem2*>(smraw);
  const int tid = threadIdx.y * BX + threadIdx.x;
  if ((int)blockIdx.x >= nwork) return;
  const int nk = (nwork - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;  // this block's items
  auto witem = [&](int k) {
    return k < EQ ? S.witem[k] : work[blockIdx.x + (long long)k * gridDim.x];
  };
  for (int k = tid; k < min(nk, EQ); k += NTH) cp_async<16>(&S.witem[k], work + blockIdx.x + (long long)k * gridDim.x);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  {
    const int4 w0 = witem(0);
    args_async(chans + w0.x, S.args[0], tid);
    if (nk > 1) args_async(chans + witem(1).x, S.args[1], tid);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    stage_2d<VEC>(S.args[0], S.buf[0], w0.y, w0.z);
    cp_async_commit();
  }
  int a0 = 0;  // ring slot of item k's arguments (k mod 3)
  for (int k = 0; k < nk; ++k) {
    const int a1 = a0 == 2 ? 0 : a0 + 1, a2 = a1 == 2 ? 0 : a1 + 1;
    cp_async_wait_all();  // item k's data and item k + 1's arguments
    if (tid == 0) S.mask = 0u;
    __syncthreads();
    if (k + 1 < nk) {
      const int4 w = witem(k + 1);
      stage_2d<VEC>(S.args[a1], S.buf[(k + 1) & 1], w.y, w.z);
    }
    if (k + 2 < nk) args_async(chans + witem(k + 2).x, S.args[a2], tid);
    cp_async_commit();
    const int4 w = witem(k);
    compute_2d(S.args[a0], S.buf[k & 1], S, w.y, w.z);
    __syncthreads();
    a0 = a1;
  }
}

template <int DIM, int VEC, bool EXT>
cudaError_t launch_plane_t(const StepArgs& a, cudaStream_t s) {
  const size_t smem = sizeof(PlaneSmem);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(species_step_plane_kernel<DIM, VEC, EXT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const auto& g = a.K.g;
  dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz);
  species_step_plane_kernel<DIM, VEC, EXT><<<grid, dim3(BX, BY, 1), smem, s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int VEC>
cudaError_t launch_plane(const StepArgs& a, cudaStream_t s) {
  return a.xin ? launch_plane_t<DIM, VEC, true>(a, s) : launch_plane_t<DIM, VEC, false>(a, s);
}

constexpr int ZMARCH_KZ = 12;
template <int VEC>
cudaError_t launch_zmarch(const StepArgs& a, cudaStream_t s) {
  const size_t smem = sizeof(ZSmem);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(species_step_zmarch_kernel<VEC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const auto& g = a.K.g;
  dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + ZMARCH_KZ - 1) / ZMARCH_KZ);
  species_step_zmarch_kernel<VEC><<<grid, dim3(BX, BY, 1), smem, s>>>(a, ZMARCH_KZ);
  return cudaGetLastError();
}

template <int DIM, int VEC>
cudaError_t launch_ens(const StepArgs* chans, const int4* work, int nwork, int grid, cudaStream_t s) {
  const size_t smem = sizeof(PlaneSmem);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(ensemble_step_kernel<DIM, VEC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  ensemble_step_kernel<DIM, VEC><<<grid, dim3(BX, BY, 1), smem, s>>>(chans, work, nwork);
  return cudaGetLastError();
}

template <int VEC>
cudaError_t launch_ens2d(const StepArgs* chans, const int4* work, int nwork, int grid, cudaStream_t s) {
  const size_t smem = sizeof(EnsSmem2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(ensemble_step2d_kernel<VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  ensemble_step2d_kernel<VEC><<<grid, dim3(BX, BY, 1), smem, s>>>(chans, work, nwork);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ensemble_step(const StepArgs* chans, const int4* work, int nwork, int grid, int dim, bool vec2,
                                 cudaStream_t s) {
  if (dim == 3) return vec2 ? launch_ens<3, 2>(chans, work, nwork, grid, s) : launch_ens<3, 1>(chans, work, nwork, grid, s);
  return vec2 ? launch_ens2d<2>(chans, work, nwork, grid, s) : launch_ens2d<1>(chans, work, nwork, grid, s);
}

int ensemble_blocks_per_sm(int dim, bool vec2) {
  int n = 0;
  const size_t smem = sizeof(PlaneSmem), smem2 = sizeof(EnsSmem2);
  cudaError_t e;
  cudaFuncSetAttribute(ensemble_step_kernel<3, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(ensemble_step_kernel<3, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaFuncSetAttribute(ensemble_step2d_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  cudaFuncSetAttribute(ensemble_step2d_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  if (dim == 3)
    e = vec2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ensemble_step_kernel<3, 2>, NTH, smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ensemble_step_kernel<3, 1>, NTH, smem);
  else
    e = vec2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ensemble_step2d_kernel<2>, NTH, smem2)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ensemble_step2d_kernel<1>, NTH, smem2);
  return e == cudaSuccess ? n : 0;
}

constexpr int kTileX = BX, kTileY = BY;
int tile_x() { return kTileX; }
int tile_y() { return kTileY; }

cudaError_t launch_species_step_plane(const StepArgs& a, cudaStream_t s) {
  const bool vec2 = (a.K.g.nx % 2) == 0;
  if (a.K.g.dim == 3) {  // the TMA z march of clot_step_zmarch.cu where its alignment rules hold
    bool used = false;
    cudaError_t e = launch_zmarch_tma(a, s, &used);
    if (e != cudaSuccess || used) return e;
  }
  if (a.K.g.dim == 3) {
    if (a.xin) return cudaErrorNotSupported;  // checked by the caller: the extension takes the TMA z march
    return vec2 ? launch_zmarch<2>(a, s) : launch_zmarch<1>(a, s);
  }
  return vec2 ? launch_plane<2, 2>(a, s) : launch_plane<2, 1>(a, s);
}

}  // namespace clot

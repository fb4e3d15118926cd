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
#include "clot_cell.cuh"

namespace clot {

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

// Block-wide maximum of two non-negative floats, folded into two device words
// with atomicMax on their bit patterns (monotone for non-negative floats).
__device__ __forceinline__ void block_max2_to(float a, float b, unsigned* words) {
  __shared__ float sh[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  if (l == 0) { sh[0][w] = a; sh[1][w] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q) { a = fmaxf(a, sh[0][q]); b = fmaxf(b, sh[1][q]); }
    if (a > 0.0f) atomicMax(words, __float_as_uint(a));
    if (b > 0.0f) atomicMax(words + 1, __float_as_uint(b));
  }
}

template <int DIM, bool TRANSPORT, bool EXT = false>
__global__ void __launch_bounds__(256) species_step_kernel(StepArgs A) {
  const StepConst& K = A.K;
  const long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = P < K.g.ncell;
  const int nx = K.g.nx, ny = K.g.ny, nz = K.g.nz;
  const long long pitch = K.g.pitch;
  const int i = active ? (int)(P % nx) : 0;
  const int j = active ? (int)((P / nx) % ny) : 0;
  const int k = active ? (int)(P / ((long long)nx * ny)) : 0;
  const long long sy = nx, sz = (long long)nx * ny;
  float rmax = 0.0f, bmax = 0.0f;

  if (active) {
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
      const bool wall = over && j == 0 && !K.wall_lagged;
      const int fidx = wall ? (i - K.g.i0) + (K.g.i1 - K.g.i0 + 1) * (k - K.g.k0) : 0;
      const float e0s = wall ? A.e0[fidx] : 0.0f, c0s = wall ? A.c0[fidx] : 0.0f;
      float e0 = e0s, c0 = c0s, d[2];
      float bound;
      if (EXT) {  // the inhibitor extension's rows in the same stages, in place
        float yx[CLOT_NX];
#pragma unroll
        for (int q = 0; q < CLOT_NS; ++q) yx[q] = y[q];
        yx[XINH] = A.xin[P];
        yx[XE2I] = A.xin[pitch + P];
        bound = rxn_rk4_dev<CLOT_NX>(R, yx, adhH, A1, coh, wall, e0, c0, K.h, K.M, d);
#pragma unroll
        for (int q = 0; q < CLOT_NS; ++q) y[q] = yx[q];
        A.xout[P] = yx[XINH];
        A.xout[pitch + P] = yx[XE2I];
      } else {
        bound = rxn_rk4_dev(R, y, adhH, A1, coh, wall, e0, c0, K.h, K.M, d);
      }
      if (wall) wall_store(A, fidx, e0s, c0s, e0, c0, d);
      if (bound != 0.0f) A.bound_acc[P] += bound;
    }
#pragma unroll
    for (int q = 0; q < CLOT_NS; ++q) A.cout[q * pitch + P] = y[q];

    if (A.predict) {
      // eta for the next step: linear extrapolation in time, and the exact
      // residual of that guess against the new theta_B (App. A Eq. eta).
      const float thB = (y[CLOT_PBA] + y[CLOT_PBSE]) * K.invPmax;
      const float* __restrict__ e = A.eta;
      const float* __restrict__ ep = A.eta_prev;
      const float gP = 2.0f * __ldg(e + P) - __ldg(ep + P);
      float lx = 0.0f, ly = 0.0f, lz = 0.0f;
      if (i > 0) lx += (2.0f * __ldg(e + P - 1) - __ldg(ep + P - 1)) - gP;
      if (i < nx - 1) lx += (2.0f * __ldg(e + P + 1) - __ldg(ep + P + 1)) - gP;
      if (j > 0) ly += (2.0f * __ldg(e + P - sy) - __ldg(ep + P - sy)) - gP;
      if (j < ny - 1) ly += (2.0f * __ldg(e + P + sy) - __ldg(ep + P + sy)) - gP;
      if (DIM == 3) {
        if (k > 0) lz += (2.0f * __ldg(e + P - sz) - __ldg(ep + P - sz)) - gP;
        if (k < nz - 1) lz += (2.0f * __ldg(e + P + sz) - __ldg(ep + P + sz)) - gP;
      }
      const float r = thB - (gP - (A.ecx * lx + A.ecy * ly + A.ecz * lz));
      A.eta_next[P] = gP;
      A.eta_res[P] = r;
      rmax = fabsf(r);
      bmax = fmaxf(thB, 0.0f);
    }
  }
  if (A.predict) block_max2_to(rmax, bmax, A.eta_max);
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
  if (b.xin) {
    const int block = 256;
    const long long grid = (b.K.g.ncell + block - 1) / block;
    species_step_kernel<2, false, true><<<(unsigned)grid, block, 0, s>>>(b);
    return cudaGetLastError();
  }
  return launch_species_step(b, s);
}

// ------------------------------------------------- inhibitor extension transport

// One explicit transport pass over dt (Sec. 3.2 step 1) of the inhibitor
// extension's two rows, I and E2,inh, like the other coagulation species:
// van Leer face values and Gauss-linear diffusion with D_chem (App. D); at the
// inlet I takes the Dirichlet value I_in and E2,inh is zero-gradient, at the
// outlet both are zero-gradient, walls are impermeable (App. C table for the
// fluid-phase species).  xout = xin - dt/V (net outflow); with xavg (the
// second stage of the two-stage transport) the mean of that and xavg.
// Neighbours are read through L1 (two rows, a light pass beside the fused
// step, which reacts the rows in its RK4 stages).
__global__ void __launch_bounds__(256) ext_transport_kernel(ExtArgs a) {
  const Geom& g = a.g;
  const long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= g.ncell) return;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int i = (int)(P % nx), j = (int)((P / nx) % ny), k = (int)(P / ((long long)nx * ny));
  const long long st[3] = {1, nx, (long long)nx * ny};
  const int pos[3] = {i, j, k}, n[3] = {nx, ny, nz};
  const long long fidx[3] = {(long long)i + (long long)(nx + 1) * (j + (long long)ny * k),
                             (long long)i + (long long)nx * (j + (long long)(ny + 1) * k), P};
  const long long fstep[3] = {1, nx, (long long)nx * ny};
  const float* F[3] = {a.fx, a.fy, a.fz};
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float* x = a.xin + (long long)r * a.pitch;
    const float cP = x[P];
    float dv = 0.0f;
    for (int ax = 0; ax < g.dim; ++ax) {
      const long long s = st[ax];
      const int q = pos[ax], nn = n[ax];
      const float D = a.dcoef[ax];
      const float Flo = F[ax][fidx[ax]], Fhi = F[ax][fidx[ax] + fstep[ax]];
      float lo = 0.0f, hi = 0.0f;
      if (q > 0) {
        const float cm1 = x[P - s];
        lo = face_flux(q > 1 ? x[P - 2 * s] : cm1, cm1, cP, q + 1 < nn ? x[P + s] : cP, q > 1, q + 1 < nn, Flo, 1.0f,
                       1.0f, false, D, a.limiter, true);
      } else if (ax == 0 && !a.closed_ends) {  // inlet face, outward flux -Flo
        const float cb = r == 0 ? a.I_in : cP;
        float out = -Flo * cb;
        if (r == 0) out -= 2.0f * D * (cb - cP);
        lo = -out;
      }
      if (q + 1 < nn) {
        const float cp1 = x[P + s];
        hi = face_flux(q > 0 ? x[P - s] : cP, cP, cp1, q + 2 < nn ? x[P + 2 * s] : cp1, q > 0, q + 2 < nn, Fhi, 1.0f,
                       1.0f, false, D, a.limiter, true);
      } else if (ax == 0 && !a.closed_ends) {  // outlet: zero gradient
        hi = Fhi * cP;
      }
      dv += hi - lo;
    }
    float v = cP - a.dtV * dv;
    if (a.xavg) v = 0.5f * (a.xavg[(long long)r * a.pitch + P] + v);
    a.xout[(long long)r * a.pitch + P] = v;
  }
}

cudaError_t launch_ext_transport(const ExtArgs& a, cudaStream_t s) {
  const int block = 256;
  const long long grid = (a.g.ncell + block - 1) / block;
  ext_transport_kernel<<<(unsigned)grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace clot

// clot_eta.cu -- K2: the virtual-substance solve of App. A, Eq. eta,
//     (I - (L_eta^2 / 4) lap_h) eta = theta_B,   zero-flux boundaries,
// by conjugate gradients in one persistent cooperative launch.  Vectors are
// FP32; every dot product and norm is accumulated in FP64 and reduced in a
// fixed order, so all blocks see bit-identical scalars and the iteration is
// deterministic.  The solve is warm-started from the eta passed in and stops
// when max|r| <= max(tol * max|theta_B|, atol); since the operator is an
// M-matrix with unit row sums, max|eta - eta_exact| <= max|r|.
//
// Blocks synchronise through a sense-free generation barrier whose waits are
// bounded (2 s of globaltimer unless clot_params.wait_s says otherwise): a
// block that gives up sets ST_TIMEOUT in the status word and returns, so a
// fault can never leave the GPU spinning.  A block that returned never arrives
// at the next barrier, so every other block's next wait runs out in turn.
//
// A predicted eta (from the fused step) that misses the stopping rule is first
// corrected on a box.  Its residual r is large only where theta_B changed in a
// way the linear extrapolation did not follow -- around the clot -- and the
// correction d of A d = r decays away from there like exp(-mu n) per cell along
// an axis, cosh(mu) = 1 + 1 / (2 c_a) (the 1D Green's function of I - c_a lap_h).
// So CG runs on the bounding box of the cells with |r| > stop / (2 (1 + c)),
// c the largest c_a, widened by ln(2 c_a max|r| / stop) / mu_a cells per axis,
// with d = 0 outside, until its residual meets the stopping rule.  Then the
// true residual theta_B - A eta is recomputed on the layer of cells around the
// box, where the cut-off correction leaves its mark; every cell further out
// keeps the residual the fused step computed, below stop / 2.  If the layer
// also meets the rule the solve is done; if not, the residual is recomputed
// everywhere and CG continues on the whole mesh.  Either way the rule holds at
// exit in the same sense as without the box (the iteration's residual where
// CG ran, the computed residual elsewhere).
#include "clot_internal.cuh"

namespace clot {


__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier that also reduces: every block has written its three partial
// values (sum, sum, max) to partials[q][blk]; the last block to arrive sums
// them with all its threads (thread t takes blocks t, t + ETA_BLOCK, ..., then a
// fixed tree) -- a fixed order, so the result is deterministic -- stores the
// three results in out[0..2], then releases the others.  Waits are bounded
// (wait_ns of globaltimer, 2 s by default): a block that gives up sets
// ST_TIMEOUT and the function returns false in all its threads.
__device__ bool grid_reduce3(unsigned* bar, int* status, int nb, const double* partials, double* out,
                             double& s0, double& s1, double& m2, unsigned long long wait_ns) {
  __shared__ int ok, last;
  __shared__ unsigned gen0;
  __shared__ double sh[3][ETA_BLOCK];
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    gen0 = *((volatile unsigned*)(bar + 1));
    __threadfence();
    last = (atomicAdd(bar, 1u) == (unsigned)nb - 1) ? 1 : 0;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double a = 0.0, b = 0.0, c = 0.0;
    for (int q = threadIdx.x; q < nb; q += ETA_BLOCK) {
      a += __ldcg(partials + q);
      b += __ldcg(partials + nb + q);
      c = fmax(c, __ldcg(partials + 2 * nb + q));
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int w = ETA_BLOCK / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
        sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
        sh[2][threadIdx.x] = fmax(sh[2][threadIdx.x], sh[2][threadIdx.x + w]);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      out[0] = sh[0][0];
      out[1] = sh[1][0];
      out[2] = sh[2][0];
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    }
  } else if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned long long t0 = now_ns();
    while (*gen == gen0) {
      if (now_ns() - t0 > wait_ns) {
        atomicOr(status, ST_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  if (!ok) return false;
  s0 = __ldcg(out);
  s1 = __ldcg(out + 1);
  m2 = __ldcg(out + 2);
  return true;
}

// Block-level reduction of three values (sum, sum, max) into partials[q][blk];
// per-thread partials arrive in FP32, the block and grid sums are FP64.
__device__ void block_reduce3(double s0, double s1, double m2, double* partials, int nb) {
  __shared__ double sh[3][ETA_BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    m2 = fmax(m2, __shfl_xor_sync(0xffffffffu, m2, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sh[0][w] = s0; sh[1][w] = s1; sh[2][w] = m2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0;
    for (int q = 0; q < ETA_BLOCK / 32; ++q) { a += sh[0][q]; b += sh[1][q]; c = fmax(c, sh[2][q]); }
    partials[blockIdx.x] = a;
    partials[nb + blockIdx.x] = b;
    partials[2 * nb + blockIdx.x] = c;
  }
}

// y = (I - cL lap) x at cell P = (i, j, k) with zero-flux boundaries (missing
// neighbours contribute nothing).  x is read through L2 (__ldcg): it changes
// between phases of the same launch, so the non-coherent path must not be used.
__device__ __forceinline__ float apply_op(const EtaArgs& a, const float* x, long long P, int i, int j, int k) {
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const float xp = __ldcg(x + P);
  float lx = 0.0f, ly = 0.0f, lz = 0.0f;
  if (i > 0) lx += __ldcg(x + P - 1) - xp;
  if (i < nx - 1) lx += __ldcg(x + P + 1) - xp;
  if (j > 0) ly += __ldcg(x + P - nx) - xp;
  if (j < ny - 1) ly += __ldcg(x + P + nx) - xp;
  if (a.g.dim == 3) {
    const long long sz = (long long)nx * ny;
    if (k > 0) lz += __ldcg(x + P - sz) - xp;
    if (k < nz - 1) lz += __ldcg(x + P + sz) - xp;
  }
  return xp - (a.cx * lx + a.cy * ly + a.cz * lz);
}

// Visit every cell once: each warp takes 32-cell chunks of x rows (one
// integer division per chunk, coalesced along x).
template <class Fn>
__device__ __forceinline__ void for_cells(const EtaArgs& a, Fn fn) {
  const int nx = a.g.nx, ny = a.g.ny;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int cprw = (nx + 31) >> 5;
  const int nch = ny * a.g.nz * cprw;
  for (int ch = warp; ch < nch; ch += nwarps) {
    const int xc = ch % cprw, r = ch / cprw;
    const int j = r % ny, k = r / ny;
    const int i = xc * 32 + lane;
    if (i < nx) fn((long long)i + (long long)nx * r, i, j, k);
  }
}

// for_cells restricted to a box (32-cell chunks along x inside the box).
template <class Fn>
__device__ __forceinline__ void for_box_cells(const EtaArgs& a, const Box& b, Fn fn) {
  const int nx = a.g.nx, ny = a.g.ny;
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int bnx = b.i1 - b.i0 + 1, bny = b.j1 - b.j0 + 1;
  const int cprw = (bnx + 31) >> 5;
  const int nch = cprw * bny * (b.k1 - b.k0 + 1);
  for (int ch = warp; ch < nch; ch += nwarps) {
    const int xc = ch % cprw, r = ch / cprw;
    const int j = b.j0 + r % bny, k = b.k0 + r / bny;
    const int i = b.i0 + xc * 32 + lane;
    if (i <= b.i1) fn((long long)i + (long long)nx * (j + (long long)ny * k), i, j, k);
  }
}

// Quads: four x-consecutive cells, moved as one float4 (needs nx % 4 == 0 and
// 16-byte aligned vectors).  Thread t takes quads t, t + T, ...: a warp reads
// 512 contiguous bytes per vector, and every thread has four cells' loads in
// flight at once -- the scalar passes are bound by memory latency, not by
// bandwidth.
__device__ __forceinline__ bool al16(const void* p) { return ((unsigned long long)p & 15u) == 0; }
__device__ __forceinline__ float4 ld4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

template <class Fn>
__device__ __forceinline__ void for_quads(const EtaArgs& a, Fn fn) {
  const unsigned nqx = (unsigned)a.g.nx >> 2, ny = (unsigned)a.g.ny;
  const unsigned nq = (unsigned)(a.g.ncell >> 2);
  const unsigned T = gridDim.x * blockDim.x;
  for (unsigned qd = blockIdx.x * blockDim.x + threadIdx.x; qd < nq; qd += T) {
    const unsigned row = qd / nqx;
    fn(4ll * qd, (int)(4u * (qd - row * nqx)), (int)(row % ny), (int)(row / ny));
  }
}

// x - (cx lx + cy ly + cz lz) for the quad at P = (i..i+3, j, k), zero-flux
// walls, with the field given by a quad loader v4 and a single-cell loader v1;
// the same per-cell expression as apply_op.  Returns the quad's own values in x.
template <class V4, class V1>
__device__ __forceinline__ float4 quad_op(const EtaArgs& a, long long P, int i, int j, int k, V4 v4, V1 v1,
                                          float4& x) {
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  x = v4(P);
  float lx[4], ly[4] = {0.0f, 0.0f, 0.0f, 0.0f}, lz[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const float c[4] = {x.x, x.y, x.z, x.w};
  lx[0] = (i > 0) ? (v1(P - 1) - c[0]) + (c[1] - c[0]) : (c[1] - c[0]);
  lx[1] = (c[0] - c[1]) + (c[2] - c[1]);
  lx[2] = (c[1] - c[2]) + (c[3] - c[2]);
  lx[3] = (i + 4 < nx) ? (c[2] - c[3]) + (v1(P + 4) - c[3]) : (c[2] - c[3]);
  if (j > 0) {
    const float4 d = v4(P - nx);
    ly[0] = d.x - c[0]; ly[1] = d.y - c[1]; ly[2] = d.z - c[2]; ly[3] = d.w - c[3];
  }
  if (j < ny - 1) {
    const float4 u = v4(P + nx);
    ly[0] += u.x - c[0]; ly[1] += u.y - c[1]; ly[2] += u.z - c[2]; ly[3] += u.w - c[3];
  }
  if (a.g.dim == 3) {
    const long long sz = (long long)nx * ny;
    if (k > 0) {
      const float4 d = v4(P - sz);
      lz[0] = d.x - c[0]; lz[1] = d.y - c[1]; lz[2] = d.z - c[2]; lz[3] = d.w - c[3];
    }
    if (k < nz - 1) {
      const float4 u = v4(P + sz);
      lz[0] += u.x - c[0]; lz[1] += u.y - c[1]; lz[2] += u.z - c[2]; lz[3] += u.w - c[3];
    }
  }
  float q[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) q[m] = c[m] - (a.cx * lx[m] + a.cy * ly[m] + a.cz * lz[m]);
  return make_float4(q[0], q[1], q[2], q[3]);
}

// CG with one grid reduction per iteration (Chronopoulos and Gear's
// formulation: with s = A p carried by a recurrence, s_i = w_i + beta_i s_{i-1}
// and w = A r, the two inner products (r, r) and (w, r) of an iteration are
// taken together).  Per iteration one pass: at each cell and its neighbours
// s_i = w_i + beta_i s_{i-1} and r_{i+1} = r_i - alpha_i s_i are formed on the
// fly, the cell's p_i = r_i + beta_i p_{i-1} updates eta, and w_{i+1} = A r_{i+1}
// with (r_{i+1}, r_{i+1}), (w_{i+1}, r_{i+1}) and max |r_{i+1}| goes to the one
// reduction; then beta_{i+1} = gamma_{i+1} / gamma_i and
// alpha_{i+1} = gamma_{i+1} / (delta_{i+1} - beta_{i+1} gamma_{i+1} / alpha_i).
// Every vector is double-buffered (no block overwrites a value another block
// still reads), so the traffic per iteration is that of the two-pass form.
// On entry a.r holds r_0 (s_rr its squared norm, s_rmax its maximum).
// Returns false if a grid barrier gave up.
__device__ bool cg_single_reduction(const EtaArgs& a, bool v4, int nb, double* res, double s_rr, double& s_rmax,
                                    double stop, int& it) {
  const long long n = a.g.ncell;
  float* R[2] = {a.r, a.cg5};
  float* Sv[2] = {a.cg5 + n, a.cg5 + 2 * n};
  float* Wv[2] = {a.cg5 + 3 * n, a.cg5 + 4 * n};
  float* Pv[2] = {a.p, a.p2};
  double d0, d1, s_del;
  // w_0 = A r_0 and delta_0 = (w_0, r_0)
  {
    float del = 0.0f;
    if (v4) {
      const float* r0 = R[0];
      for_quads(a, [&](long long P, int i, int j, int k) {
        float4 x;
        const float4 w = quad_op(a, P, i, j, k, [&](long long Q) { return ld4(r0 + Q); },
                                 [&](long long Q) { return __ldcg(r0 + Q); }, x);
        st4(Wv[0] + P, w);
        del += w.x * x.x + w.y * x.y + w.z * x.z + w.w * x.w;
      });
    } else {
      for_cells(a, [&](long long P, int i, int j, int k) {
        const float w = apply_op(a, R[0], P, i, j, k);
        Wv[0][P] = w;
        del += w * __ldcg(R[0] + P);
      });
    }
    block_reduce3(del, 0.0, 0.0, a.partials, nb);
    if (!grid_reduce3(a.bar, a.status, nb, a.partials, res, s_del, d0, d1, a.wait_ns)) return false;
  }
  if (!(s_del > 0.0)) return true;
  double gamma = s_rr, alpha = s_rr / s_del, beta = 0.0;
  int cur = 0;
  while (it < a.maxit && s_rmax > stop) {
    const float al = (float)alpha, bt = (float)beta;
    const float* r = R[cur];
    const float* w = Wv[cur];
    const float* sp = Sv[cur ^ 1];
    const float* pp = Pv[cur ^ 1];
    float* rn = R[cur ^ 1];
    float* wn = Wv[cur ^ 1];
    float* sc = Sv[cur];
    float* pc = Pv[cur];
    float g = 0.0f, del = 0.0f, rm = 0.0f;
    if (v4) {
      auto s4 = [&](long long Q) {
        float4 v = ld4(w + Q);
        if (bt != 0.0f) {
          const float4 o = ld4(sp + Q);
          v.x += bt * o.x; v.y += bt * o.y; v.z += bt * o.z; v.w += bt * o.w;
        }
        return v;
      };
      auto r4 = [&](long long Q) {
        const float4 sv = s4(Q), rv = ld4(r + Q);
        return make_float4(rv.x - al * sv.x, rv.y - al * sv.y, rv.z - al * sv.z, rv.w - al * sv.w);
      };
      auto r1 = [&](long long Q) {
        const float sv = __ldcg(w + Q) + (bt != 0.0f ? bt * __ldcg(sp + Q) : 0.0f);
        return __ldcg(r + Q) - al * sv;
      };
      for_quads(a, [&](long long P, int i, int j, int k) {
        const float4 sv = s4(P), rv = ld4(r + P), e = ld4(a.eta + P);
        float4 pv = rv;
        if (bt != 0.0f) {
          const float4 o = ld4(pp + P);
          pv.x += bt * o.x; pv.y += bt * o.y; pv.z += bt * o.z; pv.w += bt * o.w;
        }
        st4(sc + P, sv);
        st4(pc + P, pv);
        st4(a.eta + P, make_float4(e.x + al * pv.x, e.y + al * pv.y, e.z + al * pv.z, e.w + al * pv.w));
        float4 x;
        const float4 wv = quad_op(a, P, i, j, k, r4, r1, x);  // x: r_{i+1} on the quad
        st4(rn + P, x);
        st4(wn + P, wv);
        g += x.x * x.x + x.y * x.y + x.z * x.z + x.w * x.w;
        del += wv.x * x.x + wv.y * x.y + wv.z * x.z + wv.w * x.w;
        rm = fmaxf(fmaxf(rm, fmaxf(fabsf(x.x), fabsf(x.y))), fmaxf(fabsf(x.z), fabsf(x.w)));
      });
    } else {
      for_cells(a, [&](long long P, int i, int j, int k) {
        const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
        auto sv = [&](long long Q) { return __ldcg(w + Q) + (bt != 0.0f ? bt * __ldcg(sp + Q) : 0.0f); };
        auto rv = [&](long long Q) { return __ldcg(r + Q) - al * sv(Q); };
        const float sP = sv(P);
        const float pP = __ldcg(r + P) + (bt != 0.0f ? bt * __ldcg(pp + P) : 0.0f);
        sc[P] = sP;
        pc[P] = pP;
        a.eta[P] = __ldcg(a.eta + P) + al * pP;
        const float rP = __ldcg(r + P) - al * sP;
        float lx = 0.0f, ly = 0.0f, lz = 0.0f;
        if (i > 0) lx += rv(P - 1) - rP;
        if (i < nx - 1) lx += rv(P + 1) - rP;
        if (j > 0) ly += rv(P - nx) - rP;
        if (j < ny - 1) ly += rv(P + nx) - rP;
        if (a.g.dim == 3) {
          const long long sz = (long long)nx * ny;
          if (k > 0) lz += rv(P - sz) - rP;
          if (k < nz - 1) lz += rv(P + sz) - rP;
        }
        const float wP = rP - (a.cx * lx + a.cy * ly + a.cz * lz);
        rn[P] = rP;
        wn[P] = wP;
        g += rP * rP;
        del += wP * rP;
        rm = fmaxf(rm, fabsf(rP));
      });
    }
    block_reduce3(g, del, rm, a.partials, nb);
    double s_g;
    if (!grid_reduce3(a.bar, a.status, nb, a.partials, res + 3 * ((it + 1) & 1), s_g, s_del, s_rmax, a.wait_ns))
      return false;
    ++it;
    beta = s_g / gamma;
    const double den = s_del - beta * s_g / alpha;
    if (!(den > 0.0) || !(s_g > 0.0)) break;
    alpha = s_g / den;
    gamma = s_g;
    cur ^= 1;
  }
  return true;
}

__global__ void __launch_bounds__(ETA_BLOCK, 2) eta_cg_kernel(EtaArgs a) {
  const int nb = gridDim.x;
  const long long pitch = a.g.pitch;
  double* res = a.partials + 3 * nb;  // three reduced scalars (written by the last block)
  double d0, d1;

  double s_rr, s_rmax, s_bmax;
  int it = 0;
  const bool v4 = (a.g.nx & 3) == 0 && (pitch & 3) == 0 && al16(a.c) && al16(a.eta) && al16(a.r) && al16(a.p) &&
                  al16(a.q) && al16(a.p2);
  bool full = !a.predicted;  // compute the residual of eta on the whole mesh first
  if (a.predicted) {
    // The previous species step stored a predicted eta (in a.eta), its
    // residual r and the maxima of |r| and theta_B.  Accept the guess if it
    // already meets the stopping rule; otherwise iterate from it.
    const float pr = __uint_as_float(__ldcg(a.maxw));
    const float pb = __uint_as_float(__ldcg(a.maxw + 1));
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      a.maxw_clear[0] = 0u;
      a.maxw_clear[1] = 0u;
      a.status[1] = 0;
    }
    if (pb > 0.0f && pr <= fmaxf(a.tol * pb, a.atol)) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.status + 3, 1);  // accepted predictions
      return;
    }
    const double stop = (double)a.inner * fmax((double)a.tol * pb, (double)a.atol);
    // Core threshold: a cell just inside the box edge with |r| <= thr gets a
    // correction of about thr, which the zero outside turns into a residual
    // of up to (1 + c) thr in the next cell out; with thr = stop / (2 (1 + c))
    // that and the decayed core correction each stay below stop / 2.
    const float cmax = fmaxf(a.cx, fmaxf(a.cy, a.cz));
    const float thr = (float)(0.5 * stop) / (1.0f + cmax);
    // sum of r^2 and the bounding box of the cells with |r| > thr, kept as
    // max(~lo) and max(hi + 1) per axis in bar[2..7] (zeroed before the launch)
    unsigned* bw = a.bar + 2;
    float rr = 0.0f;
    unsigned bl[3] = {0u, 0u, 0u}, bh[3] = {0u, 0u, 0u};
    auto mark = [&](float r, int i, int j, int k) {
      if (fabsf(r) > thr) {
        bl[0] = max(bl[0], ~(unsigned)i);
        bl[1] = max(bl[1], ~(unsigned)j);
        bl[2] = max(bl[2], ~(unsigned)k);
        bh[0] = max(bh[0], (unsigned)i + 1u);
        bh[1] = max(bh[1], (unsigned)j + 1u);
        bh[2] = max(bh[2], (unsigned)k + 1u);
      }
    };
    if (v4) {
      for_quads(a, [&](long long P, int i, int j, int k) {
        const float4 r = ld4(a.r + P);
        rr += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
        if (fmaxf(fmaxf(fabsf(r.x), fabsf(r.y)), fmaxf(fabsf(r.z), fabsf(r.w))) > thr) {
          mark(r.x, i, j, k);
          mark(r.y, i + 1, j, k);
          mark(r.z, i + 2, j, k);
          mark(r.w, i + 3, j, k);
        }
      });
    } else {
      for_cells(a, [&](long long P, int i, int j, int k) {
        const float r = __ldcg(a.r + P);
        rr += r * r;
        mark(r, i, j, k);
      });
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      bl[d] = __reduce_max_sync(0xffffffffu, bl[d]);
      bh[d] = __reduce_max_sync(0xffffffffu, bh[d]);
    }
    if ((threadIdx.x & 31) == 0 && bh[0] != 0u) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        atomicMax(bw + d, bl[d]);
        atomicMax(bw + 3 + d, bh[d]);
      }
    }
    block_reduce3(rr, 0.0, 0.0, a.partials, nb);
    if (!grid_reduce3(a.bar, a.status, nb, a.partials, res, s_rr, d0, d1, a.wait_ns)) return;
    s_rmax = pr;
    s_bmax = pb;

    Box B;
    bool use_box = false;
    const unsigned hx = __ldcg(bw + 3);
    if (pb > 0.0f && pr < 3.0e38f && hx != 0u) {
      const int mx = box_margin(a.cx, pr, (float)stop), my = box_margin(a.cy, pr, (float)stop);
      const int mz = a.g.dim == 3 ? box_margin(a.cz, pr, (float)stop) : 0;
      B.i0 = max((int)~__ldcg(bw + 0) - mx, 0);
      B.j0 = max((int)~__ldcg(bw + 1) - my, 0);
      B.k0 = max((int)~__ldcg(bw + 2) - mz, 0);
      B.i1 = min((int)hx - 1 + mx, a.g.nx - 1);
      B.j1 = min((int)__ldcg(bw + 4) - 1 + my, a.g.ny - 1);
      B.k1 = min((int)__ldcg(bw + 5) - 1 + mz, a.g.nz - 1);
      use_box = 2 * B.cells() <= a.g.ncell;
    }
    if (use_box) {
      // CG for the correction on the box, in place on eta and r, with the
      // search direction zero outside the box
      float* pold = a.p;
      float* pnew = a.p2;
      float beta = 0.0f;
      double s_rb = 0.0, s_mb = pr;
      bool first = true;
      while (it < a.maxit && s_mb > stop) {
        float pq = 0.0f, r0 = 0.0f;
        const float bt = beta;
        const float* po = pold;
        float* pn = pnew;
        for_box_cells(a, B, [&](long long P, int i, int j, int k) {
          const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
          auto pv = [&](long long Q) { return __ldcg(a.r + Q) + (bt != 0.0f ? bt * __ldcg(po + Q) : 0.0f); };
          const float pp = pv(P);
          float lx = 0.0f, ly = 0.0f, lz = 0.0f;
          if (i > 0) lx += (i - 1 >= B.i0 ? pv(P - 1) : 0.0f) - pp;
          if (i < nx - 1) lx += (i + 1 <= B.i1 ? pv(P + 1) : 0.0f) - pp;
          if (j > 0) ly += (j - 1 >= B.j0 ? pv(P - nx) : 0.0f) - pp;
          if (j < ny - 1) ly += (j + 1 <= B.j1 ? pv(P + nx) : 0.0f) - pp;
          if (a.g.dim == 3) {
            const long long sz = (long long)nx * ny;
            if (k > 0) lz += (k - 1 >= B.k0 ? pv(P - sz) : 0.0f) - pp;
            if (k < nz - 1) lz += (k + 1 <= B.k1 ? pv(P + sz) : 0.0f) - pp;
          }
          const float q = pp - (a.cx * lx + a.cy * ly + a.cz * lz);
          pn[P] = pp;
          a.q[P] = q;
          pq += pp * q;
          if (first) {
            const float r = __ldcg(a.r + P);
            r0 += r * r;
          }
        });
        block_reduce3(pq, r0, 0.0, a.partials, nb);
        double s_pq, s_r0;
        if (!grid_reduce3(a.bar, a.status, nb, a.partials, res, s_pq, s_r0, d1, a.wait_ns)) return;
        if (first) s_rb = s_r0;
        first = false;
        if (!(s_pq > 0.0)) break;
        const float alpha = (float)(s_rb / s_pq);
        float rr2 = 0.0f, rm = 0.0f;
        for_box_cells(a, B, [&](long long P, int, int, int) {
          const float pP = __ldcg(pn + P);
          a.eta[P] = __ldcg(a.eta + P) + alpha * pP;
          const float r = __ldcg(a.r + P) - alpha * __ldcg(a.q + P);
          a.r[P] = r;
          rr2 += r * r;
          rm = fmaxf(rm, fabsf(r));
        });
        block_reduce3(rr2, 0.0, rm, a.partials, nb);
        double s_rr2;
        if (!grid_reduce3(a.bar, a.status, nb, a.partials, res + 3, s_rr2, d0, s_mb, a.wait_ns)) return;
        beta = (float)(s_rr2 / s_rb);
        s_rb = s_rr2;
        float* t = pold;
        pold = pnew;
        pnew = t;
        ++it;
      }
      // The box carries the CG residual (the recursive one, as in the global
      // iteration: recomputing theta_B - A eta in FP32 there would mostly show
      // eta's own rounding, amplified up to 1 + 12 c times).  The cells just
      // outside it get the true residual, which is where cutting the
      // correction off shows; every cell further out keeps its residual <= thr.
      Box L = B;
      L.i0 = max(B.i0 - 1, 0);
      L.j0 = max(B.j0 - 1, 0);
      L.k0 = max(B.k0 - 1, 0);
      L.i1 = min(B.i1 + 1, a.g.nx - 1);
      L.j1 = min(B.j1 + 1, a.g.ny - 1);
      L.k1 = min(B.k1 + 1, a.g.nz - 1);
      float vm = 0.0f;
      for_box_cells(a, L, [&](long long P, int i, int j, int k) {
        if (B.in(i, j, k)) return;
        const float b = (__ldcg(a.c + 2 * pitch + P) + __ldcg(a.c + 3 * pitch + P)) * a.invPmax;
        const float r = b - apply_op(a, a.eta, P, i, j, k);
        a.r[P] = r;
        vm = fmaxf(vm, fabsf(r));
      });
      block_reduce3(0.0, 0.0, vm, a.partials, nb);
      double s_vm;
      if (!grid_reduce3(a.bar, a.status, nb, a.partials, res, d0, d1, s_vm, a.wait_ns)) return;
      if (s_mb <= stop && s_vm <= stop) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
          a.status[1] = it;
          atomicAdd(a.status + 2, it);
          atomicAdd(a.status + 4, 1);  // predictions corrected on a box
        }
        return;
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.status + 5, 1);  // box corrections not enough
      full = true;  // continue on the whole mesh from the improved eta
    }
  }
  if (full) {
    // r = theta_B - A eta
    float rr = 0.0f, rmax = 0.0f, bmax = 0.0f;
    if (v4) {
      const float* eta = a.eta;
      for_quads(a, [&](long long P, int i, int j, int k) {
        const float4 b2 = ld4(a.c + 2 * pitch + P), b3 = ld4(a.c + 3 * pitch + P);
        float4 x;
        const float4 q = quad_op(a, P, i, j, k, [&](long long Q) { return ld4(eta + Q); },
                                 [&](long long Q) { return __ldcg(eta + Q); }, x);
        const float b[4] = {(b2.x + b3.x) * a.invPmax, (b2.y + b3.y) * a.invPmax, (b2.z + b3.z) * a.invPmax,
                            (b2.w + b3.w) * a.invPmax};
        const float r[4] = {b[0] - q.x, b[1] - q.y, b[2] - q.z, b[3] - q.w};
        st4(a.r + P, make_float4(r[0], r[1], r[2], r[3]));
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          rr += r[m] * r[m];
          rmax = fmaxf(rmax, fabsf(r[m]));
          bmax = fmaxf(bmax, fabsf(b[m]));
        }
      });
    } else {
      for_cells(a, [&](long long P, int i, int j, int k) {
        const float b = (__ldcg(a.c + 2 * pitch + P) + __ldcg(a.c + 3 * pitch + P)) * a.invPmax;
        const float r = b - apply_op(a, a.eta, P, i, j, k);
        a.r[P] = r;
        rr += r * r;
        rmax = fmaxf(rmax, fabsf(r));
        bmax = fmaxf(bmax, fabsf(b));
      });
    }
    block_reduce3(rr, bmax, rmax, a.partials, nb);
    // the max slot carries max|r|; max theta_B rides in the second (sum) slot
    // as a per-block max folded below
    if (!grid_reduce3(a.bar, a.status, nb, a.partials, res, s_rr, d0, s_rmax, a.wait_ns)) return;
    block_reduce3(0.0, 0.0, bmax, a.partials, nb);
    if (!grid_reduce3(a.bar, a.status, nb, a.partials, res + 3, d0, d1, s_bmax, a.wait_ns)) return;
  }

  if (s_bmax == 0.0) {  // theta_B = 0 everywhere: eta = 0
    for_cells(a, [&](long long P, int, int, int) { a.eta[P] = 0.0f; });
  } else if (a.cg5) {
    const double stop = (double)a.inner * fmax((double)a.tol * s_bmax, (double)a.atol);
    if (!cg_single_reduction(a, v4 && al16(a.cg5) && (a.g.ncell & 3) == 0, nb, res, s_rr, s_rmax, stop, it)) return;
  } else {
    // CG with the search-direction update folded into the operator pass:
    // p_new = r + beta p_old is formed on the fly at each cell and its
    // neighbours (p_old and p_new live in two buffers, so no block overwrites
    // a value another block still reads).  Two grid reductions per iteration.
    const double stop = (double)a.inner * fmax((double)a.tol * s_bmax, (double)a.atol);
    float* pold = a.p;
    float* pnew = a.p2;
    float beta = 0.0f;  // first direction: p = r
    while (it < a.maxit && s_rmax > stop) {
      float pq = 0.0f;
      const float bt = beta;
      const float* po = pold;
      float* pn = pnew;
      if (v4) {
        auto pv4 = [&](long long Q) {
          float4 v = ld4(a.r + Q);
          if (bt != 0.0f) {
            const float4 o = ld4(po + Q);
            v.x += bt * o.x; v.y += bt * o.y; v.z += bt * o.z; v.w += bt * o.w;
          }
          return v;
        };
        auto pv1 = [&](long long Q) { return __ldcg(a.r + Q) + (bt != 0.0f ? bt * __ldcg(po + Q) : 0.0f); };
        for_quads(a, [&](long long P, int i, int j, int k) {
          float4 pp;
          const float4 q = quad_op(a, P, i, j, k, pv4, pv1, pp);
          st4(pn + P, pp);
          st4(a.q + P, q);
          pq += pp.x * q.x + pp.y * q.y + pp.z * q.z + pp.w * q.w;
        });
      } else {
        for_cells(a, [&](long long P, int i, int j, int k) {
          const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
          auto pv = [&](long long Q) { return __ldcg(a.r + Q) + (bt != 0.0f ? bt * __ldcg(po + Q) : 0.0f); };
          const float pp = pv(P);
          float lx = 0.0f, ly = 0.0f, lz = 0.0f;
          if (i > 0) lx += pv(P - 1) - pp;
          if (i < nx - 1) lx += pv(P + 1) - pp;
          if (j > 0) ly += pv(P - nx) - pp;
          if (j < ny - 1) ly += pv(P + nx) - pp;
          if (a.g.dim == 3) {
            const long long sz = (long long)nx * ny;
            if (k > 0) lz += pv(P - sz) - pp;
            if (k < nz - 1) lz += pv(P + sz) - pp;
          }
          const float q = pp - (a.cx * lx + a.cy * ly + a.cz * lz);
          pn[P] = pp;
          a.q[P] = q;
          pq += pp * q;
        });
      }
      block_reduce3(pq, 0.0, 0.0, a.partials, nb);
      double s_pq;
      if (!grid_reduce3(a.bar, a.status, nb, a.partials, res, s_pq, d0, d1, a.wait_ns)) return;
      const float alpha = (float)(s_rr / s_pq);
      float rr2 = 0.0f, rm = 0.0f;
      if (v4) {
        for_quads(a, [&](long long P, int, int, int) {
          const float4 pP = ld4(pn + P), e = ld4(a.eta + P), r0 = ld4(a.r + P), q = ld4(a.q + P);
          st4(a.eta + P, make_float4(e.x + alpha * pP.x, e.y + alpha * pP.y, e.z + alpha * pP.z, e.w + alpha * pP.w));
          const float4 r = make_float4(r0.x - alpha * q.x, r0.y - alpha * q.y, r0.z - alpha * q.z, r0.w - alpha * q.w);
          st4(a.r + P, r);
          rr2 += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
          rm = fmaxf(fmaxf(rm, fmaxf(fabsf(r.x), fabsf(r.y))), fmaxf(fabsf(r.z), fabsf(r.w)));
        });
      } else {
        for_cells(a, [&](long long P, int, int, int) {
          const float pP = __ldcg(pn + P);
          a.eta[P] = __ldcg(a.eta + P) + alpha * pP;
          const float r = __ldcg(a.r + P) - alpha * __ldcg(a.q + P);
          a.r[P] = r;
          rr2 += r * r;
          rm = fmaxf(rm, fabsf(r));
        });
      }
      block_reduce3(rr2, 0.0, rm, a.partials, nb);
      double s_rr2;
      if (!grid_reduce3(a.bar, a.status, nb, a.partials, res + 3, s_rr2, d0, s_rmax, a.wait_ns)) return;
      beta = (float)(s_rr2 / s_rr);
      s_rr = s_rr2;
      float* t = pold;
      pold = pnew;
      pnew = t;
      ++it;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.status[1] = it;
    atomicAdd(a.status + 2, it);  // iterations summed over solves
  }
}

int eta_max_grid(int* grid_out) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eta_cg_kernel, ETA_BLOCK, 0) != cudaSuccess)
    return -1;
  *grid_out = sms * (per_sm < 1 ? 1 : per_sm);
  return 0;
}

cudaError_t launch_eta_solve(const EtaArgs& a, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 8 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  EtaArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)eta_cg_kernel, dim3(grid), dim3(ETA_BLOCK), args, 0, s);
}

}  // namespace clot

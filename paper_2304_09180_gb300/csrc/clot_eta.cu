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
// bounded (~2 s of globaltimer): a block that gives up sets ST_TIMEOUT in the
// status word and returns, so a fault can never leave the GPU spinning.
#include "clot_internal.cuh"

namespace clot {

constexpr int ETA_BLOCK = 256;

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier that also reduces: every block has written its three partial
// values (sum, sum, max) to partials[q][blk]; the last block to arrive sums
// them with all its threads (thread t takes blocks t, t + 256, ..., then a
// fixed tree) -- a fixed order, so the result is deterministic -- stores the
// three results in out[0..2], then releases the others.  Waits are bounded
// (~2 s of globaltimer): a block that gives up sets ST_TIMEOUT and the
// function returns false in all its threads.
__device__ bool grid_reduce3(unsigned* bar, int* status, int nb, const double* partials, double* out,
                             double& s0, double& s1, double& m2) {
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
      if (now_ns() - t0 > 2000000000ull) {
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

__global__ void __launch_bounds__(ETA_BLOCK) eta_cg_kernel(EtaArgs a) {
  const int nb = gridDim.x;
  const long long pitch = a.g.pitch;
  double* res = a.partials + 3 * nb;  // three reduced scalars (written by the last block)
  double d0, d1;

  double s_rr, s_rmax, s_bmax;
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
    float rr = 0.0f;
    for_cells(a, [&](long long P, int, int, int) {
      const float r = __ldcg(a.r + P);
      rr += r * r;
    });
    block_reduce3(rr, 0.0, 0.0, a.partials, nb);
    if (!grid_reduce3(a.bar, a.status, nb, a.partials, res, s_rr, d0, d1)) return;
    s_rmax = pr;
    s_bmax = pb;
  } else {
    // r = theta_B - A eta
    float rr = 0.0f, rmax = 0.0f, bmax = 0.0f;
    for_cells(a, [&](long long P, int i, int j, int k) {
      const float b = (__ldcg(a.c + 2 * pitch + P) + __ldcg(a.c + 3 * pitch + P)) * a.invPmax;
      const float r = b - apply_op(a, a.eta, P, i, j, k);
      a.r[P] = r;
      rr += r * r;
      rmax = fmaxf(rmax, fabsf(r));
      bmax = fmaxf(bmax, fabsf(b));
    });
    block_reduce3(rr, bmax, rmax, a.partials, nb);
    // the max slot carries max|r|; max theta_B rides in the second (sum) slot
    // as a per-block max folded below
    if (!grid_reduce3(a.bar, a.status, nb, a.partials, res, s_rr, d0, s_rmax)) return;
    block_reduce3(0.0, 0.0, bmax, a.partials, nb);
    if (!grid_reduce3(a.bar, a.status, nb, a.partials, res + 3, d0, d1, s_bmax)) return;
  }

  int it = 0;
  if (s_bmax == 0.0) {  // theta_B = 0 everywhere: eta = 0
    for_cells(a, [&](long long P, int, int, int) { a.eta[P] = 0.0f; });
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
      block_reduce3(pq, 0.0, 0.0, a.partials, nb);
      double s_pq;
      if (!grid_reduce3(a.bar, a.status, nb, a.partials, res, s_pq, d0, d1)) return;
      const float alpha = (float)(s_rr / s_pq);
      float rr2 = 0.0f, rm = 0.0f;
      for_cells(a, [&](long long P, int, int, int) {
        const float pP = __ldcg(pn + P);
        a.eta[P] = __ldcg(a.eta + P) + alpha * pP;
        const float r = __ldcg(a.r + P) - alpha * __ldcg(a.q + P);
        a.r[P] = r;
        rr2 += r * r;
        rm = fmaxf(rm, fabsf(r));
      });
      block_reduce3(rr2, 0.0, rm, a.partials, nb);
      double s_rr2;
      if (!grid_reduce3(a.bar, a.status, nb, a.partials, res + 3, s_rr2, d0, s_rmax)) return;
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

int eta_max_grid(int block, int* grid_out) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, eta_cg_kernel, block, 0) != cudaSuccess)
    return -1;
  *grid_out = sms * (per_sm < 1 ? 1 : per_sm);
  return 0;
}

cudaError_t launch_eta_solve(const EtaArgs& a, int grid, int block, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  EtaArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel((const void*)eta_cg_kernel, dim3(grid), dim3(block), args, 0, s);
}

}  // namespace clot

// clot_eta.cu -- K2: the virtual-substance solve of App. A, Eq. eta,
//     (I - (L_eta^2 / 4) lap_h) eta = theta_B,   zero-flux boundaries,
// by conjugate gradients in one persistent cooperative launch.  Vectors are
// FP32; every dot product and norm is accumulated in FP64 and reduced in a
// fixed order, so all blocks see bit-identical scalars and the iteration is
// deterministic.  The solve is warm-started from the eta passed in and stops
// when max|r| <= tol * max|theta_B|; since the operator is an M-matrix with
// unit row sums, max|eta - eta_exact| <= max|r|.
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

// Returns false (in every thread of the block) if the wait timed out.
__device__ bool grid_barrier(unsigned* bar, int* status, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = now_ns();
      while (*gen == g) {
        if (now_ns() - t0 > 2000000000ull) {
          atomicOr(status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Block-level reduction of three values (sum, sum, max) into partials[k][blk].
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
  __syncthreads();
}

// Every block sums the partials in the same order -> identical results.
__device__ void grid_combine3(const double* partials, int nb, double& s0, double& s1, double& m2) {
  __shared__ double res[3];
  if (threadIdx.x < 32) {
    double a = 0, b = 0, c = 0;
    for (int q = threadIdx.x; q < nb; q += 32) {
      a += __ldcg(partials + q);
      b += __ldcg(partials + nb + q);
      c = fmax(c, __ldcg(partials + 2 * nb + q));
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
      c = fmax(c, __shfl_xor_sync(0xffffffffu, c, o));
    }
    if (threadIdx.x == 0) { res[0] = a; res[1] = b; res[2] = c; }
  }
  __syncthreads();
  s0 = res[0];
  s1 = res[1];
  m2 = res[2];
  __syncthreads();
}

// y = (I - cL lap) x at cell P with zero-flux boundaries (missing neighbours
// contribute nothing).  x is read through L2 (__ldcg): it changes between
// phases of the same launch, so the non-coherent path must not be used.
__device__ __forceinline__ float apply_op(const EtaArgs& a, const float* x, long long P) {
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int i = (int)(P % nx), j = (int)((P / nx) % ny), k = (int)(P / ((long long)nx * ny));
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

__global__ void __launch_bounds__(ETA_BLOCK) eta_cg_kernel(EtaArgs a) {
  const int nb = gridDim.x;
  const long long n = a.g.ncell, pitch = a.g.pitch;
  const long long stride = (long long)nb * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;

  // r = theta_B - A eta, p = r
  double rr = 0.0, bb = 0.0, rmax = 0.0, bmax = 0.0;
  for (long long P = t0; P < n; P += stride) {
    const float b = (__ldcg(a.c + 2 * pitch + P) + __ldcg(a.c + 3 * pitch + P)) * a.invPmax;
    const float r = b - apply_op(a, a.eta, P);
    a.r[P] = r;
    a.p[P] = r;
    rr += (double)r * r;
    rmax = fmax(rmax, fabs((double)r));
    bmax = fmax(bmax, fabs((double)b));
  }
  block_reduce3(rr, bb, fmax(rmax, 0.0), a.partials, nb);
  // second slot carries bmax through a separate combine below
  if (!grid_barrier(a.bar, a.status, nb)) return;
  double s_rr, s_dummy, s_rmax;
  grid_combine3(a.partials, nb, s_rr, s_dummy, s_rmax);
  if (!grid_barrier(a.bar, a.status, nb)) return;
  block_reduce3(0.0, 0.0, bmax, a.partials, nb);
  if (!grid_barrier(a.bar, a.status, nb)) return;
  double s_bmax;
  grid_combine3(a.partials, nb, s_dummy, s_dummy, s_bmax);

  int it = 0;
  if (s_bmax == 0.0) {  // theta_B = 0 everywhere: eta = 0
    for (long long P = t0; P < n; P += stride) a.eta[P] = 0.0f;
  } else {
    const double stop = (double)a.tol * s_bmax;
    while (it < a.maxit && s_rmax > stop) {
      if (!grid_barrier(a.bar, a.status, nb)) return;  // p complete
      double pq = 0.0;
      for (long long P = t0; P < n; P += stride) {
        const float q = apply_op(a, a.p, P);
        a.q[P] = q;
        pq += (double)__ldcg(a.p + P) * q;
      }
      block_reduce3(pq, 0.0, 0.0, a.partials, nb);
      if (!grid_barrier(a.bar, a.status, nb)) return;
      double s_pq, d0, d1;
      grid_combine3(a.partials, nb, s_pq, d0, d1);
      const float alpha = (float)(s_rr / s_pq);
      double rr2 = 0.0, rm = 0.0;
      for (long long P = t0; P < n; P += stride) {
        const float pP = __ldcg(a.p + P);
        a.eta[P] = __ldcg(a.eta + P) + alpha * pP;
        const float r = __ldcg(a.r + P) - alpha * __ldcg(a.q + P);
        a.r[P] = r;
        rr2 += (double)r * r;
        rm = fmax(rm, fabs((double)r));
      }
      if (!grid_barrier(a.bar, a.status, nb)) return;  // everyone has read partials
      block_reduce3(rr2, 0.0, rm, a.partials, nb);
      if (!grid_barrier(a.bar, a.status, nb)) return;
      double s_rr2, d2;
      grid_combine3(a.partials, nb, s_rr2, d2, s_rmax);
      const float beta = (float)(s_rr2 / s_rr);
      s_rr = s_rr2;
      for (long long P = t0; P < n; P += stride) a.p[P] = __ldcg(a.r + P) + beta * __ldcg(a.p + P);
      ++it;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.status[1] = it;
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

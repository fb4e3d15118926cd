// clot_aux.cu -- K3 ADP-release sampling (Sec. 2 Eq. ADP_source, Sec. 3.2
// Eq. sigma_disc), K4 FP64 conservation diagnostics (invariants of App. A/B)
// and the one-off face-flux validation used by clot_species_step.
#include <float.h>

#include <algorithm>

#include "clot_internal.cuh"

namespace clot {

constexpr int AUX_BLOCK = 256;

// ------------------------------------------------------------------ sigma

__global__ void sigma_init_kernel(SigmaArgs a) {
  const long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= a.ncell) return;
  a.bound_acc[P] = 0.0f;
}

// New sample r = (platelets newly bound since the last sample) / (t - t_last)
// = Pmax (theta_B - theta_B,last) / (t - t_last) into ring slot `head`, then
// sigma = sum_lag w[lag] r(lag) over the stored samples, where
// w[lag] = A_hat * dtau * R(lag dtau) with half weight at lag 0 and lag N_tau:
// the trapezoid sum of Eq. sigma_disc regrouped by sample.  The newly-bound
// count is accumulated from the RK4 increments (bound_acc), which avoids the
// cancellation of differencing two FP32 states.
__global__ void sigma_sample_kernel(SigmaArgs a) {
  const long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= a.ncell) return;
  const float r = a.bound_acc[P] * a.inv_dt_sample;
  a.bound_acc[P] = 0.0f;
  a.hist[(long long)a.head * a.ncell + P] = r;
  float s = 0.0f;
  for (int lag = 0; lag < a.nvalid; ++lag) {
    int slot = a.head - lag;
    if (slot < 0) slot += a.nslot;
    s += a.w[lag] * a.hist[(long long)slot * a.ncell + P];
  }
  a.sigma[P] = s;
}

cudaError_t launch_sigma_init(const SigmaArgs& a, cudaStream_t s) {
  const long long grid = (a.ncell + AUX_BLOCK - 1) / AUX_BLOCK;
  sigma_init_kernel<<<(unsigned)grid, AUX_BLOCK, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sigma_sample(const SigmaArgs& a, cudaStream_t s) {
  const long long grid = (a.ncell + AUX_BLOCK - 1) / AUX_BLOCK;
  sigma_sample_kernel<<<(unsigned)grid, AUX_BLOCK, 0, s>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------ deviation form (shifts)

// dst[i] = src[i] + r for i < n (in place when dst == src): the entry and
// return shifts of the S1, S2 rows and of the inlet values under CLOT_DEVIATION.
__global__ void shift_kernel(float* dst, const float* src, long long n, float r) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i] + r;
}

cudaError_t launch_shift(float* dst, const float* src, long long n, float r, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long grid = std::min<long long>((n + AUX_BLOCK - 1) / AUX_BLOCK, 4096);
  shift_kernel<<<(unsigned)grid, AUX_BLOCK, 0, s>>>(dst, src, n, r);
  return cudaGetLastError();
}

// ------------------------------------------------------------ diagnostics

// Block-reduce 8 values (5 sums, min, count, max) with warp shuffles.
__device__ void reduce8(double (&v)[8], double* partials, int nb) {
  __shared__ double sh[8][AUX_BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double x = __shfl_xor_sync(0xffffffffu, v[q], o);
      v[q] = q == 5 ? fmin(v[q], x) : q == 7 ? fmax(v[q], x) : v[q] + x;
    }
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int q = 0; q < 8; ++q) sh[q][w] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < 8; ++q) {
      double a = sh[q][0];
      for (int k = 1; k < AUX_BLOCK / 32; ++k)
        a = q == 5 ? fmin(a, sh[q][k]) : q == 7 ? fmax(a, sh[q][k]) : a + sh[q][k];
      partials[(long long)q * nb + blockIdx.x] = a;
    }
  }
}

// Per cell the species groups are summed in FP32 (the state is FP32) and the
// sums accumulated over the thread's cells in FP64; the volume and area
// factors are applied once per thread.  Minimum, non-finite count and
// maximum theta_T are taken in FP32 (exact).  GB300's FP64 rate is a small
// fraction of its FP32 rate, so FP64 is kept to the accumulations.
// Compensated FP32 running sum (Neumaier's variant of Kahan summation): s + c
// carries the sum of the added terms to within about one FP32 rounding of
// the sum itself, independent of the number of terms (plus second-order terms
// in the unit roundoff), so a thread's partial keeps FP64-level accuracy
// without an FP64 operation per cell (FP64 runs at a small fraction of the
// FP32 rate on this GPU).  Branch-free form.
struct CSum {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__global__ void __launch_bounds__(AUX_BLOCK) diag_partial_kernel(DiagArgs a) {
  const int nb = gridDim.x;
  double w1 = 0.0, w3 = 0.0;
  CSum s0, s1, s2, s4, s2x;
  float mn = FLT_MAX, mx = -FLT_MAX, bad = 0.0f;
  const long long stride = (long long)nb * blockDim.x, pitch = a.pitch;
  const float ip = (float)a.invPmax;
  auto value = [&](float v) {
    if (!isfinite(v)) bad += 1.0f;
    else mn = fminf(mn, v);
  };
  auto cell = [&](const float (&y)[CLOT_NS]) {
    const float plt = (y[CLOT_PMU] + y[CLOT_PMA]) + (y[CLOT_PBA] + y[CLOT_PBSE]);
    const float cc = y[CLOT_C1] + y[CLOT_C2];
    s0.add(plt);
    s1.add(((y[CLOT_S1] + y[CLOT_E1]) + (y[CLOT_S1B] + y[CLOT_E1B])) + cc);
    s2.add(((y[CLOT_S2] + y[CLOT_E2]) + (y[CLOT_S2B] + y[CLOT_E2B])) + cc);
    s4.add(y[CLOT_ADP]);
    mx = fmaxf(mx, plt * ip);
#pragma unroll
    for (int q = 0; q < CLOT_NS; ++q) value(y[q]);
  };
  auto ext = [&](float xi, float xe) {  // inhibitor extension: E2,inh closes family 2
    s2x.add(xe);
    value(xi);
    value(xe);
  };
  // Quads of four consecutive cells as float4 (15 loads of 16 bytes in flight
  // per thread: the pass is bound by the bytes each SM keeps in flight), then
  // the cells of a ragged tail one by one.
  long long done = 0;
  auto al16 = [](const void* q) { return ((unsigned long long)q & 15u) == 0; };
  if (pitch % 4 == 0 && al16(a.c) && (!a.ext || al16(a.ext))) {
    const long long n4 = a.ncell / 4;
    for (long long Q = (long long)blockIdx.x * blockDim.x + threadIdx.x; Q < n4; Q += stride) {
      float4 v[CLOT_NS];
#pragma unroll
      for (int q = 0; q < CLOT_NS; ++q) v[q] = __ldcs(reinterpret_cast<const float4*>(a.c + q * pitch) + Q);
      float y[CLOT_NS];
#pragma unroll
      for (int q = 0; q < CLOT_NS; ++q) y[q] = v[q].x;
      cell(y);
#pragma unroll
      for (int q = 0; q < CLOT_NS; ++q) y[q] = v[q].y;
      cell(y);
#pragma unroll
      for (int q = 0; q < CLOT_NS; ++q) y[q] = v[q].z;
      cell(y);
#pragma unroll
      for (int q = 0; q < CLOT_NS; ++q) y[q] = v[q].w;
      cell(y);
      if (a.ext) {
        const float4 xi = __ldcs(reinterpret_cast<const float4*>(a.ext) + Q);
        const float4 xe = __ldcs(reinterpret_cast<const float4*>(a.ext + pitch) + Q);
        ext(xi.x, xe.x);
        ext(xi.y, xe.y);
        ext(xi.z, xe.z);
        ext(xi.w, xe.w);
      }
    }
    done = 4 * n4;
  }
  for (long long P = done + (long long)blockIdx.x * blockDim.x + threadIdx.x; P < a.ncell; P += stride) {
    float y[CLOT_NS];
#pragma unroll
    for (int q = 0; q < CLOT_NS; ++q) y[q] = __ldcs(a.c + q * pitch + P);
    cell(y);
    if (a.ext) ext(__ldcs(a.ext + P), __ldcs(a.ext + pitch + P));
  }
  for (long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x; f < a.n_inj; f += stride) {
    const float e0 = a.e0[f], c0 = a.c0[f];
    w1 += (double)c0;
    w3 += (double)e0 + (double)c0;
    if (!isfinite(e0)) bad += 1.0f; else mn = fminf(mn, e0);
    if (!isfinite(c0)) bad += 1.0f; else mn = fminf(mn, c0);
  }
  double v[8] = {a.V * s0.value(), a.V * s1.value() + a.A * w1, a.V * (s2.value() + s2x.value()), a.A * w3,
                 a.V * s4.value(), mn == FLT_MAX ? DBL_MAX : (double)mn, (double)bad,
                 mx == -FLT_MAX ? -DBL_MAX : (double)mx};
  reduce8(v, a.partials, nb);
}

// The block partials reduced by one block in a fixed order: thread t combines
// blocks t, t + 256, ... in turn, then a fixed tree (deterministic).
__global__ void __launch_bounds__(AUX_BLOCK) diag_final_kernel(const double* partials, int nb, double* out) {
  __shared__ double sh[8][AUX_BLOCK];
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double acc = q == 5 ? DBL_MAX : q == 7 ? -DBL_MAX : 0.0;
    for (int b = t; b < nb; b += AUX_BLOCK) {
      const double x = partials[(long long)q * nb + b];
      acc = q == 5 ? fmin(acc, x) : q == 7 ? fmax(acc, x) : acc + x;
    }
    sh[q][t] = acc;
  }
  __syncthreads();
  for (int w = AUX_BLOCK / 2; w > 0; w >>= 1) {
    if (t < w)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const double x = sh[q][t + w];
        sh[q][t] = q == 5 ? fmin(sh[q][t], x) : q == 7 ? fmax(sh[q][t], x) : sh[q][t] + x;
      }
    __syncthreads();
  }
  if (t < 8) out[t] = sh[t][0];
}

cudaError_t launch_diagnostics(const DiagArgs& a, int nblocks, cudaStream_t s) {
  diag_partial_kernel<<<nblocks, AUX_BLOCK, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, AUX_BLOCK, 0, s>>>(a.partials, nblocks, a.out);
  return cudaGetLastError();
}

// ------------------------------------------------------------ flux check

// Per cell: total outflow rate / V (Courant number per unit dt), relative net
// outflow |sum F_out| / sum |F|, and the largest |F| on wall faces.
__global__ void __launch_bounds__(AUX_BLOCK) flux_check_kernel(FluxCheckArgs a) {
  const int nb = gridDim.x;
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  // FP32 arithmetic on the FP32 fluxes (FP64 runs at a small fraction of the
  // FP32 rate here): the outflow and the face-flux magnitudes carry relative
  // errors of a few 2^-24, far inside the Courant bound's margin, and the net
  // flux, a near-cancellation, is summed with compensation (its error is about
  // one rounding of the net value itself, not of the total flux).
  float cour = 0.0f, divr = 0.0f, wall = 0.0f;
  const float invV = (float)a.invV;
  const long long stride = (long long)nb * blockDim.x;
  for (long long P = (long long)blockIdx.x * blockDim.x + threadIdx.x; P < a.g.ncell; P += stride) {
    const int i = (int)(P % nx), j = (int)((P / nx) % ny), k = (int)(P / ((long long)nx * ny));
    const long long fxl = (long long)i + (long long)(nx + 1) * (j + (long long)ny * k);
    const long long fyl = (long long)i + (long long)nx * (j + (long long)(ny + 1) * k);
    float fo[6];
    int nf = 4;
    fo[0] = -a.fx[fxl];
    fo[1] = a.fx[fxl + 1];
    fo[2] = -a.fy[fyl];
    fo[3] = a.fy[fyl + nx];
    if (a.g.dim == 3) {
      fo[4] = -a.fz[P];
      fo[5] = a.fz[P + (long long)nx * ny];
      nf = 6;
    }
    float out = 0.0f, tot = 0.0f;
    CSum net;
    for (int q = 0; q < nf; ++q) {
      out += fo[q] > 0.0f ? fo[q] : 0.0f;
      net.add(fo[q]);
      tot += fabsf(fo[q]);
    }
    cour = fmaxf(cour, out * invV);
    // inlet / outlet cells exchange with the outside: only interior balance counts
    if (i > 0 && i < nx - 1 && tot > 0.0f) divr = fmaxf(divr, fabsf(net.s + net.c) / tot);
    if (j == 0) wall = fmaxf(wall, fabsf(fo[2]));
    if (j == ny - 1) wall = fmaxf(wall, fabsf(fo[3]));
    if (a.g.dim == 3) {
      if (k == 0) wall = fmaxf(wall, fabsf(fo[4]));
      if (k == nz - 1) wall = fmaxf(wall, fabsf(fo[5]));
    }
  }
  double v[3] = {(double)cour, (double)divr, (double)wall};
  __shared__ double sh[3][AUX_BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1)
    for (int q = 0; q < 3; ++q) v[q] = fmax(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 3; ++q) sh[q][threadIdx.x >> 5] = v[q];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) {
      double m = 0.0;
      for (int w = 0; w < AUX_BLOCK / 32; ++w) m = fmax(m, sh[q][w]);
      a.partials[(long long)q * nb + blockIdx.x] = m;
    }
}

__global__ void flux_final_kernel(const double* partials, int nb, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int q = 0; q < 3; ++q) {
    double m = 0.0;
    for (int b = 0; b < nb; ++b) m = fmax(m, partials[(long long)q * nb + b]);
    out[q] = m;
  }
}

cudaError_t launch_flux_check(const FluxCheckArgs& a, int nblocks, cudaStream_t s) {
  flux_check_kernel<<<nblocks, AUX_BLOCK, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  flux_final_kernel<<<1, 32, 0, s>>>(a.partials, nblocks, a.out);
  return cudaGetLastError();
}

}  // namespace clot

// clot_surrogate.cu -- the learned reaction surrogate: a 32 -> 64 -> 64 -> 16
// GELU MLP on the tensor cores (bfloat16 operands, FP32 accumulation) that
// corrects the explicit-Euler increment of the reaction system of App. A /
// App. B over one step, with an RK4 fallback (Sec. 3.2 step 2) per cell; and
// its training (pair generation, forward/backward, Adam).
//
// Tensor-core mapping: mma.sync m16n8k16 bf16 -> f32.  A warp owns 16-row
// tiles (cells or samples).  The FP32 accumulator of one layer, after gelu and
// a bf16 pack, is exactly the A fragment of the next layer (two adjacent
// 8-column accumulator tiles form one 16-deep k-step), so activations never
// leave registers.  Weights are packed once per block into shared memory in
// B-fragment order (one 64-bit load per lane per MMA, conflict-free).
// Training keeps each 64-sample chunk's activations and gradients transposed
// in shared memory and forms the weight gradients as a second set of MMAs
// contracting over the samples; block partial sums go to a workspace that a
// second kernel reduces (fixed order, deterministic) and feeds to Adam.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include <cuda_bf16.h>

#include "clot_model.cuh"

namespace clot {
namespace {

constexpr int NP = CLOT_MLP_NPARAM;
constexpr int WSTRIDE = 7424;           // floats per block partial (NP gradients + loss, padded)
constexpr int MAX_GRAD_BLOCKS = 512;
constexpr float GELU_C = 0.7978845608028654f;  // sqrt(2 / pi)
constexpr float GELU_A = 0.044715f;
constexpr float RATE_K = 1e3f;  // relative-rate features: sign(q) log1p(RATE_K |q|)

// Output o (0..13) -> species row (ADP, row 4, has no reaction term).
__host__ __device__ constexpr int rrow(int o) { return o < 4 ? o : o + 1; }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) in FP32 with tanhf
// (training, where the backward pass needs the same activation as gelu').
__device__ __forceinline__ float gelu_f32(float z) {
  const float u = GELU_C * fmaf(GELU_A * z, z * z, z);
  const float hz = 0.5f * z;
  return fmaf(hz, tanhf(u), hz);
}

// The same function on a pair of bfloat16 values in packed bf16x2 arithmetic
// with the hardware tanh approximation (inference): z2 = z z,
// u = z (C + A C z2), g = z/2 + (z/2) tanh(u).  Each operation rounds to
// bfloat16, so g carries a few bf16 units of error; its consumer (the next
// product) takes bf16 operands anyway.
__device__ __forceinline__ uint32_t bfma2(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t btanh2(uint32_t a) {
  uint32_t d;
  asm("tanh.approx.bf16x2 %0, %1;" : "=r"(d) : "r"(a));
  return d;
}
struct Gelu2K {
  uint32_t c, ac, half, nzero;  // packed C, A C, 0.5, -0.0
  __device__ Gelu2K()
      : c(pack_bf16(GELU_C, GELU_C)), ac(pack_bf16(GELU_A * GELU_C, GELU_A * GELU_C)),
        half(pack_bf16(0.5f, 0.5f)), nzero(0x80008000u) {}
};
__device__ __forceinline__ uint32_t gelu_bf16x2(uint32_t z, const Gelu2K& k) {
  const uint32_t z2 = bfma2(z, z, k.nzero);
  const uint32_t u = bfma2(z, bfma2(z2, k.ac, k.c), k.nzero);
  const uint32_t hz = bfma2(z, k.half, k.nzero);
  return bfma2(hz, btanh2(u), hz);
}

__device__ __forceinline__ float gelu_grad(float z) {
  const float z2 = z * z;
  const float t = tanhf(GELU_C * fmaf(GELU_A * z, z2, z));
  return fmaf(0.5f, t, 0.5f) + 0.5f * z * (1.0f - t * t) * GELU_C * fmaf(3.0f * GELU_A, z2, 1.0f);
}

// B fragments of a K x N operand B(k, n) for m16n8k16: entry
// ((ks NT + nt) 32 + lane) holds {B(16ks+2q, n), B(16ks+2q+1, n)} and
// {B(16ks+2q+8, n), B(16ks+2q+9, n)}, n = 8nt + g, g = lane / 4, q = lane % 4.
// B(k, n) = W[k ld + n], or W[n ld + k] when TRANS (the transposed weight).
template <int K, int N, bool TRANS>
__device__ void build_bfrag(uint2* dst, const float* __restrict__ W, int ld) {
  constexpr int NT = N / 8, TOT = (K / 16) * NT * 32;
  for (int idx = threadIdx.x; idx < TOT; idx += blockDim.x) {
    const int lane = idx & 31, f = idx >> 5, nt = f % NT, ks = f / NT;
    const int n = 8 * nt + (lane >> 2), k = 16 * ks + 2 * (lane & 3);
    auto at = [&](int kk) { return TRANS ? __ldg(W + n * ld + kk) : __ldg(W + kk * ld + n); };
    dst[idx] = make_uint2(pack_bf16(at(k), at(k + 1)), pack_bf16(at(k + 8), at(k + 9)));
  }
}

struct MlpSmem {
  uint2 w1[2 * 8 * 32];   // W1: K 32, N 64
  uint2 w2[4 * 8 * 32];   // W2: K 64, N 64
  uint2 w3[4 * 2 * 32];   // W3: K 64, N 16
  float b1[64], b2[64], b3[16];
};

__device__ void load_mlp(MlpSmem& S, const float* __restrict__ w) {
  build_bfrag<32, 64, false>(S.w1, w + CLOT_MLP_OFF_W1, 64);
  build_bfrag<64, 64, false>(S.w2, w + CLOT_MLP_OFF_W2, 64);
  build_bfrag<64, 16, false>(S.w3, w + CLOT_MLP_OFF_W3, 16);
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    S.b1[i] = __ldg(w + CLOT_MLP_OFF_B1 + i);
    S.b2[i] = __ldg(w + CLOT_MLP_OFF_B2 + i);
    if (i < 16) S.b3[i] = __ldg(w + CLOT_MLP_OFF_B3 + i);
  }
}

template <int NT>
__device__ __forceinline__ void bias_init(float (&acc)[NT][4], const float* b, int q) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const float2 v = *reinterpret_cast<const float2*>(b + 8 * nt + 2 * q);
    acc[nt][0] = v.x; acc[nt][1] = v.y; acc[nt][2] = v.x; acc[nt][3] = v.y;
  }
}

template <int NT>
__device__ __forceinline__ void zero_acc(float (&acc)[NT][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.0f;
}

template <int KS, int NT>
__device__ __forceinline__ void mma_layer(float (&acc)[NT][4], const uint32_t (&a)[KS][4],
                                          const uint2* __restrict__ wf, int lane) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const uint2 b = wf[(ks * NT + nt) * 32 + lane];
      mma_bf16(acc[nt], a[ks], b.x, b.y);
    }
}

// Accumulator tiles (16 x 8 NT) -> A fragments of the next product
// (16 x 16 NT/2), rounded to bf16: ACT 0 as is, 2 through gelu_f32.
template <int NT, int ACT>
__device__ __forceinline__ void to_afrag(uint32_t (&a)[NT / 2][4], const float (&acc)[NT][4]) {
  auto f = [](float z) { return ACT == 0 ? z : gelu_f32(z); };
#pragma unroll
  for (int ks = 0; ks < NT / 2; ++ks) {
    a[ks][0] = pack_bf16(f(acc[2 * ks][0]), f(acc[2 * ks][1]));
    a[ks][1] = pack_bf16(f(acc[2 * ks][2]), f(acc[2 * ks][3]));
    a[ks][2] = pack_bf16(f(acc[2 * ks + 1][0]), f(acc[2 * ks + 1][1]));
    a[ks][3] = pack_bf16(f(acc[2 * ks + 1][2]), f(acc[2 * ks + 1][3]));
  }
}

// The same with gelu_bf16x2 on the bf16-rounded pre-activations (inference).
template <int NT>
__device__ __forceinline__ void to_afrag_gelu2(uint32_t (&a)[NT / 2][4], const float (&acc)[NT][4],
                                               const Gelu2K& k) {
#pragma unroll
  for (int ks = 0; ks < NT / 2; ++ks) {
    a[ks][0] = gelu_bf16x2(pack_bf16(acc[2 * ks][0], acc[2 * ks][1]), k);
    a[ks][1] = gelu_bf16x2(pack_bf16(acc[2 * ks][2], acc[2 * ks][3]), k);
    a[ks][2] = gelu_bf16x2(pack_bf16(acc[2 * ks + 1][0], acc[2 * ks + 1][1]), k);
    a[ks][3] = gelu_bf16x2(pack_bf16(acc[2 * ks + 1][2], acc[2 * ks + 1][3]), k);
  }
}

// A fragments of a 16-row tile stored row-major in shared memory as bf16
// with a row stride of LD elements.
template <int KS, int LD>
__device__ __forceinline__ void load_afrag(uint32_t (&a)[KS][4], const uint16_t* tile, int lane) {
  const int g = lane >> 2, q = lane & 3;
  const uint32_t* t = reinterpret_cast<const uint32_t*>(tile);
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    a[ks][0] = t[(g * LD + 16 * ks + 2 * q) >> 1];
    a[ks][1] = t[((g + 8) * LD + 16 * ks + 2 * q) >> 1];
    a[ks][2] = t[(g * LD + 16 * ks + 2 * q + 8) >> 1];
    a[ks][3] = t[((g + 8) * LD + 16 * ks + 2 * q + 8) >> 1];
  }
}

// A fragments of feature rows row0 .. row0+15 of x ([n][32] FP32, global).
__device__ __forceinline__ void load_afrag_x(uint32_t (&a)[2][4], const float* __restrict__ x, long long row0,
                                             long long n, int lane) {
  const int g = lane >> 2, q = lane & 3;
  const long long r0 = row0 + g, r1 = row0 + g + 8;
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    const int col = 16 * ks + 2 * q;
    const float2 z = make_float2(0.0f, 0.0f);
    const float2 v00 = r0 < n ? __ldg(reinterpret_cast<const float2*>(x + r0 * 32 + col)) : z;
    const float2 v01 = r0 < n ? __ldg(reinterpret_cast<const float2*>(x + r0 * 32 + col + 8)) : z;
    const float2 v10 = r1 < n ? __ldg(reinterpret_cast<const float2*>(x + r1 * 32 + col)) : z;
    const float2 v11 = r1 < n ? __ldg(reinterpret_cast<const float2*>(x + r1 * 32 + col + 8)) : z;
    a[ks][0] = pack_bf16(v00.x, v00.y);
    a[ks][1] = pack_bf16(v10.x, v10.y);
    a[ks][2] = pack_bf16(v01.x, v01.y);
    a[ks][3] = pack_bf16(v11.x, v11.y);
  }
}

// The inference network on T 16-row tiles: layer-1 A fragments in, the
// 16 x 16 output accumulators out.  Each weight fragment is loaded from shared
// memory once and used for all T tiles.
template <int T>
__device__ __forceinline__ void mlp_tiles(const MlpSmem& S, const uint32_t (&a1)[T][2][4], float (&o)[T][2][4],
                                          int lane, const Gelu2K& gk) {
  const int q = lane & 3;
  float z[T][8][4];
  uint32_t a[T][4][4];
#pragma unroll
  for (int t = 0; t < T; ++t) bias_init<8>(z[t], S.b1, q);
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const uint2 b = S.w1[(ks * 8 + nt) * 32 + lane];
#pragma unroll
      for (int t = 0; t < T; ++t) mma_bf16(z[t][nt], a1[t][ks], b.x, b.y);
    }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    to_afrag_gelu2<8>(a[t], z[t], gk);
    bias_init<8>(z[t], S.b2, q);
  }
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const uint2 b = S.w2[(ks * 8 + nt) * 32 + lane];
#pragma unroll
      for (int t = 0; t < T; ++t) mma_bf16(z[t][nt], a[t][ks], b.x, b.y);
    }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    to_afrag_gelu2<8>(a[t], z[t], gk);
    bias_init<2>(o[t], S.b3, q);
  }
#pragma unroll
  for (int ks = 0; ks < 4; ++ks)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const uint2 b = S.w3[(ks * 2 + nt) * 32 + lane];
#pragma unroll
      for (int t = 0; t < T; ++t) mma_bf16(o[t][nt], a[t][ks], b.x, b.y);
    }
}

// ------------------------------------------------------------------ warp-level network (mma.sync)

// forward

__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ w, const float* __restrict__ x,
                                                          long long n, float* __restrict__ out) {
  __shared__ MlpSmem S;
  load_mlp(S, w);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
  const Gelu2K gk;
  const long long ntile = (n + 15) / 16;
  for (long long t = (long long)blockIdx.x * 4 + warp; t < ntile; t += (long long)gridDim.x * 4) {
    uint32_t a[1][2][4];
    load_afrag_x(a[0], x, t * 16, n, lane);
    float ot[1][2][4];
    mlp_tiles<1>(S, a, ot, lane, gk);
    const float (&o)[2][4] = ot[0];
    const long long r0 = t * 16 + g, r1 = r0 + 8;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      if (r0 < n) *reinterpret_cast<float2*>(out + r0 * 16 + 8 * nt + 2 * q) = make_float2(o[nt][0], o[nt][1]);
      if (r1 < n) *reinterpret_cast<float2*>(out + r1 * 16 + 8 * nt + 2 * q) = make_float2(o[nt][2], o[nt][3]);
    }
  }
}


constexpr int XS_LD = 40;  // bf16 per feature row in shared memory (32 + 8: conflict-free A loads)
constexpr int VS_LD = 17;  // floats per output row in shared memory

constexpr int ES_LD = 15;  // Euler increments (14) and rho per cell row in shared memory (odd: conflict-free)

// One reaction solve over dt per cell with the surrogate where it applies.
// Thread per cell, 32 cells per warp iteration (two 16-row tiles through the
// network); persistent over the cells.  Three phases per iteration keep the
// register footprint small: (1) per cell, the Euler increments E and
// rho = max |E_s| / (|c_s| + floor_s) to shared memory and the features to the
// warp's tile; (2) the warp's network on 32 rows; (3) per cell, the state read
// again (an L1 hit), dc = E + rho v (|E| + floor) and the acceptance test
// |dc_s| <= tol (|c_s| + floor_s) for every reacting species.  Cells at rest
// (rho = 0) are left as they are; accepted cells are written; every other
// cell (adhesion layer, injury wall, rejected) is appended to a compacted
// list that surrogate_fallback_kernel integrates with RK4 in full warps.
__global__ void __launch_bounds__(128, 4) surrogate_react_kernel(const SurrArgs A) {
  __shared__ MlpSmem S;
  __shared__ __align__(16) uint16_t xs_all[4][32 * XS_LD];
  __shared__ float vs_all[4][32 * VS_LD];
  __shared__ float es_all[4][32 * ES_LD];
  load_mlp(S, A.w);
  for (int i = threadIdx.x; i < 4 * 32 * XS_LD; i += blockDim.x) (&xs_all[0][0])[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
  uint16_t* xs = xs_all[warp];
  float* vs = vs_all[warp];
  float* es = es_all[warp] + lane * ES_LD;
  const Geom& G = A.g;
  const RxnConst& R = A.r;
  unsigned n_ind = 0, n_reg = 0;
  const long long nchunk = (G.ncell + 31) / 32;
  for (long long ch = (long long)blockIdx.x * 4 + warp; ch < nchunk; ch += (long long)gridDim.x * 4) {
    __syncwarp();
    const long long P = ch * 32 + lane;
    const bool active = P < G.ncell;
    bool region = false, rest = true;
    if (active) {
      const int i = (int)(P % G.nx);
      const int j = (int)((P / G.nx) % G.ny);
      const int k = (int)(P / ((long long)G.nx * G.ny));
      region = i >= G.i0 && i <= G.i1 && k >= G.k0 && k <= G.k1 && (j <= G.hadh_jmax || j == 0);
    }
    if (active && !region) {  // phase 1
      float y[CLOT_NS], f[CLOT_NS];
#pragma unroll
      for (int s = 0; s < CLOT_NS; ++s) {
        y[s] = A.c[s * G.pitch + P];
        f[s] = 0.0f;
      }
      const float gP = affinity(R, __ldg(A.eta + P));
      const float A1 = R.k_adp * y[CLOT_ADP] / (R.adp_star + y[CLOT_ADP]);
      float fe0, fc0;
      rxn_rhs<false>(R, y, 0.0f, A1, R.kcohPmax * gP, 0.0f, 0.0f, f, fe0, fc0);
      float rho = 0.0f;
      float xf[32];
#pragma unroll
      for (int o = 0; o < 14; ++o) {
        const int s = rrow(o);
        const float E = A.dt * f[s];
        es[o] = E;
        const float q = __fdividef(E, fabsf(y[s]) + A.floor_s[s]);  // relative Euler rate
        rho = fmaxf(rho, fabsf(q));
        xf[17 + o] = copysignf(__logf(1.0f + RATE_K * fabsf(q)), q);
        rest = rest && E == 0.0f;
      }
      es[14] = rho;
      if (!rest) {
#pragma unroll
        for (int s = 0; s < CLOT_NS; ++s) xf[s] = __logf(1.0f + fmaxf(y[s], 0.0f) * A.inv_scale[s]);
        xf[15] = gP;
        xf[16] = A.xdt;
        xf[31] = 0.0f;
        uint32_t* row = reinterpret_cast<uint32_t*>(xs + lane * XS_LD);
#pragma unroll
        for (int p = 0; p < 16; ++p) row[p] = pack_bf16(xf[2 * p], xf[2 * p + 1]);
      }
    }
    const bool net = active && !region && !rest;
    if (__any_sync(0xffffffffu, net)) {  // phase 2 (warp-uniform)
      __syncwarp();
      const Gelu2K gk;
      uint32_t a[2][2][4];
      load_afrag<2, XS_LD>(a[0], xs, lane);
      load_afrag<2, XS_LD>(a[1], xs + 16 * XS_LD, lane);
      float o[2][2][4];
      mlp_tiles<2>(S, a, o, lane, gk);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          vs[(16 * mt + g) * VS_LD + 8 * nt + 2 * q] = o[mt][nt][0];
          vs[(16 * mt + g) * VS_LD + 8 * nt + 2 * q + 1] = o[mt][nt][1];
          vs[(16 * mt + g + 8) * VS_LD + 8 * nt + 2 * q] = o[mt][nt][2];
          vs[(16 * mt + g + 8) * VS_LD + 8 * nt + 2 * q + 1] = o[mt][nt][3];
        }
      __syncwarp();
    }
    bool accept = active && !region;  // rest cells: accepted unchanged
    if (net) {  // phase 3
      float y[CLOT_NS], dc[14];
#pragma unroll
      for (int s = 0; s < CLOT_NS; ++s) y[s] = A.c[s * G.pitch + P];
      const float rho = es[14];
#pragma unroll
      for (int o = 0; o < 14; ++o) {
        const int s = rrow(o);
        const float E = es[o];
        dc[o] = fmaf(rho * vs[lane * VS_LD + o], fabsf(E) + A.floor_s[s], E);
        accept = accept && fabsf(dc[o]) <= A.tol * (fabsf(y[s]) + A.floor_s[s]);  // false for NaN
      }
      if (accept) {
#pragma unroll
        for (int o = 0; o < 14; ++o) A.c[rrow(o) * G.pitch + P] = y[rrow(o)] + dc[o];
        const float bound = dc[2] + dc[3];  // outputs 2, 3 are P^{b,a}, P^{b,se}
        if (bound != 0.0f) A.bound_acc[P] += bound;
      }
    }
    const bool fb = active && !accept;
    const unsigned mask = __ballot_sync(0xffffffffu, fb);
    if (mask) {  // warp-aggregated append to the fallback list
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(A.counts + 2, (unsigned long long)__popc(mask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (fb) A.list[base + __popc(mask & ((1u << lane) - 1u))] = (int)P;
    }
    if (active) {
      const int fl = region ? 2 : accept ? 0 : 1;
      if (A.flag) A.flag[P] = (uint8_t)fl;
      n_ind += fl == 1;
      n_reg += fl == 2;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n_ind += __shfl_xor_sync(0xffffffffu, n_ind, off);
    n_reg += __shfl_xor_sync(0xffffffffu, n_reg, off);
  }
  if (lane == 0 && (n_ind | n_reg)) {
    atomicAdd(A.counts, (unsigned long long)n_ind);
    atomicAdd(A.counts + 1, (unsigned long long)n_reg);
  }
}

// ------------------------------------------------------------------ tcgen05 network
//
// The network on the fifth-generation tensor cores: one CTA of 128 threads
// takes 128 rows (cells or feature rows) at a time, thread t owning row t.
// Operands are bf16 in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, K-adjacent core matrices 128 bytes
// apart (the descriptor's leading offset), 8-row groups KC x 128 bytes apart
// (its stride offset).  Each layer is M = 128 x N x K issued as K / 16
// tcgen05.mma instructions by one thread into a tensor-memory accumulator
// (layer 1: columns 0..63, layer 2: 64..127, layer 3: 0..15), completion
// through tcgen05.commit on an mbarrier; each thread then reads its own row
// of the accumulator (tcgen05.ld 32x32b), adds the bias, applies gelu in packed
// bf16x2 and writes its row of the next layer's operand.  Waits are bounded
// (1 s of globaltimer): on expiry the CTA records ST_TIMEOUT and stops.
constexpr unsigned TC_COLS = 128;        // tensor-memory columns per CTA
constexpr int TC_SMEM = 48 * 1024;       // dynamic shared memory per CTA: at most 4 CTAs (512 columns) per SM

struct TcSmem {
  unsigned char w1[64 * 32 * 2];    // B of layer 1: N 64 x K 32
  unsigned char w2[64 * 64 * 2];    // N 64 x K 64
  unsigned char w3[16 * 64 * 2];    // N 16 x K 64
  unsigned char a1[128 * 32 * 2];   // features, M 128 x K 32
  unsigned char a2[128 * 64 * 2];   // h1, then h2: M 128 x K 64
  float b1[64], b2[64], b3[16];
  unsigned long long bar;
  unsigned tmem;
};
static_assert(sizeof(TcSmem) + 1024 <= TC_SMEM, "tcgen05 shared memory");

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr unsigned tc_idesc(unsigned M, unsigned N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Byte offset of element (row, k) in a K-major operand with kc core matrices along K.
__device__ __forceinline__ unsigned kmaj(int row, int k, int kc) {
  return (unsigned)((row >> 3) * (kc * 128) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void tc_mma(unsigned dtm, unsigned long long ad, unsigned long long bd, unsigned idesc,
                                       int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

// Thread 0: D(columns dcol..) = A (M 128 x K, kc core matrices) times B^T (N x K).
__device__ __forceinline__ void tc_layer(const TcSmem& S, unsigned dcol, const unsigned char* a, const unsigned char* bw,
                                         int kc, unsigned n) {
  const unsigned idesc = tc_idesc(128, n);
  for (int s = 0; s < kc / 2; ++s)
    tc_mma(S.tmem + dcol, smem_desc(su32(a) + s * 256, 128, kc * 128), smem_desc(su32(bw) + s * 256, 128, kc * 128),
           idesc, s);
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(&S.bar))
               : "memory");
}

// All threads: wait (bounded) for the next phase of the CTA's mbarrier.
__device__ __forceinline__ bool tc_wait(const TcSmem& S, unsigned& phase) {
  const unsigned bar = su32(&S.bar);
  auto done = [&]() {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(bar), "r"(phase)
                 : "memory");
    return ok != 0;
  };
  bool ok = done();
  if (!ok) {
    const unsigned long long t0 = gtimer();
    while (!(ok = done()))
      if (gtimer() - t0 > 1000000000ull) break;
  }
  phase ^= 1u;
  tc_fence_after();
  return ok;
}

// Thread's row, 32 accumulator columns from column col.
__device__ __forceinline__ void tc_ld32(unsigned taddr, float (&v)[32]) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tc_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Per CTA, once: weights in B layout, biases, mbarrier, tensor memory.
__device__ __forceinline__ void tc_setup(TcSmem& S, const float* __restrict__ w) {
  const int t = threadIdx.x;
  for (int i = t; i < 64 * 32; i += blockDim.x) {  // W1[k][n], k < 32
    const int n = i & 63, k = i >> 6;
    *reinterpret_cast<__nv_bfloat16*>(S.w1 + kmaj(n, k, 4)) = __float2bfloat16_rn(__ldg(w + CLOT_MLP_OFF_W1 + i));
  }
  for (int i = t; i < 64 * 64; i += blockDim.x) {
    const int n = i & 63, k = i >> 6;
    *reinterpret_cast<__nv_bfloat16*>(S.w2 + kmaj(n, k, 8)) = __float2bfloat16_rn(__ldg(w + CLOT_MLP_OFF_W2 + i));
  }
  for (int i = t; i < 64 * 16; i += blockDim.x) {  // W3[k][n], n < 16
    const int n = i & 15, k = i >> 4;
    *reinterpret_cast<__nv_bfloat16*>(S.w3 + kmaj(n, k, 8)) = __float2bfloat16_rn(__ldg(w + CLOT_MLP_OFF_W3 + i));
  }
  for (int i = t; i < 64; i += blockDim.x) {
    S.b1[i] = __ldg(w + CLOT_MLP_OFF_B1 + i);
    S.b2[i] = __ldg(w + CLOT_MLP_OFF_B2 + i);
    if (i < 16) S.b3[i] = __ldg(w + CLOT_MLP_OFF_B3 + i);
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(&S.bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (t < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(&S.tmem)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void tc_teardown(TcSmem& S) {
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(S.tmem), "r"(TC_COLS) : "memory");
  }
}

// Row t of a K-major operand with kc core matrices along K from 2 kc packed bf16 pairs.
__device__ __forceinline__ void store_row(unsigned char* op, int t, int kc, const uint32_t* pk) {
  for (int c = 0; c < kc; ++c)
    *reinterpret_cast<uint4*>(op + kmaj(t, c * 8, kc)) = make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
}

// 32 accumulator columns + bias -> gelu (bf16x2) -> 16 packed pairs.
__device__ __forceinline__ void gelu_pack32(const float (&z)[32], const float* b, const Gelu2K& gk, uint32_t* out) {
#pragma unroll
  for (int j = 0; j < 16; ++j) out[j] = gelu_bf16x2(pack_bf16(z[2 * j] + b[2 * j], z[2 * j + 1] + b[2 * j + 1]), gk);
}

// The three layers for the CTA's 128 rows, whose features are in S.a1.  v
// receives the thread's 16 outputs.  Returns false on a timed-out wait.
__device__ __forceinline__ bool tc_network(TcSmem& S, unsigned& phase, float (&v)[16], const Gelu2K& gk) {
  const int t = threadIdx.x;
  const unsigned lane_base = (unsigned)((t >> 5) * 32) << 16;
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  if (t == 0) {
    tc_fence_after();
    tc_layer(S, 0, S.a1, S.w1, 4, 64);
  }
  if (!__syncthreads_and(tc_wait(S, phase))) return false;
  uint32_t pk[32];
  {
    float z[32];
    tc_ld32(S.tmem + lane_base + 0, z);
    gelu_pack32(z, S.b1, gk, pk);
    tc_ld32(S.tmem + lane_base + 32, z);
    gelu_pack32(z, S.b1 + 32, gk, pk + 16);
  }
  store_row(S.a2, t, 8, pk);
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  if (t == 0) {
    tc_fence_after();
    tc_layer(S, 64, S.a2, S.w2, 8, 64);
  }
  if (!__syncthreads_and(tc_wait(S, phase))) return false;
  {
    float z[32];
    tc_ld32(S.tmem + lane_base + 64, z);
    gelu_pack32(z, S.b2, gk, pk);
    tc_ld32(S.tmem + lane_base + 96, z);
    gelu_pack32(z, S.b2 + 32, gk, pk + 16);
  }
  store_row(S.a2, t, 8, pk);  // layer 2 has finished reading h1
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  if (t == 0) {
    tc_fence_after();
    tc_layer(S, 0, S.a2, S.w3, 8, 16);
  }
  if (!__syncthreads_and(tc_wait(S, phase))) return false;
  tc_ld16(S.tmem + lane_base + 0, v);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] += S.b3[j];
  tc_fence_before();
  return true;
}

__device__ __forceinline__ TcSmem& tc_smem(unsigned char* raw) {
  return *reinterpret_cast<TcSmem*>(raw + ((1024u - (su32(raw) & 1023u)) & 1023u));
}

// ------------------------------------------------------------------ forward

__global__ void __launch_bounds__(128, 4) mlp_forward_tc_kernel(const float* __restrict__ w,
                                                                const float* __restrict__ x, long long n,
                                                                float* __restrict__ out, int* status) {
  extern __shared__ unsigned char tc_raw[];
  TcSmem& S = tc_smem(tc_raw);
  tc_setup(S, w);
  const int t = threadIdx.x;
  const Gelu2K gk;
  unsigned phase = 0;
  const long long nchunk = (n + 127) / 128;
  for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const long long row = ch * 128 + t;
    uint32_t pk[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const float2 v = row < n ? __ldg(reinterpret_cast<const float2*>(x + row * 32) + j) : make_float2(0.f, 0.f);
      pk[j] = pack_bf16(v.x, v.y);
    }
    store_row(S.a1, t, 4, pk);
    float v[16];
    if (!tc_network(S, phase, v, gk)) {
      if (t == 0 && status) atomicOr(status, ST_TIMEOUT);
      break;
    }
    if (row < n) {
      float4* o = reinterpret_cast<float4*>(out + row * 16);
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
    }
  }
  tc_teardown(S);
}

// ------------------------------------------------------------------ inference

// One reaction solve over dt per cell with the surrogate where it applies.
// CTA of 128 threads, one cell each, persistent over 128-cell chunks.  Per
// chunk: (1) per cell, the Euler increments E and rho = max |E_s| / (|c_s| +
// floor_s) in registers and the features to row t of the tile; (2) the
// network on the tensor cores if any cell of the chunk needs it; (3) per
// cell, dc = E + rho v (|E| + floor) and the acceptance test |dc_s| <= tol
// (|c_s| + floor_s) for every reacting species.  Cells at rest (rho = 0) are
// left as they are; accepted cells are written; every other cell (adhesion
// layer, injury wall, rejected) is appended to a compacted list that
// surrogate_fallback_kernel integrates with RK4 in full warps.
__global__ void __launch_bounds__(128, 4) surrogate_react_tc_kernel(const SurrArgs A) {
  extern __shared__ unsigned char tc_raw[];
  TcSmem& S = tc_smem(tc_raw);
  tc_setup(S, A.w);
  const int t = threadIdx.x, lane = t & 31;
  const Geom& G = A.g;
  const RxnConst& R = A.r;
  const Gelu2K gk;
  unsigned phase = 0;
  unsigned n_ind = 0, n_reg = 0;
  const long long nchunk = (G.ncell + 127) / 128;
  for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const long long P = ch * 128 + t;
    const bool active = P < G.ncell;
    bool region = false, rest = true;
    float E[14], rho = 0.0f;
#pragma unroll
    for (int o = 0; o < 14; ++o) E[o] = 0.0f;
    uint32_t pk[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) pk[j] = 0u;
    if (active) {
      const int i = (int)(P % G.nx);
      const int j = (int)((P / G.nx) % G.ny);
      const int k = (int)(P / ((long long)G.nx * G.ny));
      region = i >= G.i0 && i <= G.i1 && k >= G.k0 && k <= G.k1 && (j <= G.hadh_jmax || j == 0);
    }
    if (active && !region) {  // phase 1
      float y[CLOT_NS], f[CLOT_NS];
#pragma unroll
      for (int s = 0; s < CLOT_NS; ++s) {
        y[s] = A.c[s * G.pitch + P];
        f[s] = 0.0f;
      }
      const float gP = affinity(R, __ldg(A.eta + P));
      const float A1 = R.k_adp * y[CLOT_ADP] / (R.adp_star + y[CLOT_ADP]);
      float fe0, fc0;
      rxn_rhs<false>(R, y, 0.0f, A1, R.kcohPmax * gP, 0.0f, 0.0f, f, fe0, fc0);
      float xf[32];
#pragma unroll
      for (int o = 0; o < 14; ++o) {
        const int s = rrow(o);
        E[o] = A.dt * f[s];
        const float q = __fdividef(E[o], fabsf(y[s]) + A.floor_s[s]);  // relative Euler rate
        rho = fmaxf(rho, fabsf(q));
        xf[17 + o] = copysignf(__logf(1.0f + RATE_K * fabsf(q)), q);
        rest = rest && E[o] == 0.0f;
      }
#pragma unroll
      for (int s = 0; s < CLOT_NS; ++s) xf[s] = __logf(1.0f + fmaxf(y[s], 0.0f) * A.inv_scale[s]);
      xf[15] = gP;
      xf[16] = A.xdt;
      xf[31] = 0.0f;
#pragma unroll
      for (int j = 0; j < 16; ++j) pk[j] = pack_bf16(xf[2 * j], xf[2 * j + 1]);
    }
    const bool net = active && !region && !rest;
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = 0.0f;
    if (__syncthreads_or(net)) {  // phase 2 (CTA-uniform)
      store_row(S.a1, t, 4, pk);
      if (!tc_network(S, phase, v, gk)) {
        if (t == 0 && A.status) atomicOr(A.status, ST_TIMEOUT);
        break;
      }
    }
    bool accept = active && !region;  // rest cells: accepted unchanged
    if (net) {  // phase 3
      float dc[14];
#pragma unroll
      for (int o = 0; o < 14; ++o) {
        const int s = rrow(o);
        const float y = A.c[s * G.pitch + P];
        dc[o] = fmaf(rho * v[o], fabsf(E[o]) + A.floor_s[s], E[o]);
        accept = accept && fabsf(dc[o]) <= A.tol * (fabsf(y) + A.floor_s[s]);  // false for NaN
      }
      if (accept) {
#pragma unroll
        for (int o = 0; o < 14; ++o) A.c[rrow(o) * G.pitch + P] += dc[o];
        const float bound = dc[2] + dc[3];  // outputs 2, 3 are P^{b,a}, P^{b,se}
        if (bound != 0.0f) A.bound_acc[P] += bound;
      }
    }
    const bool fb = active && !accept;
    const unsigned mask = __ballot_sync(0xffffffffu, fb);
    if (mask) {  // warp-aggregated append to the fallback list
      const int leader = __ffs(mask) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(A.counts + 2, (unsigned long long)__popc(mask));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (fb) A.list[base + __popc(mask & ((1u << lane) - 1u))] = (int)P;
    }
    if (active) {
      const int fl = region ? 2 : accept ? 0 : 1;
      if (A.flag) A.flag[P] = (uint8_t)fl;
      n_ind += fl == 1;
      n_reg += fl == 2;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n_ind += __shfl_xor_sync(0xffffffffu, n_ind, off);
    n_reg += __shfl_xor_sync(0xffffffffu, n_reg, off);
  }
  if (lane == 0 && (n_ind | n_reg)) {
    atomicAdd(A.counts, (unsigned long long)n_ind);
    atomicAdd(A.counts + 1, (unsigned long long)n_reg);
  }
  tc_teardown(S);
}

// RK4 (M steps of h, Sec. 3.2 step 2) for the cells listed by
// surrogate_react_kernel, as clot_reaction_step does it, including the
// injury-wall exchange of floor cells over the patch.
__global__ void __launch_bounds__(128) surrogate_fallback_kernel(const SurrArgs A) {
  const Geom& G = A.g;
  const RxnConst& R = A.r;
  const long long n = (long long)*reinterpret_cast<volatile const unsigned long long*>(A.counts + 2);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long P = A.list[idx];
    float y[CLOT_NS];
#pragma unroll
    for (int s = 0; s < CLOT_NS; ++s) y[s] = A.c[s * G.pitch + P];
    const int i = (int)(P % G.nx);
    const int j = (int)((P / G.nx) % G.ny);
    const int k = (int)(P / ((long long)G.nx * G.ny));
    const bool over = i >= G.i0 && i <= G.i1 && k >= G.k0 && k <= G.k1;
    const float adhH = (over && j <= G.hadh_jmax) ? R.kadh : 0.0f;
    const float coh = R.kcohPmax * affinity(R, __ldg(A.eta + P));
    const float A1 = R.k_adp * y[CLOT_ADP] / (R.adp_star + y[CLOT_ADP]);
    const bool wall = over && j == 0;
    const int fidx = wall ? (i - G.i0) + (G.i1 - G.i0 + 1) * (k - G.k0) : 0;
    float e0 = wall ? A.e0[fidx] : 0.0f, c0 = wall ? A.c0[fidx] : 0.0f;
    const float bound = rxn_rk4(R, y, adhH, A1, coh, wall, e0, c0, A.h, A.M);
    if (wall) {
      A.e0[fidx] = e0;
      A.c0[fidx] = c0;
    }
#pragma unroll
    for (int s = 0; s < CLOT_NS; ++s)
      if (s != CLOT_ADP) A.c[s * G.pitch + P] = y[s];
    if (bound != 0.0f) A.bound_acc[P] += bound;
  }
}

// ------------------------------------------------------------------ training pairs

struct PairArgs {
  const float* __restrict__ c0;
  const float* __restrict__ eta;
  float* __restrict__ x;
  float* __restrict__ y;
  long long n, pitch;
  double dt, h;
  float xdt;
  int M;
  float inv_scale[CLOT_NS], floor_s[CLOT_NS];
  RxnConst r;
};

// Features and targets of one cell, in double precision (the target is the
// RK4 correction of Euler divided by rho, so it needs the increments to well
// below rho relative; FP32 would leave an error of order 1e-7 / rho): E =
// dt f(c0), the RK4 increment over M steps of h (summed per step),
// rho = max |E_s| / (|c0_s| + floor_s) and v = (dRK4 - E) / (rho (|E| + floor))
// (0 where rho = 0).  Training-data generation, not a per-step path.
__global__ void __launch_bounds__(128) surrogate_pairs_kernel(const PairArgs A) {
  const RxnConst& R = A.r;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < A.n;
       p += (long long)gridDim.x * blockDim.x) {
    double y0[CLOT_NS], y[CLOT_NS], d[CLOT_NS], f[CLOT_NS];
#pragma unroll
    for (int s = 0; s < CLOT_NS; ++s) {
      y0[s] = (double)__ldg(A.c0 + s * A.pitch + p);
      y[s] = y0[s];
      d[s] = 0.0;
      f[s] = 0.0;
    }
    const double eta = (double)__ldg(A.eta + p);
    const double u = eta - (double)R.eta_t;
    const double gP = u > 0.0 ? (double)R.g0 * u * u * u / ((double)R.eta_star3 + u * u * u) : 0.0;
    const double coh = (double)R.kcohPmax * gP;
    const double A1 = (double)R.k_adp * y0[CLOT_ADP] / ((double)R.adp_star + y0[CLOT_ADP]);
    const double zero = 0.0;
    double fe0, fc0;
    rxn_rhs<false, double>(R, y0, zero, A1, coh, zero, zero, f, fe0, fc0);
    const double h = A.h, h2 = 0.5 * h, h6 = h / 6.0;
    for (int m = 0; m < A.M; ++m) {
      double yt[CLOT_NS], acc[CLOT_NS], k[CLOT_NS];
#pragma unroll
      for (int s = 0; s < CLOT_NS; ++s) k[s] = 0.0;
      rxn_rhs<false, double>(R, y, zero, A1, coh, zero, zero, k, fe0, fc0);
#pragma unroll
      for (int s = 0; s < CLOT_NS; ++s) { acc[s] = k[s]; yt[s] = s == CLOT_ADP ? y[s] : y[s] + h2 * k[s]; }
      rxn_rhs<false, double>(R, yt, zero, A1, coh, zero, zero, k, fe0, fc0);
#pragma unroll
      for (int s = 0; s < CLOT_NS; ++s) { acc[s] += 2.0 * k[s]; yt[s] = s == CLOT_ADP ? y[s] : y[s] + h2 * k[s]; }
      rxn_rhs<false, double>(R, yt, zero, A1, coh, zero, zero, k, fe0, fc0);
#pragma unroll
      for (int s = 0; s < CLOT_NS; ++s) { acc[s] += 2.0 * k[s]; yt[s] = s == CLOT_ADP ? y[s] : y[s] + h * k[s]; }
      rxn_rhs<false, double>(R, yt, zero, A1, coh, zero, zero, k, fe0, fc0);
#pragma unroll
      for (int s = 0; s < CLOT_NS; ++s)
        if (s != CLOT_ADP) {
          const double inc = h6 * (acc[s] + k[s]);
          y[s] += inc;
          d[s] += inc;
        }
    }
    float xf[32];
#pragma unroll
    for (int s = 0; s < CLOT_NS; ++s) xf[s] = (float)log1p(fmax(y0[s], 0.0) * (double)A.inv_scale[s]);
    xf[15] = (float)gP;
    xf[16] = A.xdt;
    xf[31] = 0.0f;
    double E[14];
    double rho = 0.0;
#pragma unroll
    for (int o = 0; o < 14; ++o) {
      const int s = rrow(o);
      E[o] = A.dt * f[s];
      const double q = E[o] / (fabs(y0[s]) + (double)A.floor_s[s]);
      rho = fmax(rho, fabs(q));
      xf[17 + o] = (float)copysign(log1p((double)RATE_K * fabs(q)), q);
    }
    float4* xr = reinterpret_cast<float4*>(A.x + p * 32);
#pragma unroll
    for (int c = 0; c < 8; ++c) xr[c] = make_float4(xf[4 * c], xf[4 * c + 1], xf[4 * c + 2], xf[4 * c + 3]);
    float t[16];
#pragma unroll
    for (int o = 0; o < 14; ++o) {
      const int s = rrow(o);
      t[o] = rho > 0.0 ? (float)((d[s] - E[o]) / (rho * (fabs(E[o]) + (double)A.floor_s[s]))) : 0.0f;
    }
    t[14] = t[15] = 0.0f;
    float4* yr = reinterpret_cast<float4*>(A.y + p * 16);
#pragma unroll
    for (int c = 0; c < 4; ++c) yr[c] = make_float4(t[4 * c], t[4 * c + 1], t[4 * c + 2], t[4 * c + 3]);
  }
}

// ------------------------------------------------------------------ training

constexpr int T_LD = 72;  // bf16 per row of the transposed chunk tiles (64 samples + 8: conflict-free)

struct TrainSmem {
  uint2 w1[2 * 8 * 32], w2[4 * 8 * 32], w3[4 * 2 * 32];  // forward B fragments
  uint2 w3t[1 * 8 * 32];                                 // W3^T: K 16, N 64
  uint2 w2t[4 * 8 * 32];                                 // W2^T: K 64, N 64
  float b1[64], b2[64], b3[16];
  // bf16 operands of the chunk, transposed: [feature][sample]
  uint16_t xT[32 * T_LD], h1T[64 * T_LD], h2T[64 * T_LD], dT[16 * T_LD], dz2T[64 * T_LD], dz1T[64 * T_LD];
  float gw[NP];  // block gradient sums (before the 2 / (B 14) scale)
  float gb[4][64 + 64 + 16];  // per-warp bias gradient sums (b1, b2, b3), added up in warp order at the end
  float lw[4];                // per-warp loss sums
};

// Stores bf16 A fragments of a 16-row tile transposed: T[feature][col0 + row].
template <int KS>
__device__ __forceinline__ void store_afrag_T(uint16_t* T, const uint32_t (&a)[KS][4], int col0, int lane) {
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int ks = 0; ks < KS; ++ks)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = col0 + g + ((r & 1) ? 8 : 0);
      const int feat = 16 * ks + 2 * q + ((r & 2) ? 8 : 0);
      T[feat * T_LD + row] = (uint16_t)(a[ks][r] & 0xffffu);
      T[(feat + 1) * T_LD + row] = (uint16_t)(a[ks][r] >> 16);
    }
}

// Column sums of a 16 x 8NT accumulator over its 16 rows, added to dst[col]
// (a warp-private row: lanes 0..3 own distinct columns, so plain adds).
template <int NT>
__device__ __forceinline__ void colsum_add(float* dst, const float (&acc)[NT][4], int lane) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    float s0 = acc[nt][0] + acc[nt][2], s1 = acc[nt][1] + acc[nt][3];
#pragma unroll
    for (int off = 4; off < 32; off <<= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, off);
      s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    if (lane < 4) {
      dst[8 * nt + 2 * lane] += s0;
      dst[8 * nt + 2 * lane + 1] += s1;
    }
  }
}

// dst[(16 mt + r) ldo + 8 nt + c] += sum over the 64 chunk samples of
// AT[16 mt + r][s] BT[8 nt + c][s] for the listed tiles (one warp's disjoint
// part of a weight gradient).
template <int MT0, int MT, int NT0, int NT>
__device__ __forceinline__ void wgrad(float* dst, int ldo, const uint16_t* AT, const uint16_t* BT, int lane) {
  const int g = lane >> 2, q = lane & 3;
  const uint32_t* Bw = reinterpret_cast<const uint32_t*>(BT);
#pragma unroll
  for (int mt = MT0; mt < MT0 + MT; ++mt) {
    uint32_t a[4][4];
    load_afrag<4, T_LD>(a, AT + mt * 16 * T_LD, lane);
#pragma unroll
    for (int nt = NT0; nt < NT0 + NT; ++nt) {
      float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t b0 = Bw[((8 * nt + g) * T_LD + 16 * ks + 2 * q) >> 1];
        const uint32_t b1 = Bw[((8 * nt + g) * T_LD + 16 * ks + 2 * q + 8) >> 1];
        mma_bf16(c, a[ks], b0, b1);
      }
      float* d0 = dst + (16 * mt + g) * ldo + 8 * nt + 2 * q;
      float* d1 = d0 + 8 * ldo;
      d0[0] += c[0];
      d0[1] += c[1];
      d1[0] += c[2];
      d1[1] += c[3];
    }
  }
}

// Block partial gradients of the loss over rows [0, n) of x, y (64-row chunks,
// grid-strided); work[blockIdx][0..NP) gradients (unscaled), [NP] the sum of squares.
__global__ void __launch_bounds__(128, 1) mlp_grad_kernel(const float* __restrict__ w, const float* __restrict__ x,
                                                          const float* __restrict__ yv, long long n,
                                                          float* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  build_bfrag<32, 64, false>(S.w1, w + CLOT_MLP_OFF_W1, 64);
  build_bfrag<64, 64, false>(S.w2, w + CLOT_MLP_OFF_W2, 64);
  build_bfrag<64, 16, false>(S.w3, w + CLOT_MLP_OFF_W3, 16);
  build_bfrag<16, 64, true>(S.w3t, w + CLOT_MLP_OFF_W3, 16);
  build_bfrag<64, 64, true>(S.w2t, w + CLOT_MLP_OFF_W2, 64);
  for (int i = threadIdx.x; i < 64; i += blockDim.x) {
    S.b1[i] = __ldg(w + CLOT_MLP_OFF_B1 + i);
    S.b2[i] = __ldg(w + CLOT_MLP_OFF_B2 + i);
    if (i < 16) S.b3[i] = __ldg(w + CLOT_MLP_OFF_B3 + i);
  }
  for (int i = threadIdx.x; i < NP; i += blockDim.x) S.gw[i] = 0.0f;
  for (int i = threadIdx.x; i < 4 * (64 + 64 + 16); i += blockDim.x) (&S.gb[0][0])[i] = 0.0f;
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
  const int col0 = 16 * warp;
  float lsum = 0.0f;
  const long long nchunk = (n + 63) / 64;
  for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const long long row0 = ch * 64 + col0;
    // forward (FP32 pre-activations kept in registers for gelu')
    uint32_t a1[2][4];
    load_afrag_x(a1, x, row0, n, lane);
    store_afrag_T<2>(S.xT, a1, col0, lane);
    float z1[8][4], z2[8][4], o[2][4];
    uint32_t h[4][4];
    bias_init<8>(z1, S.b1, q);
    mma_layer<2, 8>(z1, a1, S.w1, lane);
    to_afrag<8, 2>(h, z1);
    store_afrag_T<4>(S.h1T, h, col0, lane);
    bias_init<8>(z2, S.b2, q);
    mma_layer<4, 8>(z2, h, S.w2, lane);
    to_afrag<8, 2>(h, z2);
    store_afrag_T<4>(S.h2T, h, col0, lane);
    bias_init<2>(o, S.b3, q);
    mma_layer<4, 2>(o, h, S.w3, lane);
    // residual d = v - target (rows >= n and columns 14, 15 zero)
    const long long r0 = row0 + g, r1 = r0 + 8;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int col = 8 * nt + 2 * q + (e & 1);
        const long long row = (e & 2) ? r1 : r0;
        const float d = (row < n && col < 14) ? o[nt][e] - __ldg(yv + row * 16 + col) : 0.0f;
        o[nt][e] = d;
        lsum = fmaf(d, d, lsum);
      }
    colsum_add<2>(S.gb[warp] + 128, o, lane);
    uint32_t da[1][4];
    to_afrag<2, 0>(da, o);
    store_afrag_T<1>(S.dT, da, col0, lane);
    // dh2 = d W3^T; dz2 = dh2 gelu'(z2)
    float gacc[8][4];
    zero_acc<8>(gacc);
    mma_layer<1, 8>(gacc, da, S.w3t, lane);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) gacc[nt][e] *= gelu_grad(z2[nt][e]);
    colsum_add<8>(S.gb[warp] + 64, gacc, lane);
    to_afrag<8, 0>(h, gacc);
    store_afrag_T<4>(S.dz2T, h, col0, lane);
    // dh1 = dz2 W2^T; dz1 = dh1 gelu'(z1)
    zero_acc<8>(gacc);
    mma_layer<4, 8>(gacc, h, S.w2t, lane);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) gacc[nt][e] *= gelu_grad(z1[nt][e]);
    colsum_add<8>(S.gb[warp], gacc, lane);
    to_afrag<8, 0>(h, gacc);
    store_afrag_T<4>(S.dz1T, h, col0, lane);
    __syncthreads();
    // weight gradients over the chunk: each warp a disjoint 16-wide slice
    switch (warp) {  // template tile indices need compile-time constants
      case 0:
        wgrad<0, 2, 0, 2>(S.gw + CLOT_MLP_OFF_W1, 64, S.xT, S.dz1T, lane);
        wgrad<0, 4, 0, 2>(S.gw + CLOT_MLP_OFF_W2, 64, S.h1T, S.dz2T, lane);
        wgrad<0, 1, 0, 2>(S.gw + CLOT_MLP_OFF_W3, 16, S.h2T, S.dT, lane);
        break;
      case 1:
        wgrad<0, 2, 2, 2>(S.gw + CLOT_MLP_OFF_W1, 64, S.xT, S.dz1T, lane);
        wgrad<0, 4, 2, 2>(S.gw + CLOT_MLP_OFF_W2, 64, S.h1T, S.dz2T, lane);
        wgrad<1, 1, 0, 2>(S.gw + CLOT_MLP_OFF_W3, 16, S.h2T, S.dT, lane);
        break;
      case 2:
        wgrad<0, 2, 4, 2>(S.gw + CLOT_MLP_OFF_W1, 64, S.xT, S.dz1T, lane);
        wgrad<0, 4, 4, 2>(S.gw + CLOT_MLP_OFF_W2, 64, S.h1T, S.dz2T, lane);
        wgrad<2, 1, 0, 2>(S.gw + CLOT_MLP_OFF_W3, 16, S.h2T, S.dT, lane);
        break;
      default:
        wgrad<0, 2, 6, 2>(S.gw + CLOT_MLP_OFF_W1, 64, S.xT, S.dz1T, lane);
        wgrad<0, 4, 6, 2>(S.gw + CLOT_MLP_OFF_W2, 64, S.h1T, S.dz2T, lane);
        wgrad<3, 1, 0, 2>(S.gw + CLOT_MLP_OFF_W3, 16, S.h2T, S.dT, lane);
        break;
    }
    __syncthreads();
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if (lane == 0) S.lw[warp] = lsum;
  __syncthreads();
  // bias gradients: the four warps' sums in a fixed order (deterministic)
  for (int i = threadIdx.x; i < 64 + 64 + 16; i += blockDim.x) {
    const float v = ((S.gb[0][i] + S.gb[1][i]) + S.gb[2][i]) + S.gb[3][i];
    const int dst = i < 64 ? CLOT_MLP_OFF_B1 + i : i < 128 ? CLOT_MLP_OFF_B2 + (i - 64) : CLOT_MLP_OFF_B3 + (i - 128);
    S.gw[dst] = v;
  }
  __syncthreads();
  float* out = work + (size_t)blockIdx.x * WSTRIDE;
  for (int i = threadIdx.x; i < NP; i += blockDim.x) out[i] = S.gw[i];
  if (threadIdx.x == 0) out[NP] = ((S.lw[0] + S.lw[1]) + S.lw[2]) + S.lw[3];
}

// Sum of the block partials (fixed order), scaled: grad = gscale sum, loss =
// lscale sum; optional Adam step on w with moments m, v.
__global__ void mlp_reduce_adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                                       const float* __restrict__ work, int nblk, float gscale, float lscale,
                                       float lr, float bc1, float bc2, float* __restrict__ grad,
                                       float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > NP) return;
  float s = 0.0f;
  for (int b = 0; b < nblk; ++b) s += work[(size_t)b * WSTRIDE + p];
  if (p == NP) {
    if (loss) *loss = s * lscale;
    return;
  }
  const float gr = s * gscale;
  if (grad) grad[p] = gr;
  if (m) {
    const float mn = fmaf(0.9f, m[p], 0.1f * gr);
    const float vn = fmaf(0.999f, v[p], 0.001f * gr * gr);
    m[p] = mn;
    v[p] = vn;
    w[p] -= lr * (mn / bc1) / (sqrtf(vn / bc2) + 1e-8f);
  }
}

int g_sms = 0;
int sm_count() {
  if (g_sms <= 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  return g_sms;
}

int grad_blocks(long long n) {
  const long long nchunk = (n + 63) / 64;
  return (int)std::max<long long>(1, std::min<long long>(nchunk, std::min(2 * sm_count(), MAX_GRAD_BLOCKS)));
}

cudaError_t launch_grad(const float* w, const float* x, const float* y, long long n, float* work, int nblk,
                        cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TrainSmem));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  mlp_grad_kernel<<<nblk, 128, sizeof(TrainSmem), s>>>(w, x, y, n, work);
  return cudaGetLastError();
}

int err(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

bool scales_ok(const clot_mlp* mlp) {
  for (int s = 0; s < CLOT_NS; ++s)
    if (!(mlp->scale[s] > 0.0f) || !isfinite(mlp->scale[s])) return false;
  return true;
}

}  // namespace

void surrogate_fill_consts(const clot_mlp* mlp, double dt, float* inv_scale, float* floor_s, float* xdt) {
  for (int s = 0; s < CLOT_NS; ++s) {
    inv_scale[s] = (float)(1.0 / (double)mlp->scale[s]);
    floor_s[s] = (float)(1e-6 * (double)mlp->scale[s]);
  }
  *xdt = (float)log(dt / 1e-5);
}

// Persistent grid of at most 4 CTAs per SM (the shared-memory size caps the
// residency at 4, so the 128 tensor-memory columns of each always fit).
template <class Kern>
int tc_grid(Kern kern, long long chunks, cudaError_t* err) {
  *err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  if (*err != cudaSuccess) return 0;
  *err = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (*err != cudaSuccess) return 0;
  return (int)std::max<long long>(1, std::min<long long>(chunks, 4LL * sm_count()));
}

cudaError_t launch_surrogate_react(const SurrArgs& a, cudaStream_t s) {
  cudaError_t e;
  if (a.engine == CLOT_MLP_ENGINE_TCGEN05) {
    const int grid = tc_grid(surrogate_react_tc_kernel, (a.g.ncell + 127) / 128, &e);
    if (e != cudaSuccess) return e;
    surrogate_react_tc_kernel<<<grid, 128, TC_SMEM, s>>>(a);
    return cudaGetLastError();
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, surrogate_react_kernel, 128, 0);
  if (e != cudaSuccess) return e;
  const long long need = (a.g.ncell + 127) / 128;
  const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)std::max(per_sm, 1) * sm_count()));
  surrogate_react_kernel<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_surrogate_fallback(const SurrArgs& a, cudaStream_t s) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, surrogate_fallback_kernel, 128, 0);
  if (e != cudaSuccess) return e;
  const long long need = (a.g.ncell + 127) / 128;
  const int grid = (int)std::max<long long>(1, std::min<long long>(need, (long long)std::max(per_sm, 1) * sm_count()));
  surrogate_fallback_kernel<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace clot

using namespace clot;

#define SURR_CUDA(expr)                                                  \
  do {                                                                   \
    cudaError_t e_ = (expr);                                             \
    if (e_ != cudaSuccess) {                                             \
      char b_[256];                                                      \
      snprintf(b_, sizeof(b_), "%s: %s", #expr, cudaGetErrorString(e_)); \
      set_last_error(b_);                                                \
      return CLOT_ECUDA;                                                 \
    }                                                                    \
  } while (0)

extern "C" int clot_surrogate_pairs(const clot_params* p, const clot_mlp* mlp, const float* c0, const float* eta,
                                    int64_t n, int64_t pitch, double dt, float* x, float* y, void* stream) {
  if (!p || !mlp || !c0 || !eta || !x || !y) return err(CLOT_EINVAL, "null argument");
  if (n < 0 || pitch < n) return err(CLOT_EINVAL, "need 0 <= n <= pitch");
  if (!(dt > 0) || p->M_rxn < 1) return err(CLOT_EINVAL, "need dt > 0 and M_rxn >= 1");
  if (!scales_ok(mlp)) return err(CLOT_EINVAL, "surrogate scales must be finite and > 0");
  if (check_params_common(p)) return CLOT_EINVAL;
  if (n == 0) return CLOT_OK;
  PairArgs A{};
  memset(&A, 0, sizeof(A));
  A.c0 = c0;
  A.eta = eta;
  A.x = x;
  A.y = y;
  A.n = n;
  A.pitch = pitch;
  A.dt = dt;
  A.M = p->M_rxn;
  A.h = dt / p->M_rxn;
  clot_mesh_desc d;
  memset(&d, 0, sizeof(d));
  d.hy = 1.0;  // wall terms are not used here
  A.r = make_rxn_const(d, p);
  surrogate_fill_consts(mlp, dt, A.inv_scale, A.floor_s, &A.xdt);
  const int grid = (int)std::min<long long>((n + 127) / 128, 16LL * sm_count());
  surrogate_pairs_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(A);
  SURR_CUDA(cudaGetLastError());
  return CLOT_OK;
}

extern "C" int clot_surrogate_forward(const clot_mlp* mlp, const float* x, int64_t n, float* out, void* stream) {
  if (!mlp || !mlp->w || !x || !out) return err(CLOT_EINVAL, "null argument");
  if (mlp->engine != CLOT_MLP_ENGINE_MMA && mlp->engine != CLOT_MLP_ENGINE_TCGEN05)
    return err(CLOT_EINVAL, "unknown network engine");
  if (n < 0) return err(CLOT_EINVAL, "n < 0");
  if (n == 0) return CLOT_OK;
  if (mlp->engine == CLOT_MLP_ENGINE_TCGEN05) {
    cudaError_t e;
    const int grid = tc_grid(mlp_forward_tc_kernel, (n + 127) / 128, &e);
    SURR_CUDA(e);
    mlp_forward_tc_kernel<<<grid, 128, TC_SMEM, (cudaStream_t)stream>>>(mlp->w, x, n, out, nullptr);
  } else {
    const long long ntile = (n + 15) / 16;
    const int grid = (int)std::min<long long>((ntile + 3) / 4, 8LL * sm_count());
    mlp_forward_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(mlp->w, x, n, out);
  }
  SURR_CUDA(cudaGetLastError());
  return CLOT_OK;
}

extern "C" int64_t clot_surrogate_workspace(int64_t n) {
  if (n <= 0) return 0;
  const long long nchunk = (n + 63) / 64;
  return (int64_t)std::min<long long>(nchunk, MAX_GRAD_BLOCKS) * WSTRIDE;
}

extern "C" int clot_surrogate_grad(const clot_mlp* mlp, const float* x, const float* y, int64_t n, float* work,
                                   int64_t work_floats, float* grad, float* loss, void* stream) {
  if (!mlp || !mlp->w || !x || !y || !work || !grad) return err(CLOT_EINVAL, "null argument");
  if (n < 1) return err(CLOT_EINVAL, "need n >= 1");
  const int nblk = grad_blocks(n);
  if (work_floats < (int64_t)nblk * WSTRIDE) return err(CLOT_EINVAL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  SURR_CUDA(launch_grad(mlp->w, x, y, n, work, nblk, s));
  const double B14 = (double)n * 14.0;
  mlp_reduce_adam_kernel<<<(NP + 1 + 255) / 256, 256, 0, s>>>(nullptr, nullptr, nullptr, work, nblk,
                                                               (float)(2.0 / B14), (float)(1.0 / B14), 0.0f, 1.0f,
                                                               1.0f, grad, loss);
  SURR_CUDA(cudaGetLastError());
  return CLOT_OK;
}

extern "C" int clot_surrogate_train(const clot_mlp* mlp, float* m, float* v, int t0, float lr, const float* x,
                                    const float* y, int64_t n, int64_t batch, int nsteps, float* work,
                                    int64_t work_floats, float* loss, void* stream) {
  if (!mlp || !mlp->w || !m || !v || !x || !y || !work) return err(CLOT_EINVAL, "null argument");
  if (batch < 1 || n < batch || n % batch != 0) return err(CLOT_EINVAL, "n must be a positive multiple of batch");
  if (nsteps < 0 || t0 < 0 || !(lr >= 0.0f)) return err(CLOT_EINVAL, "need nsteps >= 0, t0 >= 0, lr >= 0");
  const int nblk = grad_blocks(batch);
  if (work_floats < (int64_t)nblk * WSTRIDE) return err(CLOT_EINVAL, "workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const double B14 = (double)batch * 14.0;
  for (int st = 0; st < nsteps; ++st) {
    const long long off = ((long long)st * batch) % n;
    SURR_CUDA(launch_grad(mlp->w, x + off * 32, y + off * 16, batch, work, nblk, s));
    const int t = t0 + st + 1;
    const double bc1 = 1.0 - pow(0.9, t), bc2 = 1.0 - pow(0.999, t);
    mlp_reduce_adam_kernel<<<(NP + 1 + 255) / 256, 256, 0, s>>>(
        mlp->w, m, v, work, nblk, (float)(2.0 / B14), (float)(1.0 / B14), lr, (float)bc1, (float)bc2, nullptr,
        loss ? loss + st : nullptr);
    SURR_CUDA(cudaGetLastError());
  }
  return CLOT_OK;
}

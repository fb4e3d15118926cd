// clot_ensemble.cu -- many independent channels (meshes) advanced together.
//
// Every channel is a full species-step problem of its own (mesh, state,
// fluxes, inlet values, time step; Sec. 3.2).  Per step the ensemble issues
// two launches for all channels at once (or, inside the replayed graph, for
// each of up to four chains of channels holding equal shares of the cells,
// on parallel graph branches):
//   1. eta_block_cg_kernel: one block per channel solves (App. A Eq. eta)
//      by conjugate gradients with block-level (deterministic) reductions,
//      accepting the eta predicted by the previous fused step when it already
//      meets the stopping rule;
//   2. the persistent fused-step kernel (clot_step_tiled.cu) over a work list
//      of (channel, tile) items of all channels.
// The per-step kernel arguments repeat with period 6 (state ping-pong x eta
// buffer rotation), so they are uploaded once per call and a 6-step CUDA graph
// is replayed.  An autotuner picks the persistent grid size and the order of
// the work list by timing candidates on the actual ensemble.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "clot_internal.cuh"

namespace clot {
namespace {

constexpr int EB = 1024;  // threads per channel block of the eta solve
constexpr int MAXCH = 4;  // most chains of channels on parallel graph branches

// Sum, sum, max over the block (FP32 inputs, FP64 accumulation), returned to
// every thread; fixed shuffle / tree order -> deterministic.
__device__ void block_all_reduce3(float a, float b, float c, double& sa, double& sb, double& mc) {
  __shared__ double sh[3][EB / 32];
  __shared__ double res[3];
  double da = a, db = b, dc = c;
  for (int o = 16; o > 0; o >>= 1) {
    da += __shfl_xor_sync(0xffffffffu, da, o);
    db += __shfl_xor_sync(0xffffffffu, db, o);
    dc = fmax(dc, __shfl_xor_sync(0xffffffffu, dc, o));
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[0][w] = da;
    sh[1][w] = db;
    sh[2][w] = dc;
  }
  __syncthreads();
  if (w == 0) {
    double x = l < EB / 32 ? sh[0][l] : 0.0, y = l < EB / 32 ? sh[1][l] : 0.0, z = l < EB / 32 ? sh[2][l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
      z = fmax(z, __shfl_xor_sync(0xffffffffu, z, o));
    }
    if (l == 0) {
      res[0] = x;
      res[1] = y;
      res[2] = z;
    }
  }
  __syncthreads();
  sa = res[0];
  sb = res[1];
  mc = res[2];
  __syncthreads();
}

__device__ __forceinline__ float op_at(const EtaArgs& a, const float* x, int P) {
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int i = P % nx, j = (P / nx) % ny, k = P / (nx * ny);
  const float xp = x[P];
  float lx = 0.0f, ly = 0.0f, lz = 0.0f;
  if (i > 0) lx += x[P - 1] - xp;
  if (i < nx - 1) lx += x[P + 1] - xp;
  if (j > 0) ly += x[P - nx] - xp;
  if (j < ny - 1) ly += x[P + nx] - xp;
  if (a.g.dim == 3) {
    if (k > 0) lz += x[P - nx * ny] - xp;
    if (k < nz - 1) lz += x[P + nx * ny] - xp;
  }
  return xp - (a.cx * lx + a.cy * ly + a.cz * lz);
}

// A pass over the channel's n cells in which every thread keeps U cells'
// loads in flight: load(P) for P, P + EB, ..., P + (U - 1) EB first, then
// use(P, value) for each (one block per channel leaves few warps per SM, so a
// pass that waits for each cell's loads in turn is bound by memory latency).
template <int U = 2, class L, class F>
__device__ __forceinline__ void passU(int n, L load, F use) {
  for (int P0 = threadIdx.x; P0 < n; P0 += U * EB) {
    decltype(load(0)) v[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (P0 + u * EB < n) v[u] = load(P0 + u * EB);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (P0 + u * EB < n) use(P0 + u * EB, v[u]);
  }
}

// A cell's value and its neighbours' (the cell's own value where the mesh
// ends: the zero-flux walls of Eq. eta), and the operator applied to them
// with the same arithmetic as op_at.
struct Nb {
  float c, w, e, s, n, b, t;
};
__device__ __forceinline__ Nb load_nb(const EtaArgs& a, const float* x, int P) {
  const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
  const int i = P % nx, j = (P / nx) % ny, k = P / (nx * ny);
  Nb v;
  v.c = x[P];
  v.w = i > 0 ? x[P - 1] : v.c;
  v.e = i < nx - 1 ? x[P + 1] : v.c;
  v.s = j > 0 ? x[P - nx] : v.c;
  v.n = j < ny - 1 ? x[P + nx] : v.c;
  v.b = (a.g.dim == 3 && k > 0) ? x[P - nx * ny] : v.c;
  v.t = (a.g.dim == 3 && k < nz - 1) ? x[P + nx * ny] : v.c;
  return v;
}
__device__ __forceinline__ float op_nb(const EtaArgs& a, const Nb& v) {
  const float lx = (v.w - v.c) + (v.e - v.c), ly = (v.s - v.c) + (v.n - v.c), lz = (v.b - v.c) + (v.t - v.c);
  return v.c - (a.cx * lx + a.cy * ly + a.cz * lz);
}

// One block per channel: (I - L^2/4 lap) eta = theta_B by CG (App. A Eq. eta),
// same stopping rule and prediction acceptance as the single-mesh solver.
__global__ void __launch_bounds__(EB) eta_block_cg_kernel(const EtaArgs* __restrict__ chans) {
  __shared__ __align__(16) EtaArgs a;
  {
    const int* src = reinterpret_cast<const int*>(chans + blockIdx.x);
    int* dst = reinterpret_cast<int*>(&a);
    for (int q = threadIdx.x; q < (int)(sizeof(EtaArgs) / sizeof(int)); q += EB) dst[q] = src[q];
  }
  __syncthreads();
  const int n = (int)a.g.ncell;
  const long long pitch = a.g.pitch;
  // the element-wise passes move quads of four cells as float4 when they can
  auto al16 = [](const void* q) { return ((unsigned long long)q & 15u) == 0; };
  const bool v4 = n % 4 == 0 && al16(a.r) && al16(a.p) && al16(a.q) && al16(a.eta);
  const int n4 = n / 4;
  auto ld4 = [](const float* q, int Q) { return *reinterpret_cast<const float4*>(q + 4 * Q); };
  auto st4 = [](float* q, int Q, float4 v) { *reinterpret_cast<float4*>(q + 4 * Q) = v; };
  double s_rr, s_rmax, s_bmax, d0, d1;
  int it = 0;
  bool fresh = !a.predicted;
  if (a.predicted) {
    const float pr = __uint_as_float(a.maxw[0]), pb = __uint_as_float(a.maxw[1]);
    __syncthreads();
    if (threadIdx.x == 0) {
      a.maxw_clear[0] = 0u;
      a.maxw_clear[1] = 0u;
      a.status[1] = 0;
    }
    if (pb > 0.0f && pr <= fmaxf(a.tol * pb, a.atol)) {
      if (threadIdx.x == 0) a.status[3] += 1;
      return;
    }
    // The prediction's residual is large only where theta_B changed in a way
    // the extrapolation did not follow: correct eta by CG on the box around
    // the cells with |r| > thr, widened by the decay length of the correction
    // (the same rule as the single-mesh solver's box correction), then check
    // the true residual on the layer around the box.
    const double stop = (double)a.inner * fmax((double)a.tol * pb, (double)a.atol);
    const float cmax = fmaxf(a.cx, fmaxf(a.cy, a.cz));
    const float thr = (float)(0.5 * stop) / (1.0f + cmax);
    __shared__ unsigned sb[6];  // max(~lo), max(hi + 1) per axis of the cells with |r| > thr
    if (threadIdx.x < 6) sb[threadIdx.x] = 0u;
    __syncthreads();
    const int nx = a.g.nx, ny = a.g.ny;
    unsigned bl[3] = {0u, 0u, 0u}, bh[3] = {0u, 0u, 0u};
    float rr = 0.0f;
    auto mark = [&](int P, float r) {
      rr += r * r;
      if (fabsf(r) > thr) {
        const unsigned i = (unsigned)(P % nx), j = (unsigned)((P / nx) % ny), k = (unsigned)(P / (nx * ny));
        bl[0] = max(bl[0], ~i);
        bl[1] = max(bl[1], ~j);
        bl[2] = max(bl[2], ~k);
        bh[0] = max(bh[0], i + 1u);
        bh[1] = max(bh[1], j + 1u);
        bh[2] = max(bh[2], k + 1u);
      }
    };
    if (v4) {
      passU<1>(n4, [&](int Q) { return ld4(a.r, Q); }, [&](int Q, float4 r) {
        st4(a.p, Q, r);
        mark(4 * Q, r.x);
        mark(4 * Q + 1, r.y);
        mark(4 * Q + 2, r.z);
        mark(4 * Q + 3, r.w);
      });
    } else {
      passU(n, [&](int P) { return a.r[P]; }, [&](int P, float r) {
        a.p[P] = r;
        mark(P, r);
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
        atomicMax(&sb[d], bl[d]);
        atomicMax(&sb[3 + d], bh[d]);
      }
    }
    block_all_reduce3(rr, 0.0f, 0.0f, s_rr, d0, d1);  // its barriers publish sb
    s_rmax = pr;
    s_bmax = pb;
    Box B;
    bool use_box = false;
    if (pb > 0.0f && pr < 3.0e38f && sb[3] != 0u) {
      const int mx = box_margin(a.cx, pr, (float)stop), my = box_margin(a.cy, pr, (float)stop);
      const int mz = a.g.dim == 3 ? box_margin(a.cz, pr, (float)stop) : 0;
      B.i0 = max((int)~sb[0] - mx, 0);
      B.j0 = max((int)~sb[1] - my, 0);
      B.k0 = max((int)~sb[2] - mz, 0);
      B.i1 = min((int)sb[3] - 1 + mx, a.g.nx - 1);
      B.j1 = min((int)sb[4] - 1 + my, a.g.ny - 1);
      B.k1 = min((int)sb[5] - 1 + mz, a.g.nz - 1);
      use_box = 2 * B.cells() <= a.g.ncell;
    }
    if (use_box) {
      const int bnx = B.i1 - B.i0 + 1, bny = B.j1 - B.j0 + 1;
      const int nb = (int)B.cells();
      const int sz = nx * ny;
      auto cell = [&](int q, int& i, int& j, int& k) {
        i = B.i0 + q % bnx;
        j = B.j0 + (q / bnx) % bny;
        k = B.k0 + q / (bnx * bny);
        return i + nx * (j + ny * k);
      };
      // CG for the correction on the box (search direction zero outside it),
      // in place on eta and r; the search directions alternate between p, p2
      float* pold = a.p;
      float* pnew = a.p2;
      float beta = 0.0f;
      double s_rb = 0.0, s_mb = pr;
      bool first = true;
      while (it < a.maxit && s_mb > stop) {
        float pq = 0.0f, r0 = 0.0f;
        for (int q = threadIdx.x; q < nb; q += EB) {
          int i, j, k;
          const int P = cell(q, i, j, k);
          auto pv = [&](int Q) { return a.r[Q] + (beta != 0.0f ? beta * pold[Q] : 0.0f); };
          const float pp = pv(P);
          float lx = 0.0f, ly = 0.0f, lz = 0.0f;
          if (i > 0) lx += (i - 1 >= B.i0 ? pv(P - 1) : 0.0f) - pp;
          if (i < nx - 1) lx += (i + 1 <= B.i1 ? pv(P + 1) : 0.0f) - pp;
          if (j > 0) ly += (j - 1 >= B.j0 ? pv(P - nx) : 0.0f) - pp;
          if (j < ny - 1) ly += (j + 1 <= B.j1 ? pv(P + nx) : 0.0f) - pp;
          if (a.g.dim == 3) {
            if (k > 0) lz += (k - 1 >= B.k0 ? pv(P - sz) : 0.0f) - pp;
            if (k < a.g.nz - 1) lz += (k + 1 <= B.k1 ? pv(P + sz) : 0.0f) - pp;
          }
          const float qv = pp - (a.cx * lx + a.cy * ly + a.cz * lz);
          pnew[P] = pp;
          a.q[P] = qv;
          pq += pp * qv;
          if (first) r0 += a.r[P] * a.r[P];
        }
        double s_pq, s_r0;
        block_all_reduce3(pq, r0, 0.0f, s_pq, s_r0, d1);
        if (first) s_rb = s_r0;
        first = false;
        if (!(s_pq > 0.0)) break;
        const float alpha = (float)(s_rb / s_pq);
        float rr2 = 0.0f, rm = 0.0f;
        for (int q = threadIdx.x; q < nb; q += EB) {
          int i, j, k;
          const int P = cell(q, i, j, k);
          a.eta[P] += alpha * pnew[P];
          const float r = a.r[P] - alpha * a.q[P];
          a.r[P] = r;
          rr2 += r * r;
          rm = fmaxf(rm, fabsf(r));
        }
        double s_rr2;
        block_all_reduce3(rr2, 0.0f, rm, s_rr2, d0, s_mb);
        beta = (float)(s_rr2 / s_rb);
        s_rb = s_rr2;
        float* t = pold;
        pold = pnew;
        pnew = t;
        ++it;
      }
      // the true residual on the layer of cells around the box
      Box L = B;
      L.i0 = max(B.i0 - 1, 0);
      L.j0 = max(B.j0 - 1, 0);
      L.k0 = max(B.k0 - 1, 0);
      L.i1 = min(B.i1 + 1, a.g.nx - 1);
      L.j1 = min(B.j1 + 1, a.g.ny - 1);
      L.k1 = min(B.k1 + 1, a.g.nz - 1);
      const int lnx = L.i1 - L.i0 + 1, lny = L.j1 - L.j0 + 1;
      const int nl = (int)L.cells();
      float vm = 0.0f;
      for (int q = threadIdx.x; q < nl; q += EB) {
        const int i = L.i0 + q % lnx, j = L.j0 + (q / lnx) % lny, k = L.k0 + q / (lnx * lny);
        if (B.in(i, j, k)) continue;
        const int P = i + nx * (j + ny * k);
        const float b = (a.c[2 * pitch + P] + a.c[3 * pitch + P]) * a.invPmax;
        const float r = b - op_at(a, a.eta, P);
        a.r[P] = r;
        vm = fmaxf(vm, fabsf(r));
      }
      double s_vm;
      block_all_reduce3(0.0f, 0.0f, vm, d0, d1, s_vm);
      if (s_mb <= stop && s_vm <= stop) {
        if (threadIdx.x == 0) {
          a.status[1] = it;
          a.status[2] += it;
        }
        return;
      }
      fresh = true;  // continue on the whole channel from the improved eta
    }
  }
  if (fresh) {
    float rr = 0.0f, rm = 0.0f, bm = 0.0f;
    struct Fr {
      Nb x;
      float ba, bse;
    };
    passU(n, [&](int P) { return Fr{load_nb(a, a.eta, P), a.c[2 * pitch + P], a.c[3 * pitch + P]}; },
          [&](int P, const Fr& v) {
            const float b = (v.ba + v.bse) * a.invPmax;
            const float r = b - op_nb(a, v.x);
            a.r[P] = r;
            a.p[P] = r;
            rr += r * r;
            rm = fmaxf(rm, fabsf(r));
            bm = fmaxf(bm, fabsf(b));
          });
    block_all_reduce3(rr, 0.0f, rm, s_rr, d0, s_rmax);
    block_all_reduce3(0.0f, 0.0f, bm, d0, d1, s_bmax);
  }
  if (s_bmax == 0.0) {
    for (int P = threadIdx.x; P < n; P += EB) a.eta[P] = 0.0f;
  } else {
    const double stop = (double)a.inner * fmax((double)a.tol * s_bmax, (double)a.atol);
    while (it < a.maxit && s_rmax > stop) {
      __syncthreads();  // p complete
      float pq = 0.0f;
      passU(n, [&](int P) { return load_nb(a, a.p, P); },
            [&](int P, const Nb& v) {
              const float q = op_nb(a, v);
              a.q[P] = q;
              pq += v.c * q;
            });
      double s_pq;
      block_all_reduce3(pq, 0.0f, 0.0f, s_pq, d0, d1);
      const float alpha = (float)(s_rr / s_pq);
      float rr2 = 0.0f, rm = 0.0f;
      auto upd = [&](float r0, float qq) {
        const float r = r0 - alpha * qq;
        rr2 += r * r;
        rm = fmaxf(rm, fabsf(r));
        return r;
      };
      if (v4) {
        struct Q4 {
          float4 e, p, r, q;
        };
        passU<1>(n4, [&](int Q) { return Q4{ld4(a.eta, Q), ld4(a.p, Q), ld4(a.r, Q), ld4(a.q, Q)}; },
                 [&](int Q, const Q4& v) {
                   st4(a.eta, Q, make_float4(v.e.x + alpha * v.p.x, v.e.y + alpha * v.p.y, v.e.z + alpha * v.p.z,
                                             v.e.w + alpha * v.p.w));
                   const float4 r = make_float4(upd(v.r.x, v.q.x), upd(v.r.y, v.q.y), upd(v.r.z, v.q.z),
                                                upd(v.r.w, v.q.w));
                   st4(a.r, Q, r);
                 });
      } else {
        passU(n, [&](int P) { return make_float4(a.eta[P], a.p[P], a.r[P], a.q[P]); },
              [&](int P, const float4& v) {
                a.eta[P] = v.x + alpha * v.y;
                a.r[P] = upd(v.z, v.w);
              });
      }
      double s_rr2;
      block_all_reduce3(rr2, 0.0f, rm, s_rr2, d0, s_rmax);
      const float beta = (float)(s_rr2 / s_rr);
      s_rr = s_rr2;
      if (v4) {
        struct RP {
          float4 r, p;
        };
        passU<1>(n4, [&](int Q) { return RP{ld4(a.r, Q), ld4(a.p, Q)}; }, [&](int Q, const RP& v) {
          st4(a.p, Q, make_float4(v.r.x + beta * v.p.x, v.r.y + beta * v.p.y, v.r.z + beta * v.p.z,
                                  v.r.w + beta * v.p.w));
        });
      } else {
        passU(n, [&](int P) { return make_float2(a.r[P], a.p[P]); },
              [&](int P, const float2& v) { a.p[P] = v.x + beta * v.y; });
      }
      ++it;
    }
  }
  if (threadIdx.x == 0) {
    a.status[1] = it;
    a.status[2] += it;
  }
}

}  // namespace
}  // namespace clot

using namespace clot;

struct clot_ensemble {
  int nchan = 0, dim = 2;
  bool vec2 = true;
  int device = 0, sms = 1;
  std::vector<clot_mesh_desc> desc;
  std::vector<Geom> geom;
  std::vector<long long> off_state, off_cell;
  float* scratch = nullptr;   // per channel [15][pitch]
  float* eta_ws = nullptr;    // per channel [2][ncell]
  float* cg = nullptr;        // per channel [4][ncell]
  unsigned* maxw = nullptr;   // per channel [4]
  int* status = nullptr;      // per channel [4]
  double* partials = nullptr; // reductions of the diagnostics / flux checks
  int aux_blocks = 1;
  int4* work = nullptr;
  int nwork = 0;
  // Chains of the replayed graph: chain q holds channels [cb[q], cb[q + 1])
  // (about 1 / chains of the cells each) and work items [wb[q], wb[q + 1]).
  int chains = 2;             // 1: one branch for all channels; 2 .. MAXCH: parallel graph branches
  int cb[MAXCH + 1] = {};
  int wb[MAXCH + 1] = {};
  int order = 0;              // 0 channel-major, 1 largest channels first, tiles interleaved
  int grid = 0;               // persistent grid of the fused step
  StepArgs* step_dev = nullptr;  // [7][nchan]
  EtaArgs* eta_dev = nullptr;    // [7][nchan]
  std::vector<StepArgs> step_host;
  std::vector<EtaArgs> eta_host;
  std::vector<const float*> vfx, vfy, vfz;
  std::vector<double> vdt;
  cudaStream_t cap_stream = nullptr, cap_side[MAXCH - 1] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[MAXCH - 1] = {};
  cudaGraphExec_t graph = nullptr;
  int graph_grid = -1, graph_nwork = -1, graph_chains = -1;
};

static int efail(int code, const char* fmt, ...) {
  char msg[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  set_last_error(msg);
  return code;
}
#define ECUDA(expr)                                                                         \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) return efail(CLOT_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

static void ens_free(clot_ensemble* e) {
  if (!e) return;
  if (e->graph) cudaGraphExecDestroy(e->graph);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  for (int q = 0; q < MAXCH - 1; ++q) {
    if (e->cap_side[q]) cudaStreamDestroy(e->cap_side[q]);
    if (e->ev_join[q]) cudaEventDestroy(e->ev_join[q]);
  }
  if (e->ev_fork) cudaEventDestroy(e->ev_fork);
  cudaFree(e->scratch);
  cudaFree(e->eta_ws);
  cudaFree(e->cg);
  cudaFree(e->maxw);
  cudaFree(e->status);
  cudaFree(e->partials);
  cudaFree(e->work);
  cudaFree(e->step_dev);
  cudaFree(e->eta_dev);
  delete e;
}

// Chain boundaries for e->chains chains (fewer when there are fewer
// channels): cb[q] is the first channel index whose prefix holds q / chains
// of the cells, every chain keeping at least one channel.
static void split_chains(clot_ensemble* e) {
  const int n = std::max(1, std::min(e->chains, e->nchan));
  long long tot = 0;
  for (auto& g : e->geom) tot += g.ncell;
  e->cb[0] = 0;
  long long acc = 0;
  int c = 0;
  for (int q = 1; q < n; ++q) {
    while (c < e->nchan - (n - q) && acc * n < tot * q) acc += e->geom[c++].ncell;
    if (c == e->cb[q - 1]) acc += e->geom[c++].ncell;  // chain q - 1 keeps one channel at least
    e->cb[q] = c;
  }
  for (int q = n; q <= MAXCH; ++q) e->cb[q] = e->nchan;
}

// Work list: every (channel, tile column, tile row, plane) item, chain by
// chain.  Within each chain, order 0: channel by channel; order 1: channels by
// decreasing size, items of different channels interleaved round-robin
// (spreads big channels over the launch).
static void build_work(clot_ensemble* e, std::vector<int4>& w) {
  w.clear();
  const int TX = tile_x(), TY = tile_y();
  std::vector<std::vector<int4>> per(e->nchan);
  for (int c = 0; c < e->nchan; ++c) {
    const Geom& g = e->geom[c];
    for (int k = 0; k < g.nz; ++k)
      for (int by = 0; by < (g.ny + TY - 1) / TY; ++by)
        for (int bx = 0; bx < (g.nx + TX - 1) / TX; ++bx) per[c].push_back(make_int4(c, bx, by, k));
  }
  e->wb[0] = 0;
  for (int part = 0; part < MAXCH; ++part) {
    const int lo = e->cb[part], hi = e->cb[part + 1];
    if (e->order == 0) {
      for (int c = lo; c < hi; ++c) w.insert(w.end(), per[c].begin(), per[c].end());
    } else {
      std::vector<int> idx(hi - lo);
      std::iota(idx.begin(), idx.end(), lo);
      std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return per[a].size() > per[b].size(); });
      size_t maxlen = 0;
      for (int c : idx) maxlen = std::max(maxlen, per[c].size());
      for (size_t r = 0; r < maxlen; ++r)
        for (int c : idx)
          if (r < per[c].size()) w.push_back(per[c][r]);
    }
    e->wb[part + 1] = (int)w.size();
  }
}

static int upload_work(clot_ensemble* e) {
  std::vector<int4> w;
  build_work(e, w);
  e->nwork = (int)w.size();
  ECUDA(cudaMemcpy(e->work, w.data(), sizeof(int4) * w.size(), cudaMemcpyHostToDevice));
  return CLOT_OK;
}

extern "C" int clot_ensemble_create(const clot_mesh_desc* descs, int nchan, clot_ensemble** out) {
  if (!descs || !out || nchan < 1) return efail(CLOT_EINVAL, "need descs, out and nchan >= 1");
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return efail(CLOT_ECUDA, "no CUDA device");
  clot_ensemble* e = new clot_ensemble();
  e->nchan = nchan;
  e->dim = descs[0].dim;
  long long st = 0, cl = 0, cellmax = 0;
  for (int c = 0; c < nchan; ++c) {
    const clot_mesh_desc& d = descs[c];
    if (d.dim != 2 && d.dim != 3) { ens_free(e); return efail(CLOT_EINVAL, "channel %d: dim must be 2 or 3", c); }
    if (d.dim != e->dim) { ens_free(e); return efail(CLOT_EINVAL, "channels must share one dimension"); }
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || (d.dim == 2 && d.nz != 1) || !(d.hx > 0 && d.hy > 0 && d.hz > 0)) {
      ens_free(e);
      return efail(CLOT_EINVAL, "channel %d: bad sizes", c);
    }
    e->desc.push_back(d);
    e->geom.push_back(make_geom(d));
    if (d.nx % 2) e->vec2 = false;
    e->off_state.push_back(st);
    e->off_cell.push_back(cl);
    st += CLOT_NS * e->geom.back().pitch;
    cl += (e->geom.back().ncell + 31) / 32 * 32;
    cellmax = std::max(cellmax, e->geom.back().ncell);
  }
  if (cellmax >= (1LL << 31)) { ens_free(e); return efail(CLOT_EINVAL, "channel too large"); }
  if (cudaGetDevice(&e->device) != cudaSuccess) { ens_free(e); return efail(CLOT_ECUDA, "cudaGetDevice failed"); }
  cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, e->device);
  e->aux_blocks = std::max(1, std::min(8 * e->sms, (int)((cellmax + 255) / 256)));
  int ntile = 0;
  for (auto& g : e->geom) ntile += g.nz * ((g.ny + tile_y() - 1) / tile_y()) * ((g.nx + tile_x() - 1) / tile_x());
  const size_t nbytes_state = sizeof(float) * st, ncl = (size_t)cl;
  if (cudaMalloc(&e->scratch, nbytes_state) != cudaSuccess ||
      cudaMalloc(&e->eta_ws, sizeof(float) * 2 * ncl) != cudaSuccess ||
      cudaMalloc(&e->cg, sizeof(float) * 4 * ncl) != cudaSuccess ||
      cudaMalloc(&e->maxw, sizeof(unsigned) * 4 * nchan) != cudaSuccess ||
      cudaMalloc(&e->status, sizeof(int) * 4 * nchan) != cudaSuccess ||
      cudaMalloc(&e->partials, sizeof(double) * (8 * e->aux_blocks + 8)) != cudaSuccess ||
      cudaMalloc(&e->work, sizeof(int4) * ntile) != cudaSuccess ||
      cudaMalloc(&e->step_dev, sizeof(StepArgs) * 7 * nchan) != cudaSuccess ||
      cudaMalloc(&e->eta_dev, sizeof(EtaArgs) * 7 * nchan) != cudaSuccess) {
    ens_free(e);
    cudaGetLastError();
    return efail(CLOT_ENOMEM, "device allocation of the ensemble workspace failed");
  }
  if (cudaMemset(e->maxw, 0, sizeof(unsigned) * 4 * nchan) != cudaSuccess ||
      cudaMemset(e->status, 0, sizeof(int) * 4 * nchan) != cudaSuccess ||
      cudaMemset(e->cg, 0, sizeof(float) * 4 * ncl) != cudaSuccess ||
      cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) != cudaSuccess) {
    ens_free(e);
    return efail(CLOT_ECUDA, "ensemble workspace initialisation failed");
  }
  for (int q = 0; q < MAXCH - 1; ++q)
    if (cudaStreamCreateWithFlags(&e->cap_side[q], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_join[q], cudaEventDisableTiming) != cudaSuccess) {
      ens_free(e);
      return efail(CLOT_ECUDA, "ensemble workspace initialisation failed");
    }
  split_chains(e);
  e->order = 1;
  const int bps = std::max(1, ensemble_blocks_per_sm(e->dim, e->vec2));
  e->grid = e->sms * bps;
  int rc = upload_work(e);
  if (rc) { ens_free(e); return rc; }
  e->vfx.assign(nchan, nullptr);
  e->vfy.assign(nchan, nullptr);
  e->vfz.assign(nchan, nullptr);
  e->vdt.assign(nchan, 0.0);
  *out = e;
  return CLOT_OK;
}

extern "C" void clot_ensemble_destroy(clot_ensemble* e) { ens_free(e); }

extern "C" int clot_ensemble_info(const clot_ensemble* e, int chan, clot_mesh_info_t* o) {
  if (!e || !o || chan < 0 || chan >= e->nchan) return efail(CLOT_EINVAL, "bad ensemble, channel or output");
  const Geom& g = e->geom[chan];
  memset(o, 0, sizeof(*o));
  o->ncell = g.ncell;
  o->pitch = g.pitch;
  o->nfx = (long long)(g.nx + 1) * g.ny * g.nz;
  o->nfy = (long long)g.nx * (g.ny + 1) * g.nz;
  o->nfz = g.dim == 3 ? (long long)g.nx * g.ny * (g.nz + 1) : 0;
  o->n_inj = g.n_inj;
  o->inj_i0 = g.i0;
  o->inj_i1 = g.i1;
  o->inj_k0 = g.k0;
  o->inj_k1 = g.k1;
  o->hadh_jmax = g.hadh_jmax;
  o->n_hadh = (g.hadh_jmax >= 0 && g.n_inj > 0) ? (g.hadh_jmax + 1) * g.n_inj : 0;
  return CLOT_OK;
}

static int check_channel(const clot_ensemble* e, int c, const clot_channel* ch) {
  const clot_fields& f = ch->fields;
  if (!f.c || !f.eta || !f.sigma || !f.hist || !f.bound_acc) return efail(CLOT_EINVAL, "channel %d: null field", c);
  if (e->geom[c].n_inj > 0 && (!f.e0 || !f.c0)) return efail(CLOT_EINVAL, "channel %d: null e0/c0", c);
  if (!ch->fluxes.fx || !ch->fluxes.fy || (e->dim == 3 && !ch->fluxes.fz))
    return efail(CLOT_EINVAL, "channel %d: null flux", c);
  if (!ch->pmu_in || !ch->s1_in || !ch->s2_in) return efail(CLOT_EINVAL, "channel %d: null inlet profile", c);
  if (!(ch->dt > 0)) return efail(CLOT_EINVAL, "channel %d: dt must be > 0", c);
  if (f.ext) return efail(CLOT_EINVAL, "channel %d: the ensemble launch does not carry the inhibitor extension", c);
  return CLOT_OK;
}

static int validate_channel(clot_ensemble* e, int c, const clot_channel* ch, const clot_params* p,
                            cudaStream_t s) {
  const clot_fluxes& fl = ch->fluxes;
  if (e->vfx[c] == fl.fx && e->vfy[c] == fl.fy && e->vfz[c] == fl.fz && e->vdt[c] == ch->dt) return CLOT_OK;
  const clot_mesh_desc& d = e->desc[c];
  FluxCheckArgs a{};
  a.fx = fl.fx;
  a.fy = fl.fy;
  a.fz = fl.fz;
  a.g = e->geom[c];
  a.partials = e->partials;
  a.out = e->partials + 8 * e->aux_blocks;
  a.invV = 1.0 / (d.hx * d.hy * d.hz);
  ECUDA(launch_flux_check(a, e->aux_blocks, s));
  double o[3];
  ECUDA(cudaMemcpyAsync(o, a.out, sizeof(o), cudaMemcpyDeviceToHost, s));
  ECUDA(cudaStreamSynchronize(s));
  if (o[2] != 0.0) return efail(CLOT_EINVAL, "channel %d: wall faces carry nonzero flux", c);
  if (o[1] > 1e-5) return efail(CLOT_EINVAL, "channel %d: fluxes are not divergence-free", c);
  const double Dmax = std::max(p->D_P, std::max(p->D_adp, p->D_chem));
  double diff = 2 * Dmax * ch->dt * (1 / (d.hx * d.hx) + 1 / (d.hy * d.hy));
  if (d.dim == 3) diff += 2 * Dmax * ch->dt / (d.hz * d.hz);
  if (ch->dt * o[0] + diff > 1.0 + 1e-9) return efail(CLOT_EINVAL, "channel %d: dt above the stability bound", c);
  e->vfx[c] = fl.fx;
  e->vfy[c] = fl.fy;
  e->vfz[c] = fl.fz;
  e->vdt[c] = ch->dt;
  return CLOT_OK;
}

// Kernel arguments of version v (0: first step of a call; 1..6: steps
// n >= 1 with v = 1 + (n - 1) mod 6) for every channel.
static void fill_versions(clot_ensemble* e, const clot_channel* ch, const clot_params* p) {
  const int N = e->nchan;
  e->step_host.assign(7 * (size_t)N, StepArgs());
  e->eta_host.assign(7 * (size_t)N, EtaArgs());
  const double cl = p->L_eta * p->L_eta / 4.0;
  const bool do_eta = !(p->flags & CLOT_NO_ETA);
  for (int c = 0; c < N; ++c) {
    const Geom& g = e->geom[c];
    const clot_mesh_desc& d = e->desc[c];
    const clot_fields& f = ch[c].fields;
    float* S = e->scratch + e->off_state[c];
    float* W1 = e->eta_ws + 2 * e->off_cell[c];
    float* W2 = W1 + g.ncell;
    float* cg = e->cg + 4 * e->off_cell[c];
    unsigned* mw = e->maxw + 4 * c;
    int* st = e->status + 4 * c;
    for (int v = 0; v < 7; ++v) {
      const int n = v;  // a representative step index of this version
      StepArgs& A = e->step_host[(size_t)v * N + c];
      memset(&A, 0, sizeof(A));
      A.K = make_step_const(g, d, p, ch[c].dt);
      A.K.has_sigma = (!(p->flags & CLOT_NO_SIGMA) && f.n_samples > 0) ? 1 : 0;
      const bool even = (n % 2) == 0;
      A.cin = even ? f.c : S;
      A.cout = even ? S : f.c;
      A.fx = ch[c].fluxes.fx;
      A.fy = ch[c].fluxes.fy;
      A.fz = ch[c].fluxes.fz;
      A.sigma = f.sigma;
      A.pmu_in = ch[c].pmu_in;
      A.s1_in = ch[c].s1_in;
      A.s2_in = ch[c].s2_in;
      A.e0 = f.e0;
      A.c0 = f.c0;
      A.bound_acc = f.bound_acc;
      float *ecur, *eprev, *enext;
      if (n == 0) { ecur = f.eta; eprev = f.eta; enext = W1; }
      else {
        const int m = (n - 1) % 3;
        if (m == 0) { ecur = W1; eprev = f.eta; enext = W2; }
        else if (m == 1) { ecur = W2; eprev = W1; enext = f.eta; }
        else { ecur = f.eta; eprev = W2; enext = W1; }
      }
      A.eta = ecur;
      A.ecx = (float)(cl / (d.hx * d.hx));
      A.ecy = (float)(cl / (d.hy * d.hy));
      A.ecz = (float)(d.dim == 3 ? cl / (d.hz * d.hz) : 0.0);
      A.predict = do_eta ? 1 : 0;
      A.eta_prev = eprev;
      A.eta_next = enext;
      A.eta_res = cg;
      A.eta_max = mw + 2 * (n & 1);
      EtaArgs& E = e->eta_host[(size_t)v * N + c];
      memset(&E, 0, sizeof(E));
      E.c = A.cin;
      E.eta = ecur;
      E.r = cg;
      E.p = cg + g.ncell;
      E.q = cg + 2 * g.ncell;
      E.p2 = cg + 3 * g.ncell;
      E.status = st;
      E.g = g;
      E.cx = A.ecx;
      E.cy = A.ecy;
      E.cz = A.ecz;
      E.invPmax = (float)(1.0 / p->Pmax);
      E.tol = (float)p->eta_tol;
      E.atol = (float)p->eta_atol;
      E.inner = 1.0f;
      E.maxit = p->eta_maxit;
      E.wait_ns = eta_wait_ns(p->wait_s);
      E.predicted = n > 0 ? 1 : 0;
      E.maxw = mw + 2 * ((n - 1) & 1);
      E.maxw_clear = mw + 2 * (n & 1);
    }
  }
}

static int upload_versions(clot_ensemble* e, cudaStream_t s) {
  ECUDA(cudaMemcpyAsync(e->step_dev, e->step_host.data(), sizeof(StepArgs) * e->step_host.size(),
                        cudaMemcpyHostToDevice, s));
  ECUDA(cudaMemcpyAsync(e->eta_dev, e->eta_host.data(), sizeof(EtaArgs) * e->eta_host.size(),
                        cudaMemcpyHostToDevice, s));
  ECUDA(cudaStreamSynchronize(s));  // host staging arrays are reused
  return CLOT_OK;
}

// One step (version v) of channels [c0, c1), whose work items are
// work[w0, w1), with `grid` persistent blocks.
static cudaError_t launch_part(clot_ensemble* e, int v, bool eta, int c0, int c1, int w0, int w1, int grid,
                               cudaStream_t s) {
  if (c1 <= c0) return cudaSuccess;
  if (eta) {
    eta_block_cg_kernel<<<c1 - c0, EB, 0, s>>>(e->eta_dev + (size_t)v * e->nchan + c0);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return launch_ensemble_step(e->step_dev + (size_t)v * e->nchan, e->work + w0, w1 - w0, std::max(1, grid), e->dim,
                              e->vec2, s);
}

static cudaError_t launch_version(clot_ensemble* e, int v, bool eta, cudaStream_t s) {
  return launch_part(e, v, eta, 0, e->nchan, 0, e->nwork, e->grid, s);
}

// A 6-step graph (versions 1..6), captured on a private stream.  With two
// or more chains the channels of each chain advance through the six steps on
// a branch of their own (fork and join by events), so the eta solve of one
// chain can run beside the fused step of another; each chain's fused step
// gets the share of the persistent grid that its work items are of all items.
static int ensure_graph(clot_ensemble* e, bool eta) {
  int n = 0;
  while (n < MAXCH && e->cb[n + 1] > e->cb[n]) ++n;
  if (e->graph && e->graph_grid == e->grid && e->graph_nwork == e->nwork && e->graph_chains == n) return CLOT_OK;
  if (e->graph) {
    cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
  }
  cudaGraph_t g = nullptr;
  ECUDA(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t err = cudaSuccess;
  if (n == 1) {
    for (int v = 1; v <= 6 && err == cudaSuccess; ++v) err = launch_version(e, v, eta, e->cap_stream);
  } else {
    int gq[MAXCH], gsum = 0;
    for (int q = 0; q < n; ++q) {
      const long long items = e->wb[q + 1] - e->wb[q];
      gq[q] = q + 1 < n ? (int)((e->grid * items + e->nwork / 2) / e->nwork) : e->grid - gsum;
      gsum += gq[q];
    }
    auto st = [&](int q) { return q == 0 ? e->cap_stream : e->cap_side[q - 1]; };
    err = cudaEventRecord(e->ev_fork, e->cap_stream);
    for (int q = 1; q < n && err == cudaSuccess; ++q) err = cudaStreamWaitEvent(st(q), e->ev_fork, 0);
    for (int v = 1; v <= 6 && err == cudaSuccess; ++v)
      for (int q = 0; q < n && err == cudaSuccess; ++q)
        err = launch_part(e, v, eta, e->cb[q], e->cb[q + 1], e->wb[q], e->wb[q + 1], gq[q], st(q));
    for (int q = 1; q < n && err == cudaSuccess; ++q) {
      err = cudaEventRecord(e->ev_join[q - 1], st(q));
      if (err == cudaSuccess) err = cudaStreamWaitEvent(e->cap_stream, e->ev_join[q - 1], 0);
    }
  }
  if (err != cudaSuccess) {
    cudaStreamEndCapture(e->cap_stream, &g);
    if (g) cudaGraphDestroy(g);
    return efail(CLOT_ECUDA, "graph capture: %s", cudaGetErrorString(err));
  }
  ECUDA(cudaStreamEndCapture(e->cap_stream, &g));
  err = cudaGraphInstantiate(&e->graph, g, 0);
  cudaGraphDestroy(g);
  if (err != cudaSuccess) {
    e->graph = nullptr;
    return efail(CLOT_ECUDA, "graph instantiate: %s", cudaGetErrorString(err));
  }
  e->graph_grid = e->grid;
  e->graph_nwork = e->nwork;
  e->graph_chains = n;
  return CLOT_OK;
}

extern "C" int clot_ensemble_set_chains(clot_ensemble* e, int chains) {
  if (!e || chains < 1 || chains > MAXCH) return efail(CLOT_EINVAL, "chains must be 1 .. %d", MAXCH);
  ECUDA(cudaDeviceSynchronize());  // no launch may still read the work list
  e->chains = chains;
  split_chains(e);
  return upload_work(e);
}

extern "C" int clot_ensemble_run(clot_ensemble* e, clot_channel* ch, const clot_params* p, int nsteps,
                                 void* stream) {
  if (!e || !ch) return efail(CLOT_EINVAL, "null argument");
  int rc;
  if ((rc = check_params_common(p))) return rc;
  if (nsteps < 0) return efail(CLOT_EINVAL, "nsteps must be >= 0");
  if (p->flags & (CLOT_HEUN | CLOT_STRANG | CLOT_DEVIATION))
    return efail(CLOT_EINVAL, "the ensemble launch runs the one-stage step on the full-value state (no CLOT_HEUN / "
                              "CLOT_STRANG / CLOT_DEVIATION)");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != e->device) return efail(CLOT_EINVAL, "wrong device");
  cudaStream_t s = (cudaStream_t)stream;
  for (int c = 0; c < e->nchan; ++c)
    if ((rc = check_channel(e, c, &ch[c]))) return rc;
  if (nsteps == 0) return CLOT_OK;
  if (!(p->flags & CLOT_NO_TRANSPORT))
    for (int c = 0; c < e->nchan; ++c)
      if ((rc = validate_channel(e, c, &ch[c], p, s))) return rc;
  if ((p->flags & CLOT_NO_TRANSPORT) && (p->flags & CLOT_NO_REACTION))
    return efail(CLOT_EINVAL, "the ensemble needs transport or reaction");
  const bool eta = !(p->flags & CLOT_NO_ETA);
  const bool sig = !(p->flags & CLOT_NO_SIGMA);
  SigmaArgs sw{};
  memset(&sw, 0, sizeof(sw));
  sigma_weights(p, &sw);

  fill_versions(e, ch, p);
  if ((rc = upload_versions(e, s))) return rc;
  ECUDA(cudaMemsetAsync(e->maxw, 0, sizeof(unsigned) * 4 * e->nchan, s));
  const bool use_graph = nsteps > 7;
  if (use_graph && (rc = ensure_graph(e, eta))) return rc;

  // ADP release: per channel, the sampling steps depend on its own dt
  auto sample_due = [&](int c) {
    return sig && ch[c].fields.t + 1e-6 * ch[c].dt >= (ch[c].fields.n_samples + 1) * p->sigma_dt;
  };
  auto do_sigma = [&](int step_parity) -> int {
    bool changed = false;
    for (int c = 0; c < e->nchan; ++c) {
      clot_fields& f = ch[c].fields;
      SigmaArgs a = sw;
      a.sigma = f.sigma;
      a.hist = f.hist;
      a.bound_acc = f.bound_acc;
      a.ncell = e->geom[c].ncell;
      if (sig && f.t_last < 0) {
        ECUDA(launch_sigma_init(a, s));
        f.t_last = f.t;
      }
      if (sample_due(c)) {
        a.head = f.n_samples == 0 ? 0 : (f.head + 1) % a.nslot;
        a.nvalid = std::min(f.n_samples + 1, a.nslot);
        a.inv_dt_sample = (float)(1.0 / (f.t - f.t_last));
        ECUDA(launch_sigma_sample(a, s));
        if (f.n_samples == 0) changed = true;
        f.head = a.head;
        f.n_samples += 1;
        f.t_last = f.t;
      }
    }
    (void)step_parity;
    if (changed) {
      fill_versions(e, ch, p);
      return upload_versions(e, s);
    }
    return CLOT_OK;
  };
  // steps until some channel samples (the graph is replayed only in between)
  auto steps_to_sample = [&]() {
    long long best = 1LL << 40;
    if (!sig) return best;
    for (int c = 0; c < e->nchan; ++c) {
      const clot_fields& f = ch[c].fields;
      const double tn = (f.n_samples + 1) * p->sigma_dt;
      const long long k = (long long)ceil((tn - f.t - 1e-6 * ch[c].dt) / ch[c].dt);
      best = std::min(best, std::max(0LL, k));
    }
    return best;
  };

  int n = 0;
  while (n < nsteps) {
    const long long due = steps_to_sample();
    if (n >= 1 && use_graph && (n - 1) % 6 == 0 && n + 6 <= nsteps && due >= 6) {
      ECUDA(cudaGraphLaunch(e->graph, s));
      for (int c = 0; c < e->nchan; ++c)
        for (int j = 0; j < 6; ++j) ch[c].fields.t += ch[c].dt;
      n += 6;
      continue;
    }
    if ((rc = do_sigma(n))) return rc;
    const int v = n == 0 ? 0 : 1 + (n - 1) % 6;
    ECUDA(launch_version(e, v, eta, s));
    for (int c = 0; c < e->nchan; ++c) ch[c].fields.t += ch[c].dt;
    ++n;
  }
  // results back into the caller's buffers
  for (int c = 0; c < e->nchan; ++c) {
    const Geom& g = e->geom[c];
    clot_fields& f = ch[c].fields;
    if (nsteps % 2)
      ECUDA(cudaMemcpyAsync(f.c, e->scratch + e->off_state[c], sizeof(float) * CLOT_NS * g.pitch,
                            cudaMemcpyDeviceToDevice, s));
    if (eta && nsteps >= 2) {
      const int m = (nsteps - 2) % 3;  // eta used by the last step
      const float* W1 = e->eta_ws + 2 * e->off_cell[c];
      const float* used = m == 0 ? W1 : m == 1 ? W1 + g.ncell : f.eta;
      if (used != f.eta)
        ECUDA(cudaMemcpyAsync(f.eta, used, sizeof(float) * g.ncell, cudaMemcpyDeviceToDevice, s));
    }
  }
  return CLOT_OK;
}

extern "C" int clot_ensemble_diagnostics(clot_ensemble* e, int chan, const clot_fields* f, const clot_params* p,
                                         double out[8], void* stream) {
  if (!e || !f || !out || !p || chan < 0 || chan >= e->nchan) return efail(CLOT_EINVAL, "bad argument");
  const clot_mesh_desc& d = e->desc[chan];
  DiagArgs a{};
  a.c = f->c;
  a.e0 = f->e0;
  a.c0 = f->c0;
  a.ncell = e->geom[chan].ncell;
  a.pitch = e->geom[chan].pitch;
  a.n_inj = e->geom[chan].n_inj;
  a.V = d.hx * d.hy * d.hz;
  a.A = d.hx * d.hz;
  a.invPmax = 1.0 / p->Pmax;
  a.partials = e->partials;
  a.out = e->partials + 8 * e->aux_blocks;
  cudaStream_t s = (cudaStream_t)stream;
  ECUDA(launch_diagnostics(a, e->aux_blocks, s));
  ECUDA(cudaMemcpyAsync(out, a.out, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ECUDA(cudaStreamSynchronize(s));
  return CLOT_OK;
}

// Autotuner: for each candidate (persistent grid of 1, 2 or 3 x the resident
// blocks, work-list order 0 or 1) time `trials` fused-step launches on the
// current state (the kernel writes the ensemble's scratch; the state it
// updates in place -- E0, C0, the bound-platelet accumulator -- is saved and
// restored), keep the fastest.
extern "C" int clot_ensemble_tune(clot_ensemble* e, clot_channel* ch, const clot_params* p, int trials,
                                  clot_tune_t* out, void* stream) {
  if (!e || !ch || !out || trials < 1) return efail(CLOT_EINVAL, "bad argument");
  int rc;
  if ((rc = check_params_common(p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  for (int c = 0; c < e->nchan; ++c)
    if ((rc = check_channel(e, c, &ch[c]))) return rc;
  for (int c = 0; c < e->nchan; ++c)
    if ((rc = validate_channel(e, c, &ch[c], p, s))) return rc;
  // save in-place state into the CG workspace (4 ncell per channel: e0, c0 need n_inj <= ncell)
  for (int c = 0; c < e->nchan; ++c) {
    const Geom& g = e->geom[c];
    float* tmp = e->cg + 4 * e->off_cell[c];
    ECUDA(cudaMemcpyAsync(tmp, ch[c].fields.bound_acc, sizeof(float) * g.ncell, cudaMemcpyDeviceToDevice, s));
    if (g.n_inj) {
      ECUDA(cudaMemcpyAsync(tmp + g.ncell, ch[c].fields.e0, sizeof(float) * g.n_inj, cudaMemcpyDeviceToDevice, s));
      ECUDA(cudaMemcpyAsync(tmp + 2 * g.ncell, ch[c].fields.c0, sizeof(float) * g.n_inj, cudaMemcpyDeviceToDevice, s));
    }
  }
  clot_params q = *p;
  q.flags |= CLOT_NO_ETA;  // time the fused step alone
  fill_versions(e, ch, &q);
  // version 0 reads the caller's state and writes the scratch
  if ((rc = upload_versions(e, s))) return rc;
  const int bps = std::max(1, ensemble_blocks_per_sm(e->dim, e->vec2));
  const int grids[3] = {e->sms * bps, 2 * e->sms * bps, 3 * e->sms * bps};
  cudaEvent_t a, b;
  ECUDA(cudaEventCreate(&a));
  ECUDA(cudaEventCreate(&b));
  float best = 1e30f;
  int bg = e->grid, bo = e->order, ncand = 0;
  for (int order = 0; order < 2; ++order) {
    e->order = order;
    if ((rc = upload_work(e))) return rc;
    for (int gi = 0; gi < 3; ++gi) {
      e->grid = grids[gi];
      ECUDA(launch_ensemble_step(e->step_dev, e->work, e->nwork, e->grid, e->dim, e->vec2, s));  // warm-up
      ECUDA(cudaEventRecord(a, s));
      for (int t = 0; t < trials; ++t)
        ECUDA(launch_ensemble_step(e->step_dev, e->work, e->nwork, e->grid, e->dim, e->vec2, s));
      ECUDA(cudaEventRecord(b, s));
      ECUDA(cudaEventSynchronize(b));
      float ms = 0.0f;
      ECUDA(cudaEventElapsedTime(&ms, a, b));
      ms /= trials;
      if (ncand < 6) {
        out->cand_grid[ncand] = e->grid;
        out->cand_order[ncand] = order;
        out->cand_ms[ncand] = ms;
        ++ncand;
      }
      if (ms < best) {
        best = ms;
        bg = e->grid;
        bo = order;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  e->grid = bg;
  e->order = bo;
  if ((rc = upload_work(e))) return rc;
  // restore the in-place state
  for (int c = 0; c < e->nchan; ++c) {
    const Geom& g = e->geom[c];
    const float* tmp = e->cg + 4 * e->off_cell[c];
    ECUDA(cudaMemcpyAsync(ch[c].fields.bound_acc, tmp, sizeof(float) * g.ncell, cudaMemcpyDeviceToDevice, s));
    if (g.n_inj) {
      ECUDA(cudaMemcpyAsync(ch[c].fields.e0, tmp + g.ncell, sizeof(float) * g.n_inj, cudaMemcpyDeviceToDevice, s));
      ECUDA(cudaMemcpyAsync(ch[c].fields.c0, tmp + 2 * g.ncell, sizeof(float) * g.n_inj, cudaMemcpyDeviceToDevice, s));
    }
  }
  ECUDA(cudaStreamSynchronize(s));
  out->grid = bg;
  out->order = bo;
  out->ms = best;
  out->ncand = ncand;
  return CLOT_OK;
}

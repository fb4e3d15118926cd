// clot_noalloc.cu -- clot_eta_solve_noalloc: the eta solve for callers that
// cannot allocate device memory.
//
// Some callers must not call cudaMalloc: code that runs inside another
// framework whose allocator owns the device memory (a process with a hard
// memory cap, where a stray cudaMalloc could fail or evict), real-time or
// monitoring loops where cudaMalloc's implicit device synchronisation would
// stall unrelated streams, and small tools that hold a state they did not
// create and so have no clot_mesh (whose workspace comes from cudaMalloc in
// clot_mesh_create).  This entry point runs the same conjugate-gradient
// kernel as clot_eta_solve but takes its scratch -- the CG vectors r, p, q,
// the FP64 reduction partials, the grid-barrier counters and the status words
// -- from one file-scope static __device__ array.  Every GPU that loads the
// library holds that array (about 16.1 MiB) until the process exits.
//
// Host code must not use the array's name as a device address (in host code
// it names a host-side shadow); the device address comes from
// cudaGetSymbolAddress, taken once per device with that device current, on the
// first call made on that device.
#include <stdio.h>

#include <mutex>

#include "clot_internal.cuh"

namespace clot {

constexpr long long NOALLOC_MAX_CELLS = 1ll << 20;  // 1,048,576 cells
constexpr int NOALLOC_MAX_GRID = 4096;              // blocks of the cooperative launch
constexpr int NOALLOC_MAX_DEVICES = 64;

// Layout (bytes): [r | p | q | p2] floats, then partials and reduced scalars
// (doubles), then the word block: 8 barrier words at +0 (arrival counter,
// generation, box bounds of the predicted-eta correction; cleared by
// launch_eta_solve before every launch) and 8 status words at +64 (flags,
// iterations, summed iterations, accepted predictions, box corrections and
// their fallbacks).
constexpr size_t NA_VEC_BYTES = 4 * NOALLOC_MAX_CELLS * sizeof(float);
constexpr size_t NA_PART_BYTES = (3 * NOALLOC_MAX_GRID + 8) * sizeof(double);
constexpr size_t NA_WORD_BYTES = 256;
constexpr size_t NA_STATUS_OFF = 64;
constexpr size_t NA_TOTAL_BYTES = NA_VEC_BYTES + NA_PART_BYTES + NA_WORD_BYTES;
// The eta kernel uses bar[0..7], status[0..5] and partials[0 .. 3 grid + 5].
static_assert(8 * sizeof(unsigned) <= NA_STATUS_OFF, "barrier words overlap the status words");
static_assert(NA_STATUS_OFF + 8 * sizeof(int) <= NA_WORD_BYTES, "status words overflow the word block");
static_assert((3 * NOALLOC_MAX_GRID + 6) * sizeof(double) <= NA_PART_BYTES, "partials overflow their block");
static_assert(NA_VEC_BYTES % 256 == 0 && NA_PART_BYTES % 8 == 0, "misaligned scratch blocks");

static __device__ __align__(256) unsigned char g_eta_scratch[NA_TOTAL_BYTES];

namespace {
std::mutex g_mu;
void* g_addr[NOALLOC_MAX_DEVICES] = {};
}  // namespace

}  // namespace clot

using namespace clot;

// Errors are reported through clot_last_error(), like every other entry point.
static int na_fail(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

extern "C" int clot_eta_solve_noalloc(const clot_mesh_desc* d, const float* c, int64_t pitch, float* eta,
                                      const clot_params* p, int* iters, void* stream) {
  if (!d || !c || !eta || !p) return na_fail(CLOT_EINVAL, "null argument");
  if (d->dim != 2 && d->dim != 3) return na_fail(CLOT_EINVAL, "dim must be 2 or 3");
  if (d->nx < 1 || d->ny < 1 || d->nz < 1 || (d->dim == 2 && d->nz != 1))
    return na_fail(CLOT_EINVAL, "bad cell counts");
  if (!(d->hx > 0 && d->hy > 0 && d->hz > 0)) return na_fail(CLOT_EINVAL, "cell sizes must be > 0");
  const long long ncell = (long long)d->nx * d->ny * d->nz;
  if (ncell > NOALLOC_MAX_CELLS) {
    char msg[160];
    snprintf(msg, sizeof(msg), "mesh has %lld cells; the no-allocation eta solve holds scratch for at most %lld",
             ncell, NOALLOC_MAX_CELLS);
    return na_fail(CLOT_EINVAL, msg);
  }
  if (pitch < ncell) return na_fail(CLOT_EINVAL, "pitch smaller than the cell count");
  if (!(p->Pmax > 0) || p->eta_maxit < 0) return na_fail(CLOT_EINVAL, "bad params");

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return na_fail(CLOT_ECUDA, "no usable current CUDA device");
  void* base = nullptr;
  {
    // One-time set-up per device, with that device current: the device
    // address of the static scratch array.
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* a = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&a, g_eta_scratch);
      if (e != cudaSuccess || !a) {
        char msg[160];
        snprintf(msg, sizeof(msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return na_fail(CLOT_ECUDA, msg);
      }
      g_addr[dev] = a;
    }
    base = g_addr[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  EtaArgs a{};
  a.c = c;
  a.eta = eta;
  a.r = reinterpret_cast<float*>(b);
  a.p = a.r + NOALLOC_MAX_CELLS;
  a.q = a.p + NOALLOC_MAX_CELLS;
  a.p2 = a.q + NOALLOC_MAX_CELLS;
  a.partials = reinterpret_cast<double*>(b + NA_VEC_BYTES);
  a.bar = reinterpret_cast<unsigned*>(b + NA_VEC_BYTES + NA_PART_BYTES);
  a.status = reinterpret_cast<int*>(b + NA_VEC_BYTES + NA_PART_BYTES + NA_STATUS_OFF);
  a.g.dim = d->dim;
  a.g.nx = d->nx;
  a.g.ny = d->ny;
  a.g.nz = d->nz;
  a.g.ncell = ncell;
  a.g.pitch = pitch;
  a.g.i0 = 0; a.g.i1 = -1; a.g.k0 = 0; a.g.k1 = -1; a.g.n_inj = 0; a.g.hadh_jmax = -1;
  const double cl = p->L_eta * p->L_eta / 4.0;
  a.cx = (float)(cl / (d->hx * d->hx));
  a.cy = (float)(cl / (d->hy * d->hy));
  a.cz = (float)(d->dim == 3 ? cl / (d->hz * d->hz) : 0.0);
  a.invPmax = (float)(1.0 / p->Pmax);
  a.tol = (float)p->eta_tol;
  a.atol = (float)p->eta_atol;
  a.inner = 1.0f;
  a.maxit = p->eta_maxit;
  a.wait_ns = eta_wait_ns(p->wait_s);
  a.predicted = 0;
  a.maxw = nullptr;
  a.maxw_clear = nullptr;

  int grid = 0;
  if (eta_max_grid(&grid) != 0) return na_fail(CLOT_ECUDA, "occupancy query failed");
  const long long need = (ncell + ETA_BLOCK - 1) / ETA_BLOCK;
  if (grid > NOALLOC_MAX_GRID) grid = NOALLOC_MAX_GRID;
  if (grid > need) grid = (int)need;
  if (grid < 1) grid = 1;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents.  The counters (status words
  // 1..5) must start at zero; the flags word 0 is left as it is, so that a
  // timeout of an earlier call made without iters (which cannot synchronise to
  // report it) is still reported by the next call given iters.  The barrier
  // words are cleared by launch_eta_solve; r, p, q and the partials are written
  // before they are read.
  if (cudaMemsetAsync(a.status + 1, 0, 5 * sizeof(int), s) != cudaSuccess)
    return na_fail(CLOT_ECUDA, "memset failed");
  const cudaError_t e = launch_eta_solve(a, grid, s);
  if (e != cudaSuccess) {
    char msg[160];
    snprintf(msg, sizeof(msg), "eta launch: %s", cudaGetErrorString(e));
    return na_fail(CLOT_ECUDA, msg);
  }
  if (iters) {
    int st[2] = {0, 0};
    if (cudaMemcpyAsync(st, a.status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return na_fail(CLOT_ECUDA, "status read failed");
    *iters = st[1];
    if (st[0] & ST_TIMEOUT) {
      // reported once: clear the flag for the calls that follow
      if (cudaMemsetAsync(a.status, 0, sizeof(int), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return na_fail(CLOT_ECUDA, "status clear failed");
      return na_fail(CLOT_ETIMEOUT, "eta solver grid barrier timed out (this call or an earlier one without iters)");
    }
  }
  return CLOT_OK;
}

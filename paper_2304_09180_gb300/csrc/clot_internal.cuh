// clot_internal.cuh -- structures shared by the library's translation units
// (host orchestration in clot_capi.cu, kernels in clot_step.cu, clot_eta.cu,
// clot_aux.cu).  Nothing here is visible through the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "clot.h"

namespace clot {

// Transported species (Sec. 3.2 step 1): the two mobile platelet species
// (hindered), ADP and the four fluid-phase coagulation species.
constexpr int NT = 7;
__host__ __device__ constexpr int trow(int t) {
  return t == 0 ? CLOT_PMU : t == 1 ? CLOT_PMA : t == 2 ? CLOT_ADP : t == 3 ? CLOT_S1
       : t == 4 ? CLOT_S2 : t == 5 ? CLOT_E1 : CLOT_E2;
}

struct Geom {
  int dim, nx, ny, nz;
  long long ncell, pitch;
  int i0, i1, k0, k1;  // injury face rectangle (i1 < i0: no patch)
  int n_inj;
  int hadh_jmax;       // H_adh = 1 over the patch for j <= hadh_jmax
};

// Reaction constants in FP32 (App. A, App. B, App. E), converted once per call.
struct RxnConst {
  float kadh, Pmax, kcohPmax, k_adp, adp_star, k_e2, e2_star, n1, n2;
  float kS1p, kS1m, kE1p, kE1m, kS2p, kS2m, kE2p, kE2m;
  float kC1p, kC1m, kC1cat, kC2p, kC2m, kC2cat;
  float kC0p, kC0m, kC0cat;
  float aV;   // injury face area / cell volume = 1 / hy
  float Dd;   // D_chem / (hy / 2), the Robin closure conductance
  float eta_t, eta_star3, g0;
  float kI;   // inhibitor extension: I + E2 -> E2,inh rate (used with CLOT_NX states only)
  // Deviation form (CLOT_DEVIATION): the state's S1, S2 rows hold S1 - s1_ref,
  // S2 - s2_ref; the rates are evaluated at the full values (zero otherwise).
  float s1_ref, s2_ref;
};

struct StepConst {
  Geom g;
  float dt, dtV, invPmax;
  float dcoef[NT][3];  // D_s A_a / h_a
  int limiter, closed_ends, do_transport, do_reaction, has_sigma;
  int wall_lagged;     // injury-wall exchange as a lagged transport condition (the paper's placement)
  int M;               // reaction substeps
  float h;             // reaction substep (dt / M; dt / (2 M) for each half of a Strang-split step)
  RxnConst r;
};

struct StepArgs {
  const float* __restrict__ cin;
  float* __restrict__ cout;
  // Second stage of the two-stage (Heun) transport: the state the transport
  // started from; the mobile species of the result are averaged with it
  // (null: the plain one-stage step).
  const float* __restrict__ cavg;
  // Inhibitor extension (null: the paper's model): its rows I, E2,inh after
  // their transport (read at the own cell) and where the step's result goes
  // (may equal xin: each cell reads its own value before writing it).
  const float* xin;
  float* xout;
  const float* __restrict__ fx;
  const float* __restrict__ fy;
  const float* __restrict__ fz;
  const float* __restrict__ eta;
  const float* __restrict__ sigma;
  const float* __restrict__ pmu_in;
  const float* __restrict__ s1_in;
  const float* __restrict__ s2_in;
  float* e0;
  float* c0;
  // Low words of E0, C0 (CLOT_DEVIATION; null otherwise): each step's
  // increment is added in FP64 to the pair (e0 + e0lo) and the pair rounded
  // back to two floats.
  float* e0lo;
  float* c0lo;
  float* bound_acc;            // += newly bound platelets (RK4 increments of Pba + Pbse)
  // eta prediction for the next step (predict != 0): guess = 2 eta - eta_prev,
  // residual of the guess against the new theta_B, block maxima of |r| and theta_B.
  const float* __restrict__ eta_prev;
  float* eta_next;
  float* eta_res;
  unsigned* eta_max;           // [2]: max |r|, max theta_B (float bit patterns, atomicMax)
  float ecx, ecy, ecz;         // (L_eta^2 / 4) / h_a^2
  int predict;
  int* status;                 // device status word: ST_TIMEOUT when a bounded wait gives up (may be null)
  StepConst K;
};

// Device status word bits (mesh workspace, read by clot_device_status).
constexpr int ST_TIMEOUT = 1;

// Grid-barrier wait bound of the eta solver from clot_params.wait_s: <= 0 (or
// not a number) selects 2 s, anything above 10 s is cut to 10 s.
inline unsigned long long eta_wait_ns(double wait_s) {
  if (!(wait_s > 0.0)) return 2000000000ull;
  if (wait_s > 10.0) return 10000000000ull;
  const double ns = wait_s * 1e9;
  return ns < 1.0 ? 1ull : (unsigned long long)ns;
}

// Kernel launchers (defined in the .cu files; all stream-ordered).
cudaError_t launch_species_step(const StepArgs& a, cudaStream_t s);
// Tiled fused step (clot_step_tiled.cu): one z plane per block, the plane
// tile with its halo in shared memory, z neighbours from L2.
cudaError_t launch_species_step_plane(const StepArgs& a, cudaStream_t s);
// 3D fused step marching in z with TMA-staged planes (clot_step_zmarch.cu);
// *used = false (nothing launched) when the mesh or pointers miss its
// alignment rules (nx % 4, 16-byte bases) or the driver lacks tensor maps.
cudaError_t launch_zmarch_tma(const StepArgs& a, cudaStream_t s, bool* used);
// Persistent fused step over a work list of (channel, tile column, tile row,
// plane) items of several meshes (clot_step_tiled.cu).
cudaError_t launch_ensemble_step(const StepArgs* chans, const int4* work, int nwork, int grid, int dim, bool vec2,
                                 cudaStream_t s);
int ensemble_blocks_per_sm(int dim, bool vec2);
int tile_x();
int tile_y();
cudaError_t launch_reaction_only(const StepArgs& a, cudaStream_t s);

// Transport of the inhibitor extension's two rows (clot_step.cu).
struct ExtArgs {
  const float* xin;   // [2][pitch] I, E2,inh at the start of the pass
  float* xout;        // [2][pitch] after it
  const float* xavg;  // second stage of the two-stage transport: average with this (else null)
  const float* fx;
  const float* fy;
  const float* fz;
  Geom g;
  long long pitch;
  float dtV, I_in;
  float dcoef[3];     // D_chem A_a / h_a
  int limiter, closed_ends;
};
cudaError_t launch_ext_transport(const ExtArgs& a, cudaStream_t s);

struct EtaArgs {
  const float* __restrict__ c;  // state (reads Pba, Pbse)
  float* eta;
  float* r;
  float* p;
  float* q;
  float* p2;                    // second search-direction buffer (p_old / p_new alternate)
  float* cg5;                   // [5][ncell] second r, two s, two w buffers of the single-reduction CG
                                // (null: the two-reduction CG)
  double* partials;             // [3][gridDim] + 6 reduced scalars
  unsigned* bar;                // [8] arrive counter, generation, box bounds of the predicted-eta fix
  int* status;                  // [0] flags, [1] iterations, [2] summed iterations, [3] accepted predictions,
                                // [4] predictions corrected on a box, [5] box corrections that fell back
  Geom g;
  float cx, cy, cz;             // (L_eta^2 / 4) / h_a^2
  float invPmax;
  float tol;                    // acceptance: max|r| <= max(tol max theta_B, atol)
  float atol;
  float inner;                  // CG iterates down to inner * that threshold
  int maxit;
  int predicted;                // r and eta hold a predicted guess and its residual
  unsigned long long wait_ns;   // bound of each grid-barrier wait (globaltimer ns)
  const unsigned* maxw;         // [2] max |r|, max theta_B of the prediction
  unsigned* maxw_clear;         // [2] the other maxima set, zeroed for the next step
};
// The box correction of a predicted eta (App. A Eq. eta; used by the
// single-mesh solver and the ensemble's block-per-channel solver): an
// axis-aligned box of cells, bounds inclusive.
struct Box {
  int i0, i1, j0, j1, k0, k1;
  __device__ bool in(int i, int j, int k) const {
    return i >= i0 && i <= i1 && j >= j0 && j <= j1 && k >= k0 && k <= k1;
  }
  __device__ long long cells() const { return (long long)(i1 - i0 + 1) * (j1 - j0 + 1) * (k1 - k0 + 1); }
};

// Cells a correction confined to [lo, hi] must extend over along an axis with
// coupling c so that c |d| at the box edge stays below stop / 2: the decay rate
// mu per cell of the 1D Green's function, cosh(mu) = 1 + 1 / (2c), and
// |d| <= max|r| (the operator is an M-matrix with unit row sums).
__device__ __forceinline__ int box_margin(float c, float rmax, float stop) {
  if (!(c > 0.0f)) return 0;
  const float mu = acoshf(1.0f + 0.5f / c);
  const float n = logf(fmaxf(2.0f * c * rmax / stop, 1.0f)) / mu;
  return (int)fminf(ceilf(n) + 1.0f, 1.0e6f);
}

// Threads per block of the eta CG kernel (its block reductions assume it):
// two 512-thread blocks per SM cost fewer grid-barrier arrivals than five of
// 256 at the same per-pass bandwidth.
constexpr int ETA_BLOCK = 512;
cudaError_t launch_eta_solve(const EtaArgs& a, int grid, cudaStream_t s);
int eta_max_grid(int* grid_out);

struct SigmaArgs {
  float* sigma;
  float* hist;
  float* bound_acc;
  long long ncell;
  float inv_dt_sample;
  int head, nslot, nvalid;      // ring slot of the new sample; slots; samples to sum
  float w[CLOT_NTAU_MAX + 1];   // w[lag] = A_hat * trapezoid weight * R(lag dtau)
};
cudaError_t launch_sigma_init(const SigmaArgs& a, cudaStream_t s);
cudaError_t launch_sigma_sample(const SigmaArgs& a, cudaStream_t s);

struct DiagArgs {
  const float* __restrict__ c;
  const float* __restrict__ e0;
  const float* __restrict__ c0;
  const float* __restrict__ ext;  // [2][pitch] inhibitor extension rows (I, E2,inh) or null
  long long ncell, pitch;
  int n_inj;
  double V, A, invPmax;
  double* partials;             // [8][nblocks]
  double* out;                  // [8]
};
cudaError_t launch_diagnostics(const DiagArgs& a, int nblocks, cudaStream_t s);
// dst[i] = src[i] + r, i < n (the shifts of the deviation form)
cudaError_t launch_shift(float* dst, const float* src, long long n, float r, cudaStream_t s);

struct FluxCheckArgs {
  const float* fx;
  const float* fy;
  const float* fz;
  Geom g;
  double* partials;             // [3][nblocks]: max |F|/V, max |div|, max |F| on walls
  double* out;                  // [4]
  double invV;
};
cudaError_t launch_flux_check(const FluxCheckArgs& a, int nblocks, cudaStream_t s);

// Reaction surrogate (clot_surrogate.cu): one reaction solve over dt with the
// MLP increment where it applies (first launch) and RK4 on the compacted list
// of the other cells (second launch), in place on c.
struct SurrArgs {
  float* c;                    // [CLOT_NS][pitch], updated in place (pointwise)
  const float* __restrict__ eta;
  float* e0;
  float* c0;
  float* bound_acc;
  uint8_t* flag;               // [ncell] or null
  unsigned long long* counts;  // [3] indicator fallbacks, region fallbacks, fallback-list length
  int* list;                   // [ncell] cells for the RK4 fallback (compacted)
  const float* w;              // CLOT_MLP_NPARAM parameters
  int* status;                 // device status word (ST_TIMEOUT), may be null
  int engine;                  // CLOT_MLP_ENGINE_*
  Geom g;
  RxnConst r;
  float h;                     // RK4 step of the fallback
  int M;                       // RK4 steps of the fallback
  float dt, xdt, tol;          // dt = h M, xdt = log(dt / 1e-5)
  float inv_scale[CLOT_NS], floor_s[CLOT_NS];  // 1 / scale_s, 1e-6 scale_s
};
cudaError_t launch_surrogate_react(const SurrArgs& a, cudaStream_t s);
cudaError_t launch_surrogate_fallback(const SurrArgs& a, cudaStream_t s);
void surrogate_fill_consts(const clot_mlp* mlp, double dt, float* inv_scale, float* floor_s, float* xdt);

// Sets the message returned by clot_last_error() on this thread.
void set_last_error(const char* msg);

// Host-side builders shared by the single-mesh and ensemble entry points
// (clot_capi.cu): injury rectangle and adhesion region of a mesh, FP32
// step / reaction constants, parameter checks, ADP-release weights.
Geom make_geom(const clot_mesh_desc& d);
RxnConst make_rxn_const(const clot_mesh_desc& d, const clot_params* p);
StepConst make_step_const(const Geom& g, const clot_mesh_desc& d, const clot_params* p, double dt);
int check_params_common(const clot_params* p);
void sigma_weights(const clot_params* p, SigmaArgs* a);

}  // namespace clot

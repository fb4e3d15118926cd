// clot_capi.cu -- host side of the C ABI declared in include/clot.h: argument
// validation, mesh geometry (injury rectangle, adhesion region), workspace,
// FP64 -> FP32 parameter conversion and the per-step launch sequence
// (eta solve -> sigma sample when due -> fused species step).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>

#include "clot_internal.cuh"

using namespace clot;

static thread_local char g_err[512] = "";

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CUDA_OK(expr)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) return fail(CLOT_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

struct clot_mesh {
  clot_mesh_desc desc;
  Geom g;
  int device;
  float* scratch;      // [CLOT_NS][pitch] ping-pong partner of fields.c
  float* stage;        // [CLOT_NS][pitch] first-stage result of the two-stage (Heun) transport
  float* xws;          // [2][2][pitch] inhibitor extension rows after transport, and their first Heun stage
  float* dev_in;       // [2][ny nz] inlet S1, S2 minus their references (CLOT_DEVIATION)
  float* wall_lo;      // [2][max(n_inj, 1)] low words of E0, C0 (CLOT_DEVIATION)
  float* cg;           // [9][ncell] eta solver r, p, q, p2 and the single-reduction CG's five more
  float* eta_ws;       // [2][ncell] eta buffers of the step-to-step prediction
  unsigned* maxw;      // [4] two sets of (max |r|, max theta_B) of the prediction
  double* partials;
  double* dout;        // [8]
  unsigned* bar;       // [8] grid barrier words, box bounds of the eta correction
  int* status;         // [8] flags, last eta iterations, summed iterations, accepted predictions, box fixes, box fallbacks
  unsigned long long* scount;  // [4] surrogate fallback counters and list length
  // eta prediction carried from one clot_species_step call to the next
  int pred_valid;
  const float* pred_c;     // the fields' state and eta buffers it belongs to
  const float* pred_eta;
  double pred_t, pred_dt;  // time of the next step, its dt
  float* pred_guess;       // workspace buffer holding the predicted eta of that step
  int pred_sel;            // maxima set the last fused step wrote
  int eta_grid;
  int aux_blocks;
  const float* vfx[2];  // the last two validated (fluxes, dt) sets (double-buffered uploads)
  const float* vfy[2];
  const float* vfz[2];
  double vdt[2];
  int validated[2];
  int vnext;
  int ntau;
  // tracing (clot_profile_begin / _end)
  int prof_on, prof_cap, prof_n;
  cudaEvent_t* prof_ev;  // [2 * prof_cap]
  int* prof_kind;        // [prof_cap]
  int prof_count[4];
};

enum { K_STEP = 0, K_ETA = 1, K_SIGMA = 2, K_OTHER = 3 };

// Launch `fn` bracketed by timing events when profiling is on.
template <class F>
static cudaError_t traced(clot_mesh* m, int kind, cudaStream_t s, F fn) {
  if (!m->prof_on) return fn();
  m->prof_count[kind] += 1;
  if (m->prof_n >= m->prof_cap) return fn();
  cudaError_t e = cudaEventRecord(m->prof_ev[2 * m->prof_n], s);
  if (e != cudaSuccess) return e;
  e = fn();
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(m->prof_ev[2 * m->prof_n + 1], s);
  m->prof_kind[m->prof_n] = kind;
  m->prof_n += 1;
  return e;
}

static void prof_free(clot_mesh* m) {
  if (m->prof_ev) {
    for (int q = 0; q < 2 * m->prof_cap; ++q) cudaEventDestroy(m->prof_ev[q]);
    delete[] m->prof_ev;
    delete[] m->prof_kind;
  }
  m->prof_ev = nullptr;
  m->prof_kind = nullptr;
  m->prof_cap = 0;
  m->prof_on = 0;
}

extern "C" const char* clot_last_error(void) { return g_err; }

void clot::set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

static void free_mesh(clot_mesh* m) {
  if (!m) return;
  prof_free(m);
  cudaFree(m->scratch);
  cudaFree(m->stage);
  cudaFree(m->xws);
  cudaFree(m->dev_in);
  cudaFree(m->wall_lo);
  cudaFree(m->cg);
  cudaFree(m->eta_ws);
  cudaFree(m->maxw);
  cudaFree(m->partials);
  cudaFree(m->dout);
  cudaFree(m->bar);
  cudaFree(m->status);
  cudaFree(m->scount);
  delete m;
}

Geom clot::make_geom(const clot_mesh_desc& dd) {
  const clot_mesh_desc* d = &dd;
  Geom g;
  memset(&g, 0, sizeof(g));
  g.dim = d->dim;
  g.nx = d->nx;
  g.ny = d->ny;
  g.nz = d->nz;
  g.ncell = (long long)d->nx * d->ny * d->nz;
  g.pitch = (g.ncell + 31) / 32 * 32;
  // Injury faces: floor faces whose centre x (and z in 3D) lies in the patch
  // intervals -- a contiguous rectangle of (i, k).
  g.i0 = 0; g.i1 = -1;
  for (int i = 0; i < d->nx; ++i) {
    const double xc = (i + 0.5) * d->hx;
    if (xc >= d->inj_x0 && xc <= d->inj_x1) {
      if (g.i1 < g.i0) g.i0 = i;
      g.i1 = i;
    }
  }
  g.k0 = 0; g.k1 = d->nz - 1;
  if (d->dim == 3) {
    g.k1 = -1;
    for (int k = 0; k < d->nz; ++k) {
      const double zc = (k + 0.5) * d->hz;
      if (zc >= d->inj_z0 && zc <= d->inj_z1) {
        if (g.k1 < g.k0) g.k0 = k;
        g.k1 = k;
      }
    }
  }
  if (g.i1 < g.i0 || g.k1 < g.k0) { g.i0 = 0; g.i1 = -1; g.k0 = 0; g.k1 = -1; }
  g.n_inj = (g.i1 >= g.i0 && g.k1 >= g.k0) ? (g.i1 - g.i0 + 1) * (g.k1 - g.k0 + 1) : 0;
  // Adhesion region (App. A, Sec. 3.1): over the patch, cell centre within p_diam of the wall.
  g.hadh_jmax = -1;
  for (int j = 0; j < d->ny; ++j)
    if ((j + 0.5) * d->hy <= d->p_diam) g.hadh_jmax = j;

  return g;
}

extern "C" int clot_mesh_create(const clot_mesh_desc* d, clot_mesh** out) {
  if (!d || !out) return fail(CLOT_EINVAL, "null argument");
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return fail(CLOT_EINVAL, "dim must be 2 or 3 (got %d)", d->dim);
  if (d->nx < 1 || d->ny < 1 || d->nz < 1) return fail(CLOT_EINVAL, "cell counts must be >= 1");
  if (d->dim == 2 && d->nz != 1) return fail(CLOT_EINVAL, "2D meshes need nz = 1");
  if (!(d->hx > 0 && d->hy > 0 && d->hz > 0)) return fail(CLOT_EINVAL, "cell sizes must be > 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) return fail(CLOT_ECUDA, "no CUDA device");

  clot_mesh* m = new clot_mesh();
  memset(m, 0, sizeof(*m));
  m->desc = *d;
  m->g = clot::make_geom(*d);
  const Geom& g = m->g;
  CUDA_OK(cudaGetDevice(&m->device));
  int grid = 0;
  if (eta_max_grid(&grid) != 0) { free_mesh(m); return fail(CLOT_ECUDA, "occupancy query failed"); }
  // Blocks of the eta solve: about four cells per thread where the mesh is
  // small enough to leave SMs unused.  Each CG iteration pays for two or three
  // grid barriers, whose cost grows with the number of arriving blocks; on the
  // 1024 x 256 channel one block per 2048 cells took 0.91 ms of eta per primed
  // step against 1.23 ms with one per 512 cells (and 1.10 with one per 8192).
  const long long need = (g.ncell + 4 * ETA_BLOCK - 1) / (4 * ETA_BLOCK);
  m->eta_grid = (int)std::min<long long>(grid, std::max<long long>(need, 1));
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  m->aux_blocks = (int)std::min<long long>(std::max(sms, 1) * 8, std::max<long long>((g.ncell + 255) / 256, 1));

  const size_t npart = (size_t)std::max(3 * m->eta_grid + 8, 8 * m->aux_blocks);
  if (cudaMalloc(&m->scratch, sizeof(float) * CLOT_NS * g.pitch) != cudaSuccess ||
      cudaMalloc(&m->stage, sizeof(float) * CLOT_NS * g.pitch) != cudaSuccess ||
      cudaMalloc(&m->xws, sizeof(float) * 4 * g.pitch) != cudaSuccess ||
      cudaMalloc(&m->dev_in, sizeof(float) * 2 * (size_t)g.ny * g.nz) != cudaSuccess ||
      cudaMalloc(&m->wall_lo, sizeof(float) * 2 * (size_t)std::max(g.n_inj, 1)) != cudaSuccess ||
      cudaMalloc(&m->cg, sizeof(float) * 9 * g.ncell) != cudaSuccess ||
      cudaMalloc(&m->eta_ws, sizeof(float) * 2 * g.ncell) != cudaSuccess ||
      cudaMalloc(&m->maxw, sizeof(unsigned) * 4) != cudaSuccess ||
      cudaMalloc(&m->partials, sizeof(double) * npart) != cudaSuccess ||
      cudaMalloc(&m->dout, sizeof(double) * 8) != cudaSuccess ||
      cudaMalloc(&m->bar, sizeof(unsigned) * 8) != cudaSuccess ||
      cudaMalloc(&m->status, sizeof(int) * 8) != cudaSuccess ||
      cudaMalloc(&m->scount, sizeof(unsigned long long) * 4) != cudaSuccess) {
    free_mesh(m);
    cudaGetLastError();
    return fail(CLOT_ENOMEM, "device allocation of the mesh workspace failed");
  }
  if (cudaMemset(m->bar, 0, 8 * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(m->status, 0, 8 * sizeof(int)) != cudaSuccess ||
      cudaMemset(m->cg, 0, sizeof(float) * 4 * g.ncell) != cudaSuccess ||
      cudaMemset(m->maxw, 0, sizeof(unsigned) * 4) != cudaSuccess) {
    free_mesh(m);
    return fail(CLOT_ECUDA, "workspace initialisation failed");
  }
  *out = m;
  return CLOT_OK;
}

extern "C" void clot_mesh_destroy(clot_mesh* m) { free_mesh(m); }

extern "C" int clot_mesh_info(const clot_mesh* m, clot_mesh_info_t* o) {
  if (!m || !o) return fail(CLOT_EINVAL, "null argument");
  const Geom& g = m->g;
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
  o->ntau = m->ntau;
  return CLOT_OK;
}

static int check_device(const clot_mesh* m) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(CLOT_ECUDA, "cudaGetDevice failed");
  if (dev != m->device) return fail(CLOT_EINVAL, "mesh belongs to device %d, current is %d", m->device, dev);
  return CLOT_OK;
}

int clot::check_params_common(const clot_params* p) {
  if (!p) return fail(CLOT_EINVAL, "null params");
  if (p->M_rxn < 1) return fail(CLOT_EINVAL, "M_rxn must be >= 1");
  if (p->limiter != 0 && p->limiter != 1) return fail(CLOT_EINVAL, "limiter must be 0 or 1");
  if (!(p->Pmax > 0)) return fail(CLOT_EINVAL, "Pmax must be > 0");
  if (!(p->sigma_dt > 0 && p->sigma_tf > 0)) return fail(CLOT_EINVAL, "sigma_dt, sigma_tf must be > 0");
  const int ntau = (int)floor(p->sigma_tf / p->sigma_dt + 0.5);
  if (ntau < 1 || ntau > CLOT_NTAU_MAX)
    return fail(CLOT_EINVAL, "sigma_tf / sigma_dt = %d outside [1, %d]", ntau, CLOT_NTAU_MAX);
  if (!(p->eta_t < 1.0)) return fail(CLOT_EINVAL, "eta_t must be < 1");
  return CLOT_OK;
}

static int check_params(const clot_mesh* m, const clot_params* p) {
  (void)m;
  return check_params_common(p);
}

RxnConst clot::make_rxn_const(const clot_mesh_desc& d, const clot_params* p) {
  RxnConst r{};
  r.kadh = (float)p->kadh;
  r.Pmax = (float)p->Pmax;
  r.kcohPmax = (float)p->kcohPmax;
  r.k_adp = (float)p->k_adp;
  r.adp_star = (float)p->adp_star;
  r.k_e2 = (float)p->k_e2;
  r.e2_star = (float)p->e2_star;
  r.n1 = (float)(p->N1 / p->N_A);
  r.n2 = (float)(p->N2 / p->N_A);
  r.kS1p = (float)p->kS1p; r.kS1m = (float)p->kS1m;
  r.kE1p = (float)p->kE1p; r.kE1m = (float)p->kE1m;
  r.kS2p = (float)p->kS2p; r.kS2m = (float)p->kS2m;
  r.kE2p = (float)p->kE2p; r.kE2m = (float)p->kE2m;
  r.kC1p = (float)p->kC1p; r.kC1m = (float)p->kC1m; r.kC1cat = (float)p->kC1cat;
  r.kC2p = (float)p->kC2p; r.kC2m = (float)p->kC2m; r.kC2cat = (float)p->kC2cat;
  r.kC0p = (float)p->kC0p; r.kC0m = (float)p->kC0m; r.kC0cat = (float)p->kC0cat;
  r.aV = (float)(1.0 / d.hy);
  r.Dd = (float)(p->D_chem / (0.5 * d.hy));
  r.eta_t = (float)p->eta_t;
  r.eta_star3 = (float)(p->eta_star * p->eta_star * p->eta_star);
  const double u1 = 1.0 - p->eta_t;
  r.g0 = (float)((p->eta_star * p->eta_star * p->eta_star + u1 * u1 * u1) / (u1 * u1 * u1));
  r.kI = (float)p->kI;
  return r;
}

StepConst clot::make_step_const(const Geom& g, const clot_mesh_desc& d, const clot_params* p, double dt) {
  StepConst K;
  memset(&K, 0, sizeof(K));
  K.g = g;
  const double V = d.hx * d.hy * d.hz;
  const double h[3] = {d.hx, d.hy, d.hz};
  K.dt = (float)dt;
  K.dtV = (float)(dt / V);
  K.invPmax = (float)(1.0 / p->Pmax);
  for (int t = 0; t < NT; ++t) {
    const double D = t < 2 ? p->D_P : t == 2 ? p->D_adp : p->D_chem;
    for (int a = 0; a < 3; ++a) K.dcoef[t][a] = (float)(D * (V / h[a]) / h[a]);
  }
  K.limiter = p->limiter;
  K.closed_ends = (p->flags & CLOT_CLOSED_ENDS) ? 1 : 0;
  K.do_transport = (p->flags & CLOT_NO_TRANSPORT) ? 0 : 1;
  K.do_reaction = (p->flags & CLOT_NO_REACTION) ? 0 : 1;
  K.wall_lagged = (p->flags & CLOT_WALL_LAGGED) ? 1 : 0;
  K.M = p->M_rxn;
  K.h = (float)(dt / p->M_rxn);
  K.r = make_rxn_const(d, p);
  return K;
}

static StepConst make_step(const clot_mesh* m, const clot_params* p, double dt) {
  return make_step_const(m->g, m->desc, p, dt);
}

static int validate_fluxes(clot_mesh* m, const clot_fluxes* fl, const clot_params* p, double dt,
                           cudaStream_t s) {
  for (int q = 0; q < 2; ++q)
    if (m->validated[q] && m->vfx[q] == fl->fx && m->vfy[q] == fl->fy && m->vfz[q] == fl->fz && m->vdt[q] == dt)
      return CLOT_OK;
  FluxCheckArgs a{};
  a.fx = fl->fx;
  a.fy = fl->fy;
  a.fz = fl->fz;
  a.g = m->g;
  a.partials = m->partials;
  a.out = m->dout;
  a.invV = 1.0 / (m->desc.hx * m->desc.hy * m->desc.hz);
  CUDA_OK(traced(m, K_OTHER, s, [&] { return launch_flux_check(a, m->aux_blocks, s); }));
  double o[8];
  CUDA_OK(cudaMemcpyAsync(o, m->dout, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (o[2] != 0.0) return fail(CLOT_EINVAL, "wall faces carry nonzero flux (max %g)", o[2]);
  if (o[1] > 1e-5) return fail(CLOT_EINVAL, "face fluxes are not divergence-free (relative %g)", o[1]);
  const double Dmax = std::max(p->D_P, std::max(p->D_adp, p->D_chem));
  const clot_mesh_desc& d = m->desc;
  double diff = 2 * Dmax * dt * (1 / (d.hx * d.hx) + 1 / (d.hy * d.hy));
  if (d.dim == 3) diff += 2 * Dmax * dt / (d.hz * d.hz);
  const double cour = dt * o[0];
  if (cour + diff > 1.0 + 1e-9)
    return fail(CLOT_EINVAL, "dt = %g too large: Courant %g + diffusion %g > 1", dt, cour, diff);
  const int q = m->vnext;
  m->vnext ^= 1;
  m->validated[q] = 1;
  m->vfx[q] = fl->fx;
  m->vfy[q] = fl->fy;
  m->vfz[q] = fl->fz;
  m->vdt[q] = dt;
  return CLOT_OK;
}

static int check_fields(const clot_mesh* m, const clot_fields* f) {
  if (!f || !f->c || !f->eta || !f->sigma || !f->hist || !f->bound_acc)
    return fail(CLOT_EINVAL, "null field pointer");
  if (f->c_next == f->c) return fail(CLOT_EINVAL, "c_next must differ from c");
  if (m->g.n_inj > 0 && (!f->e0 || !f->c0)) return fail(CLOT_EINVAL, "null e0/c0 with an injury patch");
  return CLOT_OK;
}

void clot::sigma_weights(const clot_params* p, SigmaArgs* a) {
  const int ntau = (int)floor(p->sigma_tf / p->sigma_dt + 0.5);
  a->nslot = ntau + 1;
  for (int lag = 0; lag <= ntau; ++lag) {
    const double tau = lag * p->sigma_dt;
    const double R = exp(-(tau - 3.0) * (tau - 3.0)) / sqrt(M_PI);
    const double w = (lag == 0 || lag == ntau) ? 0.5 : 1.0;
    a->w[lag] = (float)(p->A_hat * p->sigma_dt * w * R);
  }
}

static SigmaArgs make_sigma(const clot_mesh* m, const clot_fields* f, const clot_params* p) {
  SigmaArgs a{};
  memset(&a, 0, sizeof(a));
  a.sigma = f->sigma;
  a.hist = f->hist;
  a.bound_acc = f->bound_acc;
  a.ncell = m->g.ncell;
  sigma_weights(p, &a);
  return a;
}

static EtaArgs make_eta(clot_mesh* m, clot_fields* f, const clot_params* p, const float* c) {
  EtaArgs a{};
  a.c = c;
  a.eta = f->eta;
  a.r = m->cg;
  a.p = m->cg + m->g.ncell;
  a.q = m->cg + 2 * m->g.ncell;
  a.p2 = m->cg + 3 * m->g.ncell;
  a.cg5 = m->cg + 4 * m->g.ncell;
  a.partials = m->partials;
  a.bar = m->bar;
  a.status = m->status;
  a.g = m->g;
  const double cl = p->L_eta * p->L_eta / 4.0;
  a.cx = (float)(cl / (m->desc.hx * m->desc.hx));
  a.cy = (float)(cl / (m->desc.hy * m->desc.hy));
  a.cz = (float)(m->desc.dim == 3 ? cl / (m->desc.hz * m->desc.hz) : 0.0);
  a.invPmax = (float)(1.0 / p->Pmax);
  a.tol = (float)p->eta_tol;
  a.atol = (float)p->eta_atol;
  a.inner = 1.0f;
  a.maxit = p->eta_maxit;
  a.wait_ns = eta_wait_ns(p->wait_s);
  a.predicted = 0;
  a.maxw = nullptr;
  a.maxw_clear = nullptr;
  return a;
}

// Read the device status word (synchronous) and clear its flags: the timeout
// bit is reported once, by whichever call reads it.
static int read_status(clot_mesh* m, cudaStream_t s, int* iters = nullptr) {
  int st[2];
  CUDA_OK(cudaMemcpyAsync(st, m->status, sizeof(st), cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (iters) *iters = st[1];
  if (st[0] != 0) {
    CUDA_OK(cudaMemsetAsync(m->status, 0, sizeof(int), s));
    CUDA_OK(cudaStreamSynchronize(s));
  }
  if (st[0] & ST_TIMEOUT) return fail(CLOT_ETIMEOUT, "a bounded device wait timed out (eta solver grid barrier)");
  return CLOT_OK;
}

static int check_mlp(const clot_mlp* mlp) {
  if (!mlp || !mlp->w) return fail(CLOT_EINVAL, "null network");
  if (mlp->engine != CLOT_MLP_ENGINE_MMA && mlp->engine != CLOT_MLP_ENGINE_TCGEN05)
    return fail(CLOT_EINVAL, "unknown network engine %d", mlp->engine);
  for (int q = 0; q < CLOT_NS; ++q)
    if (!(mlp->scale[q] > 0.0f) || !isfinite(mlp->scale[q]))
      return fail(CLOT_EINVAL, "surrogate scales must be finite and > 0");
  return CLOT_OK;
}

// The surrogate reaction solve of a species step over dt (h = dt / M, M RK4
// steps for the fallback cells), in place on c with the step's eta.
static SurrArgs make_surr(clot_mesh* m, clot_fields* f, const clot_params* p, const clot_mlp* mlp, float* c,
                          const float* eta, double dt, float tol) {
  SurrArgs A{};
  memset(&A, 0, sizeof(A));
  A.c = c;
  A.eta = eta;
  A.e0 = f->e0;
  A.c0 = f->c0;
  A.bound_acc = f->bound_acc;
  A.counts = m->scount;
  A.list = reinterpret_cast<int*>(m->cg);  // the eta solver's vectors are free between solves
  A.w = mlp->w;
  A.status = m->status;
  A.engine = mlp->engine;
  A.g = m->g;
  A.r = make_rxn_const(m->desc, p);
  A.h = (float)(dt / p->M_rxn);
  A.M = p->M_rxn;
  A.dt = (float)dt;
  A.tol = tol;
  surrogate_fill_consts(mlp, dt, A.inv_scale, A.floor_s, &A.xdt);
  return A;
}

static int species_steps(clot_mesh* m, clot_fields* f, const clot_fluxes* fl, const clot_params* p, double dt,
                         int nsteps, cudaStream_t s, const clot_mlp* mlp, float tol);

extern "C" int clot_species_step(clot_mesh* m, clot_fields* f, const clot_fluxes* fl, const clot_params* p,
                                 double dt, int nsteps, void* stream) {
  return species_steps(m, f, fl, p, dt, nsteps, (cudaStream_t)stream, nullptr, 0.0f);
}

extern "C" int clot_species_step_surrogate(clot_mesh* m, clot_fields* f, const clot_fluxes* fl,
                                           const clot_params* p, const clot_mlp* mlp, float tol, double dt,
                                           int nsteps, int64_t counts[3], void* stream) {
  int rc;
  if ((rc = check_mlp(mlp))) return rc;
  if (!(tol >= 0.0f)) return fail(CLOT_EINVAL, "need tol >= 0");
  if (p && (p->flags & (CLOT_HEUN | CLOT_STRANG | CLOT_NO_REACTION | CLOT_DEVIATION)))
    return fail(CLOT_EINVAL, "the surrogate step runs the one-stage fractional step with its reaction, on the "
                             "full-value state (no CLOT_DEVIATION)");
  if (f && f->ext) return fail(CLOT_EINVAL, "the surrogate step does not carry the inhibitor extension");
  if (m && m->g.ncell >= (1LL << 31)) return fail(CLOT_EINVAL, "surrogate needs ncell < 2^31");
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = species_steps(m, f, fl, p, dt, nsteps, s, mlp, tol))) return rc;
  if (counts) {
    unsigned long long hc[2] = {0, 0};
    if (nsteps > 0) {
      CUDA_OK(cudaMemcpyAsync(hc, m->scount, sizeof(hc), cudaMemcpyDeviceToHost, s));
      CUDA_OK(cudaStreamSynchronize(s));
    }
    counts[1] = (int64_t)hc[0];
    counts[2] = (int64_t)hc[1];
    counts[0] = nsteps > 0 ? m->g.ncell - counts[1] - counts[2] : 0;
  }
  return CLOT_OK;
}

static int species_steps(clot_mesh* m, clot_fields* f, const clot_fluxes* fl, const clot_params* p, double dt,
                         int nsteps, cudaStream_t s, const clot_mlp* mlp, float tol) {
  if (!m || !fl) return fail(CLOT_EINVAL, "null argument");
  int rc;
  if ((rc = check_device(m)) || (rc = check_fields(m, f)) || (rc = check_params(m, p))) return rc;
  if (!(dt > 0) || nsteps < 0) return fail(CLOT_EINVAL, "need dt > 0 and nsteps >= 0");
  if (!fl->fx || !fl->fy || (m->g.dim == 3 && !fl->fz)) return fail(CLOT_EINVAL, "null flux pointer");
  if (!p->pmu_in || !p->s1_in || !p->s2_in) return fail(CLOT_EINVAL, "null inlet profile");
  const bool ext = f->ext != nullptr;
  if (ext && m->g.dim == 3 && (m->g.nx % 4 != 0 || (reinterpret_cast<uintptr_t>(f->c) & 15u) != 0))
    return fail(CLOT_EINVAL, "the inhibitor extension on a 3D mesh needs nx a multiple of 4 and 16-byte state rows");
  if (nsteps == 0) return CLOT_OK;
  if (!(p->flags & CLOT_NO_TRANSPORT) && (rc = validate_fluxes(m, fl, p, dt, s))) return rc;
  m->ntau = (int)floor(p->sigma_tf / p->sigma_dt + 0.5);

  StepArgs A{};
  memset(&A, 0, sizeof(A));
  A.fx = fl->fx;
  A.fy = fl->fy;
  A.fz = fl->fz;
  A.sigma = f->sigma;
  A.pmu_in = p->pmu_in;
  A.s1_in = p->s1_in;
  A.s2_in = p->s2_in;
  A.e0 = f->e0;
  A.c0 = f->c0;
  A.bound_acc = f->bound_acc;
  A.status = m->status;
  A.K = make_step(m, p, dt);
  const bool dev = (p->flags & CLOT_DEVIATION) != 0;
  if (dev && mlp) return fail(CLOT_EINVAL, "CLOT_DEVIATION does not apply to the surrogate step");
  const bool surr = mlp != nullptr && A.K.do_reaction;
  if (surr) A.K.do_reaction = 0;  // the fused pass transports; the surrogate pass reacts
  const bool run_k1 = A.K.do_transport || A.K.do_reaction;
  const bool heun = (p->flags & CLOT_HEUN) != 0;
  const bool strang = (p->flags & CLOT_STRANG) && A.K.do_reaction;
  if (strang) A.K.h = (float)(dt / (2.0 * p->M_rxn));  // each half: M_rxn RK4 steps of dt / (2 M_rxn)
  const bool do_eta = !(p->flags & CLOT_NO_ETA);
  // eta prediction: each fused step also extrapolates eta to the next step and
  // records the residual of that guess; the next eta solve accepts it when it
  // meets the stopping rule.  Three buffers rotate: the caller's eta and two of
  // the workspace.
  const bool predict = do_eta && run_k1 && !surr;  // the surrogate pass ends the step: no prediction
  {
    const double cl = p->L_eta * p->L_eta / 4.0;
    A.ecx = (float)(cl / (m->desc.hx * m->desc.hx));
    A.ecy = (float)(cl / (m->desc.hy * m->desc.hy));
    A.ecz = (float)(m->desc.dim == 3 ? cl / (m->desc.hz * m->desc.hz) : 0.0);
  }
  // A call that continues the previous one on the same fields (same buffers,
  // time and dt, nothing else run on the mesh in between) picks up its
  // prediction; otherwise the first solve starts from fields.eta.
  const bool cont = predict && m->pred_valid && m->pred_c == f->c && m->pred_eta == f->eta && m->pred_t == f->t &&
                    m->pred_dt == dt && !(p->flags & CLOT_ETA_FRESH);
  m->pred_valid = 0;
  float* ecur = f->eta;
  float* eprev = f->eta;
  float* ebuf[3] = {f->eta, m->eta_ws, m->eta_ws + m->g.ncell};
  bool have_pred = false;
  int sel0 = 0;
  if (cont) {
    ecur = m->pred_guess;
    have_pred = true;
    sel0 = m->pred_sel ^ 1;
  } else if (predict) {
    CUDA_OK(cudaMemsetAsync(m->maxw, 0, 4 * sizeof(unsigned), s));
  }
  // Deviation form for the length of the call: the S1, S2 rows and their
  // inlet values shifted by the references (the rates add them back), the
  // E0, C0 low words zeroed.
  const long long pitch = m->g.pitch;
  const float r1 = (float)p->S1_ref, r2 = (float)p->S2_ref;
  if (dev) {
    const long long nb = (long long)m->g.ny * m->g.nz;
    A.K.r.s1_ref = r1;
    A.K.r.s2_ref = r2;
    CUDA_OK(launch_shift(m->dev_in, p->s1_in, nb, -r1, s));
    CUDA_OK(launch_shift(m->dev_in + nb, p->s2_in, nb, -r2, s));
    A.s1_in = m->dev_in;
    A.s2_in = m->dev_in + nb;
    CUDA_OK(launch_shift(f->c + CLOT_S1 * pitch, f->c + CLOT_S1 * pitch, m->g.ncell, -r1, s));
    CUDA_OK(launch_shift(f->c + CLOT_S2 * pitch, f->c + CLOT_S2 * pitch, m->g.ncell, -r2, s));
    if (m->g.n_inj > 0) {
      CUDA_OK(cudaMemsetAsync(m->wall_lo, 0, sizeof(float) * 2 * m->g.n_inj, s));
      A.e0lo = m->wall_lo;
      A.c0lo = m->wall_lo + m->g.n_inj;
    }
  }
  int last_sel = 0;
  float* cur = f->c;
  float* nxt = f->c_next ? f->c_next : m->scratch;
  for (int step = 0; step < nsteps; ++step) {
    const int sel = (step + sel0) & 1;
    last_sel = sel;
    if (do_eta) {
      EtaArgs e = make_eta(m, f, p, cur);
      e.eta = ecur;
      e.inner = 1.0f;  // no over-solve: measured fastest (CG iterations and accepted predictions)
      if (have_pred) {
        e.predicted = 1;
        e.maxw = m->maxw + 2 * (sel ^ 1);      // written by the previous fused step
        e.maxw_clear = m->maxw + 2 * sel;      // used by this step's fused kernel
      }
      CUDA_OK(traced(m, K_ETA, s, [&] { return launch_eta_solve(e, m->eta_grid, s); }));
    }
    if (!(p->flags & CLOT_NO_SIGMA)) {
      SigmaArgs sa = make_sigma(m, f, p);
      if (f->t_last < 0) {
        CUDA_OK(traced(m, K_SIGMA, s, [&] { return launch_sigma_init(sa, s); }));
        f->t_last = f->t;
      }
      if (f->t + 1e-6 * dt >= (f->n_samples + 1) * p->sigma_dt) {
        sa.head = f->n_samples == 0 ? 0 : (f->head + 1) % sa.nslot;
        sa.nvalid = std::min(f->n_samples + 1, sa.nslot);
        sa.inv_dt_sample = (float)(1.0 / (f->t - f->t_last));
        CUDA_OK(traced(m, K_SIGMA, s, [&] { return launch_sigma_sample(sa, s); }));
        f->head = sa.head;
        f->n_samples += 1;
        f->t_last = f->t;
      }
    }
    A.K.has_sigma = (!(p->flags & CLOT_NO_SIGMA) && f->n_samples > 0) ? 1 : 0;
    // Strang splitting: the first reaction half-step, cur -> nxt; the
    // transport then starts from nxt and the step's result lands in cur
    // (whose state the half-step has consumed).
    float* c_start = cur;
    float* c_out = nxt;
    if (strang) {
      StepArgs R = A;
      R.cin = cur;
      R.cout = nxt;
      R.eta = ecur;
      R.predict = 0;
      R.cavg = nullptr;
      R.xin = f->ext;  // the extension's rows react in place (null without it)
      R.xout = f->ext;
      CUDA_OK(traced(m, K_OTHER, s, [&] { return launch_reaction_only(R, s); }));
      c_start = nxt;
      c_out = cur;
    }
    // the extension's rows: transported by their own pass (two with Heun),
    // then reacted in the fused pass's RK4 stages, which writes them back
    A.xin = A.xout = nullptr;
    if (ext) {
      A.xin = f->ext;
      A.xout = f->ext;
      if (A.K.do_transport) {
        float* xmid = m->xws;
        float* xst = m->xws + 2 * m->g.pitch;
        ExtArgs X{};
        memset(&X, 0, sizeof(X));
        X.fx = fl->fx;
        X.fy = fl->fy;
        X.fz = fl->fz;
        X.g = m->g;
        X.pitch = m->g.pitch;
        X.dtV = A.K.dtV;
        X.I_in = (float)p->I_in;
        for (int ax = 0; ax < 3; ++ax) X.dcoef[ax] = A.K.dcoef[3][ax];  // D_chem, as S1
        X.limiter = A.K.limiter;
        X.closed_ends = A.K.closed_ends;
        X.xin = f->ext;
        X.xout = heun ? xst : xmid;
        CUDA_OK(traced(m, K_OTHER, s, [&] { return launch_ext_transport(X, s); }));
        if (heun) {
          X.xin = xst;
          X.xout = xmid;
          X.xavg = f->ext;
          CUDA_OK(traced(m, K_OTHER, s, [&] { return launch_ext_transport(X, s); }));
        }
        A.xin = xmid;
      }
    }
    if (heun && A.K.do_transport) {
      // two-stage transport: stage 1 (transport only) c_start -> stage
      // buffer; stage 2 below averages its result with c_start
      StepArgs T = A;
      T.cin = c_start;
      T.cout = m->stage;
      T.eta = ecur;
      T.K.do_reaction = 0;
      T.K.wall_lagged = 0;
      T.predict = 0;
      T.cavg = nullptr;
      T.xin = T.xout = nullptr;
      CUDA_OK(traced(m, K_STEP, s, [&] { return launch_species_step_plane(T, s); }));
      A.cin = m->stage;
      A.cavg = c_start;
    } else {
      A.cin = c_start;
      A.cavg = nullptr;
    }
    A.cout = c_out;
    A.eta = ecur;
    float* enext = nullptr;
    if (predict) {
      for (float* b : ebuf)
        if (b != ecur && b != eprev) { enext = b; break; }
      A.predict = 1;
      A.eta_prev = eprev;
      A.eta_next = enext;
      A.eta_res = m->cg;
      A.eta_max = m->maxw + 2 * sel;
    }
    if (run_k1) {
      CUDA_OK(traced(m, K_STEP, s, [&] { return launch_species_step_plane(A, s); }));
      if (c_out == nxt) std::swap(cur, nxt);
    }
    if (surr) {  // reaction over dt: the network where it applies, RK4 on the fallback list
      const SurrArgs SA = make_surr(m, f, p, mlp, cur, ecur, dt, tol);
      CUDA_OK(cudaMemsetAsync(m->scount, 0, 3 * sizeof(unsigned long long), s));
      CUDA_OK(traced(m, K_OTHER, s, [&] { return launch_surrogate_react(SA, s); }));
      CUDA_OK(traced(m, K_OTHER, s, [&] { return launch_surrogate_fallback(SA, s); }));
    }
    if (predict) {
      eprev = ecur;
      ecur = enext;
      have_pred = true;
    }
    f->t += dt;
  }
  if (cur != f->c) {
    if (f->c_next) {  // the result is in the caller's partner buffer: swap the roles
      f->c_next = f->c;
      f->c = cur;
    } else {
      CUDA_OK(cudaMemcpyAsync(f->c, cur, sizeof(float) * CLOT_NS * m->g.pitch, cudaMemcpyDeviceToDevice, s));
    }
  }
  if (dev) {  // back to the full values
    CUDA_OK(launch_shift(f->c + CLOT_S1 * pitch, f->c + CLOT_S1 * pitch, m->g.ncell, r1, s));
    CUDA_OK(launch_shift(f->c + CLOT_S2 * pitch, f->c + CLOT_S2 * pitch, m->g.ncell, r2, s));
  }
  // fields->eta returns the eta used by the last step (eprev after the
  // rotation); the prediction for the next step (ecur) is kept in a workspace
  // buffer for a continuing call.
  if (predict) {
    if (ecur == f->eta) {
      float* freeb = nullptr;
      for (float* b : ebuf)
        if (b != f->eta && b != eprev) { freeb = b; break; }
      CUDA_OK(cudaMemcpyAsync(freeb, ecur, sizeof(float) * m->g.ncell, cudaMemcpyDeviceToDevice, s));
      ecur = freeb;
    }
    if (eprev != f->eta)
      CUDA_OK(cudaMemcpyAsync(f->eta, eprev, sizeof(float) * m->g.ncell, cudaMemcpyDeviceToDevice, s));
    m->pred_valid = 1;
    m->pred_c = f->c;
    m->pred_eta = f->eta;
    m->pred_t = f->t;
    m->pred_dt = dt;
    m->pred_guess = ecur;
    m->pred_sel = last_sel;
  }
  if (p->flags & CLOT_SYNC_STATUS) return read_status(m, s);
  return CLOT_OK;
}

extern "C" int clot_reaction_step(clot_mesh* m, clot_fields* f, const clot_params* p, double h, int nsub,
                                  void* stream) {
  if (!m) return fail(CLOT_EINVAL, "null mesh");
  int rc;
  if ((rc = check_device(m)) || (rc = check_fields(m, f)) || (rc = check_params(m, p))) return rc;
  if (!(h > 0) || nsub < 1) return fail(CLOT_EINVAL, "need h > 0 and nsub >= 1");
  m->pred_valid = 0;
  cudaStream_t s = (cudaStream_t)stream;
  StepArgs A{};
  memset(&A, 0, sizeof(A));
  A.eta = f->eta;
  A.e0 = f->e0;
  A.c0 = f->c0;
  A.bound_acc = f->bound_acc;
  A.K = make_step(m, p, h * nsub);
  A.K.do_reaction = 1;
  A.K.M = nsub;
  A.K.h = (float)h;
  A.cin = f->c;
  A.cout = m->scratch;
  CUDA_OK(traced(m, K_STEP, s, [&] { return launch_reaction_only(A, s); }));
  CUDA_OK(cudaMemcpyAsync(f->c, m->scratch, sizeof(float) * CLOT_NS * m->g.pitch, cudaMemcpyDeviceToDevice, s));
  return CLOT_OK;
}

extern "C" int clot_surrogate_infer(clot_mesh* m, clot_fields* f, const clot_params* p, const clot_mlp* mlp,
                                    double h, int nsub, float tol, uint8_t* flag, int64_t counts[3],
                                    void* stream) {
  if (!m || !mlp || !mlp->w) return fail(CLOT_EINVAL, "null argument");
  int rc;
  if ((rc = check_device(m)) || (rc = check_fields(m, f)) || (rc = check_params(m, p))) return rc;
  if (!(h > 0) || nsub < 1) return fail(CLOT_EINVAL, "need h > 0 and nsub >= 1");
  if (!(tol >= 0.0f)) return fail(CLOT_EINVAL, "need tol >= 0");
  m->pred_valid = 0;
  if (mlp->engine != CLOT_MLP_ENGINE_MMA && mlp->engine != CLOT_MLP_ENGINE_TCGEN05)
    return fail(CLOT_EINVAL, "unknown network engine %d", mlp->engine);
  for (int s = 0; s < CLOT_NS; ++s)
    if (!(mlp->scale[s] > 0.0f) || !isfinite(mlp->scale[s]))
      return fail(CLOT_EINVAL, "surrogate scales must be finite and > 0");
  cudaStream_t s = (cudaStream_t)stream;
  SurrArgs A{};
  memset(&A, 0, sizeof(A));
  A.c = f->c;
  A.eta = f->eta;
  A.e0 = f->e0;
  A.c0 = f->c0;
  A.bound_acc = f->bound_acc;
  A.flag = flag;
  A.counts = m->scount;
  A.list = reinterpret_cast<int*>(m->cg);  // the eta solver's vectors are free between solves
  A.w = mlp->w;
  A.status = m->status;
  A.engine = mlp->engine;
  A.g = m->g;
  A.r = make_rxn_const(m->desc, p);
  A.h = (float)h;
  A.M = nsub;
  A.dt = (float)(h * nsub);
  A.tol = tol;
  surrogate_fill_consts(mlp, h * nsub, A.inv_scale, A.floor_s, &A.xdt);
  if (m->g.ncell >= (1LL << 31)) return fail(CLOT_EINVAL, "surrogate needs ncell < 2^31");
  CUDA_OK(cudaMemsetAsync(m->scount, 0, 3 * sizeof(unsigned long long), s));
  CUDA_OK(traced(m, K_STEP, s, [&] { return launch_surrogate_react(A, s); }));
  CUDA_OK(traced(m, K_STEP, s, [&] { return launch_surrogate_fallback(A, s); }));
  if (counts) {
    unsigned long long hc[2];
    CUDA_OK(cudaMemcpyAsync(hc, m->scount, sizeof(hc), cudaMemcpyDeviceToHost, s));
    CUDA_OK(cudaStreamSynchronize(s));
    counts[1] = (int64_t)hc[0];
    counts[2] = (int64_t)hc[1];
    counts[0] = m->g.ncell - counts[1] - counts[2];
  }
  return CLOT_OK;
}

extern "C" int clot_eta_solve(clot_mesh* m, clot_fields* f, const clot_params* p, int* iters, void* stream) {
  if (!m) return fail(CLOT_EINVAL, "null mesh");
  m->pred_valid = 0;
  int rc;
  if ((rc = check_device(m)) || (rc = check_fields(m, f)) || (rc = check_params(m, p))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  EtaArgs e = make_eta(m, f, p, f->c);
  CUDA_OK(traced(m, K_ETA, s, [&] { return launch_eta_solve(e, m->eta_grid, s); }));
  if (iters) return read_status(m, s, iters);
  return CLOT_OK;
}

static int diagnostics_launch(clot_mesh* m, const clot_fields* f, const clot_params* p, cudaStream_t s) {
  int rc;
  if ((rc = check_device(m)) || (rc = check_fields(m, f))) return rc;
  if (!p || !(p->Pmax > 0)) return fail(CLOT_EINVAL, "bad params");
  DiagArgs a{};
  a.c = f->c;
  a.e0 = f->e0;
  a.c0 = f->c0;
  a.ext = f->ext;
  a.ncell = m->g.ncell;
  a.pitch = m->g.pitch;
  a.n_inj = m->g.n_inj;
  a.V = m->desc.hx * m->desc.hy * m->desc.hz;
  a.A = m->desc.hx * m->desc.hz;
  a.invPmax = 1.0 / p->Pmax;
  a.partials = m->partials;
  a.out = m->dout;
  CUDA_OK(traced(m, K_OTHER, s, [&] { return launch_diagnostics(a, m->aux_blocks, s); }));
  return CLOT_OK;
}

extern "C" int clot_diagnostics(clot_mesh* m, const clot_fields* f, const clot_params* p, double out[8],
                                void* stream) {
  if (!m || !out) return fail(CLOT_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if ((rc = diagnostics_launch(m, f, p, s))) return rc;
  CUDA_OK(cudaMemcpyAsync(out, m->dout, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_OK(cudaStreamSynchronize(s));
  if (out[6] > 0) return fail(CLOT_ENONFINITE, "%.0f non-finite values in the state", out[6]);
  return CLOT_OK;
}

extern "C" int clot_diagnostics_async(clot_mesh* m, const clot_fields* f, const clot_params* p, double* out,
                                      void* stream) {
  if (!m || !out) return fail(CLOT_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  if ((rc = diagnostics_launch(m, f, p, s))) return rc;
  CUDA_OK(cudaMemcpyAsync(out, m->dout, 8 * sizeof(double), cudaMemcpyDefault, s));
  return CLOT_OK;
}

extern "C" int clot_device_status(clot_mesh* m, int* iters, void* stream) {
  if (!m) return fail(CLOT_EINVAL, "null mesh");
  return read_status(m, (cudaStream_t)stream, iters);
}

extern "C" int clot_profile_begin(clot_mesh* m, int max_launches) {
  if (!m || max_launches < 1) return fail(CLOT_EINVAL, "need a mesh and max_launches >= 1");
  prof_free(m);
  m->prof_ev = new cudaEvent_t[2 * (size_t)max_launches];
  m->prof_kind = new int[max_launches];
  for (int q = 0; q < 2 * max_launches; ++q) {
    if (cudaEventCreate(&m->prof_ev[q]) != cudaSuccess) {
      for (int r = 0; r < q; ++r) cudaEventDestroy(m->prof_ev[r]);
      delete[] m->prof_ev;
      delete[] m->prof_kind;
      m->prof_ev = nullptr;
      m->prof_kind = nullptr;
      return fail(CLOT_ECUDA, "cudaEventCreate failed");
    }
  }
  m->prof_cap = max_launches;
  m->prof_n = 0;
  if (cudaMemset(m->status + 2, 0, 4 * sizeof(int)) != cudaSuccess) return fail(CLOT_ECUDA, "status reset failed");
  memset(m->prof_count, 0, sizeof(m->prof_count));
  m->prof_on = 1;
  return CLOT_OK;
}

extern "C" int clot_profile_end(clot_mesh* m, clot_profile_t* o, void* stream) {
  if (!m || !o) return fail(CLOT_EINVAL, "null argument");
  memset(o, 0, sizeof(*o));
  if (!m->prof_on) return fail(CLOT_EINVAL, "profiling was not started");
  CUDA_OK(cudaStreamSynchronize((cudaStream_t)stream));
  double ms[4] = {0, 0, 0, 0};
  for (int q = 0; q < m->prof_n; ++q) {
    float t = 0.0f;
    CUDA_OK(cudaEventSynchronize(m->prof_ev[2 * q + 1]));
    CUDA_OK(cudaEventElapsedTime(&t, m->prof_ev[2 * q], m->prof_ev[2 * q + 1]));
    ms[m->prof_kind[q]] += t;
  }
  o->n_step = m->prof_count[K_STEP];
  o->n_eta = m->prof_count[K_ETA];
  o->n_sigma = m->prof_count[K_SIGMA];
  o->n_other = m->prof_count[K_OTHER];
  o->ms_step = ms[K_STEP];
  o->ms_eta = ms[K_ETA];
  o->ms_sigma = ms[K_SIGMA];
  o->ms_other = ms[K_OTHER];
  o->timed = m->prof_n;
  int st[6];
  CUDA_OK(cudaMemcpy(st, m->status, sizeof(st), cudaMemcpyDeviceToHost));
  o->eta_iters = st[2];
  o->eta_accepted = st[3];
  o->eta_box = st[4];
  o->eta_box_fallback = st[5];
  prof_free(m);
  return CLOT_OK;
}

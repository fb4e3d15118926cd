/*
 * clot.h -- C ABI of the GB300 (sm_103a) clotFoam species-step library.
 *
 * One time step of the continuum clotting model of the clotFoam paper
 * (Montgomery, Municchi, Leiderman, SoftwareX) on a uniform 2D or 3D
 * finite-volume mesh with prescribed face fluxes:
 *   - explicit finite-volume transport of the seven mobile species (Sec. 3.2
 *     step 1; App. A Eqs. for P^{m,u}, P^{m,a}; Sec. 2 Eq. ADP_eqt; App. B
 *     fluid-phase equations), van Leer face values (App. D), platelet fluxes
 *     hindered by W(theta_T) with downwind / localMax face theta (Sec. 3.2);
 *   - M_rxn RK4 reaction substeps of h = dt / M_rxn (Sec. 3.2 step 2) of the
 *     platelet sources (App. A) and the 12-species coagulation model (App. B),
 *     including the reactive injury-wall fluxes and the subendothelial E0, C0;
 *   - the virtual substance eta, (I - L_eta^2/4 lap) eta = theta_B (App. A,
 *     Eq. eta), feeding the binding affinity g(eta);
 *   - the ADP release source sigma_release by the trapezoid rule over a history
 *     sampled every sigma_dt (Sec. 2 Eq. ADP_source, Sec. 3.2 Eq. sigma_disc).
 *
 * Conventions (all entry points):
 *   - Units: mm, s, nmol, platelets.  Cells are indexed cell = i + nx (j + ny k);
 *     x is the flow axis (inlet x = 0, outlet x = nx hx), y = 0 is the floor
 *     that carries the injury patch, the other sides are walls.  2D meshes have
 *     nz = 1 and unit depth hz.
 *   - Every device pointer is CALLER-OWNED device memory (e.g. torch tensors),
 *     borrowed for the duration of the call; the library never frees it.
 *   - Every call is stream-ordered on the caller's stream (a cudaStream_t passed
 *     as void*; NULL = legacy default stream) and does not synchronise unless
 *     stated.  The library allocates device memory only in clot_mesh_create.
 *   - Return 0 (CLOT_OK) or a negative clot_status; clot_last_error() gives a
 *     one-line reason (thread-local).  There is no CPU fallback: without a
 *     CUDA device every compute call returns CLOT_ECUDA.
 */
#ifndef CLOT_H
#define CLOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CLOT_NS 15          /* cell species */
#define CLOT_NTAU_MAX 64    /* maximum sigma_tf / sigma_dt */

/* Cell-species rows of the state array c (species-major). */
enum {
  CLOT_PMU = 0, CLOT_PMA, CLOT_PBA, CLOT_PBSE, CLOT_ADP, CLOT_S1, CLOT_S2, CLOT_E1, CLOT_E2,
  CLOT_S1B, CLOT_S2B, CLOT_E1B, CLOT_E2B, CLOT_C1, CLOT_C2
};

typedef enum {
  CLOT_OK = 0,
  CLOT_EINVAL = -1,      /* bad shape, null pointer, dt above the stability bound, bad fluxes */
  CLOT_ECUDA = -2,       /* a CUDA call failed (or no device) */
  CLOT_ENONFINITE = -3,  /* the device status word reports a non-finite value */
  CLOT_ETIMEOUT = -4,    /* a bounded device-side wait gave up (kernel returned early) */
  CLOT_ENOMEM = -5
} clot_status;

/* clot_params.flags */
#define CLOT_NO_TRANSPORT 1  /* skip step 1 (tests) */
#define CLOT_NO_REACTION 2   /* skip step 2 (tests) */
#define CLOT_CLOSED_ENDS 4   /* inlet and outlet are zero-flux walls (tests) */
#define CLOT_NO_ETA 8        /* use fields.eta as given, no solve */
#define CLOT_NO_SIGMA 16     /* never sample the ADP release history */
#define CLOT_ETA_FRESH 32    /* clot_species_step: do not continue the previous call's eta prediction */
#define CLOT_SYNC_STATUS 64  /* clot_species_step: synchronise at the end and report the device status word
                                (CLOT_ETIMEOUT if a bounded device wait of this or an earlier call gave up) */
/* Time-stepping options (the paper's transport is Crank-Nicolson 0.9, second order in time, App. D; the
 * default here is the first-order explicit fractional step of Sec. 3.2): */
#define CLOT_HEUN 128        /* transport by Heun's method: c1 = c + dt L(c), c2 = c1 + dt L(c1), c <- (c + c2)/2
                                (each stage a forward-Euler transport pass, so conservation and the TVD bound
                                carry over); second order in time for the transport alone */
#define CLOT_STRANG 256      /* Strang splitting: M_rxn RK4 steps of dt/(2 M_rxn) before the transport and
                                again after it, both with g(eta) of the step's eta solve; with CLOT_HEUN the
                                whole coupled step is second order in time */
#define CLOT_WALL_LAGGED 512 /* the injury-wall exchange placed as the paper's solver places it (App. C
                                boundary table, App. B): S1 and E1 wall fluxes in the explicit transport from
                                the start-of-transport S1, E0, C0, then M_rxn RK4 steps of dt/M_rxn of the
                                E0/C0 ODEs with the floor cell's S1 held at its post-transport value; the
                                reaction then runs without the wall.  Family 1 + wall C0 is conserved only to
                                O(dt) (the default couples the wall inside the RK4 stages, exactly) */
/* Precision option for long runs of many small steps (no counterpart in the paper, whose solver works
 * in FP64).  The FP32 state is rounded once per step, and a quantity that changes by less than half an
 * FP32 ulp of itself per step (the zymogens S1, S2 near their plasma values; the injury wall's E0, C0
 * near quasi-equilibrium) loses its increments to that rounding.  With CLOT_DEVIATION, for the length
 * of one clot_species_step call: the S1 and S2 rows hold S1 - S1_ref and S2 - S2_ref (clot_params;
 * shifted in place on entry and back on return, the inlet values shifted with them; the reaction
 * evaluates its rates at the full values), and E0, C0 carry an FP32 low word each (the increment of
 * every step is added in FP64 to the pair).  The state in fields is the full-value FP32 state before
 * and after each call (after an error return in the middle of a call the S1, S2 rows may still hold
 * the deviations).  Not with clot_species_step_surrogate or ensembles (CLOT_EINVAL). */
#define CLOT_DEVIATION 1024

typedef struct clot_mesh clot_mesh; /* opaque, library-owned */

/* Mesh description (read during clot_mesh_create, caller-owned). */
typedef struct {
  int dim;                      /* 2 or 3 */
  int nx, ny, nz;               /* cells; nz = 1 in 2D */
  double hx, hy, hz;            /* cell sizes, mm (hz = depth in 2D) */
  double inj_x0, inj_x1;        /* injury patch on the floor y = 0: faces whose centre */
  double inj_z0, inj_z1;        /*   x (and, in 3D, z) lies in these closed intervals */
  double p_diam;                /* H_adh = 1 within this distance of the patch (App. A) */
} clot_mesh_desc;

/* Derived mesh facts (filled by clot_mesh_info). */
typedef struct {
  int64_t ncell;                /* nx ny nz */
  int64_t pitch;                /* floats between species rows of clot_fields.c (>= ncell, multiple of 32) */
  int64_t nfx, nfy, nfz;        /* face-flux array lengths: (nx+1) ny nz, nx (ny+1) nz, nx ny (nz+1) (0 in 2D) */
  int n_inj;                    /* injury faces; E0, C0 arrays have this length */
  int inj_i0, inj_i1, inj_k0, inj_k1; /* injury faces form the rectangle [i0,i1] x [k0,k1] of floor faces,
                                         stored k-major: e0[(i - i0) + (i1 - i0 + 1)(k - k0)] */
  int hadh_jmax;                /* H_adh = 1 for cells over the patch with j <= hadh_jmax (-1: none) */
  int n_hadh;                   /* number of cells with H_adh = 1 */
  int ntau;                     /* filled by clot_species_step from the params; 0 before */
} clot_mesh_info_t;

/* Simulation state (device pointers caller-owned; scalars updated in place). */
typedef struct {
  float *c;            /* [CLOT_NS][pitch] cell species, FP32, species-major */
  float *e0, *c0;      /* [n_inj] subendothelial enzyme and complex, nmol/mm^2 */
  float *eta;          /* [ncell] virtual substance; warm start in, solution out */
  float *sigma;        /* [ncell] ADP release rate, nmol/mm^3/s (held between samples) */
  float *hist;         /* [ntau + 1][ncell] ring of newly-bound rates, platelets/mm^3/s */
  float *bound_acc;    /* [ncell] platelets/mm^3 newly bound (P^{b,a} + P^{b,se} gained) since the
                          last sample, accumulated from the RK4 increments; equals
                          Pmax (theta_B - theta_B at the last sample) in exact arithmetic */
  double t;            /* simulated time of the state */
  double t_last;       /* time of the last sample; < 0: history starts at the next step */
  int n_samples;       /* samples taken so far */
  int head;            /* ring slot of the newest sample */
  float *c_next;       /* optional [CLOT_NS][pitch] partner of c (NULL: the mesh's own buffer and a copy back
                          after an odd number of steps).  When set, clot_species_step alternates between the
                          two and swaps c and c_next on return, so that c holds the result without a copy. */
  float *ext;          /* optional [2][pitch]: the inhibitor extension's species I and E2,inh (NULL: the
                          paper's model).  The paper's example of adding a species (Sec. "Adapting the
                          framework for different clotting models"): a fluid-phase inhibitor with
                          I + E2 -> E2,inh at rate kI I E2 (clot_params.kI), transported like the other
                          coagulation species (D_chem; I with the inlet value clot_params.I_in, E2,inh
                          zero-gradient) and reacted in the same RK4 stages.  Updated in place. */
} clot_fields;

/* Face fluxes F (mm^3/s, > 0 along +axis), device, caller-owned.  Walls must
 * carry F = 0.  fz is ignored (may be NULL) in 2D. */
typedef struct {
  const float *fx; const float *fy; const float *fz;
} clot_fluxes;

/* Model parameters (App. E) and numerical settings. */
typedef struct {
  double Pmax, kadh, kcohPmax, eta_t, eta_star, L_eta;
  double k_adp, adp_star, k_e2, e2_star;
  double A_hat, sigma_tf, sigma_dt;
  double D_P, D_adp, D_chem;
  double N1, N2, N_A;
  double kC0p, kC0m, kC0cat, kC1p, kC1m, kC1cat, kC2p, kC2m, kC2cat;
  double kS1p, kS1m, kE1p, kE1m, kS2p, kS2m, kE2p, kE2m;
  double eta_tol;      /* eta solve stops at max|r| <= max(eta_tol max theta_B, eta_atol); */
  double eta_atol;     /*   max|eta - eta_exact| <= max|r| (M-matrix, unit row sums) */
  double wait_s;       /* bound of each grid-barrier wait of the eta solver, seconds (<= 0: 2 s; at most
                          10 s).  A wait that runs out sets the timeout bit of the device status word and
                          the solver's blocks return; a tiny value makes the waits give up (tests). */
  double kI;           /* inhibitor extension (fields.ext): association rate of I and fluid-phase E2 */
  double I_in;         /*   and the inlet Dirichlet value of I */
  double S1_ref, S2_ref; /* reference values of S1, S2 under CLOT_DEVIATION (typically the plasma values) */
  int M_rxn;           /* reaction substeps per step (Sec. 3.2, default 2) */
  int limiter;         /* 0 first-order upwind, 1 van Leer (App. D) */
  int flags;           /* CLOT_NO_* bits */
  int eta_maxit;       /* iteration cap of the eta solve */
  const float *pmu_in; /* [ny nz] inlet Dirichlet P^{m,u} (App. C), device */
  const float *s1_in;  /* [ny nz] inlet Dirichlet S1, device */
  const float *s2_in;  /* [ny nz] inlet Dirichlet S2, device */
} clot_params;

/* Build the mesh of the paper's channel / duct problems on a uniform
 * Cartesian grid: the injury faces on the floor (App. C boundary table), the
 * adhesion region H_adh (App. A; cells within P_diam of the injury, Sec. 3.1)
 * and the device workspace (two state buffers: the ping-pong partner and the
 * stage buffer of the two-stage transport; eta solver vectors, reduction
 * partials, barrier and status words).  Errors: CLOT_EINVAL (dim not
 * 2/3, sizes < 1, nz != 1 in 2D, h <= 0, no CUDA device), CLOT_ENOMEM.  The
 * mesh belongs to the current CUDA device and is owned by the caller until
 * clot_mesh_destroy (which frees the workspace; NULL is ignored). */
int clot_mesh_create(const clot_mesh_desc *desc, clot_mesh **out);
/* Free a mesh from clot_mesh_create (App. C geometry); NULL is ignored. */
void clot_mesh_destroy(clot_mesh *mesh);
/* Cell count, pitch, face-flux array lengths, injury rectangle and adhesion
 * region of the mesh (App. A H_adh, App. C injury faces) into *out (host).
 * Errors: CLOT_EINVAL. */
int clot_mesh_info(const clot_mesh *mesh, clot_mesh_info_t *out);

/* Advance the state by nsteps species steps of dt (Sec. 3.2):
 *   per step: [eta solve from theta_B (App. A Eq. eta)] -> [sigma sample when
 *   t has reached the next multiple of sigma_dt (Sec. 3.2 Eq. sigma_disc)] ->
 *   fused transport + M_rxn RK4 reaction + wall exchange (one kernel) -> t += dt.
 * fields->c holds the result on return (stream-ordered).  The first call with a
 * new (fluxes, dt) pair validates them once, synchronously: walls must carry
 * zero flux, |sum of a cell's net outflow| <= 1e-6 sum|F|, and
 * Courant + sum_d 2 D_max dt / h_d^2 <= 1; otherwise CLOT_EINVAL.  The last
 * two validated (fluxes, dt) sets are remembered (double-buffered uploads).
 * Each step's fused kernel also predicts eta for the next step (2 eta - eta of
 * the previous step) with its residual; the next solve accepts it when it
 * meets the stopping rule, else corrects it by CG on the box around the cells
 * whose residual exceeds half the rule's bound (widened by the decay length of
 * the operator) and, if the recomputed residual there still misses the rule,
 * by CG on the whole mesh.  The prediction carries over to the next call when
 * that call continues this one: same fields buffers c and eta, fields->t and
 * dt continuing, and no other call of this library on the mesh in between
 * (they invalidate it).  A caller that changes c or eta itself between calls
 * sets CLOT_ETA_FRESH in params->flags for the next call.
 * With CLOT_HEUN / CLOT_STRANG a step is [reaction over dt/2] -> transport
 * stage 1 (one pass) -> transport stage 2 + average + [reaction over dt/2] +
 * eta prediction (one fused pass): two or three sweeps of the state instead
 * of one, through a second workspace buffer of the mesh.
 * Errors: CLOT_EINVAL (null pointers, nsteps < 0, dt <= 0, M_rxn < 1,
 * sigma_tf/sigma_dt > CLOT_NTAU_MAX), CLOT_ECUDA; CLOT_ETIMEOUT only with
 * CLOT_SYNC_STATUS. */
int clot_species_step(clot_mesh *mesh, clot_fields *fields, const clot_fluxes *fluxes,
                      const clot_params *params, double dt, int nsteps, void *stream);

/* Reaction only (Sec. 3.2 step 2): nsub RK4 steps of size h on every cell and
 * injury face, g(eta) taken from fields->eta as given, in place on fields->c,
 * e0, c0 (with CLOT_WALL_LAGGED in params->flags the injury faces belong to the
 * transport and are left unchanged).  fields->t is not changed.
 * Errors: CLOT_EINVAL, CLOT_ECUDA. */
int clot_reaction_step(clot_mesh *mesh, clot_fields *fields, const clot_params *params,
                       double h, int nsub, void *stream);

/* eta solve alone (App. A Eq. eta) from theta_B of fields->c, warm-started from
 * fields->eta; writes fields->eta.  If iters is not NULL the call synchronises,
 * stores the iteration count and reads (and clears) the device status word:
 * CLOT_ETIMEOUT if a grid-barrier wait of the solver ran out (params->wait_s),
 * in which case fields->eta is only partly solved.
 * Errors: CLOT_EINVAL, CLOT_ECUDA, CLOT_ETIMEOUT. */
int clot_eta_solve(clot_mesh *mesh, clot_fields *fields, const clot_params *params,
                   int *iters, void *stream);

/* Conservation diagnostics in FP64 (invariants of App. A/B), synchronous;
 * out is HOST memory of 8 doubles:
 *   out[0] sum V (Pmu + Pma + Pba + Pbse)
 *   out[1] sum V (S1 + E1 + S1b + E1b + C1 + C2) + sum_injury A C0
 *   out[2] sum V (S2 + E2 + S2b + E2b + C1 + C2)
 *   out[3] sum_injury A (E0 + C0)
 *   out[4] sum V ADP
 *   out[5] minimum over all cell and wall species
 *   out[6] count of non-finite values
 *   out[7] maximum theta_T
 * With the inhibitor extension (fields->ext) out[2] includes sum V E2,inh and
 * out[5], out[6] cover its two rows.
 * out is filled in every case; the call returns CLOT_ENONFINITE when out[6] > 0.
 * Errors: CLOT_EINVAL, CLOT_ECUDA, CLOT_ENONFINITE. */
int clot_diagnostics(clot_mesh *mesh, const clot_fields *fields, const clot_params *params,
                     double out[8], void *stream);
/* clot_diagnostics (the App. A/B invariants) without synchronising: the 8 values are copied, in stream
 * order, to out -- device memory or page-locked host memory of 8 doubles --
 * so that a time loop can read each step's diagnostics without stalling the
 * GPU.  Errors: CLOT_EINVAL, CLOT_ECUDA. */
int clot_diagnostics_async(clot_mesh *mesh, const clot_fields *fields, const clot_params *params, double *out,
                           void *stream);

/* Not part of the paper: the library's own failure reporting.
 * Read and clear the mesh's device status word (synchronous).  Returns CLOT_OK,
 * CLOT_ETIMEOUT (a bounded wait of an earlier call gave up and no call has
 * reported it yet: clot_eta_solve with iters, clot_species_step with
 * CLOT_SYNC_STATUS and this call each report a timeout once) or CLOT_ECUDA;
 * *iters (optional) receives the last eta iteration count. */
int clot_device_status(clot_mesh *mesh, int *last_eta_iters, void *stream);

/* ------------------------------------------------------------------
 * Ensembles: many independent channels advanced together (batched launches).
 * Each channel is a complete species-step problem (its own mesh, state,
 * fluxes, inlet values and dt).  Per step: one launch solves eta for every
 * channel (a block per channel, same stopping rule and prediction as
 * clot_species_step), one persistent launch runs the fused step over a work
 * list of (channel, 32x8 tile, plane) items of all channels.  The step
 * pattern repeats every 6 steps and is replayed from a CUDA graph between
 * ADP-release samples.  The model is that of clot_species_step (Sec. 3.2,
 * App. A-D); results equal running each channel alone up to the rounding
 * order of the eta reductions. */
typedef struct clot_ensemble clot_ensemble; /* opaque, library-owned */

typedef struct {
  clot_fields fields;   /* device state of the channel; scalars updated in place */
  clot_fluxes fluxes;   /* its face fluxes */
  const float *pmu_in, *s1_in, *s2_in; /* its inlet Dirichlet values [ny nz] */
  double dt;            /* its time step */
} clot_channel;

/* Autotuner result: chosen persistent grid (blocks) and work-list order
 * (0 channel by channel, 1 largest channels first, interleaved), its time per
 * fused-step launch, and every candidate timed. */
typedef struct {
  int grid, order;
  float ms;
  int ncand;
  int cand_grid[6], cand_order[6];
  float cand_ms[6];
} clot_tune_t;

/* Meshes of nchan channels (each as clot_mesh_create: App. C geometry, App. A
 * H_adh); all share dim (2 or 3).  Allocates the workspace of all channels.
 * Errors: CLOT_EINVAL, CLOT_ECUDA, CLOT_ENOMEM. */
int clot_ensemble_create(const clot_mesh_desc *descs, int nchan, clot_ensemble **out);
/* Free an ensemble (its meshes' geometry, App. C, and workspace); NULL is ignored. */
void clot_ensemble_destroy(clot_ensemble *ens);
/* clot_mesh_info of channel chan (App. A H_adh, App. C injury faces).  Errors: CLOT_EINVAL. */
int clot_ensemble_info(const clot_ensemble *ens, int chan, clot_mesh_info_t *out);
/* Advance every channel by nsteps species steps (Sec. 3.2, as
 * clot_species_step) of its own dt.  params: model constants and
 * numerics shared by all channels (its inlet pointers are not used).  The first
 * call with new fluxes or dt validates each channel as clot_species_step does.
 * Errors: CLOT_EINVAL, CLOT_ECUDA. */
int clot_ensemble_run(clot_ensemble *ens, clot_channel *chans, const clot_params *params, int nsteps,
                      void *stream);
/* clot_diagnostics (App. A/B invariants) of one channel (synchronous, out in
 * host memory).  Errors: CLOT_EINVAL, CLOT_ECUDA. */
int clot_ensemble_diagnostics(clot_ensemble *ens, int chan, const clot_fields *fields,
                              const clot_params *params, double out[8], void *stream);
/* Not part of the paper: launch configuration only (the arithmetic of the
 * Sec. 3.2 step is the same for every candidate).
 * Time `trials` fused-step launches for each candidate persistent grid
 * (1, 2, 3 x the resident blocks) and work-list order, keep the fastest for
 * later runs.  Leaves the channels' state unchanged (synchronous). */
int clot_ensemble_tune(clot_ensemble *ens, clot_channel *chans, const clot_params *params, int trials,
                       clot_tune_t *out, void *stream);
/* Not part of the paper: launch schedule only (each channel's arithmetic is
 * the same, results are bitwise equal).  Inside the replayed 6-step graph the
 * channels run as `chains` chains of consecutive channel indices holding
 * about equal shares of the cells, each on a graph branch of its own, so the
 * eta solve of one chain runs beside the fused step of another; chains = 1:
 * one branch, eta of all channels then the fused step of all.  Default 2.
 * Synchronises the device (the work list is rebuilt).
 * Errors: CLOT_EINVAL (chains outside 1 .. 4), CLOT_ECUDA. */
int clot_ensemble_set_chains(clot_ensemble *ens, int chains);

/* Per-kernel timing (library tracing).  Between clot_profile_begin and
 * clot_profile_end every kernel the library launches is bracketed by a pair of
 * CUDA events recorded on the launching stream (at most max_launches pairs;
 * later launches are only counted).  clot_profile_end synchronises the stream,
 * sums the event times per kernel kind and stops recording.  Not part of the
 * paper; used by bench.py to time the dominant kernel inside a real run.
 * Errors: CLOT_EINVAL (max_launches < 1), CLOT_ECUDA. */
typedef struct {
  int n_step, n_eta, n_sigma, n_other;  /* launches per kind (species step, eta solve, sigma, other) */
  double ms_step, ms_eta, ms_sigma, ms_other; /* summed event time of the timed launches */
  int timed;                             /* launches with event pairs */
  int eta_iters;                         /* CG iterations summed over the eta solves */
  int eta_accepted;                      /* eta solves that accepted the predicted eta */
  int eta_box;                           /* eta solves that corrected the predicted eta on a box (App. A, Eq. eta) */
  int eta_box_fallback;                  /* box corrections that missed the stopping rule and continued on the mesh */
} clot_profile_t;
/* Not part of the paper (tracing): start recording; see above. */
int clot_profile_begin(clot_mesh *mesh, int max_launches);
/* Not part of the paper (tracing): stop recording and fill *out (host). */
int clot_profile_end(clot_mesh *mesh, clot_profile_t *out, void *stream);

/* eta solve for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of clot_eta_solve.  Callers such as
 * code running under another framework's allocator (a memory-capped process),
 * real-time or monitoring loops that must not take cudaMalloc's implicit device
 * synchronisation, or tools that hold a state but no clot_mesh (whose workspace
 * is allocated by clot_mesh_create) get the same solve -- from theta_B of c
 * ([CLOT_NS][pitch], device) into eta ([ncell], device, warm start in, solution
 * out), stopping rule eta_tol / eta_maxit of params -- with no allocation: the
 * CG vectors, reduction partials and barrier words live in one static device
 * array of the library, about 16.1 MiB held by every GPU that loads it until
 * the process exits.  Limits: at most 1,048,576 cells (CLOT_EINVAL otherwise).
 * The first call on each device looks up that array's device address and
 * should be made before any stream capture; the address is kept for the life
 * of the process, so after a reset of the device's primary context
 * (cudaDeviceReset) the process must be restarted before the next call.  All
 * calls share the array, so calls that overlap on the GPU (different streams
 * or threads) race; order them on one stream.  iters (optional) synchronises,
 * receives the iteration count and reports CLOT_ETIMEOUT if a grid-barrier
 * wait (params->wait_s) ran out in this call or in an earlier call made with
 * iters NULL: such a call does not synchronise, so it cannot report the
 * timeout itself; the flag stays in the shared status words until a call with
 * iters reads and clears it.  Errors: CLOT_EINVAL, CLOT_ECUDA, CLOT_ETIMEOUT;
 * the reason is in clot_last_error(). */
int clot_eta_solve_noalloc(const clot_mesh_desc *desc, const float *c, int64_t pitch, float *eta,
                           const clot_params *params, int *iters, void *stream);

/* ------------------------------------------------------------------
 * Reaction surrogate: a learned replacement of the M_rxn RK4 reaction solve
 * (Sec. 3.2 step 2) over a step dt for cells off the adhesion layer and the
 * injury wall.  The reaction system it approximates is that of App. A
 * (platelet sources) and App. B (coagulation mass action); the paper itself
 * integrates it with RK4 only, so the surrogate is an extension.
 *
 * Definition (every entry point below follows it):
 *   features x[32]: x_s = log1p(max(c_s, 0) / scale_s) for the 15 species s,
 *     x_15 = g(eta) (App. A), x_16 = log(dt / 1e-5), x_{17+o} = sign(q_s)
 *     log1p(1e3 |q_s|) with q_s = E_s / (|c_s| + 1e-6 scale_s) the relative Euler
 *     rate of reacting species o (below), x_31 = 0;
 *   network: h1 = gelu(x W1 + b1), h2 = gelu(h1 W2 + b2), v = h2 W3 + b3 with
 *     W1 32x64, W2 64x64, W3 64x16 stored [in][out] row-major, and
 *     gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)));
 *   increment: E_s = dt f_s(c) (explicit Euler on the App. A/B right-hand side,
 *     H_adh = 0, no wall) for the 14 reacting species s (ADP excluded) in row
 *     order, o = 0..13; rho = max_s |E_s| / (|c_s| + 1e-6 scale_s), the relative
 *     Euler change (a stiffness measure); dc_s = E_s + rho v_o (|E_s| + 1e-6 scale_s);
 *     v_14, v_15 unused.  A zero network is explicit Euler; a cell with f = 0
 *     (an equilibrium, which RK4 keeps) has rho = 0 and dc = 0;
 *   training target: v_o = (dc_RK4_s - E_s) / (rho (|E_s| + 1e-6 scale_s))
 *     (0 where rho = 0), of order one since RK4 corrects Euler by O(rho);
 *     loss = mean of (v - target)^2 over the batch and o = 0..13.
 * Matrix products take bfloat16 operands (x, weights, h1, h2; in the backward
 * pass the residual v - target and the pre-activation gradients) and
 * accumulate in FP32 on the tensor cores; biases, pre-activations and gelu
 * stay FP32.  The parameters are kept in FP32 (the Adam master copy). */
#define CLOT_MLP_NPARAM 7312 /* 32*64 + 64 + 64*64 + 64 + 64*16 + 16 */
#define CLOT_MLP_OFF_W1 0
#define CLOT_MLP_OFF_B1 2048
#define CLOT_MLP_OFF_W2 2112
#define CLOT_MLP_OFF_B2 6208
#define CLOT_MLP_OFF_W3 6272
#define CLOT_MLP_OFF_B3 7296

/* Tensor-core engines of the network (same arithmetic, both sm_103a):
 *   CLOT_MLP_ENGINE_MMA: warp-level mma.sync m16n8k16, 32 cells per warp, the
 *     accumulators of a layer chained in registers into the next (default);
 *   CLOT_MLP_ENGINE_TCGEN05: tcgen05.mma of M 128 rows per CTA with the
 *     accumulators in tensor memory, read back per row by tcgen05.ld. */
#define CLOT_MLP_ENGINE_MMA 0
#define CLOT_MLP_ENGINE_TCGEN05 1

typedef struct {
  float *w;                /* device, [CLOT_MLP_NPARAM] FP32 parameters packed W1 b1 W2 b2 W3 b3 */
  float scale[CLOT_NS];    /* host values: per-species concentration scale (> 0) */
  int engine;              /* CLOT_MLP_ENGINE_*, inference only (training uses mma.sync) */
} clot_mlp;

/* Training pairs.  c0: device [CLOT_NS][pitch] states of n cells off the
 * adhesion layer; eta: device [n].  For each cell the RK4 reaction solve over
 * dt (params->M_rxn steps of dt / M_rxn, the integrator of clot_reaction_step,
 * with H_adh = 0 and no wall) gives the increment dc_RK4, summed step by step
 * so that it does not cancel against c0.  Writes x: device [n][32] features
 * and y: device [n][16] targets (columns 14, 15 zero), FP32.  params supplies
 * the reaction constants (App. E); its inlet pointers are not used.
 * Errors: CLOT_EINVAL, CLOT_ECUDA. */
int clot_surrogate_pairs(const clot_params *params, const clot_mlp *mlp, const float *c0, const float *eta,
                         int64_t n, int64_t pitch, double dt, float *x, float *y, void *stream);
/* An extension, not in the paper (the surrogate of Sec. 3.2 step 2 defined above).
 * Network output for n feature rows: x device [n][32] FP32, out device
 * [n][16] FP32 (the inference kernel's arithmetic).  Errors: CLOT_EINVAL, CLOT_ECUDA. */
int clot_surrogate_forward(const clot_mlp *mlp, const float *x, int64_t n, float *out, void *stream);
/* An extension, not in the paper (surrogate training).  FP32 device floats of
 * workspace the gradient and training calls need for a batch of n rows. */
int64_t clot_surrogate_workspace(int64_t n);
/* An extension, not in the paper (surrogate training).
 * Gradient of the loss over the n rows (x [n][32], y [n][16], device) into
 * grad (device [CLOT_MLP_NPARAM]) and the loss into *loss (device float, may
 * be NULL).  work: device, clot_surrogate_workspace(n) floats.
 * Errors: CLOT_EINVAL, CLOT_ECUDA. */
int clot_surrogate_grad(const clot_mlp *mlp, const float *x, const float *y, int64_t n, float *work,
                        int64_t work_floats, float *grad, float *loss, void *stream);
/* An extension, not in the paper (surrogate training).
 * nsteps Adam steps (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, step
 * numbers t0 + 1 .. t0 + nsteps) on mlp->w with learning rate lr; step s uses
 * rows [(s batch) mod n, + batch) of x, y (n a multiple of batch).  m, v:
 * device [CLOT_MLP_NPARAM] moment buffers (zero before the first step); loss:
 * device [nsteps] (may be NULL) receives each step's batch loss before its
 * update.  work: clot_surrogate_workspace(batch) floats.
 * Errors: CLOT_EINVAL, CLOT_ECUDA. */
int clot_surrogate_train(const clot_mlp *mlp, float *m, float *v, int t0, float lr, const float *x,
                         const float *y, int64_t n, int64_t batch, int nsteps, float *work, int64_t work_floats,
                         float *loss, void *stream);
/* Reaction solve of Sec. 3.2 step 2 (App. A/B system) over dt = h nsub like
 * clot_reaction_step, with the surrogate (an extension, not in the paper)
 * where it applies: a cell off the adhesion layer and the injury wall takes
 * c + dc when the indicator max_s |dc_s| / (|c_s| + 1e-6 scale_s) over the
 * reacting species is at most tol (and finite); every other cell takes the
 * RK4 solve (nsub steps of h, as clot_reaction_step).  Two launches: the
 * network pass, which also lists the other cells, then RK4 over that list.
 * flag (device [ncell] bytes, may be NULL) receives 0 surrogate, 1 indicator
 * fallback, 2 region fallback per cell; counts (host [3], may be NULL;
 * synchronises) receives the number of cells of each kind.  fields.bound_acc
 * gains the newly bound platelets of every cell.  Uses the mesh's eta-solver
 * workspace as the list.  Errors: CLOT_EINVAL, CLOT_ECUDA. */
int clot_surrogate_infer(clot_mesh *mesh, clot_fields *fields, const clot_params *params, const clot_mlp *mlp,
                         double h, int nsub, float tol, uint8_t *flag, int64_t counts[3], void *stream);

/* The species step of Sec. 3.2 with its reaction solve (step 2, the App. A/B
 * system) taken by the surrogate where it applies -- an extension, not in the
 * paper.  Per step: the eta solve (App. A, Eq. eta) and the sigma sample as in
 * clot_species_step, the fused transport pass of clot_species_step with its
 * reaction switched off, then the reaction over dt as clot_surrogate_infer
 * does it (the network for cells off the adhesion layer and the injury wall
 * whose indicator is at most tol, M_rxn RK4 steps of dt / M_rxn for every
 * other cell, in place).  Two more sweeps of the state than the plain step:
 * the network's weights and 64-wide accumulators do not fit beside the fused
 * pass's 128 registers and ring of staged planes.  No eta prediction (each
 * solve warm-starts from the previous eta).  mlp, tol: as clot_surrogate_infer;
 * counts (host [3], may be NULL; synchronises) receives the surrogate,
 * indicator-fallback and region-fallback cells of the last step.  Uses the
 * mesh's eta-solver workspace as the fallback list.  Errors: CLOT_EINVAL
 * (also with CLOT_HEUN, CLOT_STRANG or CLOT_NO_REACTION), CLOT_ECUDA. */
int clot_species_step_surrogate(clot_mesh *mesh, clot_fields *fields, const clot_fluxes *fluxes,
                                const clot_params *params, const clot_mlp *mlp, float tol, double dt, int nsteps,
                                int64_t counts[3], void *stream);

/* Not part of the paper: one-line description of the last error on this thread. */
const char *clot_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CLOT_H */

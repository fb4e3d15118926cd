/*
 * clot_oracle.c -- plain FP64 CPU oracle for the clotFoam species step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement
 * of what the GPU path computes.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load it.  It shares no code,
 * header, table or helper with the CUDA library; neither side includes the other.
 *
 * Citations name the sections and equations of the clotFoam paper
 * (Montgomery, Municchi, Leiderman, "clotFoam: An open-source framework to
 * simulate blood clot formation under arterial flow", SoftwareX):
 *   Sec. 2        Hill activation A(c) = k c/(c*+c); ADP equation; sigma_release
 *   Sec. 3.2      fractional step (transport over dt, then M_rxn RK4 reaction
 *                 solves of h = dt/M_rxn); downwind / localMax interpolation of
 *                 theta_T for the hindered fluxes; trapezoid rule for sigma
 *   App. A        platelet aggregation (Eqs. for P^{m,u}, P^{m,a}, P^{b,a},
 *                 P^{b,se}), W(theta_T), H_adh, eta equation, g(eta)
 *   App. B        reduced coagulation (12 species) incl. the injury-wall flux BCs
 *   App. C        boundary-condition table; parabolic inlet velocity
 *   App. D        discretisation table (van Leer, Gauss linear orthogonal)
 *   App. E        parameter values
 * Readings of points the paper leaves open (explicit Euler transport at fixed
 * dt, wall reaction coupled inside the RK4 stages through a Robin closure for
 * the wall value of S1, g = 0 below eta_t, W with theta_T clamped to [0,1],
 * sigma sampled every sigma_dt, etc.) are the ones listed in the design notes.
 * Two options state alternatives beside those defaults: OR_TRANSPORT_RK2
 * (Heun's method for the transport, second order in time like the paper's
 * Crank-Nicolson, App. D) and OR_WALL_LAGGED (the wall reaction placed the way
 * the paper's solver places it: mixed transport conditions with E0, C0 of the
 * previous step, then the E0/C0 ODEs; App. B, App. C table).
 *
 * The inhibitor extension (the paper's example of adding a species: a
 * fluid-phase inhibitor I with I + E2 -> E2,inh at rate kI I E2, Sec.
 * "Adapting the framework for different clotting models") runs when the
 * fields carry its two rows (or_fields.ext): transported like the other
 * coagulation species and reacted inside the same RK4 stages.
 * Every function computes in double precision with straightforward loops.
 * Loops over independent cells carry OpenMP pragmas; the face loops of the
 * transport run the faces along one axis in order inside each row (so every
 * cell receives its face fluxes in the same order as a serial sweep), and the
 * CG dot products stay serial: the result does not depend on the number of
 * threads, bit for bit (or_set_threads; tested).
 * Parity status: all functions are pinned by the -m "not gpu" tests
 * (tests/test_oracle_*.py) against closed forms, invariants, special cases
 * and an independent stiff ODE integrator.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_NS 15
enum { PMU = 0, PMA, PBA, PBSE, ADP, S1, S2, E1, E2, S1B, S2B, E1B, E2B, C1, C2 };
/* The extensibility example of the paper (Sec. "Adapting the framework for
 * different clotting models"): a fluid-phase inhibitor I binding fluid-phase
 * thrombin for good, I + E2 -> E2,inh at rate kI I E2.  With it the state has
 * two more fluid-phase rows after the 15, I and E2,inh, transported like the
 * other coagulation species (D_chem; I with a Dirichlet inlet value I_in,
 * E2,inh zero-gradient). */
#define OR_NX 17
enum { INH = 15, E2I = 16 };

/* flags */
#define OR_NO_TRANSPORT 1
#define OR_NO_REACTION 2
#define OR_CLOSED_ENDS 4 /* inlet and outlet behave as zero-flux walls */
#define OR_NO_ETA 8      /* keep eta as given (no solve) */
#define OR_NO_SIGMA 16   /* never sample the ADP release history */
#define OR_TRANSPORT_RK2 32 /* transport by Heun's method (SSP-RK2) instead of forward Euler */
#define OR_WALL_LAGGED 64   /* injury-wall exchange as a lagged transport boundary condition */
#define OR_STRANG 128       /* Strang splitting: reaction over dt/2, transport over dt, reaction over dt/2 */

typedef struct {
  int dim, nx, ny, nz;
  double hx, hy, hz;
  double inj_x0, inj_x1, inj_z0, inj_z1;
  double p_diam;
} or_mesh;

typedef struct {
  double Pmax, kadh, kcohPmax, eta_t, eta_star, L_eta;
  double k_adp, adp_star, k_e2, e2_star;
  double A_hat, sigma_tf, sigma_dt;
  double D_P, D_adp, D_chem;
  double N1, N2, N_A;
  double kC0p, kC0m, kC0cat, kC1p, kC1m, kC1cat, kC2p, kC2m, kC2cat;
  double kS1p, kS1m, kE1p, kE1m, kS2p, kS2m, kE2p, kE2m;
  double eta_tol;
  double kI, I_in;      /* inhibitor extension: association rate, inlet value */
  int M_rxn, limiter, flags, eta_maxit;
} or_params;

typedef struct {
  double *c;            /* [15][ncell] */
  double *e0, *c0;      /* [ninj] */
  double *eta, *sigma;  /* [ncell] */
  double *hist;         /* [ntau+1][ncell] ring of newly-bound rates */
  double *thetaB_last;  /* [ncell] theta_B at the previous sample */
  double t, t_last;     /* t_last < 0: history not initialised yet */
  int n_samples, head;
  double *ext;          /* [2][ncell] I, E2,inh of the inhibitor extension, or NULL (the paper's model) */
} or_fields;

typedef struct {
  const double *fx, *fy, *fz;              /* signed face fluxes, mm^3/s */
  const double *pmu_in, *s1_in, *s2_in;    /* inlet Dirichlet values [ny*nz] */
} or_inputs;

/* ------------------------------------------------------------------ mesh */

static long ncell_of(const or_mesh *m) { return (long)m->nx * m->ny * m->nz; }

/* Threads of the parallel loops (n < 1: all the host offers); returns the count in use. */
int or_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  else omp_set_num_threads(omp_get_num_procs());
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
static long cidx(const or_mesh *m, int i, int j, int k) {
  return (long)i + (long)m->nx * ((long)j + (long)m->ny * k);
}
static int in_mesh(const or_mesh *m, int i, int j, int k) {
  return i >= 0 && i < m->nx && j >= 0 && j < m->ny && k >= 0 && k < m->nz;
}

/* Injury faces (App. B "on dOmega_inj", Sec. 3.1 injuryWalls): floor faces
 * y = 0 whose centre lies inside [inj_x0,inj_x1] x [inj_z0,inj_z1] (z test only
 * in 3D).  Enumerated k-major, then i.  Returns the count; fills fi/fk if given. */
int or_injury_faces(const or_mesh *m, int *fi, int *fk) {
  int n = 0;
  for (int k = 0; k < m->nz; ++k) {
    double zc = (k + 0.5) * m->hz;
    if (m->dim == 3 && (zc < m->inj_z0 || zc > m->inj_z1)) continue;
    for (int i = 0; i < m->nx; ++i) {
      double xc = (i + 0.5) * m->hx;
      if (xc < m->inj_x0 || xc > m->inj_x1) continue;
      if (fi) fi[n] = i;
      if (fk) fk[n] = k;
      ++n;
    }
  }
  return n;
}

/* Adhesion region H_adh (App. A, Sec. 3.1): 1 for cells whose centre lies over
 * the injury patch and within P_diam of the injured wall y = 0, else 0. */
void or_hadh(const or_mesh *m, double *H) {
  for (int k = 0; k < m->nz; ++k)
    for (int j = 0; j < m->ny; ++j)
      for (int i = 0; i < m->nx; ++i) {
        double xc = (i + 0.5) * m->hx, yc = (j + 0.5) * m->hy, zc = (k + 0.5) * m->hz;
        int over = xc >= m->inj_x0 && xc <= m->inj_x1;
        if (m->dim == 3) over = over && zc >= m->inj_z0 && zc <= m->inj_z1;
        H[cidx(m, i, j, k)] = (over && yc <= m->p_diam) ? 1.0 : 0.0;
      }
}

/* ------------------------------------------------------ model functions */

/* Hindered transport W(theta_T) = tanh(pi (1 - theta_T)) (App. A); theta_T
 * clamped to [0,1] so W stays in [0, tanh(pi)]. */
double or_W(double theta) {
  if (theta < 0) theta = 0;
  if (theta > 1) theta = 1;
  return tanh(M_PI * (1.0 - theta));
}

/* Binding affinity g(eta) (App. A) with g0 chosen so that g(1) = 1; zero at
 * and below the threshold eta_t. */
double or_g(const or_params *p, double eta) {
  double et = p->eta_t, es = p->eta_star;
  if (eta <= et) return 0.0;
  double g0 = (es * es * es + (1 - et) * (1 - et) * (1 - et)) / ((1 - et) * (1 - et) * (1 - et));
  double u = eta - et;
  return g0 * u * u * u / (es * es * es + u * u * u);
}

/* ADP release kernel R(tau) = pi^{-1/2} exp(-(tau-3)^2) (Sec. 2, Eq. ADP_source). */
double or_R(double tau) { return exp(-(tau - 3.0) * (tau - 3.0)) / sqrt(M_PI); }

/* Reaction right-hand side of one cell (App. A platelet sources, App. B mass
 * action).  For a cell on an injury face (wall != 0) the wall exchange with
 * the face species E0, C0 is included: S1 is consumed at rate (A/V) J with
 * J = kC0+ S1_w E0 - kC0- C0, E1 is produced at (A/V) kC0cat C0 (App. B BCs),
 * and E0, C0 follow their ODEs with the same wall value S1_w.  S1_w is the
 * Robin closure D (S1 - S1_w)/delta = J, delta = half the wall-normal cell size
 * (Dd = D/delta). */
void or_rhs(const or_params *p, const double *y, double H, double g, int wall,
            double e0, double c0, double aV, double Dd, double *f, double *fe0,
            double *fc0) {
  const double Pmu = y[PMU], Pma = y[PMA], Pba = y[PBA], Pbse = y[PBSE];
  const double adp = y[ADP], s1 = y[S1], s2 = y[S2], e1 = y[E1], e2 = y[E2];
  const double s1b = y[S1B], s2b = y[S2B], e1b = y[E1B], e2b = y[E2B];
  const double c1 = y[C1], c2 = y[C2];

  /* App. A: adhesion k_adh H_adh (Pmax - P^{b,se}); activation A1([ADP]) + A2(E2)
   * with Hill functions (Sec. 2); cohesion k_coh g(eta) Pmax. */
  double adh = p->kadh * H * (p->Pmax - Pbse);
  double A1 = p->k_adp * adp / (p->adp_star + adp);
  double A2 = p->k_e2 * e2 / (p->e2_star + e2);
  double coh = p->kcohPmax * g;
  f[PMU] = -adh * Pmu - (A1 + A2) * Pmu;
  f[PMA] = -adh * Pma + (A1 + A2) * Pmu - coh * Pma;
  f[PBA] = -adh * Pba + coh * Pma;
  f[PBSE] = adh * (Pmu + Pma + Pba);
  f[ADP] = 0.0; /* ADP has only the release source, added in transport (Sec. 3.2) */

  /* App. B: free binding sites of type 1 and 2 on bound platelets. */
  double sites = Pba + Pbse;
  double free1 = p->N1 / p->N_A * sites - (s1b + e1b + c1 + c2);
  double free2 = p->N2 / p->N_A * sites - (s2b + e2b + c1 + c2);
  f[S1] = -p->kS1p * free1 * s1 + p->kS1m * s1b;
  f[S2] = -p->kS2p * free2 * s2 + p->kS2m * s2b;
  f[E1] = -p->kE1p * free1 * e1 + p->kE1m * e1b;
  f[E2] = -p->kE2p * free2 * e2 + p->kE2m * e2b;
  f[S1B] = p->kS1p * free1 * s1 - p->kS1m * s1b - p->kC2p * s1b * e2b + p->kC2m * c2;
  f[S2B] = p->kS2p * free2 * s2 - p->kS2m * s2b - p->kC1p * s2b * e1b + p->kC1m * c1;
  f[E1B] = p->kE1p * free1 * e1 - p->kE1m * e1b - p->kC1p * s2b * e1b +
           (p->kC1m + p->kC1cat) * c1 + p->kC2cat * c2;
  f[E2B] = p->kE2p * free2 * e2 - p->kE2m * e2b - p->kC2p * s1b * e2b +
           (p->kC2m + p->kC2cat) * c2 + p->kC1cat * c1;
  f[C1] = p->kC1p * s2b * e1b - (p->kC1m + p->kC1cat) * c1;
  f[C2] = p->kC2p * s1b * e2b - (p->kC2m + p->kC2cat) * c2;

  if (wall) {
    double s1w = (Dd * s1 + p->kC0m * c0) / (Dd + p->kC0p * e0);
    double J = p->kC0p * s1w * e0 - p->kC0m * c0;
    f[S1] += -aV * J;
    f[E1] += aV * p->kC0cat * c0;
    *fe0 = -p->kC0p * s1w * e0 + (p->kC0m + p->kC0cat) * c0;
    *fc0 = p->kC0p * s1w * e0 - (p->kC0m + p->kC0cat) * c0;
  }
}

/* The inhibitor extension's reaction term added to a right-hand side of the
 * extended state: fluid-phase thrombin and I each lose kI I E2, E2,inh gains it
 * (the paper's reaction rate -kI I E2 for I, Sec. "Adapting the framework"). */
static void inhibit_rhs(const or_params *p, const double *y, double *f) {
  double r = p->kI * y[INH] * y[E2];
  f[E2] -= r;
  f[INH] = -r;
  f[E2I] = r;
}

/* One classic RK4 step of size h on a cell of the extended state y[OR_NX]
 * (and its wall face, if any); ext = 0 leaves y[INH], y[E2I] untouched.
 * Sec. 3.2: the coupled reaction system is advanced with RK4. */
static void rk4_cell_x(const or_params *p, double *y, int ext, double H, double g, int wall,
                       double *e0, double *c0, double aV, double Dd, double h) {
  double k[4][OR_NX], ke0[4] = {0}, kc0[4] = {0}, yt[OR_NX];
  double e0t = wall ? *e0 : 0, c0t = wall ? *c0 : 0;
  const double a[4] = {0.0, 0.5, 0.5, 1.0};
  const int n = ext ? OR_NX : OR_NS;
  for (int s = 0; s < 4; ++s) {
    for (int q = 0; q < n; ++q) yt[q] = y[q] + (s ? a[s] * h * k[s - 1][q] : 0.0);
    if (wall) {
      e0t = *e0 + (s ? a[s] * h * ke0[s - 1] : 0.0);
      c0t = *c0 + (s ? a[s] * h * kc0[s - 1] : 0.0);
    }
    or_rhs(p, yt, H, g, wall, e0t, c0t, aV, Dd, k[s], &ke0[s], &kc0[s]);
    if (ext) inhibit_rhs(p, yt, k[s]);
  }
  for (int q = 0; q < n; ++q)
    y[q] += h / 6.0 * (k[0][q] + 2 * k[1][q] + 2 * k[2][q] + k[3][q]);
  if (wall) {
    *e0 += h / 6.0 * (ke0[0] + 2 * ke0[1] + 2 * ke0[2] + ke0[3]);
    *c0 += h / 6.0 * (kc0[0] + 2 * kc0[1] + 2 * kc0[2] + kc0[3]);
  }
}

/* One classic RK4 step of size h on a cell of the paper's model (15 species). */
void or_rk4_cell(const or_params *p, double *y, double H, double g, int wall,
                 double *e0, double *c0, double aV, double Dd, double h) {
  double yx[OR_NX];
  for (int q = 0; q < OR_NS; ++q) yx[q] = y[q];
  rk4_cell_x(p, yx, 0, H, g, wall, e0, c0, aV, Dd, h);
  for (int q = 0; q < OR_NS; ++q) y[q] = yx[q];
}

/* ------------------------------------------------------------- eta solve */

/* y = (I - (L_eta^2/4) lap_h) x with zero-flux (Neumann) boundaries: a missing
 * neighbour contributes no difference (App. A, Eq. eta). */
void or_apply_eta_op(const or_mesh *m, const or_params *p, const double *x, double *y) {
  double cl = p->L_eta * p->L_eta / 4.0;
  double h[3] = {m->hx, m->hy, m->hz};
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < m->nz; ++k)
    for (int j = 0; j < m->ny; ++j)
      for (int i = 0; i < m->nx; ++i) {
        long P = cidx(m, i, j, k);
        double lap = 0.0;
        for (int a = 0; a < m->dim; ++a)
          for (int s = -1; s <= 1; s += 2) {
            int ii = i + (a == 0) * s, jj = j + (a == 1) * s, kk = k + (a == 2) * s;
            if (!in_mesh(m, ii, jj, kk)) continue;
            lap += (x[cidx(m, ii, jj, kk)] - x[P]) / (h[a] * h[a]);
          }
        y[P] = x[P] - cl * lap;
      }
}

/* Solve (I - L^2/4 lap) eta = b by conjugate gradients in FP64, starting from
 * the eta passed in, to ||r||_2 <= tol ||b||_2.  Returns iterations used. */
int or_eta_solve(const or_mesh *m, const or_params *p, const double *b, double *eta,
                 double tol, int maxit) {
  long n = ncell_of(m);
  double bb = 0;
  for (long q = 0; q < n; ++q) bb += b[q] * b[q];
  if (bb == 0.0) {
    for (long q = 0; q < n; ++q) eta[q] = 0.0;
    return 0;
  }
  double *r = malloc(n * sizeof(double)), *pp = malloc(n * sizeof(double));
  double *qv = malloc(n * sizeof(double));
  or_apply_eta_op(m, p, eta, qv);
  double rr = 0;
  for (long q = 0; q < n; ++q) {
    r[q] = b[q] - qv[q];
    pp[q] = r[q];
    rr += r[q] * r[q];
  }
  int it = 0;
  while (it < maxit && sqrt(rr) > tol * sqrt(bb)) {
    or_apply_eta_op(m, p, pp, qv);
    double pq = 0;
    for (long q = 0; q < n; ++q) pq += pp[q] * qv[q];
    double alpha = rr / pq, rr2 = 0;
#pragma omp parallel for schedule(static)
    for (long q = 0; q < n; ++q) {
      eta[q] += alpha * pp[q];
      r[q] -= alpha * qv[q];
    }
    for (long q = 0; q < n; ++q) rr2 += r[q] * r[q];
    double beta = rr2 / rr;
#pragma omp parallel for schedule(static)
    for (long q = 0; q < n; ++q) pp[q] = r[q] + beta * pp[q];
    rr = rr2;
    ++it;
  }
  free(r);
  free(pp);
  free(qv);
  return it;
}

/* -------------------------------------------------------- ADP release */

static int ntau_of(const or_params *p) { return (int)floor(p->sigma_tf / p->sigma_dt + 0.5); }

/* Take one sample of the newly-bound platelet rate and recompute sigma_release
 * (Sec. 3.2, Eq. sigma_disc):
 *   r(t_n) = Pmax (theta_B,n - theta_B,last) / (t_n - t_last)
 *   sigma(t_n) = sum_{k=0}^{N_tau-1} A_hat dtau/2 { R(t_n - tau_k) r(tau_k)
 *                                                + R(t_n - tau_{k+1}) r(tau_{k+1}) }
 * with tau_k = t_n - tau_f + k dtau; samples older than the stored history are 0. */
void or_sigma_sample(const or_mesh *m, const or_params *p, or_fields *F) {
  long n = ncell_of(m);
  int ntau = ntau_of(p), nslot = ntau + 1;
  double dtau = p->sigma_dt, tf = p->sigma_tf, tn = F->t;
  int head = (F->n_samples == 0) ? 0 : (F->head + 1) % nslot;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < n; ++q) {
    double thB = (F->c[PBA * n + q] + F->c[PBSE * n + q]) / p->Pmax;
    F->hist[(long)head * n + q] = p->Pmax * (thB - F->thetaB_last[q]) / (tn - F->t_last);
    F->thetaB_last[q] = thB;
  }
  F->head = head;
  F->n_samples += 1;
  F->t_last = tn;
#pragma omp parallel for schedule(static)
  for (long q = 0; q < n; ++q) {
    double s = 0.0;
    for (int k = 0; k < ntau; ++k) {
      double tk = tn - tf + k * dtau, tk1 = tn - tf + (k + 1) * dtau;
      int lag_k = ntau - k, lag_k1 = ntau - k - 1; /* samples back from the newest */
      double rk = 0.0, rk1 = 0.0;
      if (lag_k < F->n_samples) rk = F->hist[(long)((head - lag_k + nslot * 4) % nslot) * n + q];
      if (lag_k1 < F->n_samples) rk1 = F->hist[(long)((head - lag_k1 + nslot * 4) % nslot) * n + q];
      s += p->A_hat * dtau / 2.0 * (or_R(tn - tk) * rk + or_R(tn - tk1) * rk1);
    }
    F->sigma[q] = s;
  }
}

/* ----------------------------------------------------------- transport */

static int is_transported(int s) {
  return s == PMU || s == PMA || s == ADP || s == S1 || s == S2 || s == E1 || s == E2 || s == INH || s == E2I;
}
/* Row s of the state: the 15 species in c, the extension's two in ext. */
static const double *row_of(const double *c, const double *ext, int s, long n) {
  return s < OR_NS ? c + (long)s * n : ext + (long)(s - OR_NS) * n;
}
static double diffusivity(const or_params *p, int s) {
  if (s == PMU || s == PMA) return p->D_P;
  if (s == ADP) return p->D_adp;
  return p->D_chem;
}

/* Face value of an advected species: van Leer limited upwind-biased
 * interpolation (App. D, "Gauss vanLeer"), psi(r) = (r + |r|)/(1 + |r|),
 * r = (cU - cUU)/(cD - cU), c_f = cU + psi (cD - cU)/2. */
double or_face_value(double cUU, double cU, double cD, int limiter) {
  if (limiter == 0) return cU;
  double den = cD - cU;
  if (den == 0.0) return cU;
  double r = (cU - cUU) / den;
  double psi = (r + fabs(r)) / (1.0 + fabs(r));
  return cU + 0.5 * psi * den;
}

/* Explicit finite-volume transport over dt (Sec. 3.2 step 1, App. A/B ADR
 * fluxes, App. C BCs, App. D schemes) for the transported species, writing
 * the post-transport state to cs.  Platelet fluxes are multiplied by W of the
 * downwind theta_T (advection) and W of the larger theta_T of the two sides
 * (diffusion, localMax).  ADP receives dt * sigma (Sec. 3.2). */
static void transport_x(const or_mesh *m, const or_params *p, const or_inputs *in, const double *c,
                        const double *ext, const double *sigma, double dt, double *cs, double *ext_out);

void or_transport(const or_mesh *m, const or_params *p, const or_inputs *in,
                  const double *c, const double *sigma, double dt, double *cs) {
  transport_x(m, p, in, c, NULL, sigma, dt, cs, NULL);
}

/* The transport of the state with the extension's rows I, E2,inh when ext is
 * not NULL (written to ext_out). */
static void transport_x(const or_mesh *m, const or_params *p, const or_inputs *in, const double *c,
                        const double *ext, const double *sigma, double dt, double *cs, double *ext_out) {
  long n = ncell_of(m);
  const int nsp = ext ? OR_NX : OR_NS;
  int nn[3] = {m->nx, m->ny, m->nz};
  double h[3] = {m->hx, m->hy, m->hz};
  double V = m->hx * m->hy * m->hz;
  double *thT = malloc(n * sizeof(double));
  double *div = calloc((size_t)nsp * n, sizeof(double));
#pragma omp parallel for schedule(static)
  for (long q = 0; q < n; ++q)
    thT[q] = (c[PMU * n + q] + c[PMA * n + q] + c[PBA * n + q] + c[PBSE * n + q]) / p->Pmax;

  for (int a = 0; a < m->dim; ++a) {
    double area = V / h[a];
    const double *Fa = a == 0 ? in->fx : a == 1 ? in->fy : in->fz;
    int fn[3] = {m->nx, m->ny, m->nz};
    fn[a] += 1;
    /* one line of faces along axis a per (u, v) position of the other two
     * axes; a line only touches its own cells, and within it the faces go in
     * order, so each cell sums its face fluxes in the serial order */
    const int u = a == 0 ? 1 : 0, v = a == 2 ? 1 : 2;
    const long nlines = (long)fn[u] * fn[v];
#pragma omp parallel for schedule(static)
    for (long line = 0; line < nlines; ++line)
      for (int w = 0; w < fn[a]; ++w) {
          int ix[3];
          ix[u] = (int)(line % fn[u]);
          ix[v] = (int)(line / fn[u]);
          ix[a] = w;
          const int i = ix[0], j = ix[1], k = ix[2];
          long fidx = (long)i + (long)fn[0] * ((long)j + (long)fn[1] * k);
          double F = Fa[fidx];
          int q = a == 0 ? i : a == 1 ? j : k; /* face position along the axis */
          int il = i - (a == 0), jl = j - (a == 1), kl = k - (a == 2);
          int hasL = q > 0, hasH = q < nn[a];
          long L = hasL ? cidx(m, il, jl, kl) : -1, Hc = hasH ? cidx(m, i, j, k) : -1;

          if (hasL && hasH) { /* interior face, flux counted L -> H */
            long U = F >= 0 ? L : Hc, D = F >= 0 ? Hc : L;
            int iu = F >= 0 ? il - (a == 0) : i + (a == 0);
            int ju = F >= 0 ? jl - (a == 1) : j + (a == 1);
            int ku = F >= 0 ? kl - (a == 2) : k + (a == 2);
            long UU = in_mesh(m, iu, ju, ku) ? cidx(m, iu, ju, ku) : U;
            for (int s = 0; s < nsp; ++s) {
              if (!is_transported(s)) continue;
              const double *cc = row_of(c, ext, s, n);
              int hind = (s == PMU || s == PMA);
              double cf = or_face_value(cc[UU], cc[U], cc[D], p->limiter);
              double Wa = hind ? or_W(thT[D]) : 1.0;
              double Wd = hind ? or_W(fmax(thT[L], thT[Hc])) : 1.0;
              double phi = Wa * F * cf - Wd * diffusivity(p, s) * area / h[a] * (cc[Hc] - cc[L]);
              div[(long)s * n + L] += phi;
              div[(long)s * n + Hc] -= phi;
            }
            continue;
          }

          /* boundary face */
          long P = hasL ? L : Hc;
          double nout = hasL ? 1.0 : -1.0; /* outward normal along +axis if the cell is on the low side */
          double Fout = nout * F;
          int inlet = (a == 0 && q == 0), outlet = (a == 0 && q == nn[0]);
          if (!(inlet || outlet)) continue; /* walls: no advective (F = 0) and no diffusive flux */
          if (p->flags & OR_CLOSED_ENDS) continue;
          int jb = j, kb = k;
          for (int s = 0; s < nsp; ++s) {
            if (!is_transported(s)) continue;
            const double *cc = row_of(c, ext, s, n);
            int hind = (s == PMU || s == PMA);
            int dirichlet = inlet && (s == PMU || s == S1 || s == S2 || s == INH);
            double cb = cc[P];
            if (dirichlet) {
              long b = (long)jb + (long)m->ny * kb;
              cb = s == PMU ? in->pmu_in[b] : s == S1 ? in->s1_in[b] : s == S2 ? in->s2_in[b] : p->I_in;
            }
            double thb = thT[P];
            if (inlet) {
              long b = (long)jb + (long)m->ny * kb;
              thb = (in->pmu_in[b] + c[PMA * n + P] + c[PBA * n + P] + c[PBSE * n + P]) / p->Pmax;
            }
            double Wa = hind ? or_W(Fout > 0 ? thb : thT[P]) : 1.0;
            double Wd = hind ? or_W(fmax(thT[P], thb)) : 1.0;
            double out = Wa * Fout * cb;
            if (dirichlet) out -= Wd * diffusivity(p, s) * area * (cb - cc[P]) / (0.5 * h[a]);
            div[(long)s * n + P] += out;
          }
        }
  }
#pragma omp parallel for collapse(2) schedule(static)
  for (int s = 0; s < nsp; ++s)
    for (long q = 0; q < n; ++q) {
      double v = row_of(c, ext, s, n)[q];
      if (is_transported(s)) v -= dt / V * div[(long)s * n + q];
      if (s == ADP && sigma) v += dt * sigma[q];
      if (s < OR_NS) cs[(long)s * n + q] = v;
      else ext_out[(long)(s - OR_NS) * n + q] = v;
    }
  free(thT);
  free(div);
}

/* --------------------------------------------------------------- step */

/* Pointwise reaction solve: nsub RK4 steps of size h on every cell, with
 * g(eta) from the eta field and H_adh from the mesh (Sec. 3.2 step 2); the
 * injury-wall exchange inside the stages when couple_wall. */
static void reaction_impl(const or_mesh *m, const or_params *p, double *c, double *ext, double *e0, double *c0,
                          const double *eta, double h, int nsub, int couple_wall) {
  long n = ncell_of(m);
  double *H = malloc(n * sizeof(double));
  or_hadh(m, H);
  int ninj = or_injury_faces(m, NULL, NULL);
  int *fi = malloc((ninj + 1) * sizeof(int)), *fk = malloc((ninj + 1) * sizeof(int));
  or_injury_faces(m, fi, fk);
  long *wall_of = malloc(n * sizeof(long));
  for (long q = 0; q < n; ++q) wall_of[q] = -1;
  for (int f = 0; f < ninj; ++f) wall_of[cidx(m, fi[f], 0, fk[f])] = f;
  double aV = 1.0 / m->hy, Dd = p->D_chem / (0.5 * m->hy);
#pragma omp parallel for schedule(dynamic, 256)
  for (long q = 0; q < n; ++q) {
    double y[OR_NX] = {0};
    for (int s = 0; s < OR_NS; ++s) y[s] = c[(long)s * n + q];
    if (ext) {
      y[INH] = ext[q];
      y[E2I] = ext[n + q];
    }
    double g = or_g(p, eta ? eta[q] : 0.0);
    long f = wall_of[q];
    const int wall = couple_wall && f >= 0;
    for (int it = 0; it < nsub; ++it)
      rk4_cell_x(p, y, ext != NULL, H[q], g, wall, wall ? &e0[f] : NULL, wall ? &c0[f] : NULL, aV, Dd, h);
    for (int s = 0; s < OR_NS; ++s) c[(long)s * n + q] = y[s];
    if (ext) {
      ext[q] = y[INH];
      ext[n + q] = y[E2I];
    }
  }
  free(H);
  free(fi);
  free(fk);
  free(wall_of);
}

void or_reaction(const or_mesh *m, const or_params *p, double *c, double *e0, double *c0,
                 const double *eta, double h, int nsub) {
  reaction_impl(m, p, c, NULL, e0, c0, eta, h, nsub, 1);
}

/* or_reaction with the inhibitor extension's rows ext[2][ncell] (I, E2,inh). */
void or_reaction_x(const or_mesh *m, const or_params *p, double *c, double *ext, double *e0, double *c0,
                   const double *eta, double h, int nsub) {
  reaction_impl(m, p, c, ext, e0, c0, eta, h, nsub, 1);
}

/* The injury-wall exchange the way the paper's solver places it (App. C
 * boundary table: mixed conditions on S1 and E1 at the injury faces; E0, C0
 * advanced by their own ODEs, App. B), as a lagged alternative to coupling it
 * inside the reaction stages.  Transport part, explicit like the rest of the
 * transport: the floor cell P over face f loses dt (A/V) J of S1 and gains
 * dt (A/V) kC0cat C0 of E1, with J = kC0+ S1_w E0 - kC0- C0 and the Robin wall
 * value S1_w from the start-of-step S1_P and E0, C0 (cs holds the post-transport
 * state, c the start of the step).  Then nsub RK4 steps of the E0, C0 ODEs with
 * S1_P frozen at its post-transport value.  The two J differ, so S1 + E1 + ...
 * + (A/V) C0 is no longer conserved exactly: the defect this reading is kept
 * to measure. */
static void wall_lagged(const or_mesh *m, const or_params *p, const double *c, double *cs, double *e0,
                        double *c0, double dt, int nsub) {
  long n = ncell_of(m);
  int ninj = or_injury_faces(m, NULL, NULL);
  int *fi = malloc((ninj + 1) * sizeof(int)), *fk = malloc((ninj + 1) * sizeof(int));
  or_injury_faces(m, fi, fk);
  const double aV = 1.0 / m->hy, Dd = p->D_chem / (0.5 * m->hy);
  for (int f = 0; f < ninj; ++f) {
    long P = cidx(m, fi[f], 0, fk[f]);
    double s1w = (Dd * c[S1 * n + P] + p->kC0m * c0[f]) / (Dd + p->kC0p * e0[f]);
    double J = p->kC0p * s1w * e0[f] - p->kC0m * c0[f];
    cs[S1 * n + P] -= dt * aV * J;
    cs[E1 * n + P] += dt * aV * p->kC0cat * c0[f];
    const double s1 = cs[S1 * n + P], h = dt / nsub;
    for (int it = 0; it < nsub; ++it) {
      double ke[4], kc[4];
      for (int st = 0; st < 4; ++st) {
        const double a = st == 0 ? 0.0 : st == 3 ? 1.0 : 0.5;
        double e = e0[f] + (st ? a * h * ke[st - 1] : 0.0), cc = c0[f] + (st ? a * h * kc[st - 1] : 0.0);
        double w = (Dd * s1 + p->kC0m * cc) / (Dd + p->kC0p * e);
        double Jt = p->kC0p * w * e - p->kC0m * cc;
        ke[st] = -Jt + p->kC0cat * cc;
        kc[st] = Jt - p->kC0cat * cc;
      }
      e0[f] += h / 6.0 * (ke[0] + 2 * ke[1] + 2 * ke[2] + ke[3]);
      c0[f] += h / 6.0 * (kc[0] + 2 * kc[1] + 2 * kc[2] + kc[3]);
    }
  }
  free(fi);
  free(fk);
}

/* The full species step (Sec. 3.2) repeated nsteps times:
 *   1. theta_B from the current state; eta solve (App. A, Eq. eta)
 *   2. sigma_release sample when t has reached the next multiple of sigma_dt
 *   3. explicit transport over dt (+ dt sigma for ADP): forward Euler, or with
 *      OR_TRANSPORT_RK2 Heun's method -- c1 = c + dt L(c), c2 = c1 + dt L(c1),
 *      c <- (c + c2) / 2, second order in time like the paper's Crank-Nicolson
 *      transport (App. D) while staying explicit; each stage is the forward
 *      Euler step, so conservation and the TVD bound carry over
 *   4. M_rxn RK4 reaction steps of h = dt / M_rxn (with OR_STRANG: M_rxn steps
 *      of dt / (2 M_rxn) before the transport and again after it -- symmetric
 *      splitting, second order where the plain fractional step is first)
 *   5. t += dt
 * Returns 0, or -1 on bad arguments. */
int or_step(const or_mesh *m, const or_params *p, or_fields *F, const or_inputs *in,
            double dt, int nsteps) {
  if (!m || !p || !F || !in || dt <= 0 || nsteps < 0) return -1;
  long n = ncell_of(m);
  double *cs = malloc((size_t)OR_NS * n * sizeof(double));
  double *cs2 = (p->flags & OR_TRANSPORT_RK2) ? malloc((size_t)OR_NS * n * sizeof(double)) : NULL;
  double *xs = F->ext ? malloc((size_t)2 * n * sizeof(double)) : NULL;
  double *xs2 = (F->ext && cs2) ? malloc((size_t)2 * n * sizeof(double)) : NULL;
  const int lagged = (p->flags & OR_WALL_LAGGED) != 0;
  const int nsub = p->M_rxn > 0 ? p->M_rxn : 1;
  double *cprev = lagged ? malloc((size_t)OR_NS * n * sizeof(double)) : NULL;
  double *thB = malloc(n * sizeof(double));
  for (int step = 0; step < nsteps; ++step) {
    for (long q = 0; q < n; ++q) thB[q] = (F->c[PBA * n + q] + F->c[PBSE * n + q]) / p->Pmax;
    if (!(p->flags & OR_NO_ETA)) or_eta_solve(m, p, thB, F->eta, p->eta_tol, p->eta_maxit);
    if (!(p->flags & OR_NO_SIGMA)) {
      if (F->t_last < 0) { /* first call: the history starts from this state */
        for (long q = 0; q < n; ++q) F->thetaB_last[q] = thB[q];
        F->t_last = F->t;
      }
      if (F->t + 1e-6 * dt >= (F->n_samples + 1) * p->sigma_dt) or_sigma_sample(m, p, F);
    }
    const int strang = (p->flags & OR_STRANG) && !(p->flags & OR_NO_REACTION) && p->M_rxn > 0;
    if (strang) reaction_impl(m, p, F->c, F->ext, F->e0, F->c0, F->eta, 0.5 * dt / p->M_rxn, p->M_rxn, !lagged);
    if (!(p->flags & OR_NO_TRANSPORT)) {
      if (lagged) memcpy(cprev, F->c, (size_t)OR_NS * n * sizeof(double));
      transport_x(m, p, in, F->c, F->ext, F->sigma, dt, cs, xs);
      if (cs2) {
        transport_x(m, p, in, cs, xs, F->sigma, dt, cs2, xs2);
        for (long q = 0; q < (long)OR_NS * n; ++q) F->c[q] = 0.5 * (F->c[q] + cs2[q]);
        if (F->ext)
          for (long q = 0; q < 2 * n; ++q) F->ext[q] = 0.5 * (F->ext[q] + xs2[q]);
      } else {
        memcpy(F->c, cs, (size_t)OR_NS * n * sizeof(double));
        if (F->ext) memcpy(F->ext, xs, (size_t)2 * n * sizeof(double));
      }
      if (lagged) wall_lagged(m, p, cprev, F->c, F->e0, F->c0, dt, nsub);
    }
    if (strang)
      reaction_impl(m, p, F->c, F->ext, F->e0, F->c0, F->eta, 0.5 * dt / p->M_rxn, p->M_rxn, !lagged);
    else if (!(p->flags & OR_NO_REACTION) && p->M_rxn > 0)
      reaction_impl(m, p, F->c, F->ext, F->e0, F->c0, F->eta, dt / p->M_rxn, p->M_rxn, !lagged);
    F->t += dt;
  }
  free(cs);
  free(cs2);
  free(xs);
  free(xs2);
  free(cprev);
  free(thB);
  return 0;
}

/* Conservation diagnostics (invariants of App. A/B):
 *  out[0] sum V (Pmu + Pma + Pba + Pbse)              platelets
 *  out[1] sum V (S1 + E1 + S1b + E1b + C1 + C2) + sum A C0      family 1
 *  out[2] sum V (S2 + E2 + S2b + E2b + C1 + C2) (+ E2,inh)      family 2
 *  out[3] sum A (E0 + C0)                                        wall enzyme
 *  out[4] sum V ADP
 *  out[5] minimum over all cell species and wall species
 *  out[6] number of non-finite values
 *  out[7] maximum of theta_T */
void or_diagnostics(const or_mesh *m, const or_params *p, const or_fields *F, double *out) {
  long n = ncell_of(m);
  double V = m->hx * m->hy * m->hz, A = m->hx * m->hz;
  int ninj = or_injury_faces(m, NULL, NULL);
  const double *c = F->c;
  double s[8] = {0, 0, 0, 0, 0, INFINITY, 0, -INFINITY};
  for (long q = 0; q < n; ++q) {
    s[0] += V * (c[PMU * n + q] + c[PMA * n + q] + c[PBA * n + q] + c[PBSE * n + q]);
    s[1] += V * (c[S1 * n + q] + c[E1 * n + q] + c[S1B * n + q] + c[E1B * n + q] + c[C1 * n + q] + c[C2 * n + q]);
    s[2] += V * (c[S2 * n + q] + c[E2 * n + q] + c[S2B * n + q] + c[E2B * n + q] + c[C1 * n + q] + c[C2 * n + q]);
    s[4] += V * c[ADP * n + q];
    double th = (c[PMU * n + q] + c[PMA * n + q] + c[PBA * n + q] + c[PBSE * n + q]) / p->Pmax;
    if (th > s[7]) s[7] = th;
    for (int sp = 0; sp < OR_NS; ++sp) {
      double v = c[(long)sp * n + q];
      if (!isfinite(v)) s[6] += 1;
      else if (v < s[5]) s[5] = v;
    }
  }
  if (F->ext)   /* inhibitor extension: E2,inh closes family 2 */
    for (long q = 0; q < n; ++q) {
      s[2] += V * F->ext[n + q];
      for (int r = 0; r < 2; ++r) {
        double v = F->ext[(long)r * n + q];
        if (!isfinite(v)) s[6] += 1;
        else if (v < s[5]) s[5] = v;
      }
    }
  for (int f = 0; f < ninj; ++f) {
    s[1] += A * F->c0[f];
    s[3] += A * (F->e0[f] + F->c0[f]);
    if (!isfinite(F->e0[f])) s[6] += 1; else if (F->e0[f] < s[5]) s[5] = F->e0[f];
    if (!isfinite(F->c0[f])) s[6] += 1; else if (F->c0[f] < s[5]) s[5] = F->c0[f];
  }
  for (int q = 0; q < 8; ++q) out[q] = s[q];
}

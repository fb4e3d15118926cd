"""Seeded synthetic inputs shaped like the clotFoam workloads.

This module is the only code that both the GPU path's tests/bench and the FP64
oracle consume.  It holds none of the species-step arithmetic: it produces the
mesh descriptions, the model parameters (the paper's App. E values, as data),
the prescribed face fluxes, the inlet Dirichlet profiles and seeded initial
states.  Everything is FP64 numpy; each consumer converts as it needs.

Workload sources (clotFoam paper):
  * 2D channel with a parabolic inlet velocity u(y) (App. C, Eq.
    parabolicVelocity) and a marginated platelet inlet profile P0 c(y)
    (App. C, Eqs. plateletShapeFunction2D, the C0 normalisation);
  * 3D duct with the two-axis shape function c(y, z) (App. C, 3D subsection);
  * plasma initial values (App. E, normal concentrations table).
No dataset is involved: the paper's examples are simulated geometries, and the
channels here are seeded stand-ins of the same shape and size range.
"""
from __future__ import annotations

import math

import numpy as np

NS = 15
SPECIES = ("Pmu", "Pma", "Pba", "Pbse", "ADP", "S1", "S2", "E1", "E2",
           "S1b", "S2b", "E1b", "E2b", "C1", "C2")
IDX = {s: q for q, s in enumerate(SPECIES)}

UM = 1e-3  # one micrometre in mm


def params_default(**over) -> dict:
    """Model parameters in mm / s / nmol / platelets (App. E tables), plus the
    numerical settings of the step.  g0 and every derived constant are left to
    the consumers."""
    p = dict(
        # App. E, platelet equation parameters
        Pmax=6.67e7, P0=2.5e5, kadh=3.3212e-8, kcohPmax=1.0e4,
        eta_t=0.1, eta_star=0.4, p_diam=3.0e-3, L_eta=2.0 * 3.0e-3,
        k_adp=0.34, adp_star=2.0e-3, k_e2=0.5, e2_star=1.0e-6,
        A_hat=2.0e-8, sigma_tf=6.0, sigma_dt=0.25,
        # App. E, diffusion coefficients
        D_P=2.5e-5, D_adp=5.0e-4, D_chem=5.0e-5,
        # App. E, binding sites and Avogadro's number per nmol (App. B)
        N1=2700.0, N2=2000.0, N_A=6.02214076e14,
        # App. E, subendothelium / platelet-surface enzyme reactions
        kC0p=8.95e3, kC0m=1.0, kC0cat=1.15,
        kC1p=1.03e5, kC1m=1.0, kC1cat=30.0,
        kC2p=1.73e4, kC2m=1.0, kC2cat=0.23,
        # App. E, binding on the platelet surface
        kS1p=5.7e4, kS1m=0.17, kE1p=1.0e4, kE1m=2.5e-2,
        kS2p=1.0e4, kS2m=5.9, kE2p=1.0e4, kE2m=5.9,
        # plasma values (App. E normal concentrations)
        S1_plasma=1.7e-4, S2_plasma=1.4e-3, E0_wall=1.5e-7,
        # numerics
        M_rxn=2, limiter=1, flags=0, eta_tol=1e-13, eta_atol=1e-6, eta_maxit=100000,
        wait_s=0.0,  # library only: grid-barrier wait bound of the eta solver (0: its default)
        # the paper's example of adding a species (inhibitor I + E2 -> E2,inh at
        # rate kI I E2): no value in the paper; off unless a run sets them
        kI=0.0, I_in=0.0,
        # library only: references of the deviation form (CLOT_DEVIATION), the plasma values
        S1_ref=1.7e-4, S2_ref=1.4e-3,
    )
    p.update(over)
    return p


# ------------------------------------------------------------------ meshes

def channel2d(nx, ny, length, height, inj_frac=(1 / 3, 2 / 3), p_diam=3.0e-3):
    """2D channel [0,length] x [0,height] (mm), unit depth, injury patch on the
    floor between inj_frac[0]*length and inj_frac[1]*length."""
    return dict(dim=2, nx=int(nx), ny=int(ny), nz=1, hx=length / nx, hy=height / ny, hz=1.0,
                inj_x0=inj_frac[0] * length, inj_x1=inj_frac[1] * length,
                inj_z0=0.0, inj_z1=0.0, p_diam=p_diam)


def duct3d(nx, ny, nz, h, inj_frac=(3 / 8, 5 / 8), p_diam=3.0e-3):
    L, W = nx * h, nz * h
    return dict(dim=3, nx=int(nx), ny=int(ny), nz=int(nz), hx=h, hy=h, hz=h,
                inj_x0=inj_frac[0] * L, inj_x1=inj_frac[1] * L,
                inj_z0=0.0, inj_z1=W, p_diam=p_diam)


def ncell(desc) -> int:
    return int(desc["nx"]) * int(desc["ny"]) * int(desc.get("nz", 1))


# ------------------------------------------------------------------ fluxes

def fluxes_channel2d(desc, shear):
    """Face fluxes (mm^3/s) of the parabolic profile u(y) = -shear/(2r)(y-r)^2 +
    shear r/2 (App. C), integrated exactly over each x face; v = 0."""
    nx, ny, hy, hz = desc["nx"], desc["ny"], desc["hy"], desc["hz"]
    r = ny * hy / 2.0

    def prim(y):  # antiderivative of u
        return -shear / (6.0 * r) * (y - r) ** 3 + 0.5 * shear * r * y

    yf = np.arange(ny + 1) * hy
    col = (prim(yf[1:]) - prim(yf[:-1])) * hz           # [ny]
    fx = np.broadcast_to(col[:, None], (ny, nx + 1)).copy().reshape(-1)  # index i + (nx+1) j
    fy = np.zeros(nx * (ny + 1))
    return dict(fx=fx, fy=fy, fz=None)


def fluxes_duct3d(desc, shear):
    """Face fluxes of u = U (4y(H-y)/H^2)(4z(W-z)/W^2), U = shear H / 4 so the
    floor shear at mid-width equals `shear`; exact face integrals."""
    nx, ny, nz, h = desc["nx"], desc["ny"], desc["nz"], desc["hy"]
    H, W = ny * h, nz * h
    U = shear * H / 4.0

    def prim(s, S):  # antiderivative of 4 s (S - s) / S^2
        return 4.0 * (S * s * s / 2.0 - s ** 3 / 3.0) / (S * S)

    yf = np.arange(ny + 1) * h
    zf = np.arange(nz + 1) * h
    iy = prim(yf[1:], H) - prim(yf[:-1], H)
    iz = prim(zf[1:], W) - prim(zf[:-1], W)
    plane = U * iz[:, None] * iy[None, :]                 # [nz, ny]
    fx = np.broadcast_to(plane[:, :, None], (nz, ny, nx + 1)).copy().reshape(-1)
    fy = np.zeros(nx * (ny + 1) * nz)
    fz = np.zeros(nx * ny * (nz + 1))
    return dict(fx=fx, fy=fy, fz=fz)


def cfl_dt(desc, fluxes, cfl=0.5):
    """dt with Courant number `cfl`: dt max_f |F_f| / (A_f h) = cfl (A_f h = V)."""
    V = desc["hx"] * desc["hy"] * desc["hz"]
    fmax = max(float(np.max(np.abs(f))) for f in (fluxes["fx"], fluxes["fy"], fluxes["fz"])
               if f is not None and f.size)
    return cfl * V / fmax


def stable_dt(desc, fluxes, params, cfl=0.5):
    """Courant-0.5 dt, capped so that explicit diffusion of the fastest species
    stays well inside its bound (0.2 h^2 / D_ADP), so that the Courant number
    plus the diffusion number sum_d 2 D_max dt / h_d^2 stays <= 0.9 (the
    library rejects a sum above 1; it binds only on meshes finer than 0.2 um),
    and so that the RK4 reaction substep resolves cohesion (dt <= 1e-4 s at
    M_rxn = 2).  The benchmark channels and duct are limited by the Courant
    number alone."""
    h = min(desc["hx"], desc["hy"], desc["hz"] if desc["dim"] == 3 else desc["hy"])
    dt = min(cfl_dt(desc, fluxes, cfl), 0.2 * h * h / params["D_adp"], 1e-4)
    axes = ("hx", "hy", "hz") if desc["dim"] == 3 else ("hx", "hy")
    dmax = max(params["D_adp"], params["D_P"], params["D_chem"])
    rate = cfl / cfl_dt(desc, fluxes, cfl) + sum(2.0 * dmax / desc[a] ** 2 for a in axes)
    return min(dt, 0.9 / rate)


# ------------------------------------------------------------ inlet profile

def margination_shape(s, r, K, m=19, n=2):
    """K R^{m-1} (1 - R)^{n-1}, R = |s - r| / r (App. C)."""
    R = np.abs(s - r) / r
    return K * R ** (m - 1) * (1.0 - R) ** (n - 1)


def beta_mn(m, n):
    return math.gamma(m) * math.gamma(n) / math.gamma(m + n)


def platelet_shape(desc, y, z=None, K=330.0, m=19, n=2):
    """c(y) (2D) or c(y, z) (3D) with the normalisation C0 of App. C, whose
    integral has the closed form (1/2r) int [1 + K R^{m-1}(1-R)^{n-1}] = 1 + K B(m,n)."""
    H = desc["ny"] * desc["hy"]
    if desc["dim"] == 2 or z is None:
        C0 = 1.0 / (1.0 + K * beta_mn(m, n))
        return C0 * (1.0 + margination_shape(y, H / 2.0, K, m, n))
    W = desc["nz"] * desc["hz"]
    C0 = 1.0 / (1.0 + 2.0 * K * beta_mn(m, n))
    return C0 * (1.0 + margination_shape(y, H / 2.0, K, m, n) + margination_shape(z, W / 2.0, K, m, n))


def inlet_values(desc, params, K=None):
    """Dirichlet inlet values at the x = 0 face centres, ordered j + ny k:
    Pmu = P0 c(y[,z]); S1, S2 at their plasma values (App. C BC table)."""
    ny, nz = desc["ny"], desc.get("nz", 1)
    yc = (np.arange(ny) + 0.5) * desc["hy"]
    if desc["dim"] == 2:
        K = 330.0 if K is None else K
        shape = platelet_shape(desc, yc, K=K)
    else:
        K = 547.0 if K is None else K
        zc = (np.arange(nz) + 0.5) * desc["hz"]
        shape = platelet_shape(desc, yc[None, :], zc[:, None], K=K).reshape(-1)
    pmu = params["P0"] * np.asarray(shape, np.float64).reshape(-1)
    s1 = np.full(ny * nz, params["S1_plasma"])
    s2 = np.full(ny * nz, params["S2_plasma"])
    return dict(pmu_in=pmu, s1_in=s1, s2_in=s2)


# ----------------------------------------------------------- initial states

def cell_centres(desc):
    nx, ny, nz = desc["nx"], desc["ny"], desc.get("nz", 1)
    x = (np.arange(nx) + 0.5) * desc["hx"]
    y = (np.arange(ny) + 0.5) * desc["hy"]
    z = (np.arange(nz) + 0.5) * desc["hz"]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X.reshape(-1), Y.reshape(-1), Z.reshape(-1)


def floor_patch_mask(desc):
    """[nz, nx] boolean of floor faces whose centre lies in the injury rectangle.
    (Input-shaping only: selects which generated wall values are handed over.)"""
    nx, nz = desc["nx"], desc.get("nz", 1)
    xc = (np.arange(nx) + 0.5) * desc["hx"]
    zc = (np.arange(nz) + 0.5) * desc["hz"]
    mx = (xc >= desc["inj_x0"]) & (xc <= desc["inj_x1"])
    mz = np.ones(nz, bool) if desc["dim"] == 2 else (zc >= desc["inj_z0"]) & (zc <= desc["inj_z1"])
    return mz[:, None] & mx[None, :]


def plasma_state(desc, params, seed=0, noise=0.01, K=None):
    """Plasma initial state: Pmu = P0 c(y[,z]), S1, S2 at plasma values, E0 on
    the injury faces, everything else 0; each value x (1 + noise xi),
    xi ~ N(0,1) iid from numpy default_rng(seed).  Returns (c[15,ncell], e0, c0)."""
    rng = np.random.default_rng(seed)
    nc = ncell(desc)
    X, Y, Z = cell_centres(desc)
    c = np.zeros((NS, nc))
    if desc["dim"] == 2:
        shape = platelet_shape(desc, Y, K=330.0 if K is None else K)
    else:
        shape = platelet_shape(desc, Y, Z, K=547.0 if K is None else K)
    c[IDX["Pmu"]] = params["P0"] * shape
    c[IDX["S1"]] = params["S1_plasma"]
    c[IDX["S2"]] = params["S2_plasma"]
    c *= 1.0 + noise * rng.standard_normal((NS, nc))
    mask = floor_patch_mask(desc)
    ninj = int(mask.sum())
    e0 = params["E0_wall"] * (1.0 + noise * rng.standard_normal(ninj))
    c0 = np.zeros(ninj)
    return c, e0, c0


def primed_state(desc, params, seed=0, noise=0.01):
    """Plasma state plus a synthetic clot: theta_B = 0.9 exp(-((x-xc)/20um)^2 -
    (y/8um)^2) centred on the injury, split 80/20 P^{b,se}/P^{b,a} in the two
    floor rows and all P^{b,a} above; bound chemicals at 10-50 % of the site
    capacity; E1, E2, ADP and P^{m,a} nonzero near the clot; part of E0 as C0."""
    rng = np.random.default_rng(seed + 7919)
    c, e0, c0 = plasma_state(desc, params, seed=seed, noise=noise)
    X, Y, Z = cell_centres(desc)
    xc = 0.5 * (desc["inj_x0"] + desc["inj_x1"])
    bump = np.exp(-((X - xc) / (20 * UM)) ** 2 - (Y / (8 * UM)) ** 2)
    if desc["dim"] == 3:
        zc = 0.5 * (desc["inj_z0"] + desc["inj_z1"])
        bump = bump * np.exp(-((Z - zc) / (40 * UM)) ** 2)
    Pmax = params["Pmax"]
    thB = 0.9 * bump
    floor_rows = Y < 2.0 * desc["hy"]
    c[IDX["Pbse"]] = np.where(floor_rows, 0.8, 0.0) * thB * Pmax
    c[IDX["Pba"]] = np.where(floor_rows, 0.2, 1.0) * thB * Pmax
    c[IDX["Pma"]] = 0.05 * params["P0"] * bump * (1 + 0.1 * rng.random(X.size))
    c[IDX["Pmu"]] *= (1.0 - 0.5 * bump)
    cap1 = params["N1"] / params["N_A"] * (c[IDX["Pba"]] + c[IDX["Pbse"]])
    cap2 = params["N2"] / params["N_A"] * (c[IDX["Pba"]] + c[IDX["Pbse"]])
    u = lambda lo, hi: lo + (hi - lo) * rng.random(X.size)
    cap = np.minimum(cap1, cap2)
    c[IDX["C1"]] = 0.02 * cap * u(0.5, 1.5)
    c[IDX["C2"]] = 0.02 * cap * u(0.5, 1.5)
    c[IDX["S1b"]] = cap1 * u(0.05, 0.3)
    c[IDX["E1b"]] = cap1 * u(0.01, 0.1)
    c[IDX["S2b"]] = cap2 * u(0.05, 0.3)
    c[IDX["E2b"]] = cap2 * u(0.01, 0.1)
    c[IDX["E1"]] = 1e-7 * bump * u(0.5, 1.5)
    c[IDX["E2"]] = 5e-7 * bump * u(0.5, 1.5)
    c[IDX["ADP"]] = 1e-3 * bump * u(0.5, 1.5)
    moved = 0.2 * e0
    return c, e0 - moved, c0 + moved


def random_reaction_states(n, params, seed=0):
    """Log-uniform random single-cell states within physical ranges (for
    reaction-surrogate training data and single-cell tests)."""
    rng = np.random.default_rng(seed)
    Pmax = params["Pmax"]
    lu = lambda lo, hi, size=n: np.exp(rng.uniform(np.log(lo), np.log(hi), size))
    c = np.zeros((NS, n))
    thB = rng.uniform(0.0, 0.9, n) * (rng.random(n) < 0.7)
    split = rng.random(n)
    c[IDX["Pbse"]] = thB * Pmax * split
    c[IDX["Pba"]] = thB * Pmax * (1 - split)
    c[IDX["Pmu"]] = lu(1e4, 2e6)
    c[IDX["Pma"]] = lu(1e2, 1e6)
    c[IDX["ADP"]] = lu(1e-8, 5e-3)
    c[IDX["S1"]] = lu(1e-6, 3e-4)
    c[IDX["S2"]] = lu(1e-5, 2e-3)
    c[IDX["E1"]] = lu(1e-12, 1e-6)
    c[IDX["E2"]] = lu(1e-12, 1e-5)
    cap1 = params["N1"] / params["N_A"] * thB * Pmax
    cap2 = params["N2"] / params["N_A"] * thB * Pmax
    frac = lambda: rng.uniform(0.0, 0.2, n)
    c[IDX["S1b"]] = cap1 * frac()
    c[IDX["E1b"]] = cap1 * frac()
    c[IDX["S2b"]] = cap2 * frac()
    c[IDX["E2b"]] = cap2 * frac()
    c[IDX["C1"]] = np.minimum(cap1, cap2) * frac() * 0.5
    c[IDX["C2"]] = np.minimum(cap1, cap2) * frac() * 0.5
    eta = rng.uniform(0.0, 1.0, n)
    return c, eta


def surrogate_scale(params):
    """Per-species concentration scales of the reaction surrogate's features
    and increment floor (data of the model, not of the method): Pmax for the
    platelets, ADP* for ADP, the plasma values for S1 and S2, 1e-8 nmol/mm^3
    for the enzymes, the site capacities n_i Pmax for the bound species."""
    Pmax = params["Pmax"]
    cap1 = params["N1"] / params["N_A"] * Pmax
    cap2 = params["N2"] / params["N_A"] * Pmax
    return np.array([Pmax, Pmax, Pmax, Pmax, params["adp_star"], params["S1_plasma"], params["S2_plasma"],
                     1e-8, 1e-8, cap1, cap2, cap1, cap2, min(cap1, cap2), min(cap1, cap2)])


def surrogate_states(n, params, seed=0, plasma_frac=0.3):
    """Training / evaluation states of the reaction surrogate: the log-uniform
    random states of random_reaction_states, with a fraction plasma_frac made
    plasma-like (no bound platelets or bound chemicals, theta_B = 0)."""
    c, eta = random_reaction_states(n, params, seed=seed)
    rng = np.random.default_rng(seed + 104729)
    plasma = rng.random(n) < plasma_frac
    for name in ("Pba", "Pbse", "S1b", "S2b", "E1b", "E2b", "C1", "C2"):
        c[IDX[name], plasma] = 0.0
    eta[plasma] = rng.uniform(0.0, 0.1, int(plasma.sum()))
    return c, eta


# -------------------------------------------------------------- workloads

def config(name: str, params=None) -> dict:
    """The synthetic workloads: mesh, fluxes, inlet values, dt and step count.
    'channel_200x40'   2D 300x60 um, shear 1000/s, 200 steps
    'channel_1024x256' 2D 300x60 um, shear 1500/s, 2000 steps
    'duct_512x128x128' 3D h = 1.5 um, floor shear 1000/s, 500 steps
    'paper_128x32'     the paper's thrombosis mesh (240x60 um, 90 um patch)."""
    params = params_default() if params is None else params
    if name == "channel_200x40":
        desc, shear, nsteps = channel2d(200, 40, 300 * UM, 60 * UM), 1000.0, 200
    elif name == "channel_1024x256":
        desc, shear, nsteps = channel2d(1024, 256, 300 * UM, 60 * UM), 1500.0, 2000
    elif name == "duct_512x128x128":
        desc, shear, nsteps = duct3d(512, 128, 128, 1.5 * UM), 1000.0, 500
    elif name == "paper_128x32":
        desc = channel2d(128, 32, 240 * UM, 60 * UM, inj_frac=(75 / 240, 165 / 240))
        shear, nsteps = 1000.0, 200
    elif name.startswith("channel_"):  # channel_<nx>x<ny> at h = 1.5 um, middle-third patch
        nx, ny = (int(v) for v in name[len("channel_"):].split("x"))
        desc, shear, nsteps = channel2d(nx, ny, nx * 1.5 * UM, ny * 1.5 * UM), 1000.0, 200
    elif name.startswith("duct_"):     # duct_<nx>x<ny>x<nz> at h = 1.5 um
        nx, ny, nz = (int(v) for v in name[len("duct_"):].split("x"))
        desc, shear, nsteps = duct3d(nx, ny, nz, 1.5 * UM), 1000.0, 500
    else:
        raise KeyError(name)
    fl = fluxes_channel2d(desc, shear) if desc["dim"] == 2 else fluxes_duct3d(desc, shear)
    inl = inlet_values(desc, params)
    dt = stable_dt(desc, fl, params)
    return dict(name=name, desc=desc, shear=shear, nsteps=nsteps, dt=dt,
                fluxes=fl, inlet=inl)


def ensemble_specs(n=256, seed=0):
    """Uneven 2D channels: nx = 8 U{8..64}, ny = nx / 4, h = 1.5 um, shear
    U[500, 2000] 1/s, injury length U[0.1, 0.5] of the channel, centred."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = 8 * int(rng.integers(8, 65))
        ny = nx // 4
        shear = float(rng.uniform(500.0, 2000.0))
        frac = float(rng.uniform(0.1, 0.5))
        L, H = nx * 1.5 * UM, ny * 1.5 * UM
        desc = channel2d(nx, ny, L, H, inj_frac=(0.5 - frac / 2, 0.5 + frac / 2))
        out.append(dict(desc=desc, shear=shear, frac=frac))
    return out

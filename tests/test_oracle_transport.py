"""Pins of the oracle's explicit finite-volume transport (Sec. 3.2 step 1,
App. A/B transport terms, App. C boundary table, App. D schemes) against
closed forms and invariants that do not come from the oracle itself."""
import math

import numpy as np
import pytest
from scipy.special import comb

import oracle as O
import synthetic as S

TRANSPORTED = (O.PMU, O.PMA, O.ADP, O.S1, O.S2, O.E1, O.E2)


def row_desc(n, h=1.0, dim=2):
    """A row of n cells along x (ny = nz = 1) with no injury patch."""
    if dim == 2:
        return dict(dim=2, nx=n, ny=1, nz=1, hx=h, hy=1.0, hz=1.0,
                    inj_x0=-1.0, inj_x1=-1.0, inj_z0=0, inj_z1=0, p_diam=0.0)
    return dict(dim=3, nx=n, ny=1, nz=1, hx=h, hy=1.0, hz=1.0,
                inj_x0=-1.0, inj_x1=-1.0, inj_z0=-1.0, inj_z1=-1.0, p_diam=0.0)


def inputs_for(desc, fx, fy=None, fz=None, pmu=0.0, s1=0.0, s2=0.0):
    nx, ny, nz = desc["nx"], desc["ny"], desc["nz"]
    fx = np.broadcast_to(np.asarray(fx, float), ((nx + 1) * ny * nz,)).copy()
    fy = np.zeros(nx * (ny + 1) * nz) if fy is None else fy
    if desc["dim"] == 3 and fz is None:
        fz = np.zeros(nx * ny * (nz + 1))
    nb = ny * nz
    return dict(fx=fx, fy=fy, fz=fz, pmu_in=np.full(nb, pmu), s1_in=np.full(nb, s1),
                s2_in=np.full(nb, s2))


def tparams(**kw):
    p = S.params_default(flags=O.NO_REACTION | O.NO_ETA | O.NO_SIGMA)
    p.update(kw)
    return p


def test_closed_box_conserves_every_species():
    """Conservative form: with inlet/outlet closed and arbitrary interior
    fluxes, sum V c is unchanged for every transported species."""
    rng = np.random.default_rng(3)
    for desc in (dict(dim=2, nx=11, ny=7, nz=1, hx=0.7, hy=0.4, hz=1.0, inj_x0=-1, inj_x1=-1,
                      inj_z0=0, inj_z1=0, p_diam=0),
                 dict(dim=3, nx=6, ny=5, nz=4, hx=0.5, hy=0.3, hz=0.6, inj_x0=-1, inj_x1=-1,
                      inj_z0=-1, inj_z1=-1, p_diam=0)):
        nx, ny, nz = desc["nx"], desc["ny"], desc["nz"]
        fx = rng.normal(size=(nz, ny, nx + 1)) * 0.01
        fy = rng.normal(size=(nz, ny + 1, nx)) * 0.01
        fy[:, 0, :] = 0
        fy[:, -1, :] = 0
        fz = None
        if desc["dim"] == 3:
            fz = rng.normal(size=(nz + 1, ny, nx)) * 0.01
            fz[0] = 0
            fz[-1] = 0
            fz = fz.reshape(-1)
        inp = inputs_for(desc, 0.0, fy.reshape(-1), fz, pmu=5e6, s1=1.0, s2=1.0)
        inp["fx"] = fx.reshape(-1)
        p = tparams(flags=O.NO_REACTION | O.NO_ETA | O.NO_SIGMA | O.CLOSED_ENDS)
        nc = nx * ny * nz
        c = rng.uniform(0.1, 1.0, size=(15, nc))
        c[O.PMU] *= 1e7
        c[O.PMA] *= 1e7
        c[O.PBA] *= 1e7
        V = desc["hx"] * desc["hy"] * desc["hz"]
        sig = rng.uniform(0, 1, nc)
        out = O.transport(desc, p, c, inp, dt=0.3, sigma=sig)
        for s in range(15):
            before, after = V * c[s].sum(), V * out[s].sum()
            if s == O.ADP:
                before += 0.3 * V * sig.sum()
            assert abs(after - before) <= 1e-13 * abs(before), S.SPECIES[s]
            if s not in TRANSPORTED:
                assert np.array_equal(out[s], c[s])


@pytest.mark.parametrize("nu", [0.3, 0.5, 0.85])
def test_upwind_step_is_binomial(nu):
    """Pure upwind advection at Courant number nu of a step fed by a Dirichlet
    inlet: c_i^n = sum_k C(n,k) nu^k (1-nu)^(n-k) c0_{i-k} (c0 = 1 left of the inlet)."""
    n_cells, nsteps = 60, 25
    desc = row_desc(n_cells)
    p = tparams(limiter=0, D_chem=0.0)
    inp = inputs_for(desc, nu, s2=1.0)  # V = 1, dt = 1: F = nu
    c = np.zeros((15, n_cells))
    c0 = np.where(np.arange(n_cells) < 10, 1.0, 0.0)
    c[O.S2] = c0
    for _ in range(nsteps):
        c = O.transport(desc, p, c, inp, dt=1.0)
    ext = lambda i: 1.0 if i < 0 else c0[i]
    exact = np.array([sum(comb(nsteps, k, exact=True) * nu ** k * (1 - nu) ** (nsteps - k) * ext(i - k)
                          for k in range(nsteps + 1)) for i in range(n_cells)])
    assert np.max(np.abs(c[O.S2] - exact)) < 1e-13


def test_upwind_unit_courant_is_exact_shift():
    desc = row_desc(30)
    p = tparams(limiter=0, D_chem=0.0)
    inp = inputs_for(desc, 1.0, s1=0.0)
    rng = np.random.default_rng(0)
    c = np.zeros((15, 30))
    c[O.S1] = rng.random(30)
    ref = c[O.S1].copy()
    for _ in range(7):
        c = O.transport(desc, p, c, inp, dt=1.0)
    assert np.array_equal(c[O.S1][7:], ref[:-7])
    assert np.all(c[O.S1][:7] == 0.0)


def test_uniform_plasma_state_is_a_fixed_point():
    """A uniform state equal to the inlet values, advected by a divergence-free
    Poiseuille flux, is unchanged (inlet Dirichlet + outlet zeroGradient)."""
    p = tparams()
    cfg = S.config("channel_40x12", p)
    d = cfg["desc"]
    nc = S.ncell(d)
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    inp["pmu_in"] = np.full_like(inp["pmu_in"], 3e5)
    c = np.zeros((15, nc))
    c[O.PMU] = 3e5
    c[O.S1] = p["S1_plasma"]
    c[O.S2] = p["S2_plasma"]
    out = O.transport(d, p, c, inp, dt=cfg["dt"])
    for s in (O.PMU, O.S1, O.S2):
        assert np.max(np.abs(out[s] - c[s])) <= 1e-14 * c[s].max()
    assert np.all(out[[O.PMA, O.ADP, O.E1, O.E2]] == 0)


def _gaussian_error(n, axis, dim):
    Lx, D, s0, T = 1.0, 1e-3, 0.05, 4.0
    h = Lx / n
    shape = [2, 2, 2] if dim == 3 else [2, 2, 1]
    shape[axis] = n
    hh = [0.5, 0.5, 0.5] if dim == 3 else [0.5, 0.5, 1.0]
    hh[axis] = h
    desc = dict(dim=dim, nx=shape[0], ny=shape[1], nz=shape[2], hx=hh[0], hy=hh[1], hz=hh[2],
                inj_x0=-1, inj_x1=-1, inj_z0=-1, inj_z1=-1, p_diam=0)
    p = tparams(D_chem=D, flags=O.NO_REACTION | O.NO_ETA | O.NO_SIGMA | O.CLOSED_ENDS)
    nc = shape[0] * shape[1] * shape[2]
    inp = inputs_for(desc, 0.0)
    X, Y, Z = S.cell_centres(desc)
    coord = (X, Y, Z)[axis]
    c = np.zeros((15, nc))
    c[O.E1] = np.exp(-(coord - 0.5) ** 2 / (2 * s0 ** 2))
    dt = 0.2 * h * h / D
    nsteps = int(round(T / dt))
    dt = T / nsteps
    for _ in range(nsteps):
        c = O.transport(desc, p, c, inp, dt=dt)
    st2 = s0 ** 2 + 2 * D * T
    exact = math.sqrt(s0 ** 2 / st2) * np.exp(-(coord - 0.5) ** 2 / (2 * st2))
    return np.max(np.abs(c[O.E1] - exact))


@pytest.mark.parametrize("axis,dim", [(0, 2), (1, 2), (2, 3)])
def test_diffusion_of_gaussian_converges_second_order(axis, dim):
    """Pure diffusion of a Gaussian against the closed-form spreading Gaussian,
    with dt ~ h^2: error O(h^2) along each axis (Gauss linear orthogonal)."""
    e1, e2 = _gaussian_error(40, axis, dim), _gaussian_error(80, axis, dim)
    assert e1 < 2e-3
    assert math.log2(e1 / e2) > 1.8


def _advect_bump(n, limiter, nu_per_h=5.0):
    """Advect a smooth bump with dt ~ h^2 (Courant number nu = nu_per_h * h),
    so the first-order forward-Euler time error is below the spatial error."""
    desc = row_desc(n, h=1.0 / n)
    p = tparams(limiter=limiter, D_chem=0.0)
    u = 1.0
    nu = nu_per_h / n
    dt = nu * desc["hx"] / u
    inp = inputs_for(desc, u * 1.0)  # area = hy hz = 1
    x = (np.arange(n) + 0.5) / n
    bump = lambda x: np.where(np.abs(x - 0.3) < 0.15, np.cos(np.pi * (x - 0.3) / 0.3) ** 2, 0.0)
    c = np.zeros((15, n))
    c[O.E2] = bump(x)
    T = 0.3
    nsteps = int(round(T / dt))
    st = O.new_state(desc, p, c, np.zeros(0), np.zeros(0))
    O.step(desc, p, st, inp, dt, nsteps)
    return np.sum(np.abs(st.c[O.E2] - bump(x - u * nsteps * dt))) / n, st.c[O.E2]


def test_van_leer_is_tvd_and_beats_upwind_order():
    """Van Leer (App. D): the L1 error on a smooth bump converges at close to
    second order in space (upwind: first order); at Courant 0.5 no new extrema
    appear and the total variation does not grow."""
    ev = [_advect_bump(n, 1)[0] for n in (100, 200, 400)]
    eu = [_advect_bump(n, 0)[0] for n in (100, 200, 400)]
    rv = math.log2(ev[1] / ev[2])
    ru = math.log2(eu[1] / eu[2])
    assert rv > 1.6, (ev, rv)
    assert ru < 1.1, (eu, ru)
    assert ev[2] < 0.2 * eu[2]
    # TVD on a rough random profile
    rng = np.random.default_rng(5)
    n = 80
    desc = row_desc(n)
    p = tparams(limiter=1, D_chem=0.0)
    inp = inputs_for(desc, 0.5)
    c = np.zeros((15, n))
    c[O.E2] = rng.random(n)
    tv0 = np.sum(np.abs(np.diff(c[O.E2])))
    lo, hi = c[O.E2].min(), c[O.E2].max()
    for _ in range(20):
        c = O.transport(desc, p, c, inp, dt=1.0)
        tv = np.sum(np.abs(np.diff(c[O.E2])))
        assert tv <= tv0 + 1e-12
        assert c[O.E2].min() >= min(lo, 0.0) - 1e-14 and c[O.E2].max() <= hi + 1e-14
        tv0 = tv


def test_van_leer_face_value_special_cases():
    """psi(r) = (r+|r|)/(1+|r|): r = 1 gives psi = 1 (linear face value),
    r <= 0 gives first-order upwind, flat upwind gives upwind."""
    assert O.face_value(0.0, 1.0, 2.0) == pytest.approx(1.5, abs=1e-15)
    assert O.face_value(2.0, 1.0, 3.0) == 1.0
    assert O.face_value(1.0, 1.0, 3.0) == 1.0
    # r = 3: psi = 1.5 -> cf = cU + 0.75 (cD - cU)
    assert O.face_value(-2.0, 1.0, 2.0) == pytest.approx(1.75, abs=1e-15)
    assert O.face_value(5.0, 1.0, 1.0) == 1.0


def _platelet_row(thetas, F, D_P=0.0, limiter=0):
    n = len(thetas)
    desc = row_desc(n)
    p = tparams(limiter=limiter, D_P=D_P, Pmax=100.0)
    inp = inputs_for(desc, F)
    c = np.zeros((15, n))
    c[O.PBA] = np.asarray(thetas) * 100.0
    return desc, p, inp, c


def test_hindered_advection_uses_downwind_theta():
    """Sec. 3.2 / App. D: the advective platelet flux through a face is scaled
    by W(theta_T) of the DOWNWIND cell."""
    desc, p, inp, c = _platelet_row([0.0, 0.8, 0.2, 0.0], F=0.1)
    c[O.PMA, 1] = 1.0  # theta of cell 1 rises to 0.81
    out = O.transport(desc, p, c, inp, dt=1.0)
    th2 = 0.2
    assert out[O.PMA, 2] == pytest.approx(0.1 * math.tanh(math.pi * (1 - th2)) * 1.0, rel=1e-14)
    # reverse the flow: the flux from cell 1 into cell 0 uses W(theta_0 = 0)
    inp2 = inputs_for(desc, -0.1)
    out = O.transport(desc, p, c, inp2, dt=1.0)
    assert out[O.PMA, 0] == pytest.approx(0.1 * math.tanh(math.pi), rel=1e-14)


def test_packed_cells_block_platelets():
    """W(1) = 0: a region at the packing limit receives no platelets by
    advection or diffusion (localMax)."""
    th = [0.0] * 10 + [1.0] * 5 + [0.0] * 5
    desc, p, inp, c = _platelet_row(th, F=0.4, D_P=0.05)
    inp["pmu_in"][:] = 1.0
    c[O.PMU, :10] = 1.0
    for _ in range(30):
        c = O.transport(desc, p, c, inp, dt=1.0)
    assert np.all(c[O.PMU, 10:] == 0.0)
    assert np.all(c[O.PMU, :10] > 0.0)


def test_hindered_diffusion_uses_local_max():
    """Diffusive platelet flux scaled by W(max(theta_P, theta_N))."""
    desc, p, inp, c = _platelet_row([0.2, 0.7], F=0.0, D_P=0.01)
    p["flags"] |= O.CLOSED_ENDS  # no inlet Dirichlet diffusion
    c[O.PMU, 0] = 1.0  # theta_0 = 0.21 < theta_1 = 0.7
    out = O.transport(desc, p, c, inp, dt=1.0)
    flux = 0.01 * math.tanh(math.pi * (1 - 0.7)) * (1.0 - 0.0) / 1.0
    assert out[O.PMU, 1] == pytest.approx(flux, rel=1e-13)
    assert out[O.PMU, 0] == pytest.approx(1.0 - flux, rel=1e-13)


def test_inlet_dirichlet_diffusion_half_cell():
    """Inlet Dirichlet diffusion uses the half-cell distance (h/2)."""
    desc = row_desc(5, h=0.5)
    p = tparams(D_chem=0.01)
    inp = inputs_for(desc, 0.0, s1=2.0)
    c = np.zeros((15, 5))
    out = O.transport(desc, p, c, inp, dt=1.0)
    V = 0.5
    assert out[O.S1, 0] == pytest.approx(0.01 * 1.0 * 2.0 / 0.25 / V, rel=1e-14)
    # zeroGradient species see no inlet diffusion
    assert np.all(out[O.E1] == 0)


def test_adp_release_source_added():
    desc = row_desc(4)
    p = tparams()
    inp = inputs_for(desc, 0.0)
    c = np.zeros((15, 4))
    sig = np.array([1.0, 2.0, 3.0, 4.0])
    out = O.transport(desc, p, c, inp, dt=0.25, sigma=sig)
    assert np.allclose(out[O.ADP], 0.25 * sig, rtol=0, atol=1e-16)

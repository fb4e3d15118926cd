"""Pins of the oracle's Heun (SSP-RK2) transport option, the second-order-in-
time variant of the explicit transport (the paper's transport is Crank-
Nicolson, second order in time, App. D; the mesh convergence study shows the
forward Euler step's first-order time error in S1).

* pure diffusion of a cosine eigenmode of the zero-flux Laplacian: n Heun
  steps multiply it by R2(z)^n, R2(z) = 1 - z + z^2/2, z = D lambda dt, exactly
  (forward Euler: (1 - z)^n);
* at fixed end time the error against exp(-D lambda t) falls 4x per halving of
  dt (forward Euler 2x);
* each stage is the conservative, TVD forward Euler step, so the closed-box
  totals are unchanged and van Leer advection at Courant 0.5 makes no new
  extrema."""
import math

import numpy as np

import oracle as O
import synthetic as S


def _row(n, h=1e-3):
    return dict(dim=2, nx=n, ny=1, nz=1, hx=h, hy=1.0, hz=1.0, inj_x0=-1.0, inj_x1=-1.0, inj_z0=0, inj_z1=0,
                p_diam=0.0)


def _inputs(desc, fx=0.0):
    nx = desc["nx"]
    return dict(fx=np.full(nx + 1, float(fx)), fy=np.zeros(2 * nx), fz=None, pmu_in=np.zeros(1),
                s1_in=np.zeros(1), s2_in=np.zeros(1))


def _params(rk2, closed=True, **kw):
    flags = O.NO_REACTION | O.NO_ETA | O.NO_SIGMA | (O.CLOSED_ENDS if closed else 0) | (O.TRANSPORT_RK2 if rk2 else 0)
    p = S.params_default(flags=flags)
    p.update(kw)
    return p


def _diffuse_mode(n, k, dt, nsteps, rk2):
    desc = _row(n)
    x = (np.arange(n) + 0.5) / n
    c = np.zeros((15, n))
    c[O.S1] = 2.0 + np.cos(math.pi * k * x)
    st = O.new_state(desc, _params(rk2), c, np.zeros(0), np.zeros(0))
    O.step(desc, _params(rk2), st, _inputs(desc), dt, nsteps)
    lam = 4.0 * math.sin(math.pi * k / (2 * n)) ** 2 / desc["hx"] ** 2
    return st.c[O.S1] - 2.0, np.cos(math.pi * k * x), S.params_default()["D_chem"] * lam * dt


def test_heun_multiplies_an_eigenmode_by_its_stability_polynomial():
    for rk2, R in ((True, lambda z: 1 - z + z * z / 2), (False, lambda z: 1 - z)):
        got, mode, z = _diffuse_mode(64, 20, 2e-3, 40, rk2)
        assert 0.05 < z < 0.5
        assert np.max(np.abs(got - mode * R(z) ** 40)) < 1e-13, rk2


def test_heun_is_second_order_in_time():
    """Error of the mode amplitude at t = 0.064 s against the semi-discrete
    exact decay exp(-D lambda t) (space is exact for an eigenmode)."""
    def err(dt, rk2):
        n = int(round(0.064 / dt))
        got, mode, z = _diffuse_mode(64, 20, dt, n, rk2)
        return abs(got[0] / mode[0] - math.exp(-z * n))
    e2 = [err(dt, True) for dt in (2e-3, 1e-3, 5e-4)]
    e1 = [err(dt, False) for dt in (2e-3, 1e-3, 5e-4)]
    r2 = [math.log2(a / b) for a, b in zip(e2, e2[1:])]
    r1 = [math.log2(a / b) for a, b in zip(e1, e1[1:])]
    assert all(abs(r - 2.0) < 0.1 for r in r2), (e2, r2)
    assert all(abs(r - 1.0) < 0.1 for r in r1), (e1, r1)


def test_heun_conserves_and_stays_tvd():
    rng = np.random.default_rng(7)
    n = 80
    desc = _row(n)
    # closed box with interior fluxes: totals unchanged
    inp = _inputs(desc)
    inp["fx"] = rng.normal(size=n + 1) * 1e-7
    c = rng.uniform(0.1, 1.0, size=(15, n))
    st = O.new_state(desc, _params(True), c.copy(), np.zeros(0), np.zeros(0))
    O.step(desc, _params(True), st, inp, 1e-3, 10)
    for s in (O.PMU, O.PMA, O.ADP, O.S1, O.S2, O.E1, O.E2):
        assert abs(st.c[s].sum() - c[s].sum()) <= 1e-13 * c[s].sum(), S.SPECIES[s]
    # van Leer advection at Courant 0.5 with inflow zero: no new extrema, total variation does not grow
    V = desc["hx"] * desc["hy"] * desc["hz"]
    dt = 1e-3
    F = 0.5 * V / dt
    p = _params(True, closed=False, limiter=1, D_chem=0.0)
    c = np.zeros((15, n))
    c[O.E2] = rng.random(n)
    lo, hi = c[O.E2].min(), c[O.E2].max()
    tv0 = np.sum(np.abs(np.diff(c[O.E2])))
    st = O.new_state(desc, p, c, np.zeros(0), np.zeros(0))
    for _ in range(20):
        O.step(desc, p, st, _inputs(desc, F), dt, 1)
        e = st.c[O.E2]
        tv = np.sum(np.abs(np.diff(e)))
        assert tv <= tv0 + 1e-12
        assert e.min() >= min(lo, 0.0) - 1e-14 and e.max() <= hi + 1e-14
        tv0 = tv

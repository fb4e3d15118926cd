"""Pins of the oracle's virtual-substance solve (App. A, Eq. eta) and the ADP
release source (Sec. 2 Eq. ADP_source, Sec. 3.2 Eq. sigma_disc)."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle as O
import synthetic as S


def box(dim, nx, ny, nz, hx, hy, hz):
    return dict(dim=dim, nx=nx, ny=ny, nz=nz, hx=hx, hy=hy, hz=hz, inj_x0=-1, inj_x1=-1,
                inj_z0=-1, inj_z1=-1, p_diam=0.0)


@pytest.mark.parametrize("desc,modes", [
    (box(2, 24, 10, 1, 1.5e-3, 1.2e-3, 1.0), [(0, 0, 0), (1, 0, 0), (3, 2, 0), (23, 9, 0)]),
    (box(3, 8, 6, 5, 1.5e-3, 1.5e-3, 2.0e-3), [(1, 1, 1), (7, 0, 4), (2, 5, 3)]),
])
def test_eta_solves_cosine_modes_exactly(desc, modes):
    """cos(pi k (i+1/2)/n) satisfies the zero-flux condition and is an
    eigenvector of the discrete Laplacian with eigenvalue -4 sin^2(pi k/2n)/h^2;
    the solution of (I - L^2/4 lap) eta = theta_B is theta_B / (1 + L^2/4 lam)."""
    p = S.params_default()
    X, Y, Z = S.cell_centres(desc)
    n = (desc["nx"], desc["ny"], desc["nz"])
    h = (desc["hx"], desc["hy"], desc["hz"])
    coords = (X, Y, Z)
    cl = p["L_eta"] ** 2 / 4
    for k in modes:
        th = np.ones_like(X)
        lam = 0.0
        for a in range(desc["dim"]):
            th = th * np.cos(math.pi * k[a] * coords[a] / (n[a] * h[a]))
            lam += 4 * math.sin(math.pi * k[a] / (2 * n[a])) ** 2 / h[a] ** 2
        eta, it = O.eta_solve(desc, p, th, tol=1e-14)
        assert np.max(np.abs(eta - th / (1 + cl * lam))) < 1e-12


def test_eta_constant_field_and_maximum_principle():
    desc = box(2, 30, 12, 1, 1.5e-3, 1.5e-3, 1.0)
    p = S.params_default()
    eta, _ = O.eta_solve(desc, p, np.full(360, 0.37))
    assert np.max(np.abs(eta - 0.37)) < 1e-14
    rng = np.random.default_rng(1)
    th = rng.random(360) ** 4
    eta, _ = O.eta_solve(desc, p, th)
    assert eta.min() >= th.min() - 1e-14 and eta.max() <= th.max() + 1e-14
    assert np.max(np.abs(O.eta_op(desc, p, eta) - th)) < 1e-12
    # a point source spreads over a few L_eta/2 = 3 um and keeps its total
    # (zero-flux boundaries: the operator's columns sum to one)
    th = np.zeros(360)
    th[15] = 1.0
    eta, _ = O.eta_solve(desc, p, th)
    assert eta[15] < 1.0 and eta[16] > 0 and eta[15 + 5] < 0.1 * eta[15]
    assert eta.sum() == pytest.approx(1.0, rel=1e-12)
    assert np.all(eta > 0)


def test_eta_operator_is_symmetric_positive():
    desc = box(3, 5, 4, 3, 1e-3, 2e-3, 1.5e-3)
    p = S.params_default()
    rng = np.random.default_rng(2)
    x, y = rng.normal(size=60), rng.normal(size=60)
    assert x @ O.eta_op(desc, p, y) == pytest.approx(y @ O.eta_op(desc, p, x), rel=1e-13)
    assert x @ O.eta_op(desc, p, x) >= x @ x


def test_eta_warm_start_converges_to_same_solution():
    desc = box(2, 20, 8, 1, 1.5e-3, 1.5e-3, 1.0)
    p = S.params_default()
    th = np.random.default_rng(3).random(160)
    a, _ = O.eta_solve(desc, p, th)
    b, it = O.eta_solve(desc, p, th, eta0=a + 1e-3)
    assert np.max(np.abs(a - b)) < 1e-13 and it > 0


# -------------------------------------------------------------- sigma

def _sigma_run(rates_per_sample):
    """Drive the sampler directly: theta_B moves by rate * dtau between samples."""
    desc = box(2, 3, 1, 1, 1.0, 1.0, 1.0)
    p = S.params_default()
    nc = 3
    st = O.new_state(desc, p, np.zeros((15, nc)), np.zeros(0), np.zeros(0))
    st.t_last = 0.0
    out = []
    for m, r in enumerate(rates_per_sample, start=1):
        st.c[O.PBA] += r * p["sigma_dt"] * p["Pmax"] * np.array([1.0, 0.5, 0.0])
        st.t = m * p["sigma_dt"]
        O.sigma_sample(desc, p, st)
        out.append(st.sigma.copy())
    return p, out


def test_sigma_impulse_response_follows_R_of_the_lag():
    """A single burst of binding (rate r* over one sample interval) releases ADP
    at A_hat R(lag) r* dtau afterwards (trapezoid weights: half at lag 0 and at
    lag tau_f / dtau = 24, zero beyond)."""
    rates = [0.0] * 3 + [0.8] + [0.0] * 28
    p, out = _sigma_run(rates)
    rstar = p["Pmax"] * 0.8
    dtau = p["sigma_dt"]
    R = lambda tau: math.exp(-(tau - 3) ** 2) / math.sqrt(math.pi)
    for lag in range(0, 28):
        m = 3 + lag  # index into out of the sample taken lag samples after the burst
        w = 0.5 if lag in (0, 24) else (1.0 if lag < 24 else 0.0)
        expect = p["A_hat"] * dtau * w * R(lag * dtau) * rstar
        assert out[m][0] == pytest.approx(expect, rel=1e-12, abs=1e-300), lag
        assert out[m][1] == pytest.approx(0.5 * expect, rel=1e-12, abs=1e-300)
        assert out[m][2] == 0.0


def test_sigma_constant_binding_rate_releases_A_hat_times_rate():
    """Steady binding at rate r: sigma -> A_hat r int_0^6 R = A_hat r erf(3)
    (the trapezoid rule on this Gaussian is accurate to ~1e-5)."""
    p, out = _sigma_run([0.5] * 40)
    r = 0.5 * p["Pmax"]
    assert out[-1][0] == pytest.approx(p["A_hat"] * r * erf(3.0), rel=2e-5)
    assert out[0][0] == pytest.approx(p["A_hat"] * p["sigma_dt"] * 0.5 * math.exp(-9) / math.sqrt(math.pi) * r,
                                      rel=1e-12)
    # before any binding there is no release
    p, out = _sigma_run([0.0] * 5)
    assert all(np.all(o == 0) for o in out)


def test_step_samples_sigma_every_dtau():
    """The full step samples at t = m dtau only; the release then feeds ADP."""
    cfg = S.config("channel_20x6")
    dt = cfg["dt"]
    p = S.params_default(sigma_dt=7 * dt, sigma_tf=42 * dt, M_rxn=1)
    d = cfg["desc"]
    c, e0, c0 = S.primed_state(d, p, seed=2)
    st = O.new_state(d, p, c, e0, c0)
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    O.step(d, p, st, inp, dt, 6)
    assert st.n_samples == 0 and np.all(st.sigma == 0)
    O.step(d, p, st, inp, dt, 2)
    assert st.n_samples == 1
    O.step(d, p, st, inp, dt, 14)
    assert st.n_samples == 3 and np.any(st.sigma > 0)

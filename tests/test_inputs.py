"""Pins of the synthetic workloads and the setup quantities (App. C inlet
profiles and velocity, App. E parameters, Sec. 3.1 adhesion region) against
values printed in the paper (tests/golden/paper_values.json) and closed forms."""
import json
import math
import os

import numpy as np
import pytest
from scipy.integrate import dblquad, quad

import oracle as O
import synthetic as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_parameters_match_the_paper_tables():
    p = S.params_default()
    for k, v in GOLD["parameters"].items():
        if k.startswith("_"):
            continue
        assert p[k] == pytest.approx(v, rel=1e-15), k
    assert p["L_eta"] == pytest.approx(2 * p["p_diam"])       # App. E: L_eta = 2 P_diam
    assert p["eta_t"] + p["eta_star"] == pytest.approx(0.5)    # rapid change at eta = 0.5
    assert p["M_rxn"] == GOLD["default_M_rxn"]["value"]


def test_inlet_profile_2d_peak_ratio_and_normalisation():
    d = S.config("channel_200x40")["desc"]
    H = d["ny"] * d["hy"]
    y = np.linspace(0, H, 200001)
    c = S.platelet_shape(d, y, K=330.0)
    ratio = c.max() / S.platelet_shape(d, np.array([H / 2]), K=330.0)[0]
    assert ratio == pytest.approx(1 + 330 * (18 / 19) ** 18 / 19, rel=1e-6)   # 7.563
    assert abs(ratio - GOLD["inlet_peak_to_centre_2d"]["value"]) < 0.1
    mean = quad(lambda s: S.platelet_shape(d, np.array([s]), K=330.0)[0], 0, H, points=[H / 2],
                limit=200)[0] / H
    assert mean == pytest.approx(1.0, rel=1e-9)


def test_inlet_profile_3d_peak_ratio_and_normalisation():
    d = S.config("duct_64x32x32")["desc"]
    H, W = d["ny"] * d["hy"], d["nz"] * d["hz"]
    ys = np.linspace(0, H, 4001)
    c_peak = S.platelet_shape(d, ys, np.full_like(ys, W / 2), K=547.0).max()
    c_mid = S.platelet_shape(d, np.array([H / 2]), np.array([W / 2]), K=547.0)[0]
    assert abs(c_peak / c_mid - GOLD["inlet_peak_to_centre_3d"]["value"]) < 0.1
    mean = dblquad(lambda z, y: S.platelet_shape(d, np.array([y]), np.array([z]), K=547.0)[0],
                   0, H, 0, W, epsabs=1e-12, epsrel=1e-10)[0] / (H * W)
    assert mean == pytest.approx(1.0, rel=1e-7)


def test_parabolic_channel_flux_and_wall_shear():
    p = S.params_default()
    cfg = S.config("channel_200x40", p)
    d, fl = cfg["desc"], cfg["fluxes"]
    r = d["ny"] * d["hy"] / 2
    Q = fl["fx"].reshape(d["ny"], d["nx"] + 1)
    assert np.allclose(Q.sum(axis=0), 2 / 3 * 1000.0 * r * r * d["hz"], rtol=1e-13)
    # u(y) = -shear/(2r)(y-r)^2 + shear r/2 has du/dy(0) = shear and u_max = shear r/2
    assert np.max(Q) / (d["hy"] * d["hz"]) < 1000 * r / 2
    assert np.all(fl["fy"] == 0)
    assert cfg["dt"] == pytest.approx(5.0e-5, rel=2e-3)


def test_duct_flux_total_and_floor_shear():
    cfg = S.config("duct_64x32x32")
    d, fl = cfg["desc"], cfg["fluxes"]
    H, W = d["ny"] * d["hy"], d["nz"] * d["hz"]
    U = 1000.0 * H / 4
    plane = fl["fx"].reshape(d["nz"], d["ny"], d["nx"] + 1)
    assert np.allclose(plane.sum(axis=(0, 1)), U * 4 * H * W / 9, rtol=1e-13)
    assert np.all(fl["fy"] == 0) and np.all(fl["fz"] == 0)


def test_injury_faces_and_adhesion_region():
    d1 = S.config("channel_200x40")["desc"]
    fi, fk = O.injury_faces(d1)
    assert fi[0] == 67 and fi[-1] == 132 and len(fi) == 66 and np.all(fk == 0)
    assert O.hadh(d1).sum() == 132                    # two rows within P_diam of the wall
    dp = S.config("paper_128x32")["desc"]
    n_adh = O.hadh(dp).sum()
    assert n_adh == 96
    assert abs(n_adh - GOLD["adhesion_region_cells"]["value"]) <= 5
    d3 = S.config("duct_64x32x32")["desc"]
    fi, fk = O.injury_faces(d3)
    assert len(fi) == 16 * 32 and fi.min() == 24 and fi.max() == 39
    assert O.hadh(d3).sum() == 2 * 16 * 32
    assert S.floor_patch_mask(d3).sum() == len(fi)


def test_plasma_state_is_seeded_and_shaped():
    p = S.params_default()
    d = S.config("channel_200x40", p)["desc"]
    a = S.plasma_state(d, p, seed=4)
    b = S.plasma_state(d, p, seed=4)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    c, e0, c0 = a
    assert np.all(c[[1, 2, 3, 4, 7, 8, 9, 10, 11, 12, 13, 14]] == 0)
    assert abs(np.mean(c[S.IDX["S1"]]) / p["S1_plasma"] - 1) < 3e-3
    assert np.std(c[S.IDX["S1"]] / p["S1_plasma"]) == pytest.approx(0.01, rel=0.1)
    assert len(e0) == 66 and np.all(c0 == 0)


def test_R_is_normalised():
    v = quad(O.R, 0, 50)[0]
    assert v == pytest.approx(0.5 * (1 + math.erf(3.0)), rel=1e-12)
    assert abs(v - GOLD["R_normalised"]["value"]) < 2e-5


def _courant_and_diffusion(desc, fluxes, params, dt):
    V = desc["hx"] * desc["hy"] * desc["hz"]
    fmax = max(float(np.max(np.abs(f))) for f in (fluxes["fx"], fluxes["fy"], fluxes["fz"])
               if f is not None and f.size)
    axes = ("hx", "hy", "hz") if desc["dim"] == 3 else ("hx", "hy")
    dmax = max(params["D_adp"], params["D_P"], params["D_chem"])
    return dt * fmax / V, sum(2.0 * dmax * dt / desc[a] ** 2 for a in axes)


def test_stable_dt_stays_inside_the_explicit_bound():
    """The library rejects Courant + sum_d 2 D_max dt / h_d^2 > 1 (explicit
    transport, App. D reading); the generator keeps the sum <= 0.9 on every
    mesh, down to the paper's finest convergence mesh (0.1875 um), and leaves the
    Courant-limited workloads at Courant 0.5."""
    p = S.params_default()
    for h in (3.0, 1.5, 0.75, 0.375, 0.1875, 0.09375):
        nx, ny = int(round(120 / h)), int(round(30 / h))
        d = S.channel2d(nx, ny, 120e-3, 30e-3, inj_frac=(36 / 120, 81 / 120))
        fl = S.fluxes_channel2d(d, 1000.0)
        c, dn = _courant_and_diffusion(d, fl, p, S.stable_dt(d, fl, p))
        assert c <= 0.5 + 1e-12 and c + dn <= 0.9 + 1e-12, (h, c, dn)
    for name in ("channel_200x40", "channel_1024x256", "duct_512x128x128", "paper_128x32"):
        cfg = S.config(name, p)
        c, dn = _courant_and_diffusion(cfg["desc"], cfg["fluxes"], p, cfg["dt"])
        assert abs(c - 0.5) < 1e-9 and c + dn < 0.9, (name, c, dn)

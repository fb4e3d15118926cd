"""Pins of the oracle's inhibitor extension: the paper's example of adding a
species to the model (Sec. "Adapting the framework for different clotting
models"), a fluid-phase inhibitor I that binds fluid-phase thrombin for good,
I + E2 -> E2,inh at rate kI I E2 (reaction rate -kI I E2 for I).

* with kI = 0 and no inhibitor the extended run is the paper's model, bit for
  bit, and the two new rows stay zero;
* a well-mixed cell holding only thrombin and inhibitor follows the closed form
  of I' = E2' = -kI I E2 (I - E2 is constant):
      E2(t) = d E2(0) / ((E2(0) + d) exp(kI d t) - E2(0)),  d = I(0) - E2(0),
  to the RK4 error, which falls 16-fold per halving of the substep;
* the reaction keeps I + E2,inh and family 2 + E2,inh, so a closed channel
  with every term active conserves both totals;
* I is transported exactly like S1: with the reactions off, an I row started
  equal to the S1 row and an inlet value equal to S1's stays bit for bit equal
  to it; a uniform I at its inlet value is a fixed point of the transport."""
import numpy as np

import oracle as O
import synthetic as S


def _run(name, flags, nsteps, ext=None, seed=3, **over):
    p = S.params_default(flags=flags, **over)
    cfg = S.config(name, p)
    d = cfg["desc"]
    st = O.new_state(d, p, *S.primed_state(d, p, seed=seed), ext=ext(d, p) if callable(ext) else ext)
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    before = O.diagnostics(d, p, st)
    O.step(d, p, st, inp, cfg["dt"], nsteps)
    return st, before, O.diagnostics(d, p, st), d, p


def test_zero_rate_and_no_inhibitor_is_the_paper_model_bit_for_bit():
    for flags in (0, O.TRANSPORT_RK2 | O.STRANG, O.WALL_LAGGED):
        a, _, _, d, _ = _run("channel_60x16", flags, 15)
        zeros = lambda d, p: np.zeros((2, S.ncell(d)))
        b, _, _, _, _ = _run("channel_60x16", flags, 15, ext=zeros, kI=0.0, I_in=0.0)
        for k in ("c", "e0", "c0", "eta"):
            assert np.array_equal(getattr(a, k), getattr(b, k)), (flags, k)
        assert np.all(b.ext == 0.0)


def test_well_mixed_thrombin_inhibition_matches_the_closed_form():
    p = S.params_default(kI=2.0e4)
    d = dict(dim=2, nx=1, ny=1, nz=1, hx=1e-3, hy=1e-3, hz=1.0,
             inj_x0=-1.0, inj_x1=-1.0, inj_z0=0.0, inj_z1=0.0, p_diam=3e-3)
    c = np.zeros((15, 1))
    E20, I0 = 2.0e-4, 5.0e-4
    c[O.E2, 0] = E20
    T = 0.2
    dd = I0 - E20
    exact = dd * E20 / ((E20 + dd) * np.exp(p["kI"] * dd * T) - E20)
    errs = []
    for nsub in (8, 16, 32):
        cc, x, _, _ = O.reaction_x(d, p, c, np.array([[I0], [0.0]]), np.zeros(0), np.zeros(0), None,
                                   T / nsub, nsub)
        errs.append(abs(cc[O.E2, 0] - exact))
        assert abs((x[O.INH, 0] - cc[O.E2, 0]) - dd) <= 1e-18          # I - E2 constant
        assert abs((cc[O.E2, 0] + x[O.E2I, 0]) - E20) <= 1e-18        # E2 + E2,inh constant
    assert errs[-1] <= 1e-7 * E20                                       # (kI I h)^4 / 120 ~ 1e-7
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0, errs                             # fourth order


def test_closed_channel_conserves_the_inhibitor_and_family_2_with_e2inh():
    def ext(d, p):
        x = np.zeros((2, S.ncell(d)))
        x[0] = 3.0e-4
        x[1] = 1.0e-5
        return x
    st, b0, b1, d, p = _run("channel_60x16", O.CLOSED_ENDS | O.NO_SIGMA, 40, ext=ext, kI=5.0e4, I_in=3.0e-4)
    V = d["hx"] * d["hy"] * d["hz"]
    inh0 = V * (3.0e-4 + 1.0e-5) * S.ncell(d)
    inh1 = V * (st.ext[0].sum() + st.ext[1].sum())
    assert abs(inh1 - inh0) <= 1e-12 * inh0
    assert abs(b1[2] - b0[2]) <= 1e-12 * b0[2]                        # family 2 + E2,inh
    assert abs(b1[1] - b0[1]) <= 1e-12 * b0[1]                        # family 1 + wall
    assert st.ext[1].sum() > 1.0e-5 * S.ncell(d) * (1 + 1e-9)         # inhibition happened


def test_inhibitor_is_transported_like_s1():
    def ext(d, p):
        c, _, _ = S.primed_state(d, p, seed=3)
        return np.stack([np.asarray(c[O.S1], np.float64), np.zeros(S.ncell(d))])
    p0 = S.params_default()
    st, _, _, d, p = _run("channel_60x16", O.NO_REACTION | O.NO_SIGMA, 30, ext=ext, kI=5.0e4,
                          I_in=p0["S1_plasma"])
    assert np.array_equal(st.ext[0], st.c[O.S1])
    uni = lambda d, p: np.stack([np.full(S.ncell(d), 3.0e-4), np.zeros(S.ncell(d))])
    st2, _, _, _, _ = _run("channel_60x16", O.NO_REACTION | O.NO_SIGMA, 30, ext=uni, kI=5.0e4, I_in=3.0e-4)
    assert np.max(np.abs(st2.ext[0] - 3.0e-4)) <= 1e-15 * 3.0e-4 * 100

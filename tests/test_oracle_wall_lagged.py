"""Pins and measurement of the oracle's lagged injury-wall option (the
paper's placement of the wall reaction: mixed boundary conditions on S1 and E1
in the transport with E0, C0 of the previous step, E0 and C0 advanced by their
own ODEs; App. B equations, App. C boundary table) against the default, the
wall exchange coupled inside the reaction's RK4 stages.

* without wall enzyme (E0 = C0 = 0) the two placements give the same state;
* both keep E0 + C0 on every face;
* the coupled placement conserves family 1, sum V (S1 + E1 + S1b + E1b + C1 +
  C2) + sum A C0, to rounding; the lagged one does not, and its defect over a
  fixed time halves with dt (first order), as does its distance to the coupled
  state."""
import numpy as np

import oracle as O
import synthetic as S


def _run(name, nsteps, dt_scale, lagged, state=None, seed=2):
    flags = O.CLOSED_ENDS | O.NO_SIGMA | (O.WALL_LAGGED if lagged else 0)
    p = S.params_default(flags=flags)
    cfg = S.config(name, p)
    d = cfg["desc"]
    c, e0, c0 = S.primed_state(d, p, seed=seed) if state is None else state
    st = O.new_state(d, p, c, e0, c0)
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    before = O.diagnostics(d, p, st)
    O.step(d, p, st, inp, cfg["dt"] * dt_scale, nsteps)
    return st, before, O.diagnostics(d, p, st)


def test_without_wall_enzyme_the_placements_agree():
    p = S.params_default()
    d = S.config("channel_60x16", p)["desc"]
    c, e0, c0 = S.primed_state(d, p, seed=4)
    state = (c, np.zeros_like(e0), np.zeros_like(c0))
    a, _, _ = _run("channel_60x16", 20, 1.0, False, state)
    b, _, _ = _run("channel_60x16", 20, 1.0, True, state)
    assert np.max(np.abs(a.c - b.c)) <= 1e-15 * np.max(np.abs(a.c))
    assert np.all(b.e0 == 0) and np.all(b.c0 == 0)


def test_both_placements_keep_the_wall_enzyme_and_the_coupled_one_family_1():
    for lagged in (False, True):
        st, before, after = _run("channel_60x16", 40, 1.0, lagged)
        assert abs(after[3] - before[3]) <= 1e-14 * before[3], lagged          # sum A (E0 + C0)
        if not lagged:
            assert abs(after[1] - before[1]) <= 1e-13 * before[1]               # family 1


def test_lagged_defect_and_distance_are_first_order_in_dt():
    defect, dist = [], []
    for k in (1, 2, 4):
        lag, b0, b1 = _run("channel_60x16", 40 * k, 1.0 / k, True)
        cpl, _, _ = _run("channel_60x16", 40 * k, 1.0 / k, False)
        defect.append(abs(b1[1] - b0[1]) / b0[1])
        dist.append(np.linalg.norm(lag.c[O.E1] - cpl.c[O.E1]) / np.linalg.norm(cpl.c[O.E1]))
    assert defect[0] > 1e-10, defect
    for e in (defect, dist):
        r = [np.log2(a / b) for a, b in zip(e, e[1:])]
        assert all(0.8 < x < 1.2 for x in r), (e, r)

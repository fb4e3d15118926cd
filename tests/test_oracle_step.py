"""Whole-step properties of the oracle (Sec. 3.2 fractional step): with the
inlet and outlet closed every linear invariant of App. A/B is conserved by the
coupled transport + reaction + wall exchange; open channels stay positive."""
import numpy as np
import pytest

import oracle as O
import synthetic as S


@pytest.mark.parametrize("name", ["channel_40x12", "duct_16x8x6"])
def test_closed_channel_conserves_all_invariants(name):
    p = S.params_default(flags=O.CLOSED_ENDS)
    cfg = S.config(name, p)
    d = cfg["desc"]
    c, e0, c0 = S.primed_state(d, p, seed=3)
    st = O.new_state(d, p, c, e0, c0)
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    before = O.diagnostics(d, p, st)
    O.step(d, p, st, inp, cfg["dt"], 25)
    after = O.diagnostics(d, p, st)
    for q in range(5):
        assert after[q] == pytest.approx(before[q], rel=1e-12), q
    assert after[6] == 0
    assert np.any(st.eta > p["eta_t"])          # cohesion is active in the primed clot
    assert np.any(st.c[O.PBA] != c[O.PBA])


def test_open_channel_stays_nonnegative_and_finite():
    p = S.params_default()
    cfg = S.config("channel_200x40", p)
    d = cfg["desc"]
    c, e0, c0 = S.primed_state(d, p, seed=1)
    st = O.new_state(d, p, c, e0, c0)
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    O.step(d, p, st, inp, cfg["dt"], 40)
    dg = O.diagnostics(d, p, st)
    assert dg[6] == 0
    assert dg[5] >= -1e-12 * p["S1_plasma"]
    assert dg[7] <= 1.0

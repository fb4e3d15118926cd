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


def test_oracle_results_do_not_depend_on_the_thread_count():
    """The OpenMP loops of the oracle keep every cell's summation order: one
    thread and all host threads give the same bits (transport with both
    options, reaction, eta solve, ADP release sampling)."""
    import oracle as O
    import synthetic as S
    import numpy as np
    out = []
    for nt in (1, 0):
        O.set_threads(nt)
        for name, flags in (("channel_60x16", O.TRANSPORT_RK2 | O.STRANG), ("duct_21x9x7", O.WALL_LAGGED)):
            p = S.params_default(flags=flags, sigma_dt=2e-4)
            cfg = S.config(name, p)
            st = O.new_state(cfg["desc"], p, *S.primed_state(cfg["desc"], p, seed=3))
            inp = dict(cfg["fluxes"])
            inp.update(cfg["inlet"])
            O.step(cfg["desc"], p, st, inp, cfg["dt"], 12)
            out.append((st.c.copy(), st.eta.copy(), st.e0.copy(), st.sigma.copy()))
    O.set_threads(0)
    for a, b in zip(out[:2], out[2:]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)

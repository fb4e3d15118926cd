"""Pins of the oracle's time-order options on the whole coupled step (Sec. 3.2
fractional step; transport App. A/B/C/D, reaction App. A/B).

The plain fractional step -- forward Euler transport, then the M_rxn RK4
reaction solves -- is first order in time twice over: in the transport and in
the splitting.  Only both changes together make the step second order: Heun
(SSP-RK2) transport and Strang splitting (reaction over dt/2, transport over
dt, reaction over dt/2).  Measured on the primed channel without ADP release,
with eta held fixed and with eta re-solved at the start of every step (the
cohesion-driven P^{m,a}, P^{b,a} included then).

Exact pin: with the transport off, Strang splitting is the plain step with
twice the RK4 substeps, bit for bit."""
import numpy as np

import oracle as O
import synthetic as S

NAME = "channel_60x16"


def _run(dt_scale, extra, nbase=40, M_rxn=2, eta=False):
    p = S.params_default(flags=O.NO_SIGMA | (0 if eta else O.NO_ETA) | extra, M_rxn=M_rxn, eta_tol=1e-13)
    cfg = S.config(NAME, p)
    d = cfg["desc"]
    c, e0, c0 = S.primed_state(d, p, seed=2, noise=0.0)
    st = O.new_state(d, p, c, e0, c0)
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    O.step(d, p, st, inp, cfg["dt"] * dt_scale, int(round(nbase / dt_scale)))
    return st


def _rates(extra, eta=False, species=("S1", "E1", "Pmu", "E2")):
    sol = {k: _run(1.0 / k, extra, eta=eta).c for k in (1, 2, 4, 16)}
    out = {}
    for s in species:
        i = S.SPECIES.index(s)
        e = [np.linalg.norm(sol[k][i] - sol[16][i]) / np.linalg.norm(sol[16][i]) for k in (1, 2, 4)]
        out[s] = [np.log2(a / b) for a, b in zip(e, e[1:])]
    return out


def test_heun_with_strang_is_second_order_and_the_plain_step_first():
    both = _rates(O.TRANSPORT_RK2 | O.STRANG)
    plain = _rates(0)
    for s in both:
        assert all(1.8 < r < 2.3 for r in both[s]), (s, both[s])
        assert all(0.9 < r < 1.4 for r in plain[s]), (s, plain[s])


def test_strang_without_transport_is_the_plain_step_with_twice_the_substeps():
    a = _run(1.0, O.STRANG | O.NO_TRANSPORT, nbase=10, M_rxn=2)
    b = _run(1.0, O.NO_TRANSPORT, nbase=10, M_rxn=4)
    assert np.array_equal(a.c, b.c) and np.array_equal(a.e0, b.e0) and np.array_equal(a.c0, b.c0)


def test_second_order_holds_with_eta_resolved_every_step():
    both = _rates(O.TRANSPORT_RK2 | O.STRANG, eta=True, species=("S1", "E1", "Pmu", "Pma", "Pba", "E2"))
    for s in both:
        assert all(1.8 < r < 2.3 for r in both[s]), (s, both[s])

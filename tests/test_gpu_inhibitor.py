"""The inhibitor extension on the GPU -- the paper's example of adding a
species (Sec. "Adapting the framework for different clotting models"): a
fluid-phase inhibitor I with I + E2 -> E2,inh at rate kI I E2, transported like
the coagulation species and reacted in the same RK4 stages -- against the
oracle's extension (tests/test_oracle_inhibitor.py pins it): the 2D channel
(plane kernel), a 3D duct (TMA z march), the second-order options (the
extension's own two-stage transport pass and the reaction half-steps), and
family 2 + E2,inh conserved in a closed channel.  kI is set large enough that
the inhibition visibly moves thrombin within the run (the paper gives no
value).  Tolerance: the parity bar, rel-L2 <= 1e-5 per species and per row."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from parity_util import rel_l2, species_errors

pytestmark = pytest.mark.gpu

TOL = 1e-5
KI, I_IN = 5.0e4, 3.0e-4


def _ext0(d, seed):
    n = S.ncell(d)
    rng = np.random.default_rng(seed)
    return np.stack([I_IN * (1.0 + 0.01 * rng.standard_normal(n)), np.zeros(n)])


def _pair(name, steps, oflags=0, gflags=0, seed=2, closed=False):
    import torch

    import paper_2304_09180_gb300 as clot
    base = O.CLOSED_ENDS | O.NO_SIGMA if closed else 0
    po = S.params_default(flags=base | oflags, kI=KI, I_in=I_IN)
    cfg = S.config(name, po)
    d = cfg["desc"]
    state = S.primed_state(d, po, seed=seed)
    x0 = _ext0(d, seed + 100)
    st = O.new_state(d, po, *state, ext=x0)
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    b0 = O.diagnostics(d, po, st)
    O.step(d, po, st, inp, cfg["dt"], steps)
    mesh = clot.Mesh(d)
    prm = clot.Params(S.params_default(kI=KI, I_in=I_IN), **cfg["inlet"], eta_tol=1e-6, flags=base | gflags)
    f = clot.Fields.from_host(mesh, prm.d, *state, ext=x0)
    g0 = clot.clot_diagnostics(mesh, f, prm)
    fl = clot.Fluxes(mesh, **cfg["fluxes"])
    for n in (steps // 2, steps - steps // 2):
        clot.clot_species_step(mesh, f, fl, prm, cfg["dt"], n)
    torch.cuda.synchronize()
    g1 = clot.clot_diagnostics(mesh, f, prm)
    return st, f.to_host(mesh), (b0, O.diagnostics(d, po, st)), (g0, g1), clot


def _check(ref, gpu):
    errs = species_errors(gpu["c"], ref.c)
    assert np.all(errs <= TOL), dict(zip(S.SPECIES, errs))
    assert rel_l2(gpu["ext"][0], ref.ext[0], I_IN) <= TOL
    assert rel_l2(gpu["ext"][1], ref.ext[1], 1e-6) <= TOL
    assert rel_l2(gpu["e0"], ref.e0) <= TOL and rel_l2(gpu["c0"], ref.c0, 1e-9) <= TOL
    assert ref.ext[1].max() > 0.0


@pytest.mark.parametrize("name,steps", [("channel_200x40", 200), ("duct_64x36x20", 20)])
def test_inhibitor_matches_oracle(name, steps):
    ref, gpu, _, _, _ = _pair(name, steps)
    _check(ref, gpu)


def test_inhibitor_with_heun_and_strang_matches_oracle():
    import paper_2304_09180_gb300 as clot
    ref, gpu, _, _, _ = _pair("channel_60x16", 60, O.TRANSPORT_RK2 | O.STRANG, clot.HEUN | clot.STRANG)
    _check(ref, gpu)


def test_inhibitor_closed_channel_keeps_family_2_with_e2inh():
    ref, gpu, (b0, b1), (g0, g1), _ = _pair("channel_60x16", 40, closed=True)
    assert abs(b1[2] - b0[2]) <= 1e-12 * b0[2]
    assert abs(g1[2] - g0[2]) <= 2e-6 * g0[2]
    _check(ref, gpu)

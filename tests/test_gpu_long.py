"""Full-length parity runs (many minutes of oracle time; run with
CLOT_LONG_TESTS=1): the 1024 x 256 channel at shear 1500/s over its full 2000
steps, FP32 GPU against the FP64 oracle (OpenMP over the host cores; its result
does not depend on the thread count), with the per-species relative L2 error
(the metric of the paper's convergence study, supporting information) and the
mass balance of each invariant reported."""
import json

import numpy as np
import pytest

import oracle as O
import synthetic as S
from parity_util import rel_l2, run_gpu, run_oracle, species_errors

pytestmark = [pytest.mark.gpu, pytest.mark.long]

TOL = 1e-5


def _balance(gpu_diag, ref_diag):
    names = ("platelets", "family1+wall", "family2", "wall enzyme", "ADP")
    return {n: float(abs(g - r) / max(abs(r), 1e-300)) for n, g, r in zip(names, gpu_diag[:5], ref_diag[:5])}


@pytest.mark.parametrize("state_kind", ["plasma", "primed"])
def test_channel_1024x256_full_2000_steps(state_kind):
    import paper_2304_09180_gb300 as clot
    O.set_threads(0)
    p = S.params_default()
    cfg = S.config("channel_1024x256", p)
    d = cfg["desc"]
    state = S.plasma_state(d, p, seed=2) if state_kind == "plasma" else S.primed_state(d, p, seed=2)
    n = cfg["nsteps"]
    ref = run_oracle(cfg, p, state, n)
    gpu = run_gpu(cfg, p, state, n, calls=4, eta_tol=1e-6)
    errs = species_errors(gpu["c"], ref.c)
    g = clot.clot_diagnostics(gpu["mesh"], gpu["fields"], gpu["params"])
    r = O.diagnostics(d, p, ref)
    out = {"config": "channel_1024x256", "state": state_kind, "steps": n,
           "rel_l2": {s: float(e) for s, e in zip(S.SPECIES, errs)},
           "e0": rel_l2(gpu["e0"], ref.e0), "c0": rel_l2(gpu["c0"], ref.c0, 1e-9),
           "eta": rel_l2(gpu["eta"], ref.eta),
           "balance_gpu_vs_oracle": _balance(g, r), "min_gpu": float(g[5]), "min_oracle": float(r[5])}
    print("RESULT " + json.dumps(out))
    assert np.all(errs <= TOL), out["rel_l2"]
    assert out["e0"] <= TOL and out["c0"] <= TOL

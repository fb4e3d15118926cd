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

TOL = 1e-5   # the parity bar of the 200-step runs


def _balance(gpu_diag, ref_diag):
    names = ("platelets", "family1+wall", "family2", "wall enzyme", "ADP")
    return {n: float(abs(g - r) / max(abs(r), 1e-300)) for n, g, r in zip(names, gpu_diag[:5], ref_diag[:5])}


def test_channel_1024x256_full_2000_steps():
    """The plasma state over the full 2000 steps, with the full-value FP32
    state and in the deviation form (CLOT_DEVIATION), against one oracle run."""
    import paper_2304_09180_gb300 as clot
    O.set_threads(0)
    p = S.params_default()
    cfg = S.config("channel_1024x256", p)
    d = cfg["desc"]
    state = S.plasma_state(d, p, seed=2)
    n = cfg["nsteps"]
    ref = run_oracle(cfg, p, state, n)
    r = O.diagnostics(d, p, ref)
    for form, flags in (("plain", 0), ("deviation", clot.DEVIATION)):
        gpu = run_gpu(cfg, p, state, n, calls=4, eta_tol=1e-6, flags=flags)
        errs = species_errors(gpu["c"], ref.c)
        g = clot.clot_diagnostics(gpu["mesh"], gpu["fields"], gpu["params"])
        out = {"config": "channel_1024x256", "state": "plasma", "form": form, "steps": n,
               "rel_l2": {s: float(e) for s, e in zip(S.SPECIES, errs)},
               "e0": rel_l2(gpu["e0"], ref.e0), "c0": rel_l2(gpu["c0"], ref.c0, 1e-9),
               "eta": rel_l2(gpu["eta"], ref.eta),
               "balance_gpu_vs_oracle": _balance(g, r), "min_gpu": float(g[5]), "min_oracle": float(r[5])}
        print("RESULT " + json.dumps(out))
        # The FP32 state is rounded once per step: over n steps a slowly varying
        # field can gather up to n roundings of 2^-24 in one direction.  Ten times
        # the 200-step horizon of the parity bar, the bound is n 2^-24 = 1.2e-4
        # (measured up to 1.7e-5 with the full-value state, in S1b and S1, which
        # change by ~1e-4 of their plasma values over the run); the invariants
        # agree to ~2e-7.
        bound = n * 2.0 ** -24
        assert np.all(errs <= bound), out["rel_l2"]
        assert out["e0"] <= bound and out["c0"] <= bound
        assert all(v <= 1e-6 for v in out["balance_gpu_vs_oracle"].values()), out["balance_gpu_vs_oracle"]


@pytest.mark.parametrize("mode", ["plain", "heun_strang", "heun_strang_deviation"])
def test_mesh_convergence_against_the_papers_finest_mesh(mode):
    """The paper's mesh study down to its finest mesh (0.1875 um; 538,261 steps
    of a 640 x 160 channel to t = 5 s).  E1 and E2 + E2^b converge at 1.4 or
    better in every mode.  S1 changes by only ~1e-4 of its plasma value, so
    its discretisation errors on the finer meshes (~3e-5) are of the size of
    what the FP32 state loses to rounding over a few hundred thousand steps:
    with the full-value FP32 state its rate flattens (1.4 plain, 1.1 with the
    second-order options, whose extra passes round more often).  In the
    deviation form (CLOT_DEVIATION) the rounding floor falls away and S1 must
    converge like the other chemicals, at 1.4 or better."""
    import paper_2304_09180_gb300 as clot
    from test_gpu_mesh_convergence import rates_against_finest
    flags = {"plain": 0, "heun_strang": clot.HEUN | clot.STRANG,
             "heun_strang_deviation": clot.HEUN | clot.STRANG | clot.DEVIATION}[mode]
    rates, errs = rates_against_finest((3.0, 1.5, 0.75, 0.375, 0.1875), flags)
    print("RESULT " + json.dumps({"mesh_study": mode, "rates": {k: float(v) for k, v in rates.items()},
                                  "errors": {k: [float(e) for e in v] for k, v in errs.items()}}))
    for s in ("E1", "E2tot"):
        assert rates[s] >= 1.4, rates
    if flags & clot.DEVIATION:
        assert rates["S1"] >= 1.4, rates

"""clot_eta_solve_noalloc: the eta solve for callers that cannot allocate
device memory (code under another framework's allocator, real-time loops that
must not take cudaMalloc's implicit synchronisation, tools without a
clot_mesh).  Its scratch is a static device array of the library, shared by
every call, so two calls in a row on different meshes must not see each
other's leftovers.  This file is collected last on purpose."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu


def test_noalloc_eta_solve_matches_the_mesh_entry_point_on_two_calls_in_a_row():
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    for name, seed in (("channel_200x40", 6), ("duct_24x12x10", 11)):
        cfg = S.config(name, p)
        d = cfg["desc"]
        c, e0, c0 = S.primed_state(d, p, seed=seed)
        mesh = clot.Mesh(d)
        f = clot.Fields.from_host(mesh, p, c, e0, c0)
        prm = clot.Params(p, **cfg["inlet"], eta_tol=1e-6)
        it_ref = clot.clot_eta_solve(mesh, f, prm)
        eta = torch.zeros_like(f.eta)
        it = clot.clot_eta_solve_noalloc(d, f.c, mesh.pitch, eta, prm)
        torch.cuda.synchronize()
        thB = (np.asarray(c, np.float32)[2].astype(np.float64) + np.asarray(c, np.float32)[3]) / p["Pmax"]
        assert it > 0 and abs(it - it_ref) <= 1
        # the tolerance of the eta parity test: 2e-6 of max theta_B
        assert np.max(np.abs(eta.double().cpu().numpy() - f.eta.double().cpu().numpy())) <= 2e-6 * thB.max()


def test_noalloc_eta_solve_rejects_meshes_above_its_scratch_size():
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config("channel_40x12", p)
    big = dict(cfg["desc"], nx=2048, ny=1024)            # 2,097,152 cells > 1,048,576
    c = torch.zeros((15, 64), dtype=torch.float32, device="cuda")
    eta = torch.zeros(64, dtype=torch.float32, device="cuda")
    prm = clot.Params(p, **cfg["inlet"])
    with pytest.raises(clot.ClotError, match="at most 1048576"):
        clot.clot_eta_solve_noalloc(big, c, 2048 * 1024, eta, prm)

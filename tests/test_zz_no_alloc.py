"""clot_eta_solve_noalloc: the eta solve for callers that cannot allocate
device memory (code under another framework's allocator, real-time loops that
must not take cudaMalloc's implicit synchronisation, tools without a
clot_mesh).  Its scratch is a static device array of the library, shared by
every call, so two calls in a row on different meshes must not see each
other's leftovers.

This file is collected last on purpose (its name sorts after every other test
file): the shared array keeps whatever the previous call left in it, so these
tests also show that a call after all the other GPU tests of the session gets
the same result as in a fresh process, and, if they fail, a run that stops at
the first failure has already run every other test."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

ETIMEOUT = -4


def _case(name, seed):
    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config(name, p)
    d = cfg["desc"]
    c, e0, c0 = S.primed_state(d, p, seed=seed)
    mesh = clot.Mesh(d)
    f = clot.Fields.from_host(mesh, p, c, e0, c0)
    prm = clot.Params(p, **cfg["inlet"], eta_tol=1e-6)
    thB = (np.asarray(c, np.float32)[2].astype(np.float64) + np.asarray(c, np.float32)[3]) / p["Pmax"]
    _case.last = (p, cfg)
    return clot, d, mesh, f, prm, thB


def test_noalloc_eta_solve_matches_the_mesh_entry_point_on_two_calls_in_a_row():
    import torch

    for name, seed in (("channel_200x40", 6), ("duct_24x12x10", 11)):
        clot, d, mesh, f, prm, thB = _case(name, seed)
        it_ref = clot.clot_eta_solve(mesh, f, prm)
        eta = torch.zeros_like(f.eta)
        it = clot.clot_eta_solve_noalloc(d, f.c, mesh.pitch, eta, prm)
        torch.cuda.synchronize()
        assert it > 0 and abs(it - it_ref) <= 1
        # the tolerance of the eta parity test: 2e-6 of max theta_B
        assert np.max(np.abs(eta.double().cpu().numpy() - f.eta.double().cpu().numpy())) <= 2e-6 * thB.max()


def test_noalloc_ragged_mesh_wide_pitch_and_no_iteration_count():
    """nx not a multiple of 4 (the solver's scalar passes) and a state pitch
    wider than the mesh needs; the second call passes no iteration count, so it
    does not synchronise and the result is read after a stream synchronise."""
    import torch

    clot, d, mesh, f, prm, thB = _case("duct_30x12x9", 4)
    clot.clot_eta_solve(mesh, f, prm)
    nc = mesh.ncell
    pitch = mesh.pitch + 96
    cw = torch.zeros((15, pitch), dtype=torch.float32, device="cuda")
    cw[:, :nc] = f.c[:, :nc]
    ref = f.eta.double().cpu().numpy()
    for want in (True, False):
        eta = torch.zeros(nc, dtype=torch.float32, device="cuda")
        it = clot.clot_eta_solve_noalloc(d, cw, pitch, eta, prm, want_iters=want)
        torch.cuda.synchronize()
        assert (it is not None and it > 0) if want else it is None
        assert np.max(np.abs(eta.double().cpu().numpy() - ref)) <= 2e-6 * thB.max()


def test_noalloc_eta_solve_rejects_meshes_above_its_scratch_size():
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config("channel_40x12", p)
    big = dict(cfg["desc"], nx=2048, ny=1024)            # 2,097,152 cells > 1,048,576
    c = torch.zeros((15, 2048 * 1024), dtype=torch.float32, device="cuda")
    eta = torch.zeros(2048 * 1024, dtype=torch.float32, device="cuda")
    prm = clot.Params(p, **cfg["inlet"])
    with pytest.raises(clot.ClotError, match="at most 1048576"):
        clot.clot_eta_solve_noalloc(big, c, 2048 * 1024, eta, prm)


def test_noalloc_timeout_without_iteration_count_is_reported_by_the_next_call():
    """A grid-barrier wait bound of 1 ns makes the solver's blocks give up
    (they return; nothing hangs).  A call without an iteration count cannot
    report that itself; the flag stays in the shared status words and the next
    call that asks for the count reports CLOT_ETIMEOUT once."""
    import torch

    clot, d, mesh, f, prm, thB = _case("channel_200x40", 9)
    p, cfg = _case.last
    fast = clot.Params(p, **cfg["inlet"], eta_tol=1e-6, wait_s=1e-9)
    eta = torch.zeros_like(f.eta)
    assert clot.clot_eta_solve_noalloc(d, f.c, mesh.pitch, eta, fast, want_iters=False) is None
    torch.cuda.synchronize()
    eta.zero_()
    with pytest.raises(clot.ClotError) as ei:
        clot.clot_eta_solve_noalloc(d, f.c, mesh.pitch, eta, prm)
    assert ei.value.code == ETIMEOUT
    it = clot.clot_eta_solve_noalloc(d, f.c, mesh.pitch, eta, prm)   # reported once, then clear
    assert it > 0

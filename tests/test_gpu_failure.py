"""Failure detection on the GPU without a GPU fault.

The eta solver's grid barrier waits at most params.wait_s; a tiny bound makes
the waits give up as soon as a block has to wait for another, the blocks
return (the kernel ends, the context stays usable) and the timeout bit of the
device status word is set.  These tests check that every entry point that
reads the status word reports it exactly once, and that the non-finite count
of the diagnostics becomes CLOT_ENONFINITE.  Nothing here faults, traps or
hangs a GPU: the waits are bounded and the solver has no copies in flight."""
import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

ETIMEOUT, ENONFINITE = -4, -3


def _setup(name="channel_200x40", seed=5):
    import paper_2304_09180_gb300 as clot
    p = S.params_default(eta_tol=1e-6)
    cfg = S.config(name, p)
    d = cfg["desc"]
    c, e0, c0 = S.primed_state(d, p, seed=seed)
    mesh = clot.Mesh(d)
    return clot, p, cfg, mesh, (c, e0, c0)


def test_eta_solve_reports_a_barrier_timeout_once_and_recovers():
    clot, p, cfg, mesh, st = _setup()
    f = clot.Fields.from_host(mesh, p, *st)
    fast = clot.Params(p, **cfg["inlet"], wait_s=1e-9)
    with pytest.raises(clot.ClotError) as ei:
        clot.clot_eta_solve(mesh, f, fast)       # cold start: many grid barriers
    assert ei.value.code == ETIMEOUT
    assert clot.clot_device_status(mesh) >= 0    # reported once: the flag was cleared
    ref = clot.Fields.from_host(mesh, p, *st)
    prm = clot.Params(p, **cfg["inlet"])
    clot.clot_eta_solve(mesh, ref, prm)          # the context and the mesh stay usable
    clot.clot_eta_solve(mesh, f, prm)
    a, b = f.eta.double().cpu().numpy(), ref.eta.double().cpu().numpy()
    assert np.max(np.abs(a - b)) <= 2e-6 * max(b.max(), 1e-30)


def test_species_step_reports_the_timeout_when_asked():
    clot, p, cfg, mesh, st = _setup()
    fl = clot.Fluxes(mesh, **cfg["fluxes"])
    f = clot.Fields.from_host(mesh, p, *st)
    prm = clot.Params(p, **cfg["inlet"], wait_s=1e-9, flags=clot.binding.SYNC_STATUS)
    with pytest.raises(clot.ClotError) as ei:
        clot.clot_species_step(mesh, f, fl, prm, cfg["dt"], 2)
    assert ei.value.code == ETIMEOUT
    clot.clot_device_status(mesh)                # already reported and cleared
    ok = clot.Params(p, **cfg["inlet"], flags=clot.binding.SYNC_STATUS)
    clot.clot_species_step(mesh, f, fl, ok, cfg["dt"], 2)


def test_device_status_reports_a_timeout_of_an_asynchronous_step():
    clot, p, cfg, mesh, st = _setup()
    fl = clot.Fluxes(mesh, **cfg["fluxes"])
    f = clot.Fields.from_host(mesh, p, *st)
    prm = clot.Params(p, **cfg["inlet"], wait_s=1e-9)
    clot.clot_species_step(mesh, f, fl, prm, cfg["dt"], 1)   # does not synchronise: returns OK
    with pytest.raises(clot.ClotError) as ei:
        clot.clot_device_status(mesh)
    assert ei.value.code == ETIMEOUT
    clot.clot_device_status(mesh)


def test_diagnostics_report_non_finite_values():
    clot, p, cfg, mesh, st = _setup()
    f = clot.Fields.from_host(mesh, p, *st)
    prm = clot.Params(p, **cfg["inlet"])
    clot.clot_diagnostics(mesh, f, prm)
    f.c[7, 123] = float("nan")
    f.c[2, 45] = float("inf")
    with pytest.raises(clot.ClotError) as ei:
        clot.clot_diagnostics(mesh, f, prm)
    assert ei.value.code == ENONFINITE
    out = clot.clot_diagnostics(mesh, f, prm, check=False)
    assert out[6] == 2

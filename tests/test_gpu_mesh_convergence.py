"""The paper's mesh convergence study (supporting information, "Mesh
convergence study") on the GPU path, with the flow frozen: a 120 x 30 um
channel with a 45 um injury, square cells of h = 3, 1.5, 0.75 and 0.375 um,
each run to t = 5 s at its own Courant-0.5 time step; errors of S1, E1, P^{m,u}
and E2 + E2^b against the finest mesh in relative l2 (the paper's E(psi_h)),
rates by a least-squares line in log-log.

Readings: the finest solution is averaged onto each coarser mesh (the cell
averages a finite-volume solution carries; sampling the coarse cells at fine
cell centres, as a point resampler does, adds an O(h) error of its own and
caps every rate near 1); initial data without noise and an injury aligned with
the coarsest cells (36 .. 81 um), so that neither seeds an O(h) error.

The paper finds second order for the fluid-phase chemicals and a super-linear
rate for the platelets.  Against the paper's finest mesh (0.1875 um, too slow for
a test) E1 converges at 2.0, E2 + E2^b at 1.7 and P^{m,u} at 2.2, while the error
of S1, which changes by only ~1e-4 of its inlet value, flattens at the finest
mesh (rate 1.1; most likely the first-order time error of the step, dt scaling
with h).  The test asserts E1 and E2 + E2^b at 1.4, S1 at first order and
P^{m,u} above 1.2."""
import math

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

UM = 1e-3
HS = (3.0, 1.5, 0.75, 0.375)


def _run(h, flags=0):
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default(eta_tol=1e-6, flags=flags)
    nx, ny = int(round(120 / h)), int(round(30 / h))
    d = S.channel2d(nx, ny, 120 * UM, 30 * UM, inj_frac=(36 / 120, 81 / 120))
    fl = S.fluxes_channel2d(d, 1000.0)
    n = math.ceil(5.0 / S.stable_dt(d, fl, p) - 1e-9)
    dt = 5.0 / n
    mesh = clot.Mesh(d)
    flx = clot.Fluxes(mesh, **fl)
    prm = clot.Params(p, **S.inlet_values(d, p))
    f = clot.Fields.from_host(mesh, p, *S.plasma_state(d, p, seed=1, noise=0.0))
    done = 0
    while done < n:
        k = min(20000, n - done)
        clot.clot_species_step(mesh, f, flx, prm, dt, k)
        done += k
    torch.cuda.synchronize()
    dg = clot.clot_diagnostics(mesh, f, prm)
    assert dg[6] == 0 and abs(f.t - 5.0) < 1e-9
    c = f.c[:, :nx * ny].double().cpu().numpy()
    ix = {s: q for q, s in enumerate(S.SPECIES)}
    out = {s: c[ix[s]].reshape(ny, nx) for s in ("S1", "E1", "Pmu")}
    out["E2tot"] = (c[ix["E2"]] + c[ix["E2b"]]).reshape(ny, nx)
    return out


def rates_against_finest(hs, flags=0):
    """Errors of the coarser meshes of hs against the finest (cell averages)
    and the least-squares rates."""
    sol = {h: _run(h, flags) for h in hs}
    ref = sol[hs[-1]]
    rates, allerrs = {}, {}
    for s in ("S1", "E1", "Pmu", "E2tot"):
        errs = []
        for h in hs[:-1]:
            m = int(round(h / hs[-1]))
            ny, nx = ref[s].shape
            avg = ref[s].reshape(ny // m, m, nx // m, m).mean(axis=(1, 3))
            errs.append(np.linalg.norm(sol[h][s] - avg) / np.linalg.norm(avg))
        allerrs[s] = errs
        rates[s] = np.polyfit(np.log(hs[:-1]), np.log(errs), 1)[0]
    return rates, allerrs


def test_mesh_convergence_rates():
    sol = {h: _run(h) for h in HS}
    ref = sol[HS[-1]]
    rates = {}
    for s in ("S1", "E1", "Pmu", "E2tot"):
        errs = []
        for h in HS[:-1]:
            m = int(round(h / HS[-1]))
            ny, nx = ref[s].shape
            avg = ref[s].reshape(ny // m, m, nx // m, m).mean(axis=(1, 3))
            errs.append(np.linalg.norm(sol[h][s] - avg) / np.linalg.norm(avg))
        assert all(b < a for a, b in zip(errs, errs[1:])), (s, errs)
        rates[s] = np.polyfit(np.log(HS[:-1]), np.log(errs), 1)[0]
    # fluid-phase chemicals: second order in the paper; S1 is bound by the time error
    for s in ("E1", "E2tot"):
        assert rates[s] >= 1.4, rates
    assert rates["S1"] >= 1.0, rates
    # platelets: super-linear in the paper
    assert rates["Pmu"] > 1.2, rates


@pytest.mark.parametrize("deviation", [False, True])
def test_mesh_convergence_with_second_order_time_stepping(deviation):
    """The same study with CLOT_HEUN | CLOT_STRANG (second order in time, like the
    paper's Crank-Nicolson transport), with the full-value FP32 state and in
    the deviation form (CLOT_DEVIATION, which keeps S1's slow increments from
    FP32 rounding): every rate at least that of the plain step's assertions,
    S1 included at 1.4."""
    import paper_2304_09180_gb300 as clot
    flags = clot.HEUN | clot.STRANG | (clot.DEVIATION if deviation else 0)
    rates, errs = rates_against_finest(HS, flags)
    print("second-order rates against 0.375 um:", rates, errs)
    for s in ("S1", "E1", "E2tot"):
        assert rates[s] >= 1.4, rates
    assert rates["Pmu"] > 1.2, rates

"""Parity of the CUDA species step (through the C ABI) with the FP64 oracle on
the same seeded inputs.  Tolerance: relative L2 per species <= 1e-5 after the
configured number of FP32 steps (rel-L2 as in the paper's convergence study),
with an RMS floor of 1e-12 of each species' natural scale."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from parity_util import SCALE, rel_l2, run_gpu, run_oracle, species_errors

pytestmark = pytest.mark.gpu

TOL = 1e-5
GPU_ETA_TOL = 1e-6


def _report(errs):
    return ", ".join(f"{n}={e:.1e}" for n, e in zip(S.SPECIES, errs))


@pytest.mark.parametrize("name,steps", [("channel_200x40", 200), ("paper_128x32", 200)])
def test_plasma_channel_matches_oracle(name, steps):
    p = S.params_default()
    cfg = S.config(name, p)
    state = S.plasma_state(cfg["desc"], p, seed=1)
    ref = run_oracle(cfg, p, state, steps)
    gpu = run_gpu(cfg, p, state, steps, eta_tol=GPU_ETA_TOL)
    errs = species_errors(gpu["c"], ref.c)
    assert np.all(errs <= TOL), _report(errs)
    assert rel_l2(gpu["e0"], ref.e0) <= TOL and rel_l2(gpu["c0"], ref.c0, 1e-9) <= TOL


@pytest.mark.parametrize("seed", [0, 3])
def test_primed_clot_matches_oracle(seed):
    """Stiff path: cohesion (eta > eta_t), binding near saturation, ADP and
    thrombin activation, wall complex -- 200 steps of the 200x40 channel."""
    p = S.params_default()
    cfg = S.config("channel_200x40", p)
    state = S.primed_state(cfg["desc"], p, seed=seed)
    ref = run_oracle(cfg, p, state, 200)
    gpu = run_gpu(cfg, p, state, 200, eta_tol=GPU_ETA_TOL)
    errs = species_errors(gpu["c"], ref.c)
    assert np.all(errs <= TOL), _report(errs)
    assert rel_l2(gpu["eta"], ref.eta) <= 1e-5
    assert rel_l2(gpu["e0"], ref.e0) <= TOL and rel_l2(gpu["c0"], ref.c0) <= TOL


@pytest.mark.parametrize("name", ["channel_4x4", "channel_37x11", "duct_5x3x3", "duct_21x9x7"])
def test_small_and_ragged_meshes_elementwise(name):
    p = S.params_default()
    cfg = S.config(name, p)
    state = S.primed_state(cfg["desc"], p, seed=2)
    ref = run_oracle(cfg, p, state, 30)
    gpu = run_gpu(cfg, p, state, 30, calls=3, eta_tol=GPU_ETA_TOL)
    for s in range(15):
        scale = max(np.max(np.abs(ref.c[s])), 1e-12 * SCALE[s])
        assert np.max(np.abs(gpu["c"][s] - ref.c[s])) <= 1e-5 * scale, S.SPECIES[s]


def test_upwind_closed_box_conserves_in_fp32():
    import paper_2304_09180_gb300 as clot
    p = S.params_default(limiter=0, flags=O.CLOSED_ENDS)
    cfg = S.config("duct_24x10x8", p)
    state = S.primed_state(cfg["desc"], p, seed=4)
    gpu = run_gpu(cfg, p, state, 1, eta_tol=GPU_ETA_TOL)
    before = clot.clot_diagnostics(gpu["mesh"], gpu["fields"], gpu["params"])
    clot.clot_species_step(gpu["mesh"], gpu["fields"],
                           clot.Fluxes(gpu["mesh"], **cfg["fluxes"]), gpu["params"], cfg["dt"], 50)
    after = clot.clot_diagnostics(gpu["mesh"], gpu["fields"], gpu["params"])
    for q in range(5):
        assert after[q] == pytest.approx(before[q], rel=2e-6), q
    assert after[6] == 0


def test_diagnostics_match_oracle():
    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config("channel_37x11", p)
    state = S.primed_state(cfg["desc"], p, seed=5)
    mesh = clot.Mesh(cfg["desc"])
    f = clot.Fields.from_host(mesh, p, *state)
    prm = clot.Params(p, **cfg["inlet"])
    dg = clot.clot_diagnostics(mesh, f, prm)
    # the oracle sees the same FP32-rounded state
    c32 = [np.asarray(a, np.float32).astype(np.float64) for a in state]
    st = O.new_state(cfg["desc"], p, *c32)
    ref = O.diagnostics(cfg["desc"], p, st)
    # the kernel sums each cell's species group in FP32 (at most 3 roundings of
    # 2^-24 of the group's magnitude) and accumulates the cells in FP64
    c = c32[0]
    d = cfg["desc"]
    V = d["hx"] * d["hy"] * d["hz"]
    g = {0: [0, 1, 2, 3], 1: [5, 7, 9, 11, 13, 14], 2: [6, 8, 10, 12, 13, 14], 4: [4]}
    for q, rows in g.items():
        bound = 4 * 2.0 ** -24 * V * np.abs(c[rows]).sum() + 1e-300
        assert abs(dg[q] - ref[q]) <= bound, (q, dg[q], ref[q], bound)
    assert dg[3] == pytest.approx(ref[3], rel=1e-12)             # wall sums: FP64 per face
    assert dg[5] == ref[5] and dg[6] == ref[6]                   # minimum and non-finite count: exact
    assert dg[7] == pytest.approx(ref[7], rel=2.0 ** -22)


def test_reaction_step_matches_oracle_on_random_states():
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config("channel_96x40", p)
    d = cfg["desc"]
    nc = S.ncell(d)
    c, eta = S.random_reaction_states(nc, p, seed=9)
    e0 = np.full(int(S.floor_patch_mask(d).sum()), 1.2e-7)
    c0 = np.full_like(e0, 2e-8)
    mesh = clot.Mesh(d)
    f = clot.Fields.from_host(mesh, p, c, e0, c0, eta=eta)
    prm = clot.Params(p, **cfg["inlet"])
    h, nsub = 2e-5, 5
    clot.clot_reaction_step(mesh, f, prm, h, nsub)
    torch.cuda.synchronize()
    g = f.to_host(mesh)
    c32, eta32, e032, c032 = (np.asarray(a, np.float32).astype(np.float64) for a in (c, eta, e0, c0))
    rc, re0, rc0 = O.reaction(d, p, c32, e032, c032, eta32, h, nsub)
    errs = species_errors(g["c"], rc)
    assert np.all(errs <= TOL), _report(errs)
    assert rel_l2(g["e0"], re0) <= TOL and rel_l2(g["c0"], rc0) <= TOL


@pytest.mark.parametrize("name", ["channel_200x40", "duct_24x12x10"])
def test_eta_solve_matches_oracle(name):
    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config(name, p)
    d = cfg["desc"]
    c, e0, c0 = S.primed_state(d, p, seed=6)
    mesh = clot.Mesh(d)
    f = clot.Fields.from_host(mesh, p, c, e0, c0)
    prm = clot.Params(p, **cfg["inlet"], eta_tol=1e-6)
    it = clot.clot_eta_solve(mesh, f, prm)
    assert 0 < it < 1000
    c32 = np.asarray(c, np.float32).astype(np.float64)
    thB = (c32[O.PBA] + c32[O.PBSE]) / p["Pmax"]
    ref, _ = O.eta_solve(d, p, thB)
    gpu = f.eta.double().cpu().numpy()
    assert np.max(np.abs(gpu - ref)) <= 2e-6 * np.max(thB)
    assert clot.clot_device_status(mesh) == it


def test_sigma_release_sampling_matches_oracle():
    """ADP release with a short sampling interval so samples fire in the run."""
    cfg = S.config("channel_60x16")
    dt = cfg["dt"]
    p = S.params_default(sigma_dt=10 * dt, sigma_tf=60 * dt)
    state = S.primed_state(cfg["desc"], p, seed=7)
    ref = run_oracle(cfg, p, state, 150)
    gpu = run_gpu(cfg, p, state, 150, calls=4, eta_tol=GPU_ETA_TOL)
    # step starts t = 0 .. 149 dt: samples at t = 10 dt, 20 dt, ..., 140 dt
    assert ref.n_samples == 14 and gpu["fields"].n_samples == 14
    assert rel_l2(gpu["sigma"], ref.sigma) <= 1e-5
    errs = species_errors(gpu["c"], ref.c)
    assert np.all(errs <= TOL), _report(errs)


def test_channel_1024x256_matches_oracle_over_100_steps():
    p = S.params_default()
    cfg = S.config("channel_1024x256", p)
    state = S.plasma_state(cfg["desc"], p, seed=2)
    ref = run_oracle(cfg, p, state, 100)
    gpu = run_gpu(cfg, p, state, 100, eta_tol=GPU_ETA_TOL)
    errs = species_errors(gpu["c"], ref.c)
    assert np.all(errs <= TOL), _report(errs)


def test_primed_duct_over_several_z_runs_matches_oracle():
    """The 3D step marches runs of 16 planes per block: 37 planes (runs of 16,
    16, 5) and ragged x / y tiles, primed clot state (cohesion, binding, wall
    exchange, eta prediction), 30 steps."""
    p = S.params_default()
    cfg = S.config("duct_40x20x37", p)
    state = S.primed_state(cfg["desc"], p, seed=4)
    ref = run_oracle(cfg, p, state, 30)
    gpu = run_gpu(cfg, p, state, 30, eta_tol=GPU_ETA_TOL)
    errs = species_errors(gpu["c"], ref.c)
    assert np.all(errs <= TOL), _report(errs)
    assert rel_l2(gpu["e0"], ref.e0) <= TOL and rel_l2(gpu["c0"], ref.c0, 1e-9) <= TOL


def test_primed_duct_64x128x128_subbox_matches_oracle_over_20_steps():
    """The benchmarked duct's cross-section (128 x 128 cells of 1.5 um) on a
    64-cell-long sub-box, in the primed clot state (every mobile species,
    cohesion, binding and the wall complex active, eta corrected every step),
    20 steps through the TMA z march, against the FP64 oracle."""
    O.set_threads(0)
    p = S.params_default()
    cfg = S.config("duct_64x128x128", p)
    state = S.primed_state(cfg["desc"], p, seed=6)
    ref = run_oracle(cfg, p, state, 20)
    gpu = run_gpu(cfg, p, state, 20, calls=2, eta_tol=GPU_ETA_TOL)
    errs = species_errors(gpu["c"], ref.c)
    assert np.all(errs <= TOL), _report(errs)
    assert rel_l2(gpu["e0"], ref.e0) <= TOL and rel_l2(gpu["c0"], ref.c0, 1e-9) <= TOL
    assert rel_l2(gpu["eta"], ref.eta) <= 1e-5


def test_duct_512x128x128_full_size_matches_oracle():
    """The benchmarked 3D duct at full size, in the bench's launch
    configuration, compared element by element over two steps."""
    p = S.params_default()
    cfg = S.config("duct_512x128x128", p)
    state = S.plasma_state(cfg["desc"], p, seed=1)
    ref = run_oracle(cfg, S.params_default(eta_tol=1e-10), state, 2)
    gpu = run_gpu(cfg, p, state, 2, eta_tol=GPU_ETA_TOL)
    errs = species_errors(gpu["c"], ref.c)
    assert np.all(errs <= TOL), _report(errs)
    assert rel_l2(gpu["e0"], ref.e0) <= TOL


def test_eta_prediction_continues_across_calls():
    """Ten calls of 5 steps give the state of one call of 50 steps bit for bit
    (the eta prediction carries over between calls on the same fields), and
    CLOT_ETA_FRESH restarts it, within the parity tolerance of the continuing run."""
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config("channel_200x40", p)
    state = S.primed_state(cfg["desc"], p, seed=2)
    mesh = clot.Mesh(cfg["desc"])
    fl = clot.Fluxes(mesh, **cfg["fluxes"])
    prm = clot.Params(p, **cfg["inlet"], eta_tol=GPU_ETA_TOL)
    fresh = clot.Params(p, **cfg["inlet"], eta_tol=GPU_ETA_TOL, flags=clot.binding.ETA_FRESH)
    one = clot.Fields.from_host(mesh, p, *state)
    clot.clot_species_step(mesh, one, fl, prm, cfg["dt"], 50)
    many = clot.Fields.from_host(mesh, p, *state)
    for _ in range(10):
        clot.clot_species_step(mesh, many, fl, prm, cfg["dt"], 5)
    restart = clot.Fields.from_host(mesh, p, *state)
    for q in range(10):
        clot.clot_species_step(mesh, restart, fl, fresh if q % 2 else prm, cfg["dt"], 5)
    torch.cuda.synchronize()
    a, b, r = one.to_host(mesh), many.to_host(mesh), restart.to_host(mesh)
    assert np.array_equal(a["c"], b["c"]) and np.array_equal(a["eta"], b["eta"])
    assert np.all(species_errors(r["c"], a["c"]) <= TOL)


@pytest.mark.parametrize("name", ["channel_400x64", "duct_128x48x96"])
def test_eta_box_correction_meets_stopping_rule(name):
    """A rejected eta prediction is corrected on a box around the clot first
    (App. A, Eq. eta).  After every step the eta the step used matches the
    oracle's solve of the same theta_B within the stopping-rule bound
    (|eta - eta*| <= max|r|, M-matrix with unit row sums), and the box path
    ran."""
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config(name, p)
    d = cfg["desc"]
    mesh = clot.Mesh(d)
    fl = clot.Fluxes(mesh, **cfg["fluxes"])
    prm = clot.Params(p, **cfg["inlet"], eta_tol=GPU_ETA_TOL)
    f = clot.Fields.from_host(mesh, p, *S.primed_state(d, p, seed=5))
    clot.clot_species_step(mesh, f, fl, prm, cfg["dt"], 1)
    clot.clot_profile_begin(mesh, max_launches=64)
    worst = 0.0
    for _ in range(6):
        torch.cuda.synchronize()
        c = f.c[:, :mesh.ncell].double().cpu().numpy()
        thB = (c[O.PBA] + c[O.PBSE]) / p["Pmax"]
        clot.clot_species_step(mesh, f, fl, prm, cfg["dt"], 1)
        torch.cuda.synchronize()
        ref, _ = O.eta_solve(d, p, thB)
        err = np.max(np.abs(f.eta.double().cpu().numpy() - ref)) / np.max(thB)
        worst = max(worst, err)
    prof = clot.clot_profile_end(mesh)
    assert worst <= 2 * GPU_ETA_TOL, worst
    assert prof["eta_box"] > 0, str(prof)


def test_async_diagnostics_flux_buffers_and_state_partner():
    """clot_diagnostics_async writes what clot_diagnostics returns; stepping
    with two flux buffers in turn (double-buffered uploads) gives the state of
    one buffer; a caller-owned partner state buffer (fields.c_next) gives the
    same state without copy-back, c ending in the first buffer after an even
    number of single-step calls."""
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config("channel_200x40", p)
    state = S.primed_state(cfg["desc"], p, seed=1)
    mesh = clot.Mesh(cfg["desc"])
    prm = clot.Params(p, **cfg["inlet"], eta_tol=GPU_ETA_TOL)
    fa, fb = clot.Fluxes(mesh, **cfg["fluxes"]), clot.Fluxes(mesh, **cfg["fluxes"])
    f1 = clot.Fields.from_host(mesh, p, *state)
    f2 = clot.Fields.from_host(mesh, p, *state)
    f3 = clot.Fields.from_host(mesh, p, *state, double_buffer=True)
    f4 = clot.Fields.from_host(mesh, p, *state)
    first = f3.c.data_ptr()
    for q in range(20):  # interleaved on one mesh: every call restarts the eta prediction, alike
        clot.clot_species_step(mesh, f1, fa, prm, cfg["dt"], 1)
        clot.clot_species_step(mesh, f2, fa if q % 2 == 0 else fb, prm, cfg["dt"], 1)
    for q in range(20):  # consecutive calls: the prediction continues, alike
        clot.clot_species_step(mesh, f3, fa, prm, cfg["dt"], 1)
    for q in range(20):
        clot.clot_species_step(mesh, f4, fa, prm, cfg["dt"], 1)
    out = torch.zeros(8, dtype=torch.float64).pin_memory()
    clot.clot_diagnostics_async(mesh, f2, prm, out)
    torch.cuda.synchronize()
    ref = clot.clot_diagnostics(mesh, f2, prm)
    assert np.array_equal(out.numpy(), ref)
    a, b = f1.to_host(mesh), f2.to_host(mesh)
    assert np.array_equal(a["c"], b["c"])
    assert f3.c.data_ptr() == first
    assert np.array_equal(f3.to_host(mesh)["c"], f4.to_host(mesh)["c"])
    assert np.all(species_errors(f3.to_host(mesh)["c"], a["c"]) <= TOL)


def test_invalid_inputs_are_rejected():
    import paper_2304_09180_gb300 as clot
    p = S.params_default()
    cfg = S.config("channel_40x12", p)
    state = S.plasma_state(cfg["desc"], p, seed=1)
    mesh = clot.Mesh(cfg["desc"])
    f = clot.Fields.from_host(mesh, p, *state)
    prm = clot.Params(p, **cfg["inlet"])
    fl = clot.Fluxes(mesh, **cfg["fluxes"])
    with pytest.raises(clot.ClotError, match="EINVAL"):
        clot.clot_species_step(mesh, f, fl, prm, 5 * cfg["dt"], 1)   # Courant > 1
    bad = dict(cfg["fluxes"])
    bad["fy"] = bad["fy"].copy()
    bad["fy"][3] = 1e-9                                              # flux through the floor
    with pytest.raises(clot.ClotError, match="EINVAL"):
        clot.clot_species_step(mesh, f, clot.Fluxes(mesh, **bad), prm, cfg["dt"], 1)
    with pytest.raises(clot.ClotError, match="EINVAL"):
        clot.Mesh(dict(cfg["desc"], dim=4))
    with pytest.raises(clot.ClotError, match="EINVAL"):
        clot.clot_species_step(mesh, f, fl, clot.Params(p, **cfg["inlet"], M_rxn=0), cfg["dt"], 1)
    clot.clot_species_step(mesh, f, fl, prm, cfg["dt"], 3)            # still usable
    assert clot.clot_diagnostics(mesh, f, prm)[6] == 0

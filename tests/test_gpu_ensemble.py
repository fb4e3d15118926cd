"""The ensemble path (many uneven channels in batched launches, a replayed
CUDA graph, the autotuner) against the single-mesh path and the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import synthetic as S
from parity_util import rel_l2, run_oracle, species_errors

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _channels(specs, params, primed_every=2, seed=0):
    import paper_2304_09180_gb300 as clot
    descs = [sp["desc"] for sp in specs]
    ens = clot.Ensemble(descs)
    fields, fluxes, inlets, dts, states, cfgs = [], [], [], [], [], []
    for c, sp in enumerate(specs):
        d = sp["desc"]
        fl = S.fluxes_channel2d(d, sp["shear"]) if d["dim"] == 2 else S.fluxes_duct3d(d, sp["shear"])
        inl = S.inlet_values(d, params)
        dt = S.stable_dt(d, fl, params)
        st = (S.primed_state if c % primed_every == 0 else S.plasma_state)(d, params, seed=seed + c)
        m = ens.meshes[c]
        fields.append(clot.Fields.from_host(m, params, *st))
        fluxes.append(clot.Fluxes(m, **fl))
        inlets.append(tuple(clot.binding._dev(inl[k]) for k in ("pmu_in", "s1_in", "s2_in")))
        dts.append(dt)
        states.append(st)
        cfgs.append(dict(desc=d, fluxes=fl, inlet=inl, dt=dt))
    return ens, fields, fluxes, inlets, dts, states, cfgs


def _specs(n, seed=3, nmax=12):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = 8 * int(rng.integers(6, nmax + 1))
        ny = max(8, nx // 4)
        frac = float(rng.uniform(0.1, 0.5))
        d = S.channel2d(nx, ny, nx * 1.5 * S.UM, ny * 1.5 * S.UM, inj_frac=(0.5 - frac / 2, 0.5 + frac / 2))
        out.append(dict(desc=d, shear=float(rng.uniform(500, 2000))))
    return out


def test_ensemble_matches_single_mesh_and_oracle():
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default(eta_tol=1e-6)
    specs = _specs(7)
    ens, fields, fluxes, inlets, dts, states, cfgs = _channels(specs, p)
    nsteps = 31                                    # first step + graph replays + a ragged tail
    ens.run(fields, fluxes, inlets, dts, p, nsteps)
    torch.cuda.synchronize()
    for c in range(len(specs)):
        cfg = cfgs[c]
        mesh = clot.Mesh(cfg["desc"])
        f1 = clot.Fields.from_host(mesh, p, *states[c])
        clot.clot_species_step(mesh, f1, clot.Fluxes(mesh, **cfg["fluxes"]),
                               clot.Params(p, **cfg["inlet"]), cfg["dt"], nsteps)
        torch.cuda.synchronize()
        a, b = fields[c].to_host(ens.meshes[c]), f1.to_host(mesh)
        errs = species_errors(a["c"], b["c"])   # same kernels; eta reductions in another order
        assert np.all(errs <= TOL), (c, errs)
        assert fields[c].t == pytest.approx(f1.t, rel=1e-15)
        if c < 2:  # and against the FP64 oracle
            ref = run_oracle(dict(cfg, dt=cfg["dt"]), S.params_default(), states[c], nsteps)
            errs = species_errors(a["c"], ref.c)
            assert np.all(errs <= TOL), (c, errs)
            assert rel_l2(a["e0"], ref.e0) <= TOL


def test_ensemble_samples_adp_release_between_graph_replays():
    import torch
    p0 = S.params_default(eta_tol=1e-6)
    specs = _specs(3, seed=5)
    ens, fields, fluxes, inlets, dts, states, cfgs = _channels(specs, p0, primed_every=1)
    dtmin = min(dts)
    p = dict(p0, sigma_dt=9.5 * dtmin, sigma_tf=6 * 9.5 * dtmin)
    ens.run(fields, fluxes, inlets, dts, p, 40)
    torch.cuda.synchronize()
    for c in range(3):
        ref = run_oracle(cfgs[c], dict(S.params_default(), sigma_dt=p["sigma_dt"], sigma_tf=p["sigma_tf"]),
                         states[c], 40)
        assert fields[c].n_samples == ref.n_samples and ref.n_samples >= 1
        g = fields[c].to_host(ens.meshes[c])
        assert rel_l2(g["sigma"], ref.sigma) <= 1e-5
        assert np.all(species_errors(g["c"], ref.c) <= TOL)


def test_autotuner_keeps_state_and_results():
    import torch
    p = S.params_default(eta_tol=1e-6)
    specs = _specs(9, seed=7)
    ens, fields, fluxes, inlets, dts, states, cfgs = _channels(specs, p)
    before = [f.to_host(m) for f, m in zip(fields, ens.meshes)]
    res = ens.tune(fields, fluxes, inlets, dts, p, trials=2)
    after = [f.to_host(m) for f, m in zip(fields, ens.meshes)]
    for a, b in zip(before, after):
        for k in ("c", "e0", "c0", "eta"):
            assert np.array_equal(a[k], b[k])
    assert len(res["candidates"]) == 6
    assert (res["grid"], res["order"]) in [(q["grid"], q["order"]) for q in res["candidates"]]
    ens.run(fields, fluxes, inlets, dts, p, 13)
    ens2, f2, fl2, in2, dt2, _, _ = _channels(specs, p)
    ens2.run(f2, fl2, in2, dt2, p, 13)
    torch.cuda.synchronize()
    for c in range(len(specs)):       # the schedule changes, the arithmetic does not
        assert np.array_equal(fields[c].to_host(ens.meshes[c])["c"], f2[c].to_host(ens2.meshes[c])["c"])


@pytest.mark.parametrize("nchan", [9, 3, 1])
def test_graph_chains_give_the_same_bits(nchan):
    """Chains only move launches onto parallel graph branches: every channel's
    results with 2 and 4 chains (at most one per channel) equal those of the
    one-branch graph bit for bit (19 steps: the first step, three 6-step graph
    replays)."""
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default(eta_tol=1e-6)
    specs = _specs(nchan, seed=11)
    outs = []
    for chains in (1, 2, 4):
        ens, fields, fluxes, inlets, dts, _, _ = _channels(specs, p)
        ens.set_chains(chains)
        ens.run(fields, fluxes, inlets, dts, p, 19)
        torch.cuda.synchronize()
        outs.append([f.to_host(m) for f, m in zip(fields, ens.meshes)])
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            for k in ("c", "e0", "c0", "eta"):
                assert np.array_equal(a[k], b[k]), k
    with pytest.raises(clot.ClotError, match="EINVAL"):
        ens.set_chains(5)


@pytest.mark.parametrize("with_eta", [False, True])
def test_odd_and_ragged_channels_match_single_mesh(with_eta):
    """Channels with odd nx (the fused kernel's one-float copies), rows and
    columns that end inside a tile, and one channel smaller than a tile:
    without eta the ensemble's fused step equals the single-mesh step bit for
    bit (same cell and face code); with eta within the parity bar (eta
    reductions in another order).  13 steps: the first step, two graph
    replays."""
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default(eta_tol=1e-6)
    shapes = [(45, 11), (77, 19), (21, 5), (63, 30), (101, 9)]
    specs = []
    for q, (nx, ny) in enumerate(shapes):
        d = S.channel2d(nx, ny, nx * 1.5 * S.UM, ny * 1.5 * S.UM, inj_frac=(0.3, 0.6))
        specs.append(dict(desc=d, shear=600.0 + 300.0 * q))
    ens, fields, fluxes, inlets, dts, states, cfgs = _channels(specs, p, seed=40)
    flags = 0 if with_eta else clot.NO_ETA
    nsteps = 13
    ens.run(fields, fluxes, inlets, dts, dict(p, flags=flags), nsteps)
    torch.cuda.synchronize()
    for c in range(len(specs)):
        cfg = cfgs[c]
        mesh = clot.Mesh(cfg["desc"])
        f1 = clot.Fields.from_host(mesh, p, *states[c])
        clot.clot_species_step(mesh, f1, clot.Fluxes(mesh, **cfg["fluxes"]),
                               clot.Params(p, **cfg["inlet"], flags=flags), cfg["dt"], nsteps)
        torch.cuda.synchronize()
        a, b = fields[c].to_host(ens.meshes[c]), f1.to_host(mesh)
        if with_eta:
            errs = species_errors(a["c"], b["c"])
            assert np.all(errs <= TOL), (c, errs)
        else:
            for k in ("c", "e0", "c0"):
                assert np.array_equal(a[k], b[k]), (c, k)


def test_ensemble_rejects_mixed_dimensions():
    import paper_2304_09180_gb300 as clot
    descs = [S.config("channel_40x12")["desc"], S.config("duct_8x6x4")["desc"]]
    with pytest.raises(clot.ClotError, match="EINVAL"):
        clot.Ensemble(descs)


def test_ensemble_with_the_largest_bench_channel_matches_oracle():
    """The ensemble's uneven sizes reach 512 x 128 cells in the bench: a mix of
    a 512 x 128 primed channel, a 64 x 16 plasma channel and a ragged 200 x 52
    primed one, 25 steps through the graph-replayed launches, each channel
    against the FP64 oracle (rel-L2 <= 1e-5 per species, and eta, whose
    predictions the primed channels correct on a box around the clot)."""
    import torch
    p = S.params_default(eta_tol=1e-6)
    specs = []
    for nx, ny, frac, shear in ((512, 128, 0.5, 2000.0), (64, 16, 0.1, 500.0), (200, 52, 0.3, 1200.0)):
        d = S.channel2d(nx, ny, nx * 1.5 * S.UM, ny * 1.5 * S.UM, inj_frac=(0.5 - frac / 2, 0.5 + frac / 2))
        specs.append(dict(desc=d, shear=shear))
    ens, fields, fluxes, inlets, dts, states, cfgs = _channels(specs, p, primed_every=2, seed=11)
    nsteps = 25
    ens.run(fields, fluxes, inlets, dts, p, nsteps)
    torch.cuda.synchronize()
    O.set_threads(0)
    for c in range(len(specs)):
        ref = run_oracle(cfgs[c], S.params_default(), states[c], nsteps)
        a = fields[c].to_host(ens.meshes[c])
        errs = species_errors(a["c"], ref.c)
        assert np.all(errs <= TOL), (c, errs)
        assert rel_l2(a["e0"], ref.e0) <= TOL and rel_l2(a["c0"], ref.c0, 1e-9) <= TOL
        # eta to the solver's stopping rule: max|r| <= max(tol max theta_B, atol)
        # bounds |eta - eta_exact| (M-matrix, unit row sums); the oracle's
        # solve is tight, and the FP32 theta_B adds ~1e-6 of its maximum
        thb = (ref.c[O.PBA] + ref.c[O.PBSE]) / p["Pmax"]
        bound = 2.0 * max(1e-6 * thb.max(), p["eta_atol"]) + 1e-6 * thb.max()
        assert np.max(np.abs(a["eta"][:ref.eta.size] - ref.eta)) <= bound, c


def test_bench_ensemble_at_full_size_matches_oracle_on_sampled_channels():
    """The bench's workload in the bench's launch configuration: all 256 uneven
    plasma channels (6.8 M cells), autotuned grid, two graph chains, 13 steps
    (the first step, two 6-step graph replays); the smallest, the largest and
    two more channels against the FP64 oracle run on those channels alone."""
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default(eta_tol=1e-6)
    specs = S.ensemble_specs(256, seed=0)
    ens = clot.Ensemble([sp["desc"] for sp in specs])
    fields, fluxes, inlets, dts, states, cfgs = [], [], [], [], [], []
    for c, sp in enumerate(specs):
        d = sp["desc"]
        fl = S.fluxes_channel2d(d, sp["shear"])
        inl = S.inlet_values(d, p)
        dt = S.stable_dt(d, fl, p)
        st = S.plasma_state(d, p, seed=1000 + c)
        m = ens.meshes[c]
        fields.append(clot.Fields.from_host(m, p, *st))
        fluxes.append(clot.Fluxes(m, **fl))
        inlets.append(tuple(clot.binding._dev(inl[k]) for k in ("pmu_in", "s1_in", "s2_in")))
        dts.append(dt)
        states.append(st)
        cfgs.append(dict(desc=d, fluxes=fl, inlet=inl, dt=dt))
    ens.tune(fields, fluxes, inlets, dts, p, trials=1)
    nsteps = 13
    ens.run(fields, fluxes, inlets, dts, p, nsteps)
    torch.cuda.synchronize()
    sizes = [sp["desc"]["nx"] * sp["desc"]["ny"] for sp in specs]
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 200})
    O.set_threads(0)
    for c in picks:
        ref = run_oracle(cfgs[c], S.params_default(), states[c], nsteps)
        a = fields[c].to_host(ens.meshes[c])
        errs = species_errors(a["c"], ref.c)
        assert np.all(errs <= TOL), (c, errs)
        assert rel_l2(a["e0"], ref.e0) <= TOL and rel_l2(a["c0"], ref.c0, 1e-9) <= TOL


def test_ensemble_lagged_wall_matches_oracle():
    """CLOT_WALL_LAGGED through the ensemble launch (the paper's placement of the
    injury-wall exchange) against the oracle's OR_WALL_LAGGED."""
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default(eta_tol=1e-6, flags=clot.WALL_LAGGED)
    specs = _specs(3, seed=9)
    ens, fields, fluxes, inlets, dts, states, cfgs = _channels(specs, p, primed_every=1)
    ens.run(fields, fluxes, inlets, dts, p, 20)
    torch.cuda.synchronize()
    for c in range(3):
        ref = run_oracle(cfgs[c], S.params_default(flags=O.WALL_LAGGED), states[c], 20)
        a = fields[c].to_host(ens.meshes[c])
        assert np.all(species_errors(a["c"], ref.c) <= TOL), c
        assert rel_l2(a["e0"], ref.e0) <= TOL and rel_l2(a["c0"], ref.c0, 1e-9) <= TOL

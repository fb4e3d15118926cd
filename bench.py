#!/usr/bin/env python
"""Benchmark of the GB300 clotFoam species step.

Workload (default): the 3D duct, 512 x 128 x 128 cells of 1.5 um (8.4 M cells,
15 FP32 species, 503 MB of state -- far larger than L2), floor shear 1000/s,
plasma initial state from seed 1, dt at Courant 0.5.  One bench step is one
full species step of the hot path: eta solve, ADP-release sample check, fused
transport + RK4 reaction + wall exchange.  Metric: cell-species updates per
second (cells x 15 species x steps / time), whole job over all ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank advances its own replica of the workload (the duct
does not shard across GPUs here: replicas only); time = max over ranks.
--impl reference times the FP64 CPU oracle (test infrastructure) on the host
cores on a bounded slab of the same duct.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "species cell-updates/s (FP32 fused step, 3D duct)"
UNIT = "cell-species updates/s"
WORKLOAD = "duct_512x128x128"
# Algorithmic HBM bytes of one fused-step launch per cell on a 3D mesh: 15
# species read and written (120 B), three face fluxes (12 B), eta (4 B) and
# sigma (4 B).  2D meshes carry two face fluxes: 136 B.
BYTES_PER_CELL = 140
BYTES_PER_CELL_2D = 136


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--ensemble-steps", type=int, default=1000)
    ap.add_argument("--surrogate-steps", type=int, default=6000, help="training steps (0: skip the surrogate)")
    ap.add_argument("--primed-steps", type=int, default=100, help="steps timed in the primed clot state (0: skip)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


KERNEL_SOURCES = ("clot_step_zmarch.cu", "clot_cell.cuh", "clot_tma.cuh", "clot_model.cuh", "clot_internal.cuh")


def source_sha():
    """Hash of the fused kernel's own sources (the DRAM traffic recorded for it
    stays valid while these are unchanged)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2304_09180_gb300", "csrc")
    for fn in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, fn), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "zmarch_step_kernel_dram_traffic_duct_256x128x64.json")))[kernel]
    except Exception:
        return None
    return rec["dram_bytes_per_launch"] if rec.get("source_sha") == source_sha() else None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def slab_desc(desc, nx):
    """A slab of the duct: same cross-section, cell size, fluxes per face and
    inlet, nx cells long (the injury patch keeps its 3/8-5/8 placement)."""
    d = S.duct3d(nx, desc["ny"], desc["nz"], desc["hx"])
    return d


# ---------------------------------------------------------------- oracle

def oracle_run(desc, params, nsteps, warmup=0, seed=1):
    import oracle as O
    fl = S.fluxes_duct3d(desc, 1000.0) if desc["dim"] == 3 else S.fluxes_channel2d(desc, 1000.0)
    inl = S.inlet_values(desc, params)
    dt = S.stable_dt(desc, fl, params)
    c, e0, c0 = S.plasma_state(desc, params, seed=seed)
    st = O.new_state(desc, params, c, e0, c0)
    inp = dict(fl)
    inp.update(inl)
    if warmup:
        O.step(desc, params, st, inp, dt, warmup)
    t0 = time.perf_counter()
    O.step(desc, params, st, inp, dt, nsteps)
    return time.perf_counter() - t0


# Arm CPU part numbers (MIDR_EL1 bits 15:4) of the cores this may meet.
ARM_PARTS = {0xd40: "Arm Neoverse V1", 0xd4f: "Arm Neoverse V2", 0xd84: "Arm Neoverse V3",
             0xd0c: "Arm Neoverse N1", 0xd49: "Arm Neoverse N2", 0xd8e: "Arm Neoverse N3"}


def host_cpu():
    """The host the oracle ran on: logical CPU count and model name (best
    effort; Arm hosts list the core's part number instead of a name)."""
    info = {"nproc": os.cpu_count()}
    try:
        model, part, impl = None, None, None
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            val = line.split(":", 1)[1].strip() if ":" in line else ""
            if key in ("model name", "cpu model", "processor name") and model is None:
                model = val
            elif key == "cpu part" and part is None:
                part = int(val, 16)
            elif key == "cpu implementer" and impl is None:
                impl = int(val, 16)
        if model is None and part is not None:
            model = ARM_PARTS.get(part, f"Arm core part 0x{part:03x} (implementer 0x{impl or 0:02x})")
        if model is None:
            import platform
            model = platform.machine()
        info["model"] = model
    except Exception:
        pass
    return info


def cpu_baseline(cfg):
    """The oracle as it stands (FP64) on a bounded sample: the first steps of a
    64-cell-long slab of the duct, on one host thread (the baseline) and with
    its OpenMP loops over every host core (same results, bit for bit)."""
    import oracle as O
    O.build()
    p = S.params_default()
    desc = slab_desc(cfg["desc"], 64) if cfg["desc"]["dim"] == 3 else cfg["desc"]
    nsteps = 3
    nc = S.ncell(desc)
    O.set_threads(1)
    sec = oracle_run(desc, p, nsteps)
    allc = O.set_threads(0)
    sec_all = oracle_run(desc, p, nsteps)
    sample = (f"first {nsteps} steps of a {desc['nx']}x{desc['ny']}x{desc['nz']} slab of the duct (same cells, "
              f"fluxes, inlet), FP64")
    return {"value": nc * 15 * nsteps / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sample}, {sec:.1f} s on 1 thread", "host": host_cpu(),
            "all_cores": {"value": nc * 15 * nsteps / sec_all, "unit": UNIT, "cores": allc,
                          "sample": f"{sample}, {sec_all:.1f} s on {allc} threads"}}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    O.build()
    threads = O.set_threads(0)                   # the oracle as it stands: OpenMP over the host cores
    cfg = S.config(args.workload)
    p = S.params_default()
    # size the slab so (warmup + steps) oracle steps take a few minutes
    # (oracle: ~7.3 us per cell-step on one host core, about 0.7 x linear in threads)
    budget_s, cost_per_cell_step = 120.0, 7.5e-6 / max(1.0, 0.7 * threads)
    cells = budget_s / max(args.steps + args.warmup, 1) / cost_per_cell_step
    d = cfg["desc"]
    if d["dim"] == 3:
        nx = int(max(2, min(d["nx"], cells // (d["ny"] * d["nz"]))))
        desc = slab_desc(d, nx)
    else:
        desc = d
    sec = oracle_run(desc, p, args.steps, warmup=args.warmup)
    nc = S.ncell(desc)
    v = nc * 15 * args.steps / sec
    sample = (f"{args.steps} steps (after {args.warmup} warm-up) of a {desc['nx']}x{desc['ny']}x"
              f"{desc.get('nz', 1)} slab of the {args.workload} duct, FP64 oracle, {threads} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "sample": sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------- GPU

def combine_over_ranks(ms, units, device=None):
    """Whole-job timing across ranks: the slowest rank's time and the units
    (cells) all ranks processed.  One process per GPU; under a single process
    it returns its arguments."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def ensemble_share(nchan, rank, ws):
    """Channels of the ensemble that rank `rank` of `ws` advances."""
    return list(range(nchan))[rank::ws]


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2304_09180_gb300 as clot

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    p = S.params_default(eta_tol=1e-6)
    cfg = S.config(args.workload, p)
    d, dt = cfg["desc"], cfg["dt"]
    nc = S.ncell(d)
    c, e0, c0 = S.plasma_state(d, p, seed=1 + rank)
    mesh = clot.Mesh(d)
    fl = clot.Fluxes(mesh, **cfg["fluxes"])
    prm = clot.Params(p, **cfg["inlet"])
    f = clot.Fields.from_host(mesh, p, c, e0, c0)

    clot.clot_species_step(mesh, f, fl, prm, dt, args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    sampler = ClockSampler(vis.split(",")[local] if vis else torch.cuda.current_device())
    time.sleep(0.2)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clot.clot_profile_begin(mesh, max_launches=4 * args.steps + 16)
    ev0.record(stream)
    clot.clot_species_step(mesh, f, fl, prm, dt, args.steps)
    ev1.record(stream)
    prof = clot.clot_profile_end(mesh)
    barrier()
    clocks = sampler.stop()
    ms, cells = combine_over_ranks(ev0.elapsed_time(ev1), nc, dev)
    dg = clot.clot_diagnostics(mesh, f, prm)
    value = cells * 15 * args.steps / (ms / 1e3)

    # dominant kernel: the fused species step
    k1_ms = prof["ms_step"] / max(prof["n_step"], 1)
    bpc = BYTES_PER_CELL if d["dim"] == 3 else BYTES_PER_CELL_2D
    pk, pk_src = peaks()
    achieved = nc * bpc / (k1_ms / 1e3) / 1e9
    eta_ms = prof["ms_eta"] / max(prof["n_eta"], 1)
    traffic = recorded_traffic("species_step_3d")

    # end to end through the public API from pinned host buffers: every step
    # uploads that step's face fluxes (double-buffered, on a copy stream, so the
    # upload of step n + 1 overlaps step n) and reads its diagnostics back to
    # pinned host memory (stream-ordered, no per-step synchronisation)
    e2e = None
    if args.e2e_steps > 0:
        K = args.e2e_steps
        host = {k: torch.from_numpy(np.asarray(v, np.float32)).pin_memory()
                for k, v in cfg["fluxes"].items() if v is not None}
        c_host = torch.zeros((15, mesh.pitch), dtype=torch.float32).pin_memory()
        c_host[:, :nc] = torch.from_numpy(np.asarray(c, np.float32))
        out_host = torch.empty_like(c_host).pin_memory()
        diag_host = torch.zeros((K, 8), dtype=torch.float64).pin_memory()
        flx = [fl, clot.Fluxes(mesh, **cfg["fluxes"])]
        flux_bytes = sum(t.numel() * 4 for t in host.values())
        copy_stream = torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        used = [torch.cuda.Event(), torch.cuda.Event()]

        def upload(q):
            with torch.cuda.stream(copy_stream):
                copy_stream.wait_event(used[q])
                flx[q].fx.copy_(host["fx"], non_blocking=True)
                flx[q].fy.copy_(host["fy"], non_blocking=True)
                if "fz" in host:
                    flx[q].fz.copy_(host["fz"], non_blocking=True)
                copied[q].record(copy_stream)

        # validate the second flux buffer once (untimed, as any run does before its loop)
        f2 = clot.Fields.from_host(mesh, p, c, e0, c0, double_buffer=True)
        clot.clot_species_step(mesh, f2, flx[1], prm, dt, 1)
        f2 = clot.Fields.from_host(mesh, p, c, e0, c0, double_buffer=True)
        for q in range(2):
            used[q].record(stream)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        f2.c.copy_(c_host, non_blocking=True)
        upload(0)
        for st in range(K):
            q = st & 1
            if st + 1 < K:
                upload(q ^ 1)
            stream.wait_event(copied[q])
            clot.clot_species_step(mesh, f2, flx[q], prm, dt, 1)
            used[q].record(stream)
            clot.clot_diagnostics_async(mesh, f2, prm, diag_host[st])
        out_host.copy_(f2.c, non_blocking=True)
        torch.cuda.synchronize()
        sec, cells_e = combine_over_ranks(time.perf_counter() - t0, nc, dev)
        state_bytes = 15 * mesh.pitch * 4
        e2e = {"value": cells_e * 15 * K / sec, "unit": UNIT,
               "h2d_bytes_per_step": int(flux_bytes + state_bytes / K),
               "d2h_bytes_per_step": int(64 + state_bytes / K),
               "steps": K, "what": "per step: face fluxes H2D from pinned memory (copy stream, double-buffered), "
                                   "one clot_species_step (state double-buffered in caller buffers, eta "
                                   "prediction continuing between calls), clot_diagnostics_async D2H to pinned "
                                   "memory; state H2D before and D2H after the loop",
               "last_diagnostics_finite": bool(np.isfinite(diag_host[-1].numpy()).all())}

    # the same step in the primed clot state: every mobile species present
    # near the clot, cohesion and binding active, eta corrected every step
    primed = None
    if args.primed_steps > 0:
        fp = clot.Fields.from_host(mesh, p, *S.primed_state(d, p, seed=1 + rank))
        clot.clot_eta_solve(mesh, fp, prm)
        clot.clot_species_step(mesh, fp, fl, prm, dt, 5)
        torch.cuda.synchronize()
        barrier()
        clot.clot_profile_begin(mesh, max_launches=4 * args.primed_steps + 16)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        clot.clot_species_step(mesh, fp, fl, prm, dt, args.primed_steps)
        q1.record(stream)
        pp = clot.clot_profile_end(mesh)
        barrier()
        pms, pcells = combine_over_ranks(q0.elapsed_time(q1), nc, dev)
        k1p = pp["ms_step"] / max(pp["n_step"], 1)
        ach_p = nc * bpc / (k1p / 1e3) / 1e9
        primed = {"state": f"primed clot (seed {1 + rank}): theta_B Gaussian on the floor, bound chemicals, "
                           f"E1, E2, ADP, P^ma nonzero", "steps": args.primed_steps,
                  "ms_per_step": pms / args.primed_steps,
                  "value": pcells * 15 * args.primed_steps / (pms / 1e3), "unit": UNIT,
                  "species_step_ms": k1p, "eta_solve_ms": pp["ms_eta"] / max(pp["n_eta"], 1),
                  "eta_cg_iterations": pp["eta_iters"], "eta_predictions_accepted": pp["eta_accepted"],
                  "roofline": {"bound": "hbm", "achieved": ach_p, "peak": pk["hbm_gbs"], "unit": "GB/s",
                               "frac": ach_p / pk["hbm_gbs"], "bytes_per_cell": bpc}}
        del fp

    ens = run_ensemble(args, ws, rank) if args.ensemble_steps > 0 else None
    sur = run_surrogate(args, rank) if args.surrogate_steps > 0 else None

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(cfg)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: 3D duct {d['nx']}x{d['ny']}x{d['nz']} cells of "
                               f"{d['hx'] * 1e3:.2f} um, floor shear 1000/s, plasma state seed 1",
                   "ncell": nc, "species": 15, "dt": dt, "M_rxn": p["M_rxn"],
                   "flush": "inputs larger than L2 (503 MB state per copy)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                     "kernel": "zmarch_step_kernel (fused transport + RK4 + wall, TMA plane ring)",
                     "bytes_per_cell": bpc, "ms_per_launch": k1_ms, "peak_source": pk_src},
        "kernels": {"species_step_ms": k1_ms, "eta_solve_ms": eta_ms,
                    "sigma_ms": prof["ms_sigma"] / max(prof["n_sigma"], 1) if prof["n_sigma"] else 0.0,
                    "launches": {k: prof[k] for k in ("n_step", "n_eta", "n_sigma", "n_other")},
                    "eta_cg_iterations": prof["eta_iters"], "eta_predictions_accepted": prof["eta_accepted"],
                    "eta_box_corrections": prof["eta_box"], "eta_box_fallbacks": prof["eta_box_fallback"]},
        "gpu_launches": prof["n_step"] + prof["n_eta"] + prof["n_sigma"] + prof["n_other"],
        "clocks": clocks,
        "diagnostics": {"platelets": dg[0], "min": dg[5], "nonfinite": dg[6]},
        "e2e": e2e,
        "cpu_baseline": cpu,
        "primed": primed,
        "ensemble": ens,
        "surrogate": sur,
    }
    print(json.dumps(line))


def run_ensemble(args, ws, rank):
    """The uneven-channel ensemble: 256 independent 2D channels (nx = 8 U{8..64},
    ny = nx/4, h = 1.5 um, shear U[500, 2000]/s, injury 10-50 % of the length,
    per-channel dt at Courant 0.5), plasma states; under torchrun each rank
    takes every ws-th channel.  Autotuned, then timed over --ensemble-steps."""
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default(eta_tol=1e-6)
    allspecs = S.ensemble_specs(256, seed=0)
    specs = [allspecs[q] for q in ensemble_share(len(allspecs), rank, ws)]
    ens = clot.Ensemble([sp["desc"] for sp in specs])
    fields, fluxes, inlets, dts = [], [], [], []
    ncell = 0
    for c, sp in enumerate(specs):
        d = sp["desc"]
        fl = S.fluxes_channel2d(d, sp["shear"])
        inl = S.inlet_values(d, p)
        dts.append(S.stable_dt(d, fl, p))
        m = ens.meshes[c]
        fields.append(clot.Fields.from_host(m, p, *S.plasma_state(d, p, seed=1000 + c)))
        fluxes.append(clot.Fluxes(m, **fl))
        inlets.append(tuple(clot.binding._dev(inl[k]) for k in ("pmu_in", "s1_in", "s2_in")))
        ncell += m.ncell
    tune = ens.tune(fields, fluxes, inlets, dts, p, trials=3)
    ens.run(fields, fluxes, inlets, dts, p, 5)
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.run(fields, fluxes, inlets, dts, p, args.ensemble_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms, cells = combine_over_ranks(e0.elapsed_time(e1), ncell, torch.device("cuda"))
    cells = int(cells)
    # the same steps with the other graph schedules: 1 branch (eta of all
    # channels, then the fused step of all), 3 and 4 chains of channels
    by_chains = {}
    for nch in (1, 3, 4):
        ens.set_chains(nch)
        e0.record(stream)
        ens.run(fields, fluxes, inlets, dts, p, args.ensemble_steps)
        e1.record(stream)
        torch.cuda.synchronize()
        msq, _ = combine_over_ranks(e0.elapsed_time(e1), ncell, torch.device("cuda"))
        by_chains[nch] = msq / args.ensemble_steps
    ens.set_chains(2)
    by_chains[2] = ms / args.ensemble_steps
    bad = sum(int(ens.diagnostics(c, fields[c], p)[6]) for c in range(len(specs)))
    pk, _ = peaks()
    step_ach = cells * BYTES_PER_CELL_2D / (ms / args.ensemble_steps / 1e3) / 1e9
    kern_ach = cells * BYTES_PER_CELL_2D / (tune["ms"] / 1e3) / 1e9 if tune.get("ms") else None
    return {"workload": "256 uneven 2D channels (64x16 .. 512x128, shear 500-2000/s, injury 10-50 %)",
            "channels": 256, "cells": cells, "steps": args.ensemble_steps,
            "ms_per_step": ms / args.ensemble_steps,
            "value": cells * 15 * args.ensemble_steps / (ms / 1e3), "unit": UNIT,
            "roofline": {"bound": "hbm", "bytes_per_cell": BYTES_PER_CELL_2D, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "achieved_whole_step": step_ach, "frac_whole_step": step_ach / pk["hbm_gbs"],
                         "achieved_fused_step_kernel": kern_ach,
                         "frac_fused_step_kernel": kern_ach / pk["hbm_gbs"] if kern_ach else None,
                         "note": "whole step = block-per-channel eta CG + persistent fused step; the kernel figure "
                                 "uses the autotuner's time per fused-step launch"},
            "launch": "per step: block-per-channel eta CG + persistent fused step, 6-step CUDA graph replay with "
                      "the channels in two chains of about half the cells on parallel graph branches",
            "ms_per_step_by_chains": {str(q): by_chains[q] for q in sorted(by_chains)},
            "tune": tune, "nonfinite": bad}


def run_surrogate(args, rank):
    """The reaction surrogate: training on GPU-generated pairs, then the
    reaction solve of the 3D duct workload in a primed (clot) state, surrogate
    vs the plain FP32 RK4 reaction step (clot_reaction_step) on the same
    state: time per call and species rel-L2 of the surrogate against RK4 (and
    of explicit Euler, a zero network, for context)."""
    import torch

    import paper_2304_09180_gb300 as clot
    p = S.params_default(eta_tol=1e-6)
    scale = S.surrogate_scale(p)
    prm0 = clot.Params(p, np.zeros(1), np.zeros(1), np.zeros(1))
    rng = np.random.default_rng(7 + rank)
    w0 = np.zeros(clot.MLP_NPARAM)
    w0[0:2048] = (rng.standard_normal((32, 64)) * np.sqrt(2.0 / 31) * (np.arange(32) < 31)[:, None]).ravel()
    w0[2112:6208] = rng.standard_normal(4096) * np.sqrt(2.0 / 64)
    w0[6272:7296] = (rng.standard_normal((64, 16)) * 0.01 * (np.arange(16) < 14)[None, :]).ravel()
    mlp = clot.Mlp(w0, scale)
    zero = clot.Mlp(np.zeros(clot.MLP_NPARAM), scale)
    xs, ys = [], []
    for q, dtp in enumerate((5e-6, 1.5625e-5, 5e-5)):
        c, eta = S.surrogate_states(65536, p, seed=20 + q + 10 * rank)
        x, y = clot.clot_surrogate_pairs(prm0, zero, clot.binding._dev(c), clot.binding._dev(eta), dtp)
        xs.append(x)
        ys.append(y)
    dp = S.config("channel_200x40", p)["desc"]
    cp_, _, _ = S.primed_state(dp, p, seed=3)
    ep = np.random.default_rng(1).uniform(0, 1, cp_.shape[1])
    for dtp in (5e-6, 1.5625e-5, 5e-5):
        x, y = clot.clot_surrogate_pairs(prm0, zero, clot.binding._dev(cp_), clot.binding._dev(ep), dtp)
        xs.append(x)
        ys.append(y)
    X, Y = torch.cat(xs), torch.cat(ys).clamp(-4, 4)
    rho = (torch.expm1(X[:, 17:31].abs()) / 1e3).max(1).values
    X, Y = X[rho >= 1e-4], Y[rho >= 1e-4]
    batch = 16384
    n = (X.shape[0] // batch) * batch
    perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(rank)).cuda()
    X, Y = X[perm][:n].contiguous(), Y[perm][:n].contiguous()
    m = torch.zeros(clot.MLP_NPARAM, device="cuda")
    v = torch.zeros_like(m)
    K = args.surrogate_steps
    work = torch.empty(clot.clot_surrogate_workspace(batch), device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    losses = []
    e0.record()
    for k, lr in enumerate((2e-3, 1e-3, 5e-4)):     # step-halved learning rate
        losses.append(clot.clot_surrogate_train(mlp, m, v, k * (K // 3), lr, X, Y, batch, K // 3, work=work))
    e1.record()
    torch.cuda.synchronize()
    tms = e0.elapsed_time(e1)
    ksteps = 3 * (K // 3)
    L = torch.cat(losses).cpu().numpy()
    flop_row = 2 * (32 * 64 + 64 * 64 + 64 * 16)          # one forward pass
    train = {"pairs": int(n), "selection": "rows with relative Euler change rho >= 1e-4",
             "batch": batch, "steps": ksteps, "ms_per_step": tms / ksteps,
             "samples_per_s": batch * ksteps / (tms / 1e3),
             "tensor_tflops": 3 * flop_row * batch * ksteps / (tms / 1e3) / 1e12,
             "loss_first": float(L[:10].mean()), "loss_last": float(L[-10:].mean())}

    # held-out stiff states: what the trained network gains over explicit Euler
    ch, eh = S.surrogate_states(1 << 18, p, seed=77 + rank)
    dstrip = S.channel2d(ch.shape[1], 1, ch.shape[1] * 1.5e-3, 1.5e-3, inj_frac=(2.0, 2.0))
    mstrip = clot.Mesh(dstrip)
    fref = clot.Fields.from_host(mstrip, p, ch, np.zeros(0), np.zeros(0), eta=eh)
    clot.clot_reaction_step(mstrip, fref, prm0, 7.8125e-6, 2)
    heldout = {}
    for tol_h in (3e-2, 1.0):
        row = {}
        for name, net in (("trained", mlp), ("euler", zero)):
            fh = clot.Fields.from_host(mstrip, p, ch, np.zeros(0), np.zeros(0), eta=eh)
            cnt = clot.clot_surrogate_infer(mstrip, fh, prm0, net, 7.8125e-6, 2, tol_h, counts=True)
            a_, b_ = fh.c[:, :ch.shape[1]].double(), fref.c[:, :ch.shape[1]].double()
            e = (torch.linalg.norm(a_ - b_, dim=1) / torch.clamp(torch.linalg.norm(b_, dim=1), min=1e-300))
            row[name] = {"max_rel_l2": float(e.max()), "E2": float(e[8]), "Pba": float(e[2]),
                         "accepted": int(cnt[0])}
        heldout[str(tol_h)] = row

    cfg = S.config(args.workload, p)
    d = cfg["desc"]
    mesh = clot.Mesh(d)
    prm = clot.Params(p, **cfg["inlet"])
    st = S.primed_state(d, p, seed=1 + rank)
    base = clot.Fields.from_host(mesh, p, *st)
    clot.clot_eta_solve(mesh, base, prm)
    h, nsub, tol = cfg["dt"] / p["M_rxn"], p["M_rxn"], 1e-3
    nc = mesh.ncell

    def fresh():
        f = clot.Fields.from_host(mesh, p, *st)
        f.eta.copy_(base.eta)
        return f

    fr, fs, fz = fresh(), fresh(), fresh()
    clot.clot_reaction_step(mesh, fr, prm, h, nsub)
    counts = clot.clot_surrogate_infer(mesh, fs, prm, mlp, h, nsub, tol, counts=True)
    clot.clot_surrogate_infer(mesh, fz, prm, zero, h, nsub, tol)
    torch.cuda.synchronize()

    def rel(a, b):
        a, b = a.c[:, :nc].double(), b.c[:, :nc].double()
        nb = torch.linalg.norm(b, dim=1)
        return (torch.linalg.norm(a - b, dim=1) / torch.clamp(nb, min=1e-300)).cpu().numpy()

    err_s, err_e = rel(fs, fr), rel(fz, fr)

    def timed(fn, n=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    ms_rk = timed(lambda: clot.clot_reaction_step(mesh, fr, prm, h, nsub))
    ms_sur = timed(lambda: clot.clot_surrogate_infer(mesh, fs, prm, mlp, h, nsub, tol))
    mlp_tc = clot.Mlp(mlp.w.double().cpu().numpy(), scale, engine=clot.MLP_ENGINE_TCGEN05)
    ftc = fresh()
    ms_tc = timed(lambda: clot.clot_surrogate_infer(mesh, ftc, prm, mlp_tc, h, nsub, tol))

    # whole species steps on the primed duct: the plain fused step against
    # the surrogate step (transport pass + surrogate reaction pass), at the
    # default M_rxn and with more reaction substeps (a stiffer setting where
    # RK4 costs more and the network's cost stays the same); 20 steps each
    # from the same state, then the species rel-L2 of the two results
    fl_d = clot.Fluxes(mesh, **cfg["fluxes"])
    steps = {}
    for M in (nsub, 8, 32):
        pm = clot.Params(p, **cfg["inlet"], M_rxn=M)
        fa, fb = fresh(), fresh()
        clot.clot_species_step(mesh, fa, fl_d, pm, cfg["dt"], 2)
        clot.clot_species_step_surrogate(mesh, fb, fl_d, pm, mlp, tol, cfg["dt"], 2)
        torch.cuda.synchronize()
        a0, a1, b0, b1 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        a0.record()
        clot.clot_species_step(mesh, fa, fl_d, pm, cfg["dt"], 20)
        a1.record()
        b0.record()
        cnt_s = clot.clot_species_step_surrogate(mesh, fb, fl_d, pm, mlp, tol, cfg["dt"], 20, counts=True)
        b1.record()
        torch.cuda.synchronize()
        ms_plain, ms_surr = a0.elapsed_time(a1) / 20, b0.elapsed_time(b1) / 20
        e = rel(fb, fa)
        steps[f"M_rxn={M}"] = {"ms_plain_step": ms_plain, "ms_surrogate_step": ms_surr,
                               "speedup": ms_plain / ms_surr,
                               "counts_last_step": {"surrogate": cnt_s[0], "indicator_fallback": cnt_s[1],
                                                    "region_fallback": cnt_s[2]},
                               "rel_l2_vs_plain_after_22_steps": {"E2": float(e[8]), "Pba": float(e[2]),
                                                                  "Pbse": float(e[3]),
                                                                  "max": float(np.max(e))}}
    return {"workload": f"{args.workload} primed clot state (seed {1 + rank}), eta solved, one reaction "
                        f"solve over dt = {cfg['dt']:.4g} s (M_rxn = {nsub} RK4 steps for the plain path)",
            "tol": tol, "cells": nc, "counts": {"surrogate": counts[0], "indicator_fallback": counts[1],
                                                "region_fallback": counts[2]},
            "ms_rk4": ms_rk, "ms_surrogate": ms_sur, "speedup": ms_rk / ms_sur,
            "engine": "mma.sync (register-chained layers)", "ms_surrogate_tcgen05": ms_tc,
            "cell_updates_per_s_rk4": nc * 15 / (ms_rk / 1e3),
            "cell_updates_per_s_surrogate": nc * 15 / (ms_sur / 1e3),
            "rel_l2_vs_rk4": {sp: float(e) for sp, e in zip(S.SPECIES, err_s)},
            "rel_l2_euler_vs_rk4": {sp: float(e) for sp, e in zip(S.SPECIES, err_e)},
            "heldout_random_states": {"cells": int(ch.shape[1]), "dt": 1.5625e-5, "by_tol": heldout},
            "species_step": {"what": "20 species steps of the primed duct: plain fused step vs "
                                     "clot_species_step_surrogate (fused transport pass + surrogate reaction pass "
                                     "+ RK4 fallback list); rel-L2 of the surrogate result against the plain one",
                             "tol": tol, "by_M_rxn": steps},
            "training": train}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

"""Shared helpers of the GPU parity tests: run the same seeded input through
the CUDA library (via the C ABI binding) and through the FP64 oracle, and
measure per-species relative L2 errors (the metric of the paper's
convergence study, supporting information Eq. l2-norm) with a floor."""
import numpy as np

import oracle as O
import synthetic as S

# Natural magnitude of each species (for the relative-L2 floor): platelets at
# the normal density P0, ADP at its half-activation level, S1/S2 at plasma
# values, enzymes and bound species at the thrombin half-activation level.
SCALE = np.array([2.5e5, 2.5e5, 2.5e5, 2.5e5, 2e-3, 1.7e-4, 1.4e-3, 1e-6, 1e-6,
                  1e-6, 1e-6, 1e-6, 1e-6, 1e-6, 1e-6])
FLOOR_REL = 1e-12   # an RMS below 1e-12 of the natural scale counts as zero


def rel_l2(a, b, scale=1.0):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    floor = FLOOR_REL * scale * np.sqrt(max(b.size, 1))
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), floor))


def species_errors(gpu_c, ref_c):
    return np.array([rel_l2(gpu_c[s], ref_c[s], SCALE[s]) for s in range(15)])


def inputs_of(cfg):
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    return inp


def run_oracle(cfg, params, state, nsteps, dt=None):
    c, e0, c0 = state
    st = O.new_state(cfg["desc"], params, c, e0, c0)
    O.step(cfg["desc"], params, st, inputs_of(cfg), cfg["dt"] if dt is None else dt, nsteps)
    return st


def run_gpu(cfg, params, state, nsteps, dt=None, calls=1, **over):
    import torch

    import paper_2304_09180_gb300 as clot
    c, e0, c0 = state
    d = cfg["desc"]
    mesh = clot.Mesh(d)
    fl = clot.Fluxes(mesh, **cfg["fluxes"])
    prm = clot.Params(params, **cfg["inlet"], **over)
    f = clot.Fields.from_host(mesh, params, c, e0, c0)
    per = nsteps // calls
    for q in range(calls):
        n = per if q < calls - 1 else nsteps - per * (calls - 1)
        clot.clot_species_step(mesh, f, fl, prm, cfg["dt"] if dt is None else dt, n)
    torch.cuda.synchronize()
    out = f.to_host(mesh)
    out["fields"], out["mesh"], out["params"] = f, mesh, prm
    return out

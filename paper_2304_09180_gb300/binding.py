"""ctypes binding of the C ABI in include/clot.h.

Argument marshalling only: every step of the species update runs in the CUDA
kernels of libclot.so.  PyTorch provides device memory (tensors) and streams.
There is no CPU fallback: if the library is not built or no CUDA device is
present, loading or calling fails with an exception.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(HERE, "_build", "libclot.so")

NS = 15
SPECIES = ("Pmu", "Pma", "Pba", "Pbse", "ADP", "S1", "S2", "E1", "E2",
           "S1b", "S2b", "E1b", "E2b", "C1", "C2")
NO_TRANSPORT, NO_REACTION, CLOSED_ENDS, NO_ETA, NO_SIGMA, ETA_FRESH, SYNC_STATUS = 1, 2, 4, 8, 16, 32, 64
HEUN, STRANG, WALL_LAGGED, DEVIATION = 128, 256, 512, 1024
STATUS = {0: "CLOT_OK", -1: "CLOT_EINVAL", -2: "CLOT_ECUDA", -3: "CLOT_ENONFINITE",
          -4: "CLOT_ETIMEOUT", -5: "CLOT_ENOMEM"}


class ClotError(RuntimeError):
    """A non-zero status of a library call: .code is the CLOT_* code, the
    message carries clot_last_error()."""

    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class clot_mesh_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("inj_x0", C.c_double), ("inj_x1", C.c_double),
                ("inj_z0", C.c_double), ("inj_z1", C.c_double), ("p_diam", C.c_double)]


class clot_mesh_info_t(C.Structure):
    _fields_ = [("ncell", C.c_int64), ("pitch", C.c_int64), ("nfx", C.c_int64), ("nfy", C.c_int64),
                ("nfz", C.c_int64), ("n_inj", C.c_int), ("inj_i0", C.c_int), ("inj_i1", C.c_int),
                ("inj_k0", C.c_int), ("inj_k1", C.c_int), ("hadh_jmax", C.c_int), ("n_hadh", C.c_int),
                ("ntau", C.c_int)]


_fp = C.POINTER(C.c_float)


class clot_fields(C.Structure):
    _fields_ = [("c", _fp), ("e0", _fp), ("c0", _fp), ("eta", _fp), ("sigma", _fp), ("hist", _fp),
                ("bound_acc", _fp), ("t", C.c_double), ("t_last", C.c_double),
                ("n_samples", C.c_int), ("head", C.c_int), ("c_next", _fp), ("ext", _fp)]


class clot_fluxes(C.Structure):
    _fields_ = [("fx", _fp), ("fy", _fp), ("fz", _fp)]


PARAM_DOUBLES = ("Pmax", "kadh", "kcohPmax", "eta_t", "eta_star", "L_eta",
                 "k_adp", "adp_star", "k_e2", "e2_star",
                 "A_hat", "sigma_tf", "sigma_dt",
                 "D_P", "D_adp", "D_chem",
                 "N1", "N2", "N_A",
                 "kC0p", "kC0m", "kC0cat", "kC1p", "kC1m", "kC1cat", "kC2p", "kC2m", "kC2cat",
                 "kS1p", "kS1m", "kE1p", "kE1m", "kS2p", "kS2m", "kE2p", "kE2m",
                 "eta_tol", "eta_atol", "wait_s", "kI", "I_in", "S1_ref", "S2_ref")
PARAM_INTS = ("M_rxn", "limiter", "flags", "eta_maxit")


class clot_params(C.Structure):
    _fields_ = ([(k, C.c_double) for k in PARAM_DOUBLES] + [(k, C.c_int) for k in PARAM_INTS] +
                [("pmu_in", _fp), ("s1_in", _fp), ("s2_in", _fp)])


class clot_profile_t(C.Structure):
    _fields_ = [("n_step", C.c_int), ("n_eta", C.c_int), ("n_sigma", C.c_int), ("n_other", C.c_int),
                ("ms_step", C.c_double), ("ms_eta", C.c_double), ("ms_sigma", C.c_double),
                ("ms_other", C.c_double), ("timed", C.c_int), ("eta_iters", C.c_int),
                ("eta_accepted", C.c_int), ("eta_box", C.c_int), ("eta_box_fallback", C.c_int)]


class clot_channel(C.Structure):
    _fields_ = [("fields", clot_fields), ("fluxes", clot_fluxes), ("pmu_in", _fp), ("s1_in", _fp),
                ("s2_in", _fp), ("dt", C.c_double)]


class clot_tune_t(C.Structure):
    _fields_ = [("grid", C.c_int), ("order", C.c_int), ("ms", C.c_float), ("ncand", C.c_int),
                ("cand_grid", C.c_int * 6), ("cand_order", C.c_int * 6), ("cand_ms", C.c_float * 6)]


MLP_NPARAM = 7312


MLP_ENGINE_MMA, MLP_ENGINE_TCGEN05 = 0, 1


class clot_mlp(C.Structure):
    _fields_ = [("w", _fp), ("scale", C.c_float * NS), ("engine", C.c_int)]


_lib = None


def lib():
    """Load libclot.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(SO_PATH):
        raise RuntimeError(f"CUDA library not built: {SO_PATH} is missing "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    L = C.CDLL(SO_PATH)
    P, vp = C.POINTER, C.c_void_p
    L.clot_mesh_create.argtypes = [P(clot_mesh_desc), P(vp)]
    L.clot_mesh_destroy.argtypes = [vp]
    L.clot_mesh_destroy.restype = None
    L.clot_mesh_info.argtypes = [vp, P(clot_mesh_info_t)]
    L.clot_species_step.argtypes = [vp, P(clot_fields), P(clot_fluxes), P(clot_params), C.c_double,
                                    C.c_int, vp]
    L.clot_reaction_step.argtypes = [vp, P(clot_fields), P(clot_params), C.c_double, C.c_int, vp]
    L.clot_eta_solve.argtypes = [vp, P(clot_fields), P(clot_params), P(C.c_int), vp]
    L.clot_diagnostics.argtypes = [vp, P(clot_fields), P(clot_params), P(C.c_double), vp]
    L.clot_device_status.argtypes = [vp, P(C.c_int), vp]
    L.clot_diagnostics_async.argtypes = [vp, P(clot_fields), P(clot_params), C.c_void_p, vp]
    L.clot_profile_begin.argtypes = [vp, C.c_int]
    L.clot_profile_end.argtypes = [vp, P(clot_profile_t), vp]
    L.clot_eta_solve_noalloc.argtypes = [P(clot_mesh_desc), _fp, C.c_int64, _fp, P(clot_params),
                                         P(C.c_int), vp]
    L.clot_ensemble_create.argtypes = [P(clot_mesh_desc), C.c_int, P(vp)]
    L.clot_ensemble_destroy.argtypes = [vp]
    L.clot_ensemble_destroy.restype = None
    L.clot_ensemble_info.argtypes = [vp, C.c_int, P(clot_mesh_info_t)]
    L.clot_ensemble_run.argtypes = [vp, P(clot_channel), P(clot_params), C.c_int, vp]
    L.clot_ensemble_diagnostics.argtypes = [vp, C.c_int, P(clot_fields), P(clot_params), P(C.c_double), vp]
    L.clot_ensemble_tune.argtypes = [vp, P(clot_channel), P(clot_params), C.c_int, P(clot_tune_t), vp]
    L.clot_ensemble_set_chains.argtypes = [vp, C.c_int]
    L.clot_surrogate_pairs.argtypes = [P(clot_params), P(clot_mlp), _fp, _fp, C.c_int64, C.c_int64, C.c_double,
                                       _fp, _fp, vp]
    L.clot_surrogate_forward.argtypes = [P(clot_mlp), _fp, C.c_int64, _fp, vp]
    L.clot_surrogate_workspace.argtypes = [C.c_int64]
    L.clot_surrogate_workspace.restype = C.c_int64
    L.clot_surrogate_grad.argtypes = [P(clot_mlp), _fp, _fp, C.c_int64, _fp, C.c_int64, _fp, _fp, vp]
    L.clot_surrogate_train.argtypes = [P(clot_mlp), _fp, _fp, C.c_int, C.c_float, _fp, _fp, C.c_int64, C.c_int64,
                                       C.c_int, _fp, C.c_int64, _fp, vp]
    L.clot_surrogate_infer.argtypes = [vp, P(clot_fields), P(clot_params), P(clot_mlp), C.c_double, C.c_int,
                                       C.c_float, C.c_void_p, P(C.c_int64), vp]
    L.clot_species_step_surrogate.argtypes = [vp, P(clot_fields), P(clot_fluxes), P(clot_params), P(clot_mlp),
                                              C.c_float, C.c_double, C.c_int, P(C.c_int64), vp]
    L.clot_last_error.restype = C.c_char_p
    _lib = L
    return L


EXPORTED = ("clot_mesh_create", "clot_mesh_destroy", "clot_mesh_info", "clot_species_step",
            "clot_reaction_step", "clot_eta_solve", "clot_diagnostics", "clot_diagnostics_async", "clot_device_status",
            "clot_profile_begin", "clot_profile_end", "clot_eta_solve_noalloc", "clot_last_error",
            "clot_ensemble_create", "clot_ensemble_destroy", "clot_ensemble_info", "clot_ensemble_run",
            "clot_ensemble_diagnostics", "clot_ensemble_tune", "clot_ensemble_set_chains", "clot_surrogate_pairs",
            "clot_surrogate_forward", "clot_surrogate_workspace", "clot_surrogate_grad", "clot_surrogate_train",
            "clot_surrogate_infer", "clot_species_step_surrogate")


def _check(rc):
    if rc != 0:
        raise ClotError(rc, lib().clot_last_error().decode())


def _stream_ptr(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _fptr(t: torch.Tensor | None):
    if t is None:
        return None
    assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    return C.cast(C.c_void_p(t.data_ptr()), _fp)


def _dev(a, device="cuda"):
    return torch.as_tensor(np.ascontiguousarray(np.asarray(a, np.float64)), dtype=torch.float32,
                           device=device)


def _desc(desc: dict) -> clot_mesh_desc:
    return clot_mesh_desc(int(desc["dim"]), int(desc["nx"]), int(desc["ny"]), int(desc.get("nz", 1)),
                          float(desc["hx"]), float(desc["hy"]), float(desc.get("hz", 1.0)),
                          float(desc["inj_x0"]), float(desc["inj_x1"]),
                          float(desc.get("inj_z0", 0.0)), float(desc.get("inj_z1", 0.0)),
                          float(desc["p_diam"]))


class Mesh:
    """A uniform mesh with its device workspace (clot_mesh_create)."""

    def __init__(self, desc: dict):
        self.desc = dict(desc)
        d = _desc(desc)
        h = C.c_void_p()
        _check(lib().clot_mesh_create(C.byref(d), C.byref(h)))
        self.h = h
        self.info = clot_mesh_info_t()
        _check(lib().clot_mesh_info(self.h, C.byref(self.info)))

    @property
    def ncell(self):
        """Number of cells nx ny nz."""
        return int(self.info.ncell)

    @property
    def pitch(self):
        """Floats between species rows of the state (>= ncell, multiple of 32)."""
        return int(self.info.pitch)

    @property
    def n_inj(self):
        """Number of injury faces (length of the E0, C0 arrays)."""
        return int(self.info.n_inj)

    def injury_rect(self):
        """(i0, i1, k0, k1): the injury faces are the floor faces [i0, i1] x [k0, k1]."""
        i = self.info
        return i.inj_i0, i.inj_i1, i.inj_k0, i.inj_k1

    def close(self):
        """Free the mesh and its workspace (also done when the object is collected)."""
        if getattr(self, "h", None):
            lib().clot_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ntau_of(params: dict) -> int:
    return int(np.floor(params["sigma_tf"] / params["sigma_dt"] + 0.5))


@dataclass
class Fields:
    """Device state (clot_fields): FP32 torch tensors + host clock scalars."""
    c: torch.Tensor           # [15, pitch]
    e0: torch.Tensor
    c0: torch.Tensor
    eta: torch.Tensor
    sigma: torch.Tensor
    hist: torch.Tensor
    bound_acc: torch.Tensor
    t: float = 0.0
    t_last: float = -1.0
    n_samples: int = 0
    head: int = 0
    c_next: torch.Tensor | None = None  # optional ping-pong partner of c (no copy-back)
    ext: torch.Tensor | None = None     # optional [2, pitch] inhibitor extension rows I, E2,inh

    @staticmethod
    def from_host(mesh: Mesh, params: dict, c, e0, c0, eta=None, device="cuda",
                  double_buffer: bool = False, ext=None) -> "Fields":
        nc, pitch = mesh.ncell, mesh.pitch
        cc = torch.zeros((NS, pitch), dtype=torch.float32, device=device)
        cc[:, :nc] = _dev(np.asarray(c).reshape(NS, nc), device)
        eta_t = torch.zeros(nc, dtype=torch.float32, device=device) if eta is None else _dev(eta, device)
        n_inj = max(mesh.n_inj, 1)
        e0_t = torch.zeros(n_inj, dtype=torch.float32, device=device)
        c0_t = torch.zeros(n_inj, dtype=torch.float32, device=device)
        if mesh.n_inj:
            e0_t[:mesh.n_inj] = _dev(e0, device)
            c0_t[:mesh.n_inj] = _dev(c0, device)
        return Fields(cc, e0_t, c0_t, eta_t,
                      torch.zeros(nc, dtype=torch.float32, device=device),
                      torch.zeros((ntau_of(params) + 1, nc), dtype=torch.float32, device=device),
                      torch.zeros(nc, dtype=torch.float32, device=device),
                      c_next=torch.zeros_like(cc) if double_buffer else None,
                      ext=None if ext is None else Fields._ext(ext, nc, pitch, device))

    @staticmethod
    def _ext(ext, nc, pitch, device):
        x = torch.zeros((2, pitch), dtype=torch.float32, device=device)
        x[:, :nc] = _dev(np.asarray(ext).reshape(2, nc), device)
        return x

    def cstruct(self) -> clot_fields:
        return clot_fields(_fptr(self.c), _fptr(self.e0), _fptr(self.c0), _fptr(self.eta),
                           _fptr(self.sigma), _fptr(self.hist), _fptr(self.bound_acc),
                           self.t, self.t_last, self.n_samples, self.head, _fptr(self.c_next),
                           _fptr(self.ext))

    def absorb(self, f: clot_fields):
        self.t, self.t_last, self.n_samples, self.head = f.t, f.t_last, f.n_samples, f.head
        if self.c_next is not None and C.cast(f.c, C.c_void_p).value != self.c.data_ptr():
            self.c, self.c_next = self.c_next, self.c

    def to_host(self, mesh: Mesh):
        nc = mesh.ncell
        out = dict(c=self.c[:, :nc].double().cpu().numpy(),
                   e0=self.e0[:mesh.n_inj].double().cpu().numpy(),
                   c0=self.c0[:mesh.n_inj].double().cpu().numpy(),
                   eta=self.eta.double().cpu().numpy(), sigma=self.sigma.double().cpu().numpy())
        if self.ext is not None:
            out["ext"] = self.ext[:, :nc].double().cpu().numpy()
        return out


class Fluxes:
    """Prescribed face fluxes (mm^3/s, positive along +axis) on the device:
    fx [(nx+1) ny nz], fy [nx (ny+1) nz], fz [nx ny (nz+1)] (3D only)."""

    def __init__(self, mesh: Mesh, fx, fy, fz=None, device="cuda"):
        self.fx, self.fy = _dev(fx, device), _dev(fy, device)
        self.fz = _dev(fz, device) if fz is not None else None
        self.c = clot_fluxes(_fptr(self.fx), _fptr(self.fy), _fptr(self.fz))


class Params:
    """clot_params from a parameter dict and the inlet Dirichlet profiles."""

    def __init__(self, params: dict, pmu_in, s1_in, s2_in, device="cuda", **over):
        p = dict(params)
        for k in ("wait_s", "kI", "I_in"):
            p.setdefault(k, 0.0)
        p.update(over)
        self.d = p
        self.pmu_in, self.s1_in, self.s2_in = (_dev(a, device) for a in (pmu_in, s1_in, s2_in))
        self.c = clot_params(*[float(p[k]) for k in PARAM_DOUBLES], *[int(p[k]) for k in PARAM_INTS],
                             _fptr(self.pmu_in), _fptr(self.s1_in), _fptr(self.s2_in))


# ------------------------------------------------------------- C-ABI calls

def clot_species_step(mesh: Mesh, fields: Fields, fluxes: Fluxes, params: Params, dt: float,
                      nsteps: int, stream=None):
    """nsteps species steps of dt on fields (eta solve, ADP-release sample,
    fused transport + reaction + wall exchange), stream-ordered; fields' time
    and history scalars are updated.  Raises ClotError on invalid input."""
    f = fields.cstruct()
    _check(lib().clot_species_step(mesh.h, C.byref(f), C.byref(fluxes.c), C.byref(params.c), float(dt),
                                   int(nsteps), _stream_ptr(stream)))
    fields.absorb(f)


def clot_reaction_step(mesh: Mesh, fields: Fields, params: Params, h: float, nsub: int, stream=None):
    """The reaction alone: nsub RK4 steps of h on every cell and injury face,
    with g(eta) from fields.eta as given, in place."""
    f = fields.cstruct()
    _check(lib().clot_reaction_step(mesh.h, C.byref(f), C.byref(params.c), float(h), int(nsub),
                                    _stream_ptr(stream)))


def clot_eta_solve(mesh: Mesh, fields: Fields, params: Params, stream=None) -> int:
    """eta from theta_B of fields.c, warm-started from fields.eta; returns
    the CG iteration count (synchronises)."""
    f = fields.cstruct()
    it = C.c_int(0)
    _check(lib().clot_eta_solve(mesh.h, C.byref(f), C.byref(params.c), C.byref(it), _stream_ptr(stream)))
    return it.value


def clot_diagnostics(mesh: Mesh, fields: Fields, params: Params, stream=None, check=True) -> np.ndarray:
    """FP64 invariants (synchronous): [platelets, family 1 + wall C0, family 2,
    wall enzyme, ADP, minimum, non-finite count, max theta_T].  The library
    returns CLOT_ENONFINITE when the state holds non-finite values: raised as
    ClotError unless check=False, which returns the values anyway."""
    f = fields.cstruct()
    out = (C.c_double * 8)()
    rc = lib().clot_diagnostics(mesh.h, C.byref(f), C.byref(params.c), out, _stream_ptr(stream))
    if not (rc == -3 and not check):
        _check(rc)
    return np.array(out[:])


def clot_diagnostics_async(mesh: Mesh, fields: Fields, params: Params, out: torch.Tensor, stream=None):
    """The 8 diagnostics into out (8 float64, device or pinned host memory),
    stream-ordered, without synchronising."""
    assert out.dtype == torch.float64 and out.numel() >= 8 and (out.is_cuda or out.is_pinned())
    f = fields.cstruct()
    _check(lib().clot_diagnostics_async(mesh.h, C.byref(f), C.byref(params.c), C.c_void_p(out.data_ptr()),
                                        _stream_ptr(stream)))


def clot_device_status(mesh: Mesh, stream=None) -> int:
    """Read and clear the device status; returns the last eta iteration count,
    raises ClotError(CLOT_ETIMEOUT) if a bounded device wait gave up."""
    it = C.c_int(0)
    _check(lib().clot_device_status(mesh.h, C.byref(it), _stream_ptr(stream)))
    return it.value


def clot_profile_begin(mesh: Mesh, max_launches: int = 4096):
    """Start timing every library kernel launch with CUDA events."""
    _check(lib().clot_profile_begin(mesh.h, int(max_launches)))


def clot_profile_end(mesh: Mesh, stream=None) -> dict:
    """Stop timing; launches and summed milliseconds per kernel kind, eta
    iteration, acceptance and box-correction counts."""
    o = clot_profile_t()
    _check(lib().clot_profile_end(mesh.h, C.byref(o), _stream_ptr(stream)))
    return {k: getattr(o, k) for k, _ in clot_profile_t._fields_}


def clot_eta_solve_noalloc(desc: dict, c: torch.Tensor, pitch: int, eta: torch.Tensor, params: Params,
                           stream=None, want_iters=True) -> int | None:
    """eta solve that allocates no device memory (see include/clot.h): for
    callers that cannot call cudaMalloc.  c is the [15, pitch] state, eta the
    [ncell] warm start / result.  Returns the CG iteration count, or None with
    want_iters=False (the call then does not synchronise, and a timeout is
    reported by the next call that asks for the count).  The C side cannot
    check the tensors' sizes or devices, so this wrapper does, before any
    launch: ValueError if c has fewer than 15 * pitch floats, eta fewer than
    nx * ny * nz, or either is not on the current CUDA device."""
    ncell = int(desc["nx"]) * int(desc["ny"]) * int(desc.get("nz", 1))
    if int(pitch) < ncell:
        raise ValueError(f"pitch {pitch} is smaller than the cell count {ncell}")
    if c.numel() < NS * int(pitch):
        raise ValueError(f"c holds {c.numel()} floats, the solve reads {NS} x pitch = {NS * int(pitch)}")
    if eta.numel() < ncell:
        raise ValueError(f"eta holds {eta.numel()} floats, the mesh has {ncell} cells")
    for name, t in (("c", c), ("eta", eta)):
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 tensor")
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device")
    d = clot_mesh_desc(int(desc["dim"]), int(desc["nx"]), int(desc["ny"]), int(desc.get("nz", 1)),
                       float(desc["hx"]), float(desc["hy"]), float(desc.get("hz", 1.0)),
                       float(desc["inj_x0"]), float(desc["inj_x1"]),
                       float(desc.get("inj_z0", 0.0)), float(desc.get("inj_z1", 0.0)),
                       float(desc["p_diam"]))
    it = C.c_int(0)
    _check(lib().clot_eta_solve_noalloc(C.byref(d), _fptr(c), int(pitch), _fptr(eta), C.byref(params.c),
                                        C.byref(it) if want_iters else None, _stream_ptr(stream)))
    return it.value if want_iters else None


class _Info:
    """Mesh facts of one ensemble channel (duck-types Mesh for Fields/Fluxes)."""

    def __init__(self, info: clot_mesh_info_t):
        self.info = info

    ncell = property(lambda self: int(self.info.ncell))
    pitch = property(lambda self: int(self.info.pitch))
    n_inj = property(lambda self: int(self.info.n_inj))


class Ensemble:
    """Independent channels advanced together (clot_ensemble_*)."""

    def __init__(self, descs):
        self.descs = [dict(d) for d in descs]
        arr = (clot_mesh_desc * len(descs))(*[_desc(d) for d in descs])
        h = C.c_void_p()
        _check(lib().clot_ensemble_create(arr, len(descs), C.byref(h)))
        self.h = h
        self.meshes = []
        for c in range(len(descs)):
            info = clot_mesh_info_t()
            _check(lib().clot_ensemble_info(self.h, c, C.byref(info)))
            self.meshes.append(_Info(info))

    def __len__(self):
        return len(self.descs)

    def _channels(self, fields, fluxes, inlets, dts):
        n = len(self.descs)
        arr = (clot_channel * n)()
        for c in range(n):
            ins = inlets[c]
            arr[c] = clot_channel(fields[c].cstruct(), fluxes[c].c, _fptr(ins[0]), _fptr(ins[1]), _fptr(ins[2]),
                                  float(dts[c]))
        return arr

    @staticmethod
    def _params(params: dict) -> clot_params:
        params = dict(params)
        for k in ("wait_s", "kI", "I_in"):
            params.setdefault(k, 0.0)
        return clot_params(*[float(params[k]) for k in PARAM_DOUBLES], *[int(params[k]) for k in PARAM_INTS],
                           None, None, None)

    def run(self, fields, fluxes, inlets, dts, params: dict, nsteps: int, stream=None):
        """fields: list of Fields, fluxes: list of Fluxes, inlets: list of
        (pmu_in, s1_in, s2_in) device tensors, dts: list of floats."""
        arr = self._channels(fields, fluxes, inlets, dts)
        prm = self._params(params)
        _check(lib().clot_ensemble_run(self.h, arr, C.byref(prm), int(nsteps), _stream_ptr(stream)))
        for c in range(len(self.descs)):
            fields[c].absorb(arr[c].fields)

    def tune(self, fields, fluxes, inlets, dts, params: dict, trials: int = 3, stream=None) -> dict:
        arr = self._channels(fields, fluxes, inlets, dts)
        prm = self._params(params)
        out = clot_tune_t()
        _check(lib().clot_ensemble_tune(self.h, arr, C.byref(prm), int(trials), C.byref(out), _stream_ptr(stream)))
        return {"grid": out.grid, "order": out.order, "ms": out.ms,
                "candidates": [{"grid": out.cand_grid[q], "order": out.cand_order[q], "ms": out.cand_ms[q]}
                               for q in range(out.ncand)]}

    def set_chains(self, chains: int):
        """Launch schedule of the replayed graph: 1 .. 4 chains of channels on
        parallel branches (default 2); synchronises the device."""
        _check(lib().clot_ensemble_set_chains(self.h, int(chains)))

    def diagnostics(self, chan: int, fields, params: dict, stream=None):
        f = fields.cstruct()
        prm = self._params(params)
        out = (C.c_double * 8)()
        _check(lib().clot_ensemble_diagnostics(self.h, int(chan), C.byref(f), C.byref(prm), out,
                                               _stream_ptr(stream)))
        return np.array(out[:])

    def close(self):
        if getattr(self, "h", None):
            lib().clot_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- reaction surrogate

class Mlp:
    """The surrogate network: FP32 parameters on the device (packed W1 b1 W2
    b2 W3 b3, include/clot.h) and the per-species scales (host)."""

    def __init__(self, w, scale, device="cuda", engine=MLP_ENGINE_MMA):
        self.w = torch.as_tensor(np.asarray(w, np.float64), dtype=torch.float32, device=device).contiguous()
        assert self.w.numel() == MLP_NPARAM
        self.scale = [float(v) for v in scale]
        assert len(self.scale) == NS
        self.engine = int(engine)

    def cstruct(self) -> clot_mlp:
        return clot_mlp(_fptr(self.w), (C.c_float * NS)(*self.scale), self.engine)


def clot_surrogate_pairs(params: Params, mlp: Mlp, c0: torch.Tensor, eta: torch.Tensor, dt: float,
                         stream=None):
    """Features x [n, 32] and targets y [n, 16] of the RK4 reaction solve
    over dt (params M_rxn steps) from states c0 [15, pitch] (n = eta.numel())."""
    n = eta.numel()
    x = torch.empty((n, 32), dtype=torch.float32, device=c0.device)
    y = torch.empty((n, 16), dtype=torch.float32, device=c0.device)
    m = mlp.cstruct()
    _check(lib().clot_surrogate_pairs(C.byref(params.c), C.byref(m), _fptr(c0), _fptr(eta), n, c0.shape[1],
                                      float(dt), _fptr(x), _fptr(y), _stream_ptr(stream)))
    return x, y


def clot_surrogate_forward(mlp: Mlp, x: torch.Tensor, stream=None) -> torch.Tensor:
    n = x.shape[0]
    out = torch.empty((n, 16), dtype=torch.float32, device=x.device)
    m = mlp.cstruct()
    _check(lib().clot_surrogate_forward(C.byref(m), _fptr(x), n, _fptr(out), _stream_ptr(stream)))
    return out


def clot_surrogate_workspace(n: int) -> int:
    return int(lib().clot_surrogate_workspace(int(n)))


def clot_surrogate_grad(mlp: Mlp, x: torch.Tensor, y: torch.Tensor, work: torch.Tensor | None = None,
                        stream=None):
    """Gradient [NPARAM] and loss of the mean-square loss over the rows of x, y."""
    n = x.shape[0]
    if work is None:
        work = torch.empty(clot_surrogate_workspace(n), dtype=torch.float32, device=x.device)
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    m = mlp.cstruct()
    _check(lib().clot_surrogate_grad(C.byref(m), _fptr(x), _fptr(y), n, _fptr(work), work.numel(), _fptr(grad),
                                     _fptr(loss), _stream_ptr(stream)))
    return grad, loss


def clot_surrogate_train(mlp: Mlp, m: torch.Tensor, v: torch.Tensor, t0: int, lr: float, x: torch.Tensor,
                         y: torch.Tensor, batch: int, nsteps: int, work: torch.Tensor | None = None,
                         loss: torch.Tensor | None = None, stream=None):
    """nsteps Adam steps on mlp.w (in place); returns the per-step losses (device)."""
    n = x.shape[0]
    if work is None:
        work = torch.empty(clot_surrogate_workspace(batch), dtype=torch.float32, device=x.device)
    if loss is None:
        loss = torch.empty(max(nsteps, 1), dtype=torch.float32, device=x.device)
    c = mlp.cstruct()
    _check(lib().clot_surrogate_train(C.byref(c), _fptr(m), _fptr(v), int(t0), float(lr), _fptr(x), _fptr(y), n,
                                      int(batch), int(nsteps), _fptr(work), work.numel(), _fptr(loss),
                                      _stream_ptr(stream)))
    return loss


def clot_surrogate_infer(mesh: Mesh, fields: Fields, params: Params, mlp: Mlp, h: float, nsub: int, tol: float,
                         flag: torch.Tensor | None = None, counts: bool = False, stream=None):
    """Reaction solve over h * nsub with the surrogate where it applies (in
    place on fields).  flag: optional uint8 [ncell] tensor; counts=True
    returns (surrogate, indicator fallback, region fallback) cell counts."""
    f = fields.cstruct()
    m = mlp.cstruct()
    fl = None
    if flag is not None:
        assert flag.is_cuda and flag.dtype == torch.uint8 and flag.numel() >= mesh.ncell
        fl = C.c_void_p(flag.data_ptr())
    cnt = (C.c_int64 * 3)() if counts else None
    _check(lib().clot_surrogate_infer(mesh.h, C.byref(f), C.byref(params.c), C.byref(m), float(h), int(nsub),
                                      float(tol), fl, cnt, _stream_ptr(stream)))
    return tuple(cnt[:]) if counts else None


def clot_species_step_surrogate(mesh: Mesh, fields: Fields, fluxes: Fluxes, params: Params, mlp: Mlp, tol: float,
                                dt: float, nsteps: int, counts: bool = False, stream=None):
    """nsteps species steps whose reaction solve takes the surrogate where it
    applies (see include/clot.h); counts=True synchronises and returns the
    (surrogate, indicator fallback, region fallback) cells of the last step."""
    f = fields.cstruct()
    m = mlp.cstruct()
    cnt = (C.c_int64 * 3)() if counts else None
    _check(lib().clot_species_step_surrogate(mesh.h, C.byref(f), C.byref(fluxes.c), C.byref(params.c), C.byref(m),
                                             float(tol), float(dt), int(nsteps), cnt, _stream_ptr(stream)))
    fields.absorb(f)
    return tuple(cnt[:]) if counts else None

"""FP64 CPU oracle for the clotFoam species step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product
path (``paper_2304_09180_gb300``) never imports it, and it never imports the
product path.  It shares no code with the CUDA library: ``clot_oracle.c`` is a
separate statement of the method in plain C, compiled here with gcc.

The wrapper only marshals numpy arrays into the C structs; every step of the
method is in ``clot_oracle.c`` (see its header for the paper citations).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "clot_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libclot_oracle.so")

NS = 15
SPECIES = ("Pmu", "Pma", "Pba", "Pbse", "ADP", "S1", "S2", "E1", "E2",
           "S1b", "S2b", "E1b", "E2b", "C1", "C2")
(PMU, PMA, PBA, PBSE, ADP, S1, S2, E1, E2, S1B, S2B, E1B, E2B, C1, C2) = range(NS)
INH, E2I = 0, 1   # rows of the inhibitor extension's array (I, E2,inh)

NO_TRANSPORT, NO_REACTION, CLOSED_ENDS, NO_ETA, NO_SIGMA = 1, 2, 4, 8, 16
TRANSPORT_RK2 = 32  # Heun (SSP-RK2) transport instead of forward Euler
WALL_LAGGED = 64    # injury-wall exchange as a lagged transport boundary condition (the paper's placement)
STRANG = 128        # Strang splitting: reaction dt/2, transport dt, reaction dt/2


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops (n < 1: every host core); the
    results do not depend on it.  Returns the count in use."""
    return int(lib().or_set_threads(int(n)))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE arithmetic, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fopenmp",
                               "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("inj_x0", C.c_double), ("inj_x1", C.c_double),
                ("inj_z0", C.c_double), ("inj_z1", C.c_double),
                ("p_diam", C.c_double)]


_PARAM_DOUBLES = ("Pmax", "kadh", "kcohPmax", "eta_t", "eta_star", "L_eta",
                  "k_adp", "adp_star", "k_e2", "e2_star",
                  "A_hat", "sigma_tf", "sigma_dt",
                  "D_P", "D_adp", "D_chem",
                  "N1", "N2", "N_A",
                  "kC0p", "kC0m", "kC0cat", "kC1p", "kC1m", "kC1cat",
                  "kC2p", "kC2m", "kC2cat",
                  "kS1p", "kS1m", "kE1p", "kE1m", "kS2p", "kS2m", "kE2p", "kE2m",
                  "eta_tol", "kI", "I_in")
_PARAM_INTS = ("M_rxn", "limiter", "flags", "eta_maxit")


class Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in _PARAM_DOUBLES] + [(k, C.c_int) for k in _PARAM_INTS]


_dp = C.POINTER(C.c_double)


class Fields(C.Structure):
    _fields_ = [("c", _dp), ("e0", _dp), ("c0", _dp), ("eta", _dp), ("sigma", _dp),
                ("hist", _dp), ("thetaB_last", _dp),
                ("t", C.c_double), ("t_last", C.c_double),
                ("n_samples", C.c_int), ("head", C.c_int), ("ext", _dp)]


class Inputs(C.Structure):
    _fields_ = [("fx", _dp), ("fy", _dp), ("fz", _dp),
                ("pmu_in", _dp), ("s1_in", _dp), ("s2_in", _dp)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        P = C.POINTER
        L.or_injury_faces.argtypes = [P(Mesh), P(C.c_int), P(C.c_int)]
        L.or_injury_faces.restype = C.c_int
        L.or_hadh.argtypes = [P(Mesh), _dp]
        L.or_W.argtypes = [C.c_double]
        L.or_W.restype = C.c_double
        L.or_g.argtypes = [P(Params), C.c_double]
        L.or_g.restype = C.c_double
        L.or_R.argtypes = [C.c_double]
        L.or_R.restype = C.c_double
        L.or_rhs.argtypes = [P(Params), _dp, C.c_double, C.c_double, C.c_int, C.c_double,
                             C.c_double, C.c_double, C.c_double, _dp, _dp, _dp]
        L.or_rk4_cell.argtypes = [P(Params), _dp, C.c_double, C.c_double, C.c_int, _dp, _dp,
                                  C.c_double, C.c_double, C.c_double]
        L.or_apply_eta_op.argtypes = [P(Mesh), P(Params), _dp, _dp]
        L.or_eta_solve.argtypes = [P(Mesh), P(Params), _dp, _dp, C.c_double, C.c_int]
        L.or_eta_solve.restype = C.c_int
        L.or_sigma_sample.argtypes = [P(Mesh), P(Params), P(Fields)]
        L.or_face_value.argtypes = [C.c_double] * 3 + [C.c_int]
        L.or_face_value.restype = C.c_double
        L.or_transport.argtypes = [P(Mesh), P(Params), P(Inputs), _dp, _dp, C.c_double, _dp]
        L.or_reaction.argtypes = [P(Mesh), P(Params), _dp, _dp, _dp, _dp, C.c_double, C.c_int]
        L.or_reaction_x.argtypes = [P(Mesh), P(Params), _dp, _dp, _dp, _dp, _dp, C.c_double, C.c_int]
        L.or_step.argtypes = [P(Mesh), P(Params), P(Fields), P(Inputs), C.c_double, C.c_int]
        L.or_step.restype = C.c_int
        L.or_diagnostics.argtypes = [P(Mesh), P(Params), P(Fields), _dp]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_set_threads.restype = C.c_int
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def make_mesh(desc: dict) -> Mesh:
    return Mesh(int(desc["dim"]), int(desc["nx"]), int(desc["ny"]), int(desc.get("nz", 1)),
                float(desc["hx"]), float(desc["hy"]), float(desc.get("hz", 1.0)),
                float(desc["inj_x0"]), float(desc["inj_x1"]),
                float(desc.get("inj_z0", 0.0)), float(desc.get("inj_z1", 0.0)),
                float(desc["p_diam"]))


def make_params(params: dict) -> Params:
    p = Params()
    for k in _PARAM_DOUBLES:
        setattr(p, k, float(params[k]))
    for k in _PARAM_INTS:
        setattr(p, k, int(params[k]))
    return p


def ntau(params: dict) -> int:
    return int(np.floor(params["sigma_tf"] / params["sigma_dt"] + 0.5))


@dataclass
class State:
    """FP64 state of one simulation: cell species c[15, ncell], wall species,
    eta, sigma, the sigma history ring and the host-side clock scalars."""
    c: np.ndarray
    e0: np.ndarray
    c0: np.ndarray
    eta: np.ndarray
    sigma: np.ndarray
    hist: np.ndarray
    thetaB_last: np.ndarray
    t: float = 0.0
    t_last: float = -1.0
    n_samples: int = 0
    head: int = 0
    ext: np.ndarray | None = None   # [2, ncell] I, E2,inh of the inhibitor extension (None: the paper's model)
    _keep: list = field(default_factory=list, repr=False)

    def cfields(self) -> Fields:
        f = Fields(_ptr(self.c), _ptr(self.e0), _ptr(self.c0), _ptr(self.eta), _ptr(self.sigma),
                   _ptr(self.hist), _ptr(self.thetaB_last), self.t, self.t_last,
                   self.n_samples, self.head, _ptr(self.ext))
        return f

    def absorb(self, f: Fields):
        self.t, self.t_last, self.n_samples, self.head = f.t, f.t_last, f.n_samples, f.head

    def copy(self) -> "State":
        return State(self.c.copy(), self.e0.copy(), self.c0.copy(), self.eta.copy(),
                     self.sigma.copy(), self.hist.copy(), self.thetaB_last.copy(),
                     self.t, self.t_last, self.n_samples, self.head,
                     None if self.ext is None else self.ext.copy())


def new_state(desc: dict, params: dict, c, e0, c0, eta=None, ext=None) -> State:
    """ext: [2, ncell] initial I, E2,inh to run the inhibitor extension."""
    nc = int(desc["nx"]) * int(desc["ny"]) * int(desc.get("nz", 1))
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(NS, nc))
    e0 = np.ascontiguousarray(np.asarray(e0, dtype=np.float64))
    c0 = np.ascontiguousarray(np.asarray(c0, dtype=np.float64))
    eta = np.zeros(nc) if eta is None else np.ascontiguousarray(np.asarray(eta, np.float64))
    x = None if ext is None else np.ascontiguousarray(np.array(ext, np.float64).reshape(2, nc))
    return State(c.copy(), e0.copy(), c0.copy(), eta.copy(), np.zeros(nc),
                 np.zeros((ntau(params) + 1, nc)), np.zeros(nc), ext=x)


class Inputs_:
    """Holds numpy inputs alive while the C struct points at them."""

    def __init__(self, fx, fy, fz, pmu_in, s1_in, s2_in):
        self.arrs = [None if a is None else np.ascontiguousarray(np.asarray(a, np.float64))
                     for a in (fx, fy, fz, pmu_in, s1_in, s2_in)]
        self.c = Inputs(*[_ptr(a) for a in self.arrs])


def step(desc: dict, params: dict, st: State, inputs: dict, dt: float, nsteps: int) -> State:
    """Advance ``st`` in place by nsteps species steps; returns it."""
    m, p = make_mesh(desc), make_params(params)
    inp = Inputs_(inputs["fx"], inputs["fy"], inputs.get("fz"), inputs["pmu_in"],
                  inputs["s1_in"], inputs["s2_in"])
    f = st.cfields()
    rc = lib().or_step(C.byref(m), C.byref(p), C.byref(f), C.byref(inp.c), float(dt), int(nsteps))
    if rc != 0:
        raise ValueError(f"or_step failed ({rc})")
    st.absorb(f)
    return st


def transport(desc, params, c, inputs, dt, sigma=None):
    m, p = make_mesh(desc), make_params(params)
    c = np.ascontiguousarray(np.asarray(c, np.float64))
    out = np.empty_like(c)
    inp = Inputs_(inputs["fx"], inputs["fy"], inputs.get("fz"), inputs["pmu_in"],
                  inputs["s1_in"], inputs["s2_in"])
    sg = None if sigma is None else np.ascontiguousarray(np.asarray(sigma, np.float64))
    lib().or_transport(C.byref(m), C.byref(p), C.byref(inp.c), _ptr(c), _ptr(sg), float(dt), _ptr(out))
    return out


def reaction(desc, params, c, e0, c0, eta, h, nsub):
    """Pointwise RK4 reaction solve on copies; returns (c, e0, c0)."""
    m, p = make_mesh(desc), make_params(params)
    c = np.ascontiguousarray(np.array(c, np.float64))
    e0 = np.ascontiguousarray(np.array(e0, np.float64))
    c0 = np.ascontiguousarray(np.array(c0, np.float64))
    eta = None if eta is None else np.ascontiguousarray(np.asarray(eta, np.float64))
    lib().or_reaction(C.byref(m), C.byref(p), _ptr(c), _ptr(e0), _ptr(c0), _ptr(eta),
                      float(h), int(nsub))
    return c, e0, c0


def reaction_x(desc, params, c, ext, e0, c0, eta, h, nsub):
    """reaction() with the inhibitor extension's rows ext [2, ncell]; returns
    (c, ext, e0, c0)."""
    m, p = make_mesh(desc), make_params(params)
    c = np.ascontiguousarray(np.array(c, np.float64))
    x = np.ascontiguousarray(np.array(ext, np.float64))
    e0 = np.ascontiguousarray(np.array(e0, np.float64))
    c0 = np.ascontiguousarray(np.array(c0, np.float64))
    eta = None if eta is None else np.ascontiguousarray(np.asarray(eta, np.float64))
    lib().or_reaction_x(C.byref(m), C.byref(p), _ptr(c), _ptr(x), _ptr(e0), _ptr(c0), _ptr(eta),
                        float(h), int(nsub))
    return c, x, e0, c0


def rhs(params, y, H=0.0, g=0.0, wall=False, e0=0.0, c0=0.0, aV=0.0, Dd=1.0):
    p = make_params(params)
    y = np.ascontiguousarray(np.asarray(y, np.float64))
    f = np.zeros(NS)
    fe0, fc0 = C.c_double(0.0), C.c_double(0.0)
    lib().or_rhs(C.byref(p), _ptr(y), H, g, int(wall), e0, c0, aV, Dd, _ptr(f),
                 C.byref(fe0), C.byref(fc0))
    return f, fe0.value, fc0.value


def rk4_cell(params, y, h, nsub=1, H=0.0, g=0.0, wall=False, e0=0.0, c0=0.0, aV=0.0, Dd=1.0):
    p = make_params(params)
    y = np.ascontiguousarray(np.array(y, np.float64))
    e = C.c_double(e0)
    cc = C.c_double(c0)
    for _ in range(nsub):
        lib().or_rk4_cell(C.byref(p), _ptr(y), H, g, int(wall), C.byref(e), C.byref(cc), aV, Dd, h)
    return y, e.value, cc.value


def eta_op(desc, params, x):
    m, p = make_mesh(desc), make_params(params)
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    y = np.empty_like(x)
    lib().or_apply_eta_op(C.byref(m), C.byref(p), _ptr(x), _ptr(y))
    return y


def eta_solve(desc, params, thetaB, eta0=None, tol=1e-13, maxit=100000):
    m, p = make_mesh(desc), make_params(params)
    b = np.ascontiguousarray(np.asarray(thetaB, np.float64))
    eta = np.zeros_like(b) if eta0 is None else np.array(eta0, np.float64)
    it = lib().or_eta_solve(C.byref(m), C.byref(p), _ptr(b), _ptr(eta), tol, maxit)
    return eta, it


def sigma_sample(desc, params, st: State) -> State:
    m, p = make_mesh(desc), make_params(params)
    f = st.cfields()
    if st.t_last < 0:
        raise ValueError("history not initialised")
    lib().or_sigma_sample(C.byref(m), C.byref(p), C.byref(f))
    st.absorb(f)
    return st


def injury_faces(desc):
    m = make_mesh(desc)
    n = lib().or_injury_faces(C.byref(m), None, None)
    fi = (C.c_int * max(n, 1))()
    fk = (C.c_int * max(n, 1))()
    lib().or_injury_faces(C.byref(m), fi, fk)
    return np.array(fi[:n], np.int64), np.array(fk[:n], np.int64)


def hadh(desc):
    m = make_mesh(desc)
    nc = int(desc["nx"]) * int(desc["ny"]) * int(desc.get("nz", 1))
    H = np.zeros(nc)
    lib().or_hadh(C.byref(m), _ptr(H))
    return H


def W(theta):
    return lib().or_W(float(theta))


def g(params, eta):
    return lib().or_g(C.byref(make_params(params)), float(eta))


def R(tau):
    return lib().or_R(float(tau))


def face_value(cuu, cu, cd, limiter=1):
    return lib().or_face_value(float(cuu), float(cu), float(cd), int(limiter))


def diagnostics(desc, params, st: State) -> np.ndarray:
    m, p = make_mesh(desc), make_params(params)
    f = st.cfields()
    out = np.zeros(8)
    lib().or_diagnostics(C.byref(m), C.byref(p), C.byref(f), _ptr(out))
    return out

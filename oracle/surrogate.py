"""FP64 reference of the reaction surrogate -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and ``bench.py``'s baseline legs use this module.  The
surrogate replaces the M_rxn RK4 reaction solve of one species step (Sec. 3.2
step 2; the reaction system of App. A / App. B) by one evaluation of the
reaction right-hand side f plus a small MLP:

  features x (31, zero-padded to 32):
      x_s    = log1p(max(c_s, 0) / scale_s)           s = 0..14 (all cell species)
      x_15   = g(eta)                                  (App. A binding affinity)
      x_16   = log(dt / 1e-5)
      x_17+o = sign(q_s) log1p(1e3 |q_s|), q_s = E_s / (|c_s| + 1e-6 scale_s)
                                                       (relative Euler rate of reacting species o)
  network  h1 = gelu(x W1 + b1)    32 -> 64
           h2 = gelu(h1 W2 + b2)   64 -> 64
           v  = h2 W3 + b3         64 -> 16 (14 used: the reacting species, ADP excluded)
  increment of species s over dt:
      E_s  = dt f_s(c)                                 (explicit Euler)
      rho  = max_s |E_s| / (|c_s| + 1e-6 scale_s)      (relative Euler change, a stiffness measure)
      dc_s = E_s + rho v_s (|E_s| + 1e-6 scale_s)
  training target v_s = (dc_RK4_s - E_s) / (rho (|E_s| + 1e-6 scale_s)) (0 where
  rho = 0), loss = the mean square of (v - target) over the batch and the 14
  used outputs.

A zero network is exactly explicit Euler.  The correction RK4 makes to Euler
is of order rho relative to the Euler increment, so the targets are of order
one, and a cell with f = 0 (an equilibrium, which RK4 keeps) has rho = 0 and
dc = 0 whatever the network says.
gelu is the tanh form of the Gaussian error linear unit (Hendrycks & Gimpel):
gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).

Precision model of the GPU kernels (``bf16=True`` emulates it): the operands of
every matrix product are rounded to bfloat16 (features x, the weights, the
hidden activations h1 and h2, and in the backward pass the loss residual
out - y and the pre-activation gradients dz1, dz2); products accumulate in
wide precision; biases, pre-activations z, gelu and gelu' stay wide.  The
loss-gradient scale 2 / (B * 14) is applied after the contractions.

Every function here is float64 numpy; gradients are checked against finite
differences in tests/test_oracle_surrogate.py.
"""
from __future__ import annotations

import math

import numpy as np

NIN, NH, NOUT, NIN_PAD, NOUT_PAD = 31, 64, 14, 32, 16
# the 14 reacting species (all but ADP, row 4) in output order
REACTING = (0, 1, 2, 3, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14)
FLOOR = 1e-6
DT_REF = 1e-5
RATE_K = 1e3
GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715

# packed parameter vector: W1[32][64] b1[64] W2[64][64] b2[64] W3[64][16] b3[16]
SHAPES = (("W1", (NIN_PAD, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (NH, NOUT_PAD)), ("b3", (NOUT_PAD,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def pack(P):
    return np.concatenate([np.asarray(P[k], np.float64).reshape(-1) for k, _ in SHAPES])


def unpack(w):
    w = np.asarray(w, np.float64)
    P, o = {}, 0
    for k, s in SHAPES:
        n = int(np.prod(s))
        P[k] = w[o:o + n].reshape(s).copy()
        o += n
    return P


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.ascontiguousarray(np.asarray(a, np.float64), dtype=np.float32)
    b = a32.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    z = np.asarray(z, np.float64)
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    z = np.asarray(z, np.float64)
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def init_params(seed=0):
    """He-style initialisation; W stored [in, out]; padded rows/columns zero."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((NIN_PAD, NH)) * math.sqrt(2.0 / NIN)
    W1[NIN:] = 0.0
    W2 = rng.standard_normal((NH, NH)) * math.sqrt(2.0 / NH)
    W3 = rng.standard_normal((NH, NOUT_PAD)) * 0.01
    W3[:, NOUT:] = 0.0
    return dict(W1=W1, b1=np.zeros(NH), W2=W2, b2=np.zeros(NH), W3=W3, b3=np.zeros(NOUT_PAD))


def features(c, g, dt, scale, euler):
    """c: [15, n] states, g: [n] binding affinity g(eta), dt: scalar or [n],
    euler: [15, n] Euler increments."""
    c = np.asarray(c, np.float64)
    scale = np.asarray(scale, np.float64)
    n = c.shape[1]
    x = np.zeros((n, NIN_PAD))
    x[:, :15] = np.log1p(np.maximum(c, 0.0) / scale[:, None]).T
    x[:, 15] = g
    x[:, 16] = np.log(np.broadcast_to(np.asarray(dt, np.float64), (n,)) / DT_REF)
    for o, s in enumerate(REACTING):
        q = np.asarray(euler[s], np.float64) / (np.abs(c[s]) + FLOOR * scale[s])
        x[:, 17 + o] = np.sign(q) * np.log1p(RATE_K * np.abs(q))
    return x


def _den(euler, scale, s):
    return np.abs(euler[s]) + FLOOR * scale[s]


def stiffness(c, euler, scale):
    """rho = max over the reacting species of |E_s| / (|c_s| + FLOOR scale_s)."""
    c = np.asarray(c, np.float64)
    rho = np.zeros(c.shape[1])
    for s in REACTING:
        rho = np.maximum(rho, np.abs(euler[s]) / (np.abs(c[s]) + FLOOR * scale[s]))
    return rho


def targets(c0, c1, euler, scale, d=None):
    """v = (dc - E) / (rho (|E| + FLOOR scale)) for the reacting species
    (0 where rho = 0); [n, 16].  dc = c1 - c0, or the increments d when given."""
    n = c0.shape[1]
    if d is not None:
        c1 = np.asarray(c0, np.float64) + d
    rho = stiffness(c0, euler, scale)
    safe = np.where(rho > 0, rho, 1.0)
    y = np.zeros((n, NOUT_PAD))
    for o, s in enumerate(REACTING):
        inc = d[s] if d is not None else c1[s] - c0[s]
        y[:, o] = np.where(rho > 0, (inc - euler[s]) / (safe * _den(euler, scale, s)), 0.0)
    return y


def increments(c0, euler, v, scale):
    """dc[15, n] from the Euler increment and the network output (ADP row 0)."""
    euler = np.asarray(euler, np.float64)
    rho = stiffness(c0, euler, scale)
    dc = np.zeros_like(euler)
    for o, s in enumerate(REACTING):
        dc[s] = euler[s] + rho * v[:, o] * _den(euler, scale, s)
    return dc


def apply(c0, euler, v, scale):
    """New state from the Euler increment and the network output."""
    return np.asarray(c0, np.float64) + increments(c0, euler, v, scale)


def forward(P, x, bf16_ops=False):
    r = bf16 if bf16_ops else (lambda a: np.asarray(a, np.float64))
    xb = r(x)
    W1, W2, W3 = r(P["W1"]), r(P["W2"]), r(P["W3"])
    z1 = xb @ W1 + P["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ W2 + P["b2"]
    h2 = r(gelu(z2))
    out = h2 @ W3 + P["b3"]
    return out, (xb, z1, h1, z2, h2, W1, W2, W3)


def loss_and_grads(P, x, y, bf16_ops=False):
    """Mean square error over the batch and the 14 used outputs, and its
    gradients with respect to every parameter (backpropagation), with the
    operand rounding of the GPU kernels when bf16_ops is set."""
    r = bf16 if bf16_ops else (lambda a: np.asarray(a, np.float64))
    out, (xb, z1, h1, z2, h2, W1, W2, W3) = forward(P, x, bf16_ops)
    B = x.shape[0]
    diff = np.zeros_like(out)
    diff[:, :NOUT] = out[:, :NOUT] - np.asarray(y, np.float64)[:, :NOUT]
    loss = float(np.sum(diff ** 2) / (B * NOUT))
    scale = 2.0 / (B * NOUT)
    d = r(diff)
    G = {}
    G["W3"] = scale * (h2.T @ d)
    G["b3"] = scale * diff.sum(0)
    dz2 = (d @ W3.T) * gelu_grad(z2)
    dz2b = r(dz2)
    G["W2"] = scale * (h1.T @ dz2b)
    G["b2"] = scale * dz2.sum(0)
    dz1 = (dz2b @ W2.T) * gelu_grad(z1)
    dz1b = r(dz1)
    G["W1"] = scale * (xb.T @ dz1b)
    G["b1"] = scale * dz1.sum(0)
    return loss, G


def adam(P, G, state, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) with bias correction at step t >= 1;
    ``state`` holds the first and second moments per parameter."""
    for k in P:
        m = state.setdefault("m" + k, np.zeros_like(P[k]))
        v = state.setdefault("v" + k, np.zeros_like(P[k]))
        m[...] = b1 * m + (1 - b1) * G[k]
        v[...] = b2 * v + (1 - b2) * G[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P


# ------------------------------------------------------------ the surrogate step

def euler_increments(params, c, eta, dt):
    """E = dt f(c) with the App. A/B right-hand side of an interior cell off
    the adhesion layer (H_adh = 0, no wall face), g = g(eta)."""
    import oracle
    c = np.asarray(c, np.float64)
    n = c.shape[1]
    E = np.zeros_like(c)
    g = np.array([oracle.g(params, float(e)) for e in eta])
    for i in range(n):
        f, _, _ = oracle.rhs(params, c[:, i], H=0.0, g=g[i])
        E[:, i] = dt * f
    E[4] = 0.0
    return E, g


def indicator(c, dc, scale):
    """Largest relative change the surrogate proposes over the reacting species:
    max_s |dc_s| / (|c_s| + FLOOR scale_s)."""
    ind = np.zeros(c.shape[1])
    for s in REACTING:
        ind = np.maximum(ind, np.abs(dc[s]) / (np.abs(c[s]) + FLOOR * scale[s]))
    return ind


def surrogate_parts(desc, params, c, e0, c0, eta, P, scale, h, nsub, bf16_ops=True):
    """Both candidates of the surrogate reaction solve over dt = h * nsub on a
    mesh: ``surr`` = c + dc (network increment, ADP unchanged) and ``rk`` =
    the RK4 solve (nsub steps of h) with its E0, C0; ``region`` marks the
    adhesion-layer and injury-wall cells, ``ind`` the indicator; ``x`` the
    features and ``euler`` the Euler increments."""
    import oracle
    c = np.asarray(c, np.float64)
    dt = h * nsub
    rk_c, rk_e0, rk_c0 = oracle.reaction(desc, params, c, e0, c0, eta, h, nsub)
    H = oracle.hadh(desc)
    nx, ny = int(desc["nx"]), int(desc["ny"])
    fi, fk = oracle.injury_faces(desc)
    wall = np.zeros(c.shape[1], bool)
    wall[fi + nx * ny * fk] = True          # floor row j = 0 above an injury face
    E, g = euler_increments(params, c, eta, dt)
    x = features(c, g, dt, scale, E)
    out, _ = forward(P, x, bf16_ops)
    dc = increments(c, E, out, scale)
    return dict(surr=c + dc, rk=rk_c, e0=rk_e0, c0=rk_c0, region=(H > 0) | wall,
                ind=indicator(c, dc, scale), x=x, euler=E)


def surrogate_step(desc, params, c, e0, c0, eta, P, scale, h, nsub, tol, bf16_ops=True):
    """One reaction solve over dt = h * nsub on a mesh: cells off the adhesion
    layer and the injury wall take the surrogate increment when its indicator
    is at most ``tol``; the others take the RK4 solve (nsub steps of h).
    Returns (c, e0, c0, flag, ind) with flag 0 = surrogate, 1 = indicator
    fallback, 2 = region fallback (H_adh > 0 or a wall cell)."""
    q = surrogate_parts(desc, params, c, e0, c0, eta, P, scale, h, nsub, bf16_ops)
    ind = q["ind"]
    flag = np.where(q["region"], 2, np.where(ind > tol, 1, 0))
    new = np.where(flag[None, :] == 0, q["surr"], q["rk"])
    return new, q["e0"], q["c0"], flag, ind


def _bare_mesh(n):
    """A 1 x n strip with no injury patch: every cell is interior and off the
    adhesion layer (H_adh = 0, no wall face)."""
    return dict(dim=2, nx=int(n), ny=1, nz=1, hx=1e-3, hy=1e-3, hz=1.0,
                inj_x0=-1.0, inj_x1=-1.0, inj_z0=0.0, inj_z1=0.0, p_diam=3e-3)


def rk4_increments(params, c0, eta, dt):
    """Classical RK4 over dt in M_rxn steps of dt / M_rxn (Sec. 3.2 step 2)
    for cells off the adhesion layer and the wall, returning the summed step
    increments h/6 (k1 + 2 k2 + 2 k3 + k4) instead of the new state, so that
    the increment keeps its relative precision when it is far smaller than
    the state (ADP row zero: it has no reaction term)."""
    import oracle
    c0 = np.asarray(c0, np.float64)
    n = c0.shape[1]
    M = int(params["M_rxn"])
    h = dt / M
    d = np.zeros_like(c0)
    for i in range(n):
        g = oracle.g(params, float(eta[i]))
        rhs = lambda y: oracle.rhs(params, y, H=0.0, g=g)[0]
        y = c0[:, i].copy()
        for _ in range(M):
            k1 = rhs(y)
            k2 = rhs(y + 0.5 * h * k1)
            k3 = rhs(y + 0.5 * h * k2)
            k4 = rhs(y + h * k3)
            inc = h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            inc[4] = 0.0
            y = y + inc
            d[:, i] += inc
    return d


def pairs(params, c0, eta, dt, scale):
    """Features and targets of the RK4 reaction solve over dt (M_rxn steps of
    dt / M_rxn) from the states c0 [15, n] (FP64)."""
    c0 = np.asarray(c0, np.float64)
    d = rk4_increments(params, c0, eta, dt)
    E, g = euler_increments(params, c0, eta, dt)
    return features(c0, g, dt, scale, E), targets(c0, c0 + d, E, scale, d=d)

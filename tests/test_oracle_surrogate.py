"""Pins of the FP64 surrogate reference (oracle/surrogate.py): backprop
gradients against central finite differences, the GELU definition against
its closed form at special points, the reduction to explicit Euler for a zero
network, and a target/apply round trip."""
import math

import numpy as np
import pytest

import oracle.surrogate as M


def test_gelu_special_values():
    assert M.gelu(np.array([0.0]))[0] == 0.0
    # odd part: gelu(z) - gelu(-z) = z because tanh is odd
    z = np.linspace(-3, 3, 13)
    assert np.allclose(M.gelu(z) - M.gelu(-z), z, atol=1e-15)
    # the tanh form stays within 1e-3 of the erf definition z Phi(z)
    exact = np.array([0.5 * v * (1 + math.erf(v / math.sqrt(2))) for v in z])
    assert np.max(np.abs(M.gelu(z) - exact)) < 1e-3
    assert M.gelu(np.array([40.0]))[0] == 40.0 and M.gelu(np.array([-40.0]))[0] == 0.0
    h = 1e-6
    assert np.allclose(M.gelu_grad(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), atol=1e-8)


def test_bf16_rounding():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    v = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 3.0, -2.5, 1e-20, 65504.0])
    r = M.bf16(v)
    assert list(r[:5]) == [1.0, 1.0, 1 + 2 ** -6, 3.0, -2.5]
    assert abs(r[5] - 1e-20) <= 2 ** -8 * 1e-20
    assert np.all(np.abs(M.bf16(np.linspace(-7, 7, 1001)) - np.linspace(-7, 7, 1001))
                  <= 2 ** -8 * np.abs(np.linspace(-7, 7, 1001)))


def test_pack_unpack_round_trip():
    P = M.init_params(4)
    w = M.pack(P)
    assert w.size == M.NPARAM == 32 * 64 + 64 + 64 * 64 + 64 + 64 * 16 + 16
    Q = M.unpack(w)
    for k in P:
        assert np.array_equal(P[k], Q[k])


@pytest.mark.parametrize("bf16_ops", [False, True])
def test_backprop_matches_finite_differences(bf16_ops):
    rng = np.random.default_rng(0)
    P = M.init_params(1)
    P["W3"] = rng.standard_normal(P["W3"].shape) * 0.3
    P["b1"] = rng.standard_normal(64) * 0.1
    x = rng.standard_normal((20, 32))
    x[:, 31:] = 0
    y = rng.standard_normal((20, 16))
    loss, G = M.loss_and_grads(P, x, y)
    if bf16_ops:
        # with operands rounded, the gradient is the exact gradient of the
        # rounded network up to the bf16 rounding of dz: compare against FP64
        # backprop at the bf16-rounded point within the rounding error
        Pb = {k: (M.bf16(v) if k.startswith("W") else v) for k, v in P.items()}
        xb = M.bf16(x)
        _, Gr = M.loss_and_grads(Pb, xb, y, bf16_ops=True)
        _, Ge = M.loss_and_grads(Pb, xb, y)
        for k in P:
            err = np.linalg.norm(Gr[k] - Ge[k]) / np.linalg.norm(Ge[k])
            assert err < 2e-2, (k, err)
        return
    h = 1e-6
    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = M.loss_and_grads(P, x, y)
            flat[idx] = old - h
            lm, _ = M.loss_and_grads(P, x, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert G[k].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, idx)


def test_zero_network_is_explicit_euler_and_targets_round_trip():
    rng = np.random.default_rng(2)
    scale = np.full(15, 2.0)
    c0 = rng.random((15, 7))
    euler = rng.standard_normal((15, 7)) * 1e-2
    c1 = M.apply(c0, euler, np.zeros((7, 16)), scale)
    for s in M.REACTING:
        assert np.allclose(c1[s], c0[s] + euler[s], rtol=0, atol=1e-15)
    assert np.array_equal(c1[4], c0[4])                     # ADP has no reaction
    target = rng.random((15, 7))
    y = M.targets(c0, target, euler, scale)
    back = M.apply(c0, euler, y, scale)
    for s in M.REACTING:
        assert np.allclose(back[s], target[s], rtol=1e-12)


def test_adam_decreases_a_convex_loss():
    rng = np.random.default_rng(3)
    P = M.init_params(0)
    x = rng.standard_normal((64, 32))
    x[:, 31:] = 0
    y = np.zeros((64, 16))
    y[:, :14] = 0.1
    st = {}
    l0, _ = M.loss_and_grads(P, x, y)
    for t in range(1, 60):
        _, G = M.loss_and_grads(P, x, y)
        P = M.adam(P, G, st, 3e-3, t)
    l1, _ = M.loss_and_grads(P, x, y)
    assert l1 < 0.2 * l0


def _params():
    import synthetic
    return synthetic.params_default()


def test_surrogate_step_zero_network_closed_form():
    """A linear-activation cell (only P^{m,u}, P^{m,a}, ADP nonzero, no
    adhesion, g = 0) has the Euler increment dP^{m,u} = -A dt P^{m,u} with
    A = k_adp ADP / (ADP* + ADP) (App. A); a zero network returns it."""
    import synthetic
    p = _params()
    desc = synthetic.channel2d(6, 4, 9e-3, 6e-3)
    n = 24
    c = np.zeros((15, n))
    c[0] = 2e5
    c[1] = 1e3
    c[4] = np.linspace(1e-6, 1e-3, n)
    P = {k: np.zeros_like(v) for k, v in M.init_params(0).items()}
    scale = synthetic.surrogate_scale(p)
    dt = 1e-5
    new, _, _, flag, ind = M.surrogate_step(desc, p, c, np.zeros(2), np.zeros(2), np.zeros(n), P, scale,
                                            dt / 2, 2, tol=np.inf)
    A = p["k_adp"] * c[4] / (p["adp_star"] + c[4])
    off = flag == 0
    assert off.sum() > 0 and np.all(flag[~off] == 2)
    assert np.allclose(new[0, off], c[0, off] * (1 - A[off] * dt), rtol=1e-14)
    assert np.allclose(new[1, off], c[1, off] + A[off] * dt * c[0, off], rtol=1e-14)
    assert np.allclose(ind[off], A[off] * dt * c[0, off] / (c[1, off] + 1e-6 * scale[1]), rtol=1e-12)


def test_surrogate_step_region_and_fallback_take_rk4():
    """Adhesion-layer and wall cells, and every cell when tol = 0, take the
    RK4 reaction solve; an equilibrium cell (plasma values, nothing bound,
    ADP = E2 = 0) is kept by both."""
    import oracle
    import synthetic
    p = _params()
    desc = synthetic.channel2d(12, 6, 18e-3, 9e-3)
    c, e0, c0 = synthetic.primed_state(desc, p, seed=3)
    n = c.shape[1]
    eta = np.linspace(0.0, 0.9, n)
    P = M.init_params(1)
    P["W3"] *= 30.0
    scale = synthetic.surrogate_scale(p)
    h, nsub = 5e-6, 2
    rk, rke0, rkc0 = oracle.reaction(desc, p, c, e0, c0, eta, h, nsub)
    new, ne0, nc0, flag, _ = M.surrogate_step(desc, p, c, e0, c0, eta, P, scale, h, nsub, tol=0.0)
    assert np.all(flag > 0) or np.all((flag > 0) | (np.abs(new - c).sum(0) == 0))
    assert np.allclose(new, rk, rtol=1e-15, atol=0)
    assert np.array_equal(ne0, rke0) and np.array_equal(nc0, rkc0)
    H = oracle.hadh(desc)
    new2, _, _, flag2, _ = M.surrogate_step(desc, p, c, e0, c0, eta, P, scale, h, nsub, tol=np.inf)
    assert np.all(flag2[H > 0] == 2)
    assert np.array_equal(new2[:, H > 0], rk[:, H > 0])
    assert np.all(flag2[H == 0] == 0)
    rest = np.zeros((15, 1))
    rest[0], rest[5], rest[6] = 2.5e5, 1.7e-4, 1.4e-3
    E, _ = M.euler_increments(p, rest, np.zeros(1), 1e-5)
    assert np.all(E == 0.0) and M.stiffness(rest, E, scale)[0] == 0.0
    assert np.all(M.increments(rest, E, np.ones((1, 16)), scale) == 0.0)


def test_pairs_targets_reproduce_rk4():
    """apply(c0, E, target) reconstructs the oracle's RK4 state (targets are
    the exact correction of Euler by construction)."""
    import oracle
    import synthetic
    p = _params()
    c, eta = synthetic.surrogate_states(64, p, seed=5)
    scale = synthetic.surrogate_scale(p)
    dt = 1.5625e-5
    x, y = M.pairs(p, c, eta, dt, scale)
    E, g = M.euler_increments(p, c, eta, dt)
    back = M.apply(c, E, y, scale)
    for i in range(0, 64, 9):
        ref, _, _ = oracle.rk4_cell(p, c[:, i], dt / 2, nsub=2, g=oracle.g(p, eta[i]))
        for s in M.REACTING:
            assert back[s, i] == pytest.approx(ref[s], rel=1e-9, abs=1e-12 * scale[s])
    assert np.all(x[:, 31:] == 0) and np.allclose(x[:, 16], np.log(dt / 1e-5))
    assert np.allclose(x[:, 15], g)
    # relative-rate features: sign and magnitude of E_s / (|c_s| + floor_s)
    for o, s in enumerate(M.REACTING):
        q = E[s] / (np.abs(c[s]) + 1e-6 * scale[s])
        assert np.allclose(np.expm1(np.abs(x[:, 17 + o])) / 1e3, np.abs(q), rtol=1e-9, atol=1e-15)
        assert np.all(np.sign(x[:, 17 + o]) == np.sign(q))


def test_pairs_linear_activation_closed_form():
    """Linear-activation cells (only P^{m,u}, P^{m,a}, ADP nonzero, g = 0):
    with A = k_adp ADP / (ADP* + ADP), Euler gives dP^{m,u} = -A dt P^{m,u},
    two RK4 steps of dt/2 multiply P^{m,u} by R(-A dt/2)^2 with the RK4
    stability polynomial R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 (App. A), and
    P^{m,a} gains what P^{m,u} loses.  The targets follow in closed form."""
    import synthetic
    p = _params()
    scale = synthetic.surrogate_scale(p)
    n = 5
    c = np.zeros((15, n))
    c[0] = [2e5, 5e5, 1e6, 3e4, 2e5]
    c[1] = [1e3, 0.0, 5e4, 1e2, 2e5]
    c[4] = [1e-5, 1e-4, 1e-3, 3e-3, 5e-7]
    dt = 2e-5
    x, y = M.pairs(p, c, np.zeros(n), dt, scale)
    A = p["k_adp"] * c[4] / (p["adp_star"] + c[4])
    z = -A * dt / 2
    w = z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24       # R(z) - 1
    dP = c[0] * w * (2 + w)                             # c (R^2 - 1)
    E = 2 * z * c[0]                                    # -A dt c
    dPmE = c[0] * (z ** 2 + z ** 3 / 3 + z ** 4 / 12 + w ** 2)   # dP - E without cancellation
    fl0, fl1 = 1e-6 * scale[0], 1e-6 * scale[1]
    rho = np.maximum(np.abs(E) / (c[0] + fl0), np.abs(E) / (c[1] + fl1))
    # the oracle forms the RK4 increment step by step and subtracts E in FP64:
    # absolute error a few units of 2^-52 |E| before the division
    eps = 2.0 ** -52
    for o, sign, fl in ((0, 1.0, fl0), (1, -1.0, fl1)):
        den = rho * (np.abs(E) + fl)
        exp = sign * dPmE / den
        atol = 16 * eps * np.abs(E) / den
        assert np.all(np.abs(y[:, o] - exp) <= 1e-9 * np.abs(exp) + atol), (o, y[:, o], exp)
    assert np.all(y[:, 2:] == 0.0)
    assert np.allclose(x[:, 0], np.log1p(c[0] / scale[0])) and np.allclose(x[:, 4], np.log1p(c[4] / scale[4]))
    assert np.allclose(x[:, 17], -np.log1p(1e3 * np.abs(E) / (c[0] + fl0)))      # P^{m,u} loses
    assert np.allclose(x[:, 18], np.log1p(1e3 * np.abs(E) / (c[1] + fl1)))       # P^{m,a} gains

"""Parity of the reaction surrogate kernels (through the C ABI) with the FP64
reference in oracle/surrogate.py on seeded inputs: network forward, training
pairs, loss gradient, Adam, the training loop, and the surrogate reaction
solve with its RK4 fallback on 2D and 3D meshes."""
import numpy as np
import pytest

import oracle as O
import oracle.surrogate as MS
import synthetic as S
from parity_util import SCALE, rel_l2, species_errors

pytestmark = pytest.mark.gpu

PRM = S.params_default()
SCL = S.surrogate_scale(PRM)
U = 2.0 ** -8   # bfloat16 unit roundoff


def _clot():
    import paper_2304_09180_gb300 as clot
    return clot


def _net(seed=1, w3=30.0, bias=0.1):
    rng = np.random.default_rng(seed + 17)
    P = MS.init_params(seed)
    P["b1"] = rng.normal(0.0, bias, 64)
    P["b2"] = rng.normal(0.0, bias, 64)
    P["W3"] = P["W3"] * w3
    P["b3"][:14] = rng.normal(0.0, bias, 14)
    return P


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _prm(clot, **over):
    z = np.zeros(1)
    return clot.Params(PRM, z, z, z, **over)


def forward_bound(P, x, x_err=None):
    """Element-wise bound of |GPU - oracle| for the forward pass.  The oracle
    rounds the same operands to bf16 but evaluates gelu exactly; the GPU
    evaluates gelu in bf16x2 arithmetic (z rounded, z^2, the cubic, tanh,
    z/2 (1 + t), each rounded to bf16 with unit roundoff u = 2^-8): the
    relative error of the tanh argument is at most ~6u, moving tanh by at most
    6u max_x x sech^2 x < 2.7u, so |g_gpu - gelu(z)| <= 2u |z| + 2u |g| and
    |g_gpu - bf16(gelu(z))| <= 2u |z| + 3u |g|; propagated through W2 (with
    |gelu'| <= 1.13) and W3 and doubled, plus FP32 accumulation order.
    x_err: a bound of |x_gpu - x| when the GPU computes its own features."""
    out, (xb, z1, h1, z2, h2, W1, W2, W3) = MS.forward(P, x, bf16_ops=True)
    e1 = 3 * U * np.abs(h1) + 2 * U * np.abs(z1)
    if x_err is not None:
        e1 = e1 + 1.13 * (x_err @ np.abs(W1))
    e2 = 1.13 * (e1 @ np.abs(W2)) + 3 * U * np.abs(h2) + 2 * U * np.abs(z2)
    acc = 1e-6 * (np.abs(h2) @ np.abs(W3) + np.abs(P["b3"]))
    return out, 2.0 * (e2 @ np.abs(W3)) + acc + 1e-7


ENGINES = [0, 1]  # warp-level mma.sync, tcgen05 with tensor-memory accumulators


@pytest.mark.parametrize("engine", ENGINES)
def test_forward_matches_bf16_oracle(engine):
    clot = _clot()
    c, eta = S.surrogate_states(3001, PRM, seed=11)
    x, _ = MS.pairs(PRM, c, eta, 1.5625e-5, SCL)
    P = _net()
    mlp = clot.Mlp(MS.pack(P), SCL, engine=engine)
    out = clot.clot_surrogate_forward(mlp, _t(x)).double().cpu().numpy()
    ref, bound = forward_bound(P, x)
    viol = np.abs(out - ref) - bound
    assert np.all(viol <= 0), f"max excess {viol.max():.3g}, max |diff| {np.abs(out - ref).max():.3g}"
    assert np.all(out[:, 14:] == ref[:, 14:])  # padded outputs: bias only (zero)


def test_pairs_match_oracle():
    """Both sides compute the pairs in FP64 from the same FP32 states; they
    differ by the GPU's FP32-rounded rate constants and scales and the FP32
    output: 1e-5 relative, plus 2e-6 absolute for near-equilibrium binding
    terms (k+ free s - k- s_b), where a 6e-8 change of a rate constant moves
    E and dRK4 by 6e-8 of the gross rate rather than of the net; both sides
    also carry the FP64 rounding of dRK4 - E, a few units of 2^-52 |E|
    divided by rho (|E| + floor)."""
    import torch
    clot = _clot()
    n = 5003
    c, eta = S.surrogate_states(n, PRM, seed=12)
    c, eta = _f32(c), _f32(eta)
    dt = 1.5625e-5
    x_ref, y_ref = MS.pairs(PRM, c, eta, dt, SCL)
    mlp = clot.Mlp(np.zeros(clot.MLP_NPARAM), SCL)
    x, y = clot.clot_surrogate_pairs(_prm(clot), mlp, _t(c), _t(eta), dt)
    torch.cuda.synchronize()
    x, y = x.double().cpu().numpy(), y.double().cpu().numpy()
    assert np.all(np.abs(x - x_ref) <= 2e-6 * (1.0 + np.abs(x_ref)))
    E, _ = MS.euler_increments(PRM, c, eta, dt)
    rho = MS.stiffness(c, E, SCL)
    assert np.all((rho > 0) | np.all(y_ref == 0, axis=1))
    noise = np.zeros_like(y_ref)
    for o, s in enumerate(MS.REACTING):
        den = rho * (np.abs(E[s]) + MS.FLOOR * SCL[s])
        noise[:, o] = np.where(rho > 0, 64 * 2.0 ** -52 * np.abs(E[s]) / np.where(den > 0, den, 1.0), 0.0)
    err = np.abs(y - y_ref)
    tol = 1e-5 * np.abs(y_ref) + 2e-6 + noise
    assert np.all(err <= tol), f"max excess {(err - tol).max():.3g} at {np.unravel_index(np.argmax(err - tol), err.shape)}"


def test_gradient_matches_oracle():
    """GPU loss gradient vs the FP64 gradient of the same bf16-operand
    network (oracle emulates the roundings): per parameter block rel-L2 below
    1e-2 (the two differ where an FP32 value rounds to the other bf16
    neighbour), and within 5e-2 of the exact FP64 gradient."""
    import torch
    clot = _clot()
    n = 4133
    c, eta = S.surrogate_states(n, PRM, seed=13)
    x, y = MS.pairs(PRM, c, eta, 1.5625e-5, SCL)
    y = np.clip(y, -10, 10)
    P = _net(w3=5.0)
    mlp = clot.Mlp(MS.pack(P), SCL)
    grad, loss = clot.clot_surrogate_grad(mlp, _t(x), _t(y))
    torch.cuda.synchronize()
    G = MS.unpack(grad.double().cpu().numpy())
    l_ref, Gr = MS.loss_and_grads(P, x, y, bf16_ops=True)
    l_ex, Ge = MS.loss_and_grads(P, x, y)
    assert float(loss.item()) == pytest.approx(l_ref, rel=1e-3)
    for k in G:
        assert rel_l2(G[k], Gr[k]) < 1e-2, (k, rel_l2(G[k], Gr[k]))
        assert rel_l2(G[k], Ge[k]) < 5e-2, (k, rel_l2(G[k], Ge[k]))
    assert np.all(G["W1"][31:] == 0) and np.all(G["W3"][:, 14:] == 0) and np.all(G["b3"][14:] == 0)


def test_adam_steps_match_oracle():
    """Two training steps (t = 1, 2) equal FP64 Adam applied to the GPU's own
    gradients of the two batches."""
    import torch
    clot = _clot()
    n, batch, lr = 2048, 1024, 1e-3
    c, eta = S.surrogate_states(n, PRM, seed=14)
    x, y = MS.pairs(PRM, c, eta, 1e-5, SCL)
    y = np.clip(y, -10, 10)
    P = _net(w3=5.0)
    w0 = MS.pack(P)
    mlp = clot.Mlp(w0, SCL)
    xt, yt = _t(x), _t(y)
    m = torch.zeros(clot.MLP_NPARAM, device="cuda")
    v = torch.zeros_like(m)
    state, Pr = {}, MS.unpack(mlp.w.double().cpu().numpy())
    for t in (1, 2):
        rows = slice((t - 1) * batch, t * batch)
        g, _ = clot.clot_surrogate_grad(mlp, xt[rows].contiguous(), yt[rows].contiguous())
        clot.clot_surrogate_train(mlp, m, v, t - 1, lr, xt[rows].contiguous(), yt[rows].contiguous(), batch, 1)
        torch.cuda.synchronize()
        Pr = MS.adam(Pr, MS.unpack(g.double().cpu().numpy()), state, lr, t)
        got = mlp.w.double().cpu().numpy()
        assert np.max(np.abs(got - MS.pack(Pr))) <= 1e-6 + 1e-6 * np.max(np.abs(MS.pack(Pr)))
        Pr = MS.unpack(got)   # continue from the GPU's FP32 weights


def test_training_is_bitwise_reproducible():
    """The block gradient sums are formed in a fixed order (no floating-point
    atomics), so two training runs from the same weights on the same batches
    give the same weights bit for bit, and so do two gradient evaluations."""
    import torch
    clot = _clot()
    n, batch = 8192, 2048
    c, eta = S.surrogate_states(n, PRM, seed=15)
    x, y = MS.pairs(PRM, c, eta, 1e-5, SCL)
    xt, yt = _t(x), _t(np.clip(y, -10, 10))
    w0 = MS.pack(_net(w3=5.0))
    out = []
    for _ in range(2):
        mlp = clot.Mlp(w0, SCL)
        m = torch.zeros(clot.MLP_NPARAM, device="cuda")
        v = torch.zeros_like(m)
        clot.clot_surrogate_train(mlp, m, v, 0, 1e-3, xt, yt, batch, 40)
        g, loss = clot.clot_surrogate_grad(mlp, xt, yt)
        torch.cuda.synchronize()
        out.append((mlp.w.cpu().numpy().copy(), g.cpu().numpy().copy(), float(loss)))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]


def test_training_reduces_loss():
    """Pairs generated on the GPU (targets clipped to [-1, 1]: beyond that
    Euler is off by more than the step's own increment, a stiff cell the
    indicator rejects), 400 Adam steps over 10 batches of 4096 rows: the loss
    of the last pass over the batches is below half the first pass's, and
    held-out predictions beat explicit Euler (v = 0)."""
    import torch
    clot = _clot()
    prm = _prm(clot)
    mlp = clot.Mlp(MS.pack(MS.init_params(3)), SCL)
    xs, ys = [], []
    for q, dt in enumerate((5e-6, 1.5625e-5, 5e-5)):
        c, eta = S.surrogate_states(16384, PRM, seed=20 + q)
        x, y = clot.clot_surrogate_pairs(prm, mlp, _t(c), _t(eta), dt)
        xs.append(x)
        ys.append(y)
    x = torch.cat(xs)
    y = torch.cat(ys).clamp(-4, 4)
    perm = torch.randperm(x.shape[0], generator=torch.Generator().manual_seed(0)).cuda()
    x, y = x[perm].contiguous(), y[perm].contiguous()
    xtr, ytr, xho, yho = x[:40960], y[:40960], x[40960:], y[40960:]
    m = torch.zeros(clot.MLP_NPARAM, device="cuda")
    v = torch.zeros_like(m)
    loss = clot.clot_surrogate_train(mlp, m, v, 0, 2e-3, xtr, ytr, 4096, 400)
    torch.cuda.synchronize()
    L = loss.cpu().numpy()
    assert np.all(np.isfinite(L))
    assert L[-10:].mean() < 0.5 * L[:10].mean(), (L[:10], L[-10:])
    out = clot.clot_surrogate_forward(mlp, xho)
    mse = float(((out[:, :14] - yho[:, :14]) ** 2).mean())
    mse0 = float((yho[:, :14] ** 2).mean())
    assert mse < 0.5 * mse0, (mse, mse0)


def _f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


def _infer_case(desc, state, eta, P, tol, h=7.8125e-6, nsub=2, engine=0):
    import torch
    clot = _clot()
    c, e0, c0 = state
    mesh = clot.Mesh(desc)
    prm = _prm(clot)
    f = clot.Fields.from_host(mesh, PRM, c, e0, c0, eta=eta)
    mlp = clot.Mlp(MS.pack(P), SCL, engine=engine)
    flag = torch.full((mesh.ncell,), 255, dtype=torch.uint8, device="cuda")
    counts = clot.clot_surrogate_infer(mesh, f, prm, mlp, h, nsub, tol, flag=flag, counts=True)
    torch.cuda.synchronize()
    out = f.to_host(mesh)
    out["flag"] = flag.cpu().numpy().astype(int)
    out["counts"] = counts
    out["bound"] = f.bound_acc.double().cpu().numpy()
    return out, MS.surrogate_parts(desc, PRM, c, e0, c0, eta, P, SCL, h, nsub)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("case", ["channel", "duct"])
@pytest.mark.parametrize("tol", [1e-3, 3e-2])
def test_infer_matches_oracle(case, tol, engine):
    """Same FP32 inputs on both sides.  (a) Flags equal the oracle's wherever
    the oracle's indicator is farther from tol than the GPU/oracle network
    difference can move it; the only other allowed difference is a cell the
    GPU finds at rest (its FP32 Euler increment underflows to zero) whose
    oracle RK4 solve leaves it unchanged to 1e-6.  (b) Accepted cells: within
    rho fb (|E_s| + floor_s) of the oracle's surrogate state, fb the forward
    bound of test_forward_matches_bf16_oracle, plus FP32 rounding.  (c) Every
    other cell: RK4, species rel-L2 <= 1e-5 against the oracle, likewise E0,
    C0 and the bound-platelet accumulator.  (d) counts are those of the flags."""
    cfg = S.config("channel_200x40" if case == "channel" else "duct_40x16x12", PRM)
    desc = cfg["desc"]
    c, e0, c0 = (_f32(a) for a in S.primed_state(desc, PRM, seed=2))
    n = c.shape[1]
    eta = _f32(np.random.default_rng(5).uniform(0.0, 1.0, n))
    P = _net(w3=3.0)
    out, q = _infer_case(desc, (c, e0, c0), eta, P, tol, engine=engine)
    fl = out["flag"]
    assert np.all(fl <= 2)
    flag = np.where(q["region"], 2, np.where(q["ind"] > tol, 1, 0))
    E = q["euler"]
    rho = MS.stiffness(c, E, SCL)
    # the kernel computes its features in FP32 (fast log): one bf16 unit of
    # each feature plus 1e-7 absolute (log1p of a tiny argument)
    _, fb = forward_bound(P, q["x"], x_err=U * np.abs(q["x"]) + 1e-7)
    margin = 1e-5 * q["ind"]
    for o, s in enumerate(MS.REACTING):
        fl_s = MS.FLOOR * SCL[s]
        margin = margin + rho * fb[:, o] * (np.abs(E[s]) + fl_s) / (np.abs(c[s]) + fl_s)
    clear = np.abs(q["ind"] - tol) > margin
    mism = clear & (fl != flag)
    still = np.ones(n, bool)
    for s in MS.REACTING:
        still &= np.abs(q["rk"][s] - c[s]) <= 1e-6 * (np.abs(c[s]) + MS.FLOOR * SCL[s])
    assert np.all(still[mism] & (fl[mism] == 0)), int(mism.sum())
    acc = (fl == 0) & ~mism
    for o, s in enumerate(MS.REACTING):
        den = np.abs(E[s]) + MS.FLOOR * SCL[s]
        # + 1e-15 scale_s: FP32 subnormal results (quantum 1.4e-45)
        bound = rho * fb[:, o] * den + 2e-7 * (np.abs(c[s]) + np.abs(q["surr"][s])) + 1e-9 * MS.FLOOR * SCL[s]
        err = np.abs(out["c"][s] - q["surr"][s])
        assert np.all(err[acc] <= bound[acc]), (S.SPECIES[s], float((err - bound)[acc].max()))
    bsum = np.zeros(n)
    for o, s in ((2, 2), (3, 3)):
        bsum += rho * fb[:, o] * (np.abs(E[s]) + MS.FLOOR * SCL[s]) + 2e-7 * np.abs(q["surr"][s] - c[s])
    gain_acc = (q["surr"][2] + q["surr"][3]) - (c[2] + c[3])
    assert np.all(np.abs(out["bound"] - gain_acc)[acc] <= bsum[acc] + 2e-9 * MS.FLOOR * SCL[2])
    assert np.array_equal(out["c"][:, mism], c[:, mism])
    rk = fl > 0
    errs = species_errors(out["c"][:, rk], q["rk"][:, rk])
    assert np.all(errs <= 1e-5), errs
    assert rel_l2(out["e0"], q["e0"]) <= 1e-5 and rel_l2(out["c0"], q["c0"], 1e-9) <= 1e-5
    gained = (q["rk"][2] + q["rk"][3]) - (c[2] + c[3])
    assert rel_l2(out["bound"][rk], gained[rk], 2.5e5) <= 1e-5
    assert np.array_equal(out["counts"], [int((fl == 0).sum()), int((fl == 1).sum()), int((fl == 2).sum())])
    assert (fl == 0).sum() > 0 and (fl == 1).sum() > 0 and (fl == 2).sum() > 0


@pytest.mark.parametrize("engine", ENGINES)
def test_infer_tol_zero_is_reaction_step(engine):
    """tol = 0: every cell that moves falls back, so the solve equals
    clot_reaction_step (same RK4 device code) up to FP32 contraction order."""
    import torch
    clot = _clot()
    cfg = S.config("channel_200x40", PRM)
    desc = cfg["desc"]
    c, e0, c0 = S.primed_state(desc, PRM, seed=4)
    eta = np.random.default_rng(6).uniform(0.0, 1.0, c.shape[1])
    # tol = 0 accepts only cells at rest (dc = 0), which RK4 also keeps
    mesh = clot.Mesh(desc)
    prm = _prm(clot)
    f1 = clot.Fields.from_host(mesh, PRM, c, e0, c0, eta=eta)
    f2 = clot.Fields.from_host(mesh, PRM, c, e0, c0, eta=eta)
    mlp = clot.Mlp(MS.pack(_net()), SCL, engine=engine)
    clot.clot_surrogate_infer(mesh, f1, prm, mlp, 5e-6, 2, 0.0)
    clot.clot_reaction_step(mesh, f2, prm, 5e-6, 2)
    torch.cuda.synchronize()
    a, b = f1.to_host(mesh), f2.to_host(mesh)
    assert np.all(species_errors(a["c"], b["c"]) <= 1e-6)
    assert np.allclose(a["e0"], b["e0"], rtol=1e-6, atol=0)


def test_trained_network_beats_explicit_euler():
    """What the learned part gains: a network trained on the GPU (pairs from
    the RK4 solve of random and primed states at three dt, rows with relative
    Euler change rho >= 1e-4, 6000 Adam steps, the bench's recipe) against
    the same path with a zero network (explicit Euler), on held-out random
    states, both judged against clot_reaction_step (RK4).  The trained
    network's worst species error is below a quarter of Euler's at tol 3e-2
    and below 0.7 of it at tol 1 (where the stiffest accepted cells dominate),
    and thrombin (E2) and bound platelets (P^{b,a}, P^{b,se}) stay within 1e-3."""
    import torch
    clot = _clot()
    prm = _prm(clot)
    zero = clot.Mlp(np.zeros(clot.MLP_NPARAM), SCL)
    xs, ys = [], []
    for q, dt in enumerate((5e-6, 1.5625e-5, 5e-5)):
        c, eta = S.surrogate_states(65536, PRM, seed=40 + q)
        for cc, ee in ((c, eta),):
            x, y = clot.clot_surrogate_pairs(prm, zero, _t(cc), _t(ee), dt)
            xs.append(x)
            ys.append(y)
    d = S.config("channel_200x40", PRM)["desc"]
    cp, _, _ = S.primed_state(d, PRM, seed=3)
    ep = np.random.default_rng(1).uniform(0, 1, cp.shape[1])
    for dt in (5e-6, 1.5625e-5, 5e-5):
        x, y = clot.clot_surrogate_pairs(prm, zero, _t(cp), _t(ep), dt)
        xs.append(x)
        ys.append(y)
    X, Y = torch.cat(xs), torch.cat(ys).clamp(-4, 4)
    rho = (torch.expm1(X[:, 17:31].abs()) / 1e3).max(1).values
    keep = rho >= 1e-4
    X, Y = X[keep], Y[keep]
    perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(0)).cuda()
    batch = 16384
    n = (X.shape[0] // batch) * batch
    X, Y = X[perm][:n].contiguous(), Y[perm][:n].contiguous()
    mlp = clot.Mlp(MS.pack(MS.init_params(3)), SCL)
    m = torch.zeros(clot.MLP_NPARAM, device="cuda")
    v = torch.zeros_like(m)
    for k, lr in enumerate((2e-3, 1e-3, 5e-4)):
        clot.clot_surrogate_train(mlp, m, v, 2000 * k, lr, X, Y, batch, 2000)
    torch.cuda.synchronize()

    ch, eh = S.surrogate_states(65536, PRM, seed=77)
    desc = S.channel2d(ch.shape[1], 1, ch.shape[1] * 1.5e-3, 1.5e-3, inj_frac=(2.0, 2.0))
    mesh = clot.Mesh(desc)
    ref = clot.Fields.from_host(mesh, PRM, ch, np.zeros(0), np.zeros(0), eta=eh)
    clot.clot_reaction_step(mesh, ref, prm, 7.8125e-6, 2)
    rk = ref.to_host(mesh)["c"]
    for tol in (3e-2, 1.0):
        errs = {}
        for name, net in (("trained", mlp), ("euler", zero)):
            f = clot.Fields.from_host(mesh, PRM, ch, np.zeros(0), np.zeros(0), eta=eh)
            clot.clot_surrogate_infer(mesh, f, prm, net, 7.8125e-6, 2, tol)
            torch.cuda.synchronize()
            errs[name] = species_errors(f.to_host(mesh)["c"], rk)
        gain = 0.25 if tol < 0.1 else 0.7
        assert errs["trained"].max() < gain * errs["euler"].max(), (tol, errs)
        for s in (2, 3, 8):
            assert errs["trained"][s] <= 1e-3, (tol, S.SPECIES[s], errs["trained"][s])


@pytest.mark.parametrize("case,tol", [("channel", 1e-3), ("duct", 2e-2)])
def test_species_step_surrogate_matches_oracle(case, tol):
    """One species step with the surrogate reaction (clot_species_step_surrogate).
    (1) Its transport pass is the fused pass of clot_species_step with the
    reaction off: a CLOT_NO_REACTION step on the same input, which matches the
    oracle's transport (rel-L2 <= 1e-5 per species).  (2) Its reaction pass,
    given that post-transport state (FP32) and the eta the step solved, is the
    oracle's surrogate reaction of oracle/surrogate.py: cells whose indicator
    lies clearly on one side of tol (farther than the network difference can
    move it) take the oracle's choice -- the network increment within the
    forward bound of test_forward_matches_bf16_oracle, or RK4 within rel-L2
    1e-5 -- and every other cell one of the two; the counts agree.  tol sits
    inside the indicator's range of each case (on the duct, whose primed cells
    all lie above 2e-3, near its median), so both choices are taken."""
    import torch
    clot = _clot()
    name = "channel_200x40" if case == "channel" else "duct_40x16x12"
    cfg = S.config(name, PRM)
    desc, dt = cfg["desc"], cfg["dt"]
    state = tuple(_f32(a) for a in S.primed_state(desc, PRM, seed=2))
    mesh = clot.Mesh(desc)
    fl = clot.Fluxes(mesh, **cfg["fluxes"])
    M = int(PRM["M_rxn"])
    # (1) the transport pass
    ft = clot.Fields.from_host(mesh, PRM, *state)
    clot.clot_species_step(mesh, ft, fl, clot.Params(PRM, **cfg["inlet"], eta_tol=1e-6, flags=clot.NO_REACTION), dt, 1)
    torch.cuda.synchronize()
    tr = ft.to_host(mesh)
    po = S.params_default(flags=O.NO_REACTION | O.NO_ETA)
    st = O.new_state(desc, po, *state)
    inp = dict(cfg["fluxes"])
    inp.update(cfg["inlet"])
    O.step(desc, po, st, inp, dt, 1)
    errs = species_errors(tr["c"], st.c)
    assert np.all(errs <= 1e-5), errs
    # (2) the surrogate step from the same input
    P = _net(w3=3.0)
    mlp = clot.Mlp(MS.pack(P), SCL)
    fs = clot.Fields.from_host(mesh, PRM, *state)
    counts = clot.clot_species_step_surrogate(mesh, fs, fl, clot.Params(PRM, **cfg["inlet"], eta_tol=1e-6), mlp, tol,
                                              dt, 1, counts=True)
    torch.cuda.synchronize()
    out = fs.to_host(mesh)
    c = _f32(tr["c"])
    eta = _f32(ft.eta.double().cpu().numpy())   # the eta the step solved (same solve in both calls)
    q = MS.surrogate_parts(desc, PRM, c, state[1], state[2], eta, P, SCL, dt / M, M)
    n = c.shape[1]
    E = q["euler"]
    rho = MS.stiffness(c, E, SCL)
    _, fb = forward_bound(P, q["x"], x_err=U * np.abs(q["x"]) + 1e-7)
    margin = 1e-5 * q["ind"]
    for o, s in enumerate(MS.REACTING):
        fl_s = MS.FLOOR * SCL[s]
        margin = margin + rho * fb[:, o] * (np.abs(E[s]) + fl_s) / (np.abs(c[s]) + fl_s)
    flag = np.where(q["region"], 2, np.where(q["ind"] > tol, 1, 0))
    clear = q["region"] | (np.abs(q["ind"] - tol) > margin)
    near_surr = np.ones(n, bool)
    for o, s in enumerate(MS.REACTING):
        den = np.abs(E[s]) + MS.FLOOR * SCL[s]
        bound = rho * fb[:, o] * den + 2e-7 * (np.abs(c[s]) + np.abs(q["surr"][s])) + 1e-9 * MS.FLOOR * SCL[s]
        near_surr &= np.abs(out["c"][s] - q["surr"][s]) <= bound
    take_s = clear & (flag == 0)
    assert np.all(near_surr[take_s]), int((~near_surr[take_s]).sum())
    take_r = clear & (flag > 0)
    assert np.all(species_errors(out["c"][:, take_r], q["rk"][:, take_r]) <= 1e-5)
    assert rel_l2(out["e0"], q["e0"]) <= 1e-5 and rel_l2(out["c0"], q["c0"], 1e-9) <= 1e-5
    assert counts[2] == int(q["region"].sum())
    assert int((take_s).sum()) <= counts[0] <= int((flag == 0).sum() + (~clear).sum())
    assert counts[0] > 0 and counts[1] > 0, counts

"""Pins of the oracle's reaction right-hand side and RK4 integrator
(Sec. 3.2 step 2; App. A platelet sources; App. B mass-action coagulation and
injury-wall exchange).  Each term is isolated by zeroing the other rate
constants and compared with a closed-form solution, so a dropped term, a wrong
sign, a wrong site type or a swapped product fails at least one test."""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp

import oracle as O
import synthetic as S

ALL_RATES = ("kadh", "kcohPmax", "k_adp", "k_e2",
             "kC0p", "kC0m", "kC0cat", "kC1p", "kC1m", "kC1cat", "kC2p", "kC2m", "kC2cat",
             "kS1p", "kS1m", "kE1p", "kE1m", "kS2p", "kS2m", "kE2p", "kE2m")


def R4(z):
    """Amplification factor of classic RK4 on y' = lambda y, z = lambda h."""
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def only(**on):
    """Default parameters with every rate constant zero except those given."""
    p = S.params_default()
    for k in ALL_RATES:
        p[k] = 0.0
    for k, v in on.items():
        p[k] = S.params_default()[k] if v is True else v
    return p


def y0(**vals):
    y = np.zeros(15)
    for k, v in vals.items():
        y[S.IDX[k]] = v
    return y


def logistic(k, a, b, t):
    """x(t) of dx/dt = k (a - x)(b - x), x(0) = 0, a != b."""
    u = (b / a) * np.exp(k * (b - a) * t)
    return (b - a * u) / (1 - u)


# ------------------------------------------------------------ invariants

def test_rk4_conserves_linear_invariants():
    p = S.params_default()
    c, eta = S.random_reaction_states(300, p, seed=11)
    aV, Dd = 1 / 1.5e-3, p["D_chem"] / 0.75e-3
    for q in range(c.shape[1]):
        y = c[:, q].copy()
        H = float(q % 2)
        wall = (q % 3 == 0)
        g = O.g(p, eta[q])
        e0, c0 = (1.2e-7, 3e-8) if wall else (0.0, 0.0)
        y1, e1, c1 = O.rk4_cell(p, y, 2e-5, nsub=4, H=H, g=g, wall=wall, e0=e0, c0=c0, aV=aV, Dd=Dd)
        I = S.IDX
        plt = lambda v: v[I["Pmu"]] + v[I["Pma"]] + v[I["Pba"]] + v[I["Pbse"]]
        f1 = lambda v, cc: (v[I["S1"]] + v[I["E1"]] + v[I["S1b"]] + v[I["E1b"]] + v[I["C1"]]
                            + v[I["C2"]] + aV * cc)
        f2 = lambda v: v[I["S2"]] + v[I["E2"]] + v[I["S2b"]] + v[I["E2b"]] + v[I["C1"]] + v[I["C2"]]
        assert plt(y1) == pytest.approx(plt(y), rel=1e-14)
        assert f1(y1, c1) == pytest.approx(f1(y, c0), rel=1e-13)
        assert f2(y1) == pytest.approx(f2(y), rel=1e-13)
        if wall:
            assert e1 + c1 == pytest.approx(e0 + c0, rel=1e-14)
        assert y1[I["ADP"]] == y[I["ADP"]]


# ------------------------------------------------------------ App. A

@pytest.mark.parametrize("adp_mult,e2_mult,rate", [
    (1.0, 0.0, 0.34 / 2),          # [ADP] = ADP*: A1 = k_adp / 2
    (0.0, 1.0, 0.5 / 2),           # E2 = e2*: A2 = k_e2 / 2
    (1.0, 1.0, (0.34 + 0.5) / 2),  # both add
    (1e9, 0.0, 0.34),              # saturation: A1 -> k_adp
])
def test_activation_is_hill_and_linear_in_pmu(adp_mult, e2_mult, rate):
    p = only(k_adp=True, k_e2=True)
    y = y0(Pmu=2e5, ADP=adp_mult * p["adp_star"], E2=e2_mult * p["e2_star"])
    h, n = 0.05, 20
    y1, _, _ = O.rk4_cell(p, y, h, nsub=n)
    assert y1[S.IDX["Pmu"]] == pytest.approx(2e5 * R4(-rate * h) ** n, rel=1e-9 if adp_mult > 1e3 else 1e-14)
    assert y1[S.IDX["Pma"]] == pytest.approx(2e5 - y1[S.IDX["Pmu"]], rel=1e-13)
    assert y1[S.IDX["E2"]] == y[S.IDX["E2"]]


def test_cohesion_converts_pma_to_pba_at_kcoh_g_pmax():
    p = only(kcohPmax=True)
    g = O.g(p, 1.0)
    assert g == pytest.approx(1.0, abs=1e-15)
    y = y0(Pma=1e5)
    h, n = 1e-5, 30
    y1, _, _ = O.rk4_cell(p, y, h, nsub=n, g=g)
    assert y1[S.IDX["Pma"]] == pytest.approx(1e5 * R4(-1e4 * h) ** n, rel=1e-13)
    assert y1[S.IDX["Pba"]] == pytest.approx(1e5 - y1[S.IDX["Pma"]], rel=1e-13)


@pytest.mark.parametrize("who", ["Pmu", "Pma", "Pba"])
def test_adhesion_is_logistic_towards_pmax(who):
    """dPbse/dt = kadh (Pmax - Pbse)(Pmu + Pma + Pba), the sum being T - Pbse:
    x(t) of dx/dt = kadh (Pmax - x)(T - x)."""
    p = only(kadh=True)
    T = 3e6
    y = y0(**{who: T})
    h, n = 2e-3, 500
    y1, _, _ = O.rk4_cell(p, y, h, nsub=n, H=1.0)
    x = logistic(p["kadh"], p["Pmax"], T, h * n)
    assert y1[S.IDX["Pbse"]] == pytest.approx(x, rel=1e-11)
    assert y1[S.IDX[who]] == pytest.approx(T - x, rel=1e-11)
    # no adhesion outside the adhesion region
    y2, _, _ = O.rk4_cell(p, y, h, nsub=3, H=0.0)
    assert np.array_equal(y2, y)


def test_binding_affinity_and_hindrance_special_values():
    p = S.params_default()
    assert O.g(p, 1.0) == pytest.approx(1.0, abs=1e-15)      # g(1) = 1 (App. A)
    assert O.g(p, p["eta_t"]) == 0.0 and O.g(p, 0.05) == 0.0  # no binding below threshold
    ginf = O.g(p, 1e5)
    assert O.g(p, p["eta_t"] + p["eta_star"]) == pytest.approx(ginf / 2, rel=1e-9)
    ys = [O.g(p, e) for e in np.linspace(0.1, 1.0, 50)]
    assert all(b >= a for a, b in zip(ys, ys[1:]))
    assert O.W(0.0) == pytest.approx(math.tanh(math.pi), rel=1e-15)
    assert O.W(1.0) == 0.0 and O.W(2.0) == 0.0 and O.W(-1.0) == O.W(0.0)
    assert O.W(0.5) == pytest.approx(math.tanh(math.pi / 2), rel=1e-15)


# ------------------------------------------------------------ App. B

def test_unbinding_returns_each_bound_species_to_its_fluid_partner():
    p = only(kS1m=True, kE1m=True, kS2m=True, kE2m=True)
    y = y0(S1b=1e-6, E1b=2e-7, S2b=3e-6, E2b=4e-8)
    h, n = 0.01, 40
    y1, _, _ = O.rk4_cell(p, y, h, nsub=n)
    for b, f, k in (("S1b", "S1", "kS1m"), ("E1b", "E1", "kE1m"),
                    ("S2b", "S2", "kS2m"), ("E2b", "E2", "kE2m")):
        exp_b = y[S.IDX[b]] * R4(-p[k] * h) ** n
        assert y1[S.IDX[b]] == pytest.approx(exp_b, rel=1e-13), b
        assert y1[S.IDX[f]] == pytest.approx(y[S.IDX[b]] - exp_b, rel=1e-12), f


@pytest.mark.parametrize("fluid,bound,kp,family,others", [
    ("S1", "S1b", "kS1p", 1, ("E1b",)),
    ("E1", "E1b", "kE1p", 1, ("S1b",)),
    ("S2", "S2b", "kS2p", 2, ("E2b",)),
    ("E2", "E2b", "kE2p", 2, ("S2b",)),
])
def test_binding_consumes_free_sites_of_its_type(fluid, bound, kp, family, others):
    """Fluid species + free site -> bound species (k+ only).  Free sites of type
    i are N_i/N_A (Pba + Pbse) minus the occupied sites of that type, which
    include the other bound species of the type and both complexes C1, C2."""
    p = only(**{kp: True})
    P = 2e7
    N = p["N1"] if family == 1 else p["N2"]
    cap = N / p["N_A"] * P
    occ = {others[0]: 0.10 * cap, "C1": 0.05 * cap, "C2": 0.07 * cap}
    # type-2 (or type-1) species that must NOT count as occupying this type
    wrong = {"S2b": 0.2 * cap, "E2b": 0.1 * cap} if family == 1 else {"S1b": 0.2 * cap, "E1b": 0.1 * cap}
    s0 = 1.3 * cap
    y = y0(Pbse=0.6 * P, Pba=0.4 * P, **{fluid: s0}, **occ, **wrong)
    h, n = 2e-4, 1000
    y1, _, _ = O.rk4_cell(p, y, h, nsub=n)
    B = cap - sum(occ.values())
    x = logistic(p[kp], s0, B, h * n)
    assert y1[S.IDX[bound]] == pytest.approx(y[S.IDX[bound]] + x, rel=1e-9)
    assert y1[S.IDX[fluid]] == pytest.approx(s0 - x, rel=1e-9)


@pytest.mark.parametrize("cplx,km,kcat,sub,enz,prod", [
    ("C1", "kC1m", "kC1cat", "S2b", "E1b", "E2b"),   # S2b + E1b <-> C1 -> E1b + E2b
    ("C2", "kC2m", "kC2cat", "S1b", "E2b", "E1b"),   # S1b + E2b <-> C2 -> E2b + E1b
])
def test_complex_decay_branches_into_unbinding_and_catalysis(cplx, km, kcat, sub, enz, prod):
    p = only(**{km: True, kcat: True})
    y = y0(**{cplx: 5e-8})
    h, n = 0.002, 200
    y1, _, _ = O.rk4_cell(p, y, h, nsub=n)
    lam = p[km] + p[kcat]
    C = 5e-8 * R4(-lam * h) ** n
    d = 5e-8 - C
    assert y1[S.IDX[cplx]] == pytest.approx(C, rel=1e-13)
    assert y1[S.IDX[enz]] == pytest.approx(d, rel=1e-12)             # enzyme always returned
    assert y1[S.IDX[sub]] == pytest.approx(d * p[km] / lam, rel=1e-12)  # unbinding
    assert y1[S.IDX[prod]] == pytest.approx(d * p[kcat] / lam, rel=1e-12)  # product


@pytest.mark.parametrize("cplx,kp,a,b", [("C1", "kC1p", "S2b", "E1b"), ("C2", "kC2p", "S1b", "E2b")])
def test_complex_formation_is_bimolecular(cplx, kp, a, b):
    p = only(**{kp: True})
    A0, B0 = 2e-5, 7e-6
    y = y0(**{a: A0, b: B0})
    h, n = 1e-4, 1000
    y1, _, _ = O.rk4_cell(p, y, h, nsub=n)
    x = logistic(p[kp], A0, B0, h * n)
    assert y1[S.IDX[cplx]] == pytest.approx(x, rel=1e-9)
    assert y1[S.IDX[a]] == pytest.approx(A0 - x, rel=1e-9)
    assert y1[S.IDX[b]] == pytest.approx(B0 - x, rel=1e-9)


# ------------------------------------------------------- injury wall

def test_wall_complex_release_feeds_S1_and_E1_through_A_over_V():
    p = only(kC0m=True, kC0cat=True)
    aV, Dd = 1 / 1.5e-3, 5e-5 / 0.75e-3
    y = y0(S1=1e-4)
    h, n = 0.01, 100
    y1, e1, c1 = O.rk4_cell(p, y, h, nsub=n, wall=True, e0=1e-7, c0=5e-8, aV=aV, Dd=Dd)
    lam = p["kC0m"] + p["kC0cat"]
    C = 5e-8 * R4(-lam * h) ** n
    d = 5e-8 - C
    assert c1 == pytest.approx(C, rel=1e-13)
    assert e1 == pytest.approx(1e-7 + d, rel=1e-13)
    assert y1[S.IDX["S1"]] == pytest.approx(1e-4 + aV * d * p["kC0m"] / lam, rel=1e-12)
    assert y1[S.IDX["E1"]] == pytest.approx(aV * d * p["kC0cat"] / lam, rel=1e-12)


def test_wall_binding_bimolecular_in_the_well_mixed_limit():
    """With D/delta -> infinity the wall value equals the cell value and
    S1 + E0 -> C0 obeys dC0/dt = k+ (S1_0 - (A/V) C0)(E0_0 - C0)."""
    p = only(kC0p=True)
    aV = 1 / 1.5e-3
    S10, E00 = 1.7e-4, 1.5e-7
    y = y0(S1=S10)
    h, n = 2e-3, 1000
    y1, e1, c1 = O.rk4_cell(p, y, h, nsub=n, wall=True, e0=E00, c0=0.0, aV=aV, Dd=1e15)
    x = logistic(p["kC0p"] * aV, S10 / aV, E00, h * n)
    assert c1 == pytest.approx(x, rel=1e-9)
    assert e1 == pytest.approx(E00 - x, rel=1e-9)
    assert y1[S.IDX["S1"]] == pytest.approx(S10 - aV * x, rel=1e-9)


def test_robin_wall_value_gives_flux_continuity():
    """The wall value S1_w satisfies D (S1 - S1_w)/delta = J = k+ S1_w E0 - k- C0:
    the S1 the cell loses equals the diffusive flux to the wall, S1_w < S1
    when the wall consumes S1."""
    p = S.params_default()
    aV, Dd = 1 / 1.5e-3, p["D_chem"] / 0.75e-3
    rng = np.random.default_rng(2)
    for _ in range(20):
        y = y0(S1=rng.uniform(1e-5, 2e-4))
        e0, c0 = rng.uniform(1e-8, 1.5e-7), rng.uniform(0, 5e-8)
        fw, fe0, fc0 = O.rhs(p, y, wall=True, e0=e0, c0=c0, aV=aV, Dd=Dd)
        fn, _, _ = O.rhs(p, y)
        lam = p["kC0m"] + p["kC0cat"]
        s1w = (fc0 + lam * c0) / (p["kC0p"] * e0)
        J = -(fw[S.IDX["S1"]] - fn[S.IDX["S1"]]) / aV
        assert Dd * (y[S.IDX["S1"]] - s1w) == pytest.approx(J, rel=1e-10)
        assert fw[S.IDX["E1"]] - fn[S.IDX["E1"]] == pytest.approx(aV * p["kC0cat"] * c0, rel=1e-14)
        assert fe0 + fc0 == pytest.approx(0.0, abs=1e-25)
        if J > 0:
            assert s1w < y[S.IDX["S1"]]


# ------------------------------------------------------- integrator order

def test_rk4_is_fourth_order_against_radau():
    """Single-cell trajectories of the full coupled system (platelets, all 12
    coagulation species, injury wall) converge at fourth order to a
    tight-tolerance implicit Radau solution."""
    p = S.params_default()
    aV, Dd = 1 / 1.5e-3, p["D_chem"] / 0.75e-3
    c, eta = S.random_reaction_states(4, p, seed=5)
    for q in range(3):
        y = c[:, q].copy()
        y[S.IDX["Pbse"]] = 0.3 * p["Pmax"]
        y[S.IDX["Pba"]] = 0.3 * p["Pmax"]
        g, e0, c0 = 0.05, 1.2e-7, 2e-8
        scale = np.maximum(np.abs(np.append(y, [e0, c0])), 1e-12)

        def f(t, z):
            v = z * scale
            fy, fe, fc = O.rhs(p, v[:15], H=1.0, g=g, wall=True, e0=v[15], c0=v[16], aV=aV, Dd=Dd)
            return np.append(fy, [fe, fc]) / scale

        T = 4e-3
        ref = solve_ivp(f, (0, T), np.ones(17), method="Radau", rtol=1e-12, atol=1e-13).y[:, -1] * scale
        errs = []
        for n in (20, 40):
            y1, e1, c1 = O.rk4_cell(p, y, T / n, nsub=n, H=1.0, g=g, wall=True, e0=e0, c0=c0, aV=aV, Dd=Dd)
            errs.append(np.max(np.abs(np.append(y1, [e1, c1]) - ref) / scale))
        assert errs[1] < 1e-7
        assert errs[0] / errs[1] > 11.0, errs

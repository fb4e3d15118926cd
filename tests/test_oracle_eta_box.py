"""Pins of the two facts behind the GPU's box correction of a rejected eta
prediction (App. A, Eq. eta: (I - (L_eta^2/4) lap_h) eta = theta_B, zero-flux
walls):

* along an axis the discrete Green's function of I - c lap_h decays by
  exp(-mu) per cell, cosh(mu) = 1 + 1/(2c);
* a correction computed on the box around the cells with |r| > stop/(2(1+c)),
  widened by ln(2 c max|r| / stop)/mu cells per axis and zero outside, leaves a
  residual within the stopping rule everywhere (the box rule), while the same
  box around |r| > stop/2 does not in the worst case.

The correction is solved to 1e-14 here (CG in FP64), so what is checked is
the cut-off at the box edge, not the iteration."""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
import synthetic as S

H = 1.5e-3  # cell size (mm) of the duct and channel workloads


def _desc(dim, nx, ny, nz, h=H):
    return dict(dim=dim, nx=nx, ny=ny, nz=nz, hx=h, hy=h, hz=h if dim == 3 else 1.0, inj_x0=-1, inj_x1=-1,
                inj_z0=-1, inj_z1=-1, p_diam=0.0)


def _coupling(p, h=H):
    return p["L_eta"] ** 2 / 4 / h ** 2


def test_green_function_decays_by_exp_minus_mu_per_cell():
    """A point source on a line of cells: eta_i = A q^|i| with q the root of
    c q^2 - (1 + 2c) q + c = 0 below 1, i.e. q = exp(-mu), cosh(mu) = 1 + 1/(2c)."""
    p = S.params_default()
    n = 401
    th = np.zeros(n)
    th[n // 2] = 1.0
    eta, _ = O.eta_solve(_desc(2, n, 1, 1), p, th, tol=1e-15)
    c = _coupling(p)
    q = math.exp(-math.acosh(1.0 + 0.5 / c))
    i0 = n // 2
    ratios = eta[i0 + 1:i0 + 21] / eta[i0:i0 + 20]
    assert np.allclose(ratios, q, rtol=1e-7, atol=0.0), ratios
    assert np.allclose(eta[i0 - 20:i0][::-1], eta[i0 + 1:i0 + 21], rtol=1e-9, atol=0.0)
    assert abs(c - 4.0) < 1e-12 and abs(-math.log(q) - 0.4949) < 1e-4  # the workloads' c = L^2/4h^2 = 4


def _operator(nx, ny, nz, c):
    """I - c lap_h on an nx x ny x nz grid, zero-flux walls (missing neighbours
    contribute nothing), cell index i + nx (j + ny k)."""
    def lap1(n):
        main = -2.0 * np.ones(n)
        main[0] += 1.0
        main[-1] += 1.0
        return sp.diags([np.ones(n - 1), main, np.ones(n - 1)], [-1, 0, 1])
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    lap = sp.kron(Iz, sp.kron(Iy, lap1(nx))) + sp.kron(Iz, sp.kron(lap1(ny), Ix)) + sp.kron(lap1(nz), sp.kron(Iy, Ix))
    return (sp.identity(nx * ny * nz) - c * lap).tocsr()


def _box_correction(A, r, shape, c, stop, thr):
    """The box rule: bounding box of |r| > thr, widened per axis by
    ceil(ln(max(2 c max|r| / stop, 1)) / mu) + 1 cells, correction solved on the
    box with zero outside; returns the new residual r - A d on the whole grid."""
    nx, ny, nz = shape
    mu = math.acosh(1.0 + 0.5 / c)
    m = int(math.ceil(math.log(max(2.0 * c * np.max(np.abs(r)) / stop, 1.0)) / mu)) + 1
    k, j, i = np.unravel_index(np.nonzero(np.abs(r) > thr)[0], (nz, ny, nx))
    lo = [max(v.min() - m, 0) for v in (i, j, k)]
    hi = [min(v.max() + m, n - 1) for v, n in zip((i, j, k), shape)]
    K, J, I = np.meshgrid(np.arange(lo[2], hi[2] + 1), np.arange(lo[1], hi[1] + 1), np.arange(lo[0], hi[0] + 1),
                          indexing="ij")
    box = (I + nx * (J + ny * K)).ravel()
    d = np.zeros_like(r)
    x, info = spla.cg(A[box][:, box], r[box], rtol=1e-14, atol=0.0, maxiter=2000)
    assert info == 0
    d[box] = x
    return r - A @ d, box


def _residual(shape, pr, outside, seed):
    """Large residual (up to pr) on a 6 x 4 x 6 core near the floor; elsewhere
    the given field."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    r = outside.copy()
    core = np.zeros((nz, ny, nx), bool)
    core[20:26, 0:4, 28:34] = True
    r[core.ravel()] = pr * rng.uniform(-1.0, 1.0, core.sum())
    return r


def test_box_rule_keeps_the_residual_within_the_stopping_rule():
    p = S.params_default()
    c = _coupling(p)
    shape = (64, 32, 48)
    A = _operator(*shape, c)
    n = A.shape[0]
    stop = 1e-6
    thr = 0.5 * stop / (1.0 + c)
    rng = np.random.default_rng(11)
    for seed, pr in ((1, 1e-4), (2, 3e-5), (3, 1e-3)):
        # outside the core: random residuals up to thr, and the worst case, thr of one sign
        for outside in (rng.uniform(-thr, thr, n) * 0.999, np.full(n, 0.999 * thr)):
            r = _residual(shape, pr, outside, seed)
            r_new, box = _box_correction(A, r, shape, c, stop, thr)
            assert box.size < n
            assert np.max(np.abs(r_new)) <= stop, (seed, pr, np.max(np.abs(r_new)))


def test_box_around_half_the_rule_is_not_enough():
    """Without the 1 + c factor the cut-off correction of a one-signed residual
    just below stop/2 outside the core pushes the first cells outside the box
    over the rule: d at the box edge is about (1 - exp(-mu)) r, and the cell
    outside gets r + c d."""
    p = S.params_default()
    c = _coupling(p)
    shape = (64, 32, 48)
    A = _operator(*shape, c)
    stop = 1e-6
    r = _residual(shape, 1e-4, np.full(A.shape[0], 0.999 * 0.5 * stop), 1)
    r_new, _ = _box_correction(A, r, shape, c, stop, 0.5 * stop)
    q = math.exp(-math.acosh(1.0 + 0.5 / c))
    assert np.max(np.abs(r_new)) > stop
    assert np.max(np.abs(r_new)) <= 0.5 * stop * (1.0 + c * (1.0 - q)) * 1.01

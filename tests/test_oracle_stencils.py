"""Pins for the oracle's discretisation steps (paper Sec. 2): kNN stencils, tangent plane, PHS
RBF-FD weights, GFD weights and global assembly. Each pin is fixed by something other than the
oracle itself: a library routine (scipy cKDTree, scipy RBFInterpolator), exact polynomial
reproduction, the spectrum of the LBO on the unit sphere, or an algebraic characterisation."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from paper_2204_06154_gb300 import inputs as I


def _rand_cloud(N, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((N, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x


def test_knn_matches_kdtree(oracle):
    x = _rand_cloud(3000, 1)
    q = x[:500]
    k = 30
    idx, d2 = oracle.knn(x, q, k, self_first=False, return_d2=True)
    dd, ii = cKDTree(x).query(q, k=k)
    np.testing.assert_allclose(np.sqrt(d2), dd, rtol=0, atol=1e-14)
    # random cloud: no ties, so the index lists must be identical
    assert np.array_equal(idx, ii.astype(np.int32))
    # sorted ascending by (d2, index)
    assert np.all(np.diff(d2, axis=1) >= 0)


def test_knn_self_first_and_ties(oracle):
    # icosahedral nodes have many exactly equal distances: ties are broken by smaller index
    x, _ = I.icosahedral_sphere(2)
    idx, d2 = oracle.knn(x, x, 7, self_first=True, return_d2=True)
    assert np.array_equal(idx[:, 0], np.arange(x.shape[0]))
    for i in range(x.shape[0]):
        # brute force: all candidates sorted by (d2, index), self first
        dx = x - x[i]
        d = (dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1]) + dx[:, 2] * dx[:, 2]
        d[i] = -1.0
        order = np.lexsort((np.arange(len(d)), d))[:7]
        assert np.array_equal(idx[i], order.astype(np.int32))


def test_tangent_basis_orthonormal(oracle):
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        t1, t2 = oracle.tangent_basis(n)
        M = np.stack([t1, t2, n])
        np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-14)
    # axis-aligned normal: t1 uses the first axis with the smallest |n_a|
    t1, t2 = oracle.tangent_basis(np.array([0.0, 0.0, 1.0]))
    np.testing.assert_allclose(t1, [1, 0, 0], atol=0)
    np.testing.assert_allclose(t2, [0, 1, 0], atol=0)


def _plane_stencils(N, n, seed):
    """Scattered points on the plane z = 0 with normal e_z: the LBO is the plane Laplacian."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-1, 1, size=(N, 2))
    x = np.concatenate([xy, np.zeros((N, 1))], axis=1)
    nrm = np.tile([0.0, 0.0, 1.0], (N, 1))
    return x, nrm


@pytest.mark.parametrize("k,ell,n", [(1, 2, 30), (1, 3, 50), (3, 3, 20), (2, 4, 40)])
def test_phs_polynomial_reproduction(oracle, k, ell, n):
    """Sec. 2.2, eq. (rbf_fd_lap): the constraint rows force sum_j c_j p(x_j) = Lap p(x_c) for
    every polynomial of degree <= ell (here in the plane, where the LBO is the Laplacian)."""
    x, nrm = _plane_stencils(400, n, 7)
    idx = oracle.knn(x, x, n, self_first=True)
    w = oracle.phs_weights(x, nrm, idx, k, ell)
    rng = np.random.default_rng(1)
    for i in range(0, 400, 37):
        nb = x[idx[i]]
        c = x[i]
        for a in range(ell + 1):
            for b in range(ell + 1 - a):
                # shifted monomial (x - cx)^a (y - cy)^b: Laplacian at the centre is 2 for (2,0), (0,2)
                vals = (nb[:, 0] - c[0]) ** a * (nb[:, 1] - c[1]) ** b
                expect = 2.0 if (a, b) in ((2, 0), (0, 2)) else 0.0
                got = w[i] @ vals
                scale = np.abs(w[i]) @ np.abs(vals) + 1.0
                assert abs(got - expect) <= 1e-9 * scale, (i, a, b, got, expect)
        # a generic degree-ell polynomial with random coefficients
        coef = rng.standard_normal((ell + 1, ell + 1))
        vals = sum(coef[a, b] * nb[:, 0] ** a * nb[:, 1] ** b for a in range(ell + 1) for b in range(ell + 1 - a))
        lap = sum(coef[a, b] * (a * (a - 1) * c[0] ** max(a - 2, 0) * c[1] ** b if a >= 2 else 0.0)
                  + coef[a, b] * (b * (b - 1) * c[0] ** a * c[1] ** max(b - 2, 0) if b >= 2 else 0.0)
                  for a in range(ell + 1) for b in range(ell + 1 - a))
        assert abs(w[i] @ vals - lap) <= 1e-8 * (np.abs(w[i]).sum() + 1)


def test_phs_matches_scipy_rbf_interpolant(oracle):
    """The weights apply the 2-D Laplacian at the centre to the PHS + polynomial interpolant of
    the data (Sec. 2.2). scipy's RBFInterpolator builds the same interpolant (kernel 'cubic' =
    r^3, degree ell) with its own solver; its Laplacian at the centre is taken by a centred
    finite difference, which is exact for the polynomial part and O(h) for r^3 terms."""
    from scipy.interpolate import RBFInterpolator
    x, nrm = _plane_stencils(300, 30, 3)
    idx = oracle.knn(x, x, 30, self_first=True)
    w = oracle.phs_weights(x, nrm, idx, 1, 2)
    rng = np.random.default_rng(5)
    for i in (0, 11, 123):
        nb = x[idx[i], :2]
        u = np.sin(2 * nb[:, 0]) * np.cos(3 * nb[:, 1]) + rng.standard_normal(30) * 0.01
        s = RBFInterpolator(nb, u, kernel="cubic", degree=2)
        c = x[i, :2]

        def fd(h):
            pts = np.array([c, c + [h, 0], c - [h, 0], c + [0, h], c - [0, h]])
            v = s(pts)
            return (v[1] + v[2] + v[3] + v[4] - 4 * v[0]) / h ** 2
        # the r^3 term centred on the node makes the error linear in h: Richardson-extrapolate
        lap_fd = 2.0 * fd(1e-4) - fd(2e-4)
        got = w[i] @ u
        assert abs(got - lap_fd) <= 2e-5 * max(1.0, abs(got)), (got, lap_fd)


def test_phs_rotation_invariance(oracle):
    """Weights depend only on the geometry: rotating the cloud and normals rigidly leaves them
    unchanged (the tangent basis rotates within T_x M, to which the method is invariant)."""
    x = _rand_cloud(1500, 2)
    nrm = x.copy()
    idx = oracle.knn(x, x, 30, self_first=True)
    w = oracle.phs_weights(x, nrm, idx, 1, 2)
    q, _ = np.linalg.qr(np.random.default_rng(9).standard_normal((3, 3)))
    xr = x @ q.T
    idxr = oracle.knn(xr, xr, 30, self_first=True)
    assert np.array_equal(idx, idxr)
    wr = oracle.phs_weights(xr, xr.copy(), idxr, 1, 2)
    err = np.max(np.abs(w - wr), axis=1) / np.max(np.abs(w), axis=1)
    assert err.max() < 1e-9


def test_sphere_lbo_spectrum_converges(oracle):
    """On the unit sphere Lap_S Y_4^3 = -20 Y_4^3 (closed-form harmonic polynomial z(x^3-3xy^2)).
    The discrete D must approach this with order about ell - 1 or better (Sec. 5) as the
    icosahedral level grows (config: r^3, ell = 2, n = 30)."""
    errs = []
    for q in (3, 4, 5):
        x, nrm = I.icosahedral_sphere(q)
        idx, w, L = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, 1.0)
        y = I.y43(x)
        Dy = y - L @ y
        errs.append(np.linalg.norm(Dy + 20 * y) / np.linalg.norm(20 * y))
    assert errs[0] > errs[1] > errs[2]
    rate = math.log(errs[0] / errs[2]) / math.log(4.0)   # h halves per level: h^2 ratio 4 per level
    assert rate > 0.9, errs


def test_gfd_reproduction_and_wls_characterisation(oracle):
    """Sec. 2.3: c = W P (P^T W P)^{-1} Lap p is the unique vector with (i) P^T c = Lap p(0)
    (exactness on polynomials of degree <= ell) and (ii) W^{-1} c in range(P)."""
    x, nrm = _plane_stencils(300, 25, 4)
    n, ell, alpha = 25, 2, 4.0
    idx = oracle.knn(x, x, n, self_first=True)
    w = oracle.gfd_weights(x, nrm, idx, ell, alpha)
    # support radii (in the plane the tangent coordinates are the xy offsets)
    rho = np.array([np.max(np.linalg.norm(x[idx[i], :2] - x[i, :2], axis=1)) for i in range(300)])
    for i in (0, 17, 250):
        d = x[idx[i], :2] - x[i, :2]
        P = np.stack([d[:, 0] ** a * d[:, 1] ** (deg - a) for deg in range(ell + 1) for a in range(deg, -1, -1)], 1)
        lap = np.array([2.0 if (a, deg - a) in ((2, 0), (0, 2)) else 0.0 for deg in range(ell + 1) for a in range(deg, -1, -1)])
        np.testing.assert_allclose(P.T @ w[i], lap, atol=1e-9 * np.abs(w[i]).sum())
        Wd = np.exp(-alpha * np.sum(d * d, 1) / (rho[i] ** 2 + rho[idx[i]] ** 2))
        y = w[i] / Wd
        coef, *_ = np.linalg.lstsq(P, y, rcond=None)
        assert np.linalg.norm(P @ coef - y) <= 1e-8 * np.linalg.norm(y)


def test_assembly_constant_reproduction(oracle):
    """D 1 = 0 (constants are reproduced, Lap 1 = 0), so L 1 = 1 for L = I - mu D; the diagonal is
    present in every row and columns are ascending (Sec. 2, eq. (discrete_system))."""
    x, nrm = I.fibonacci_sphere(2000, jitter=0.1, seed=1)
    idx, w, L = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, 0.7)
    ones = np.ones(x.shape[0])
    res = L @ ones - ones
    scale = 0.7 * np.abs(w).sum(axis=1)
    assert np.all(np.abs(res) <= 1e-11 * scale)
    for i in range(0, 2000, 97):
        cols = L.indices[L.indptr[i]:L.indptr[i + 1]]
        assert np.all(np.diff(cols) > 0) and i in cols
    _, _, Dm = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, poisson=True)
    assert np.all(np.abs(Dm @ ones) <= 1e-11 * np.abs(w).sum(axis=1))


def test_singular_stencil_reported(oracle):
    """Collinear stencil nodes are not unisolvent for degree >= 1 (Sec. 2.2): error, row named."""
    x = np.zeros((40, 3))
    x[:, 0] = np.linspace(0, 1, 40)
    nrm = np.tile([0.0, 0.0, 1.0], (40, 1))
    idx = oracle.knn(x, x, 20, self_first=True)
    with pytest.raises(oracle.OracleError) as e:
        oracle.phs_weights(x, nrm, idx, 1, 2)
    assert e.value.status == 2 and e.value.row == 0


def test_weights_of_a_row_subset(oracle):
    """The row-subset entry returns the same rows as the full computation, and rejects a stencil
    table that does not hold one row per centre."""
    x, nrm = I.fibonacci_sphere(1500, jitter=0.1, seed=4)
    idx = oracle.knn(x, x, 30, self_first=True)
    w = oracle.phs_weights(x, nrm, idx, 1, 2)
    rows = np.array([1499, 0, 17, 17, 800], np.int32)
    assert np.array_equal(oracle.phs_weights(x, nrm, idx[rows], 1, 2, rows=rows), w[rows])
    with pytest.raises(ValueError):
        oracle.phs_weights(x, nrm, idx[:100], 1, 2)
    with pytest.raises(ValueError):
        oracle.phs_weights(x, nrm, idx, 1, 2, rows=rows)
    with pytest.raises(oracle.OracleError):
        oracle.phs_weights(x, nrm, idx[:1], 1, 2, rows=np.array([1500], np.int32))

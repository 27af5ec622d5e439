"""Pins for the oracle's surface Poisson solver with the mean-zero constraint (Sec. 4.4): the
bordered system of eq. (saddle_point), the bordered Galerkin operators of eq. (gco_saddle_point),
the u-only smoother and the bordered coarse solve. Checked against a dense solve of the bordered
system, a dense two-level cycle written from the equations, and the Y_5^4 test problem of Sec. 5.4
(exact solution known), whose error must fall with refinement."""
import numpy as np
import pytest

from paper_2204_06154_gb300 import inputs as I


def _poisson(oracle, q, n=30, ell=2):
    x, nrm = I.icosahedral_sphere(q)
    idx, w, L = oracle.build_operator(x, nrm, n, "rbf", 1, ell, 1.0, poisson=True)
    return x, L


def _bordered_dense(L):
    N = L.shape[0]
    B = np.zeros((N + 1, N + 1))
    B[:N, :N] = L.toarray()
    B[:N, N] = 1.0
    B[N, :N] = 1.0
    return B


def test_bordered_fgmres_matches_dense_solve(oracle):
    x, L = _poisson(oracle, 3)
    N = L.shape[0]
    H = oracle.setup(x, L, 40, bordered=True)
    assert H.p >= 2
    f = np.random.default_rng(2).standard_normal(N)
    u, lam, it, rel = oracle.fgmres_bordered(L, H, f, tol=1e-12)
    ref = np.linalg.solve(_bordered_dense(L), np.concatenate([f, [0.0]]))
    assert rel <= 1e-12
    assert np.linalg.norm(u - ref[:N]) <= 1e-9 * np.linalg.norm(ref[:N])
    assert abs(lam - ref[N]) <= 1e-9 * max(1.0, abs(ref[N]))
    assert abs(u.sum()) <= 1e-10 * np.abs(u).sum()          # the constraint


def test_bordered_two_level_cycle_dense(oracle):
    """One bordered V-cycle with p = 2 equals the cycle written with dense matrices:
    e1 = B^-1 r; t = r - L e1, s1 = s - 1.e1; [eH; mu] = Lt_H^-1 [R t; s1] with
    Lt_H = [R L P, R 1; (R 1)^T, 0]; e2 = e1 + P eH; e3 = e2 + B^-1 (r - L e2 - 1 mu)."""
    x, L = _poisson(oracle, 3)
    N = L.shape[0]
    H = oracle.setup(x, L, N // 4, seed=4, bordered=True)
    assert H.p == 2
    rng = np.random.default_rng(5)
    r, s = rng.standard_normal(N), 0.7
    e, mu = oracle.vcycle_bordered(H, r, s)
    perm = H.perm[0]
    A = H.L[0].toarray()
    q = np.argsort(H.colors[0], kind="stable")
    B = np.zeros_like(A)
    B[np.ix_(q, q)] = np.tril(A[np.ix_(q, q)])
    P = H.P[0].toarray(); R = P.T
    one = np.ones(N)
    c1 = R @ one
    LH = np.zeros((P.shape[1] + 1, P.shape[1] + 1))
    LH[:-1, :-1] = R @ A @ P
    LH[:-1, -1] = c1
    LH[-1, :-1] = c1
    rp = r[perm]
    e1 = np.linalg.solve(B, rp)
    t = rp - A @ e1
    s1 = s - one @ e1
    sol = np.linalg.solve(LH, np.concatenate([R @ t, [s1]]))
    e2 = e1 + P @ sol[:-1]
    mu_ref = sol[-1]
    e3 = e2 + np.linalg.solve(B, rp - A @ e2 - one * mu_ref)
    ref = np.empty(N); ref[perm] = e3
    assert np.linalg.norm(e - ref) <= 1e-11 * np.linalg.norm(ref)
    assert abs(mu - mu_ref) <= 1e-11 * max(1.0, abs(mu_ref))


def test_border_vectors_are_restricted_ones(oracle):
    """c_0 = 1 and c_{j+1} = R_j c_j: every c_j has the sum of the finest level's ones, since the
    interpolation rows reproduce constants (rows of P sum to 1)."""
    x, L = _poisson(oracle, 4)
    H = oracle.setup(x, L, 40, bordered=True)
    assert H.p >= 3
    for j in range(H.p):
        assert abs(H.cvec[j].sum() - L.shape[0]) <= 1e-9 * L.shape[0]
    assert np.allclose(np.asarray(H.P[0].sum(axis=1)).ravel(), 1.0, atol=1e-13)


def test_poisson_y54_error_falls_with_refinement(oracle):
    """Sec. 5.4's test problem: Lap_S u = f with u = Y_5^4 = z(x^4 - 6x^2y^2 + y^4) (up to the
    normalisation), f = -30 u on the unit sphere. The constrained solution has zero mean, and its
    error against the mean-free exact solution falls by at least 3x per icosahedral refinement
    (degree-2 polynomials)."""
    errs = []
    for q in (3, 4, 5):
        x, L = _poisson(oracle, q)
        H = oracle.setup(x, L, 250 if q > 3 else 40, bordered=True)
        Y = I.y54(x)
        u, lam, it, rel = oracle.fgmres_bordered(L, H, -30.0 * Y, tol=1e-12)
        assert rel <= 1e-12 and it <= 30
        assert abs(u.mean()) <= 1e-12 * np.abs(u).max()
        errs.append(np.linalg.norm(u - (Y - Y.mean())) / np.linalg.norm(Y))
    assert errs[0] > 3 * errs[1] > 9 * errs[2], errs

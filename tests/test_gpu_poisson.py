"""GPU parity of the surface Poisson solver with the mean-zero constraint (Sec. 4.4): the
bordered V-cycle and the bordered FGMRES against the oracle on the same operator, the Y_5^4
problem of Sec. 5.4 against its exact solution, and the argument checks. FP64 cycle within 1e-12
of the oracle's, FP32 within 1e-4; solutions within 1e-8 at a 1e-12 residual."""
import numpy as np
import pytest
import torch

from paper_2204_06154_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def M():
    from paper_2204_06154_gb300 import mgm
    mgm.lib()
    return mgm


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def H(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def poisson5(M, oracle):
    x, nrm = I.icosahedral_sphere(5)
    idx, w, L = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, 1.0, poisson=True)
    Lt = (T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), T(L.data))
    Hg = {prec: M.Hierarchy(T(x), *Lt, n_min=250, precision=prec, constraint=True) for prec in ("f64", "f32")}
    Ho = oracle.setup(x, L, 250, seed=0, bordered=True)
    return x, L, Hg, Ho


def test_bordered_vcycle_matches_oracle(poisson5, oracle):
    x, L, Hg, Ho = poisson5
    N = L.shape[0]
    rng = np.random.default_rng(7)
    r, s = rng.standard_normal(N), 0.37
    e, mu = oracle.vcycle_bordered(Ho, r, s)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-4)):
        z = H(Hg[prec].vcycle(T(np.concatenate([r, [s]]))))
        assert np.linalg.norm(z[:N] - e) <= tol * np.linalg.norm(e), prec
        assert abs(z[N] - mu) <= tol * max(abs(mu), np.linalg.norm(e) / np.sqrt(N)), prec


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_bordered_solve_matches_oracle(poisson5, oracle, prec):
    x, L, Hg, Ho = poisson5
    N = L.shape[0]
    f = np.random.default_rng(8).standard_normal(N)
    uo, lamo, ito, relo = oracle.fgmres_bordered(L, Ho, f, tol=1e-12)
    u, info = Hg[prec].solve(T(f), tol=1e-12, maxit=100)
    assert info["converged"] and info["rel_res"] <= 1e-12
    assert np.linalg.norm(H(u) - uo) <= 1e-8 * np.linalg.norm(uo)
    assert abs(info["multiplier"] - lamo) <= 1e-8 * np.linalg.norm(f) / np.sqrt(N)
    assert abs(info["iters"] - ito) <= 2, (info["iters"], ito)
    assert abs(H(u).sum()) <= 1e-9 * np.abs(H(u)).sum()


def test_poisson_y54_solution(poisson5):
    """Lap_S u = -30 Y_5^4 on the unit sphere: the constrained solution is Y_5^4 minus its mean,
    to the discretisation error of degree-2 RBF-FD at N = 10,242 (0.6% in the oracle)."""
    x, L, Hg, Ho = poisson5
    Y = I.y54(x)
    u, info = Hg["f32"].solve(T(-30.0 * Y), tol=1e-10)
    assert info["converged"]
    err = np.linalg.norm(H(u) - (Y - Y.mean())) / np.linalg.norm(Y)
    assert err < 0.01, err


def test_constrained_hierarchy_argument_checks(poisson5, M):
    x, L, Hg, Ho = poisson5
    f = T(np.ones(L.shape[0]))
    with pytest.raises(M.MGMError):
        Hg["f64"].solve(f, krylov="bicgstab")
    with pytest.raises(M.MGMError):
        M.solve_multi(Hg["f64"], torch.ones((2, L.shape[0]), dtype=torch.float64, device=DEV))

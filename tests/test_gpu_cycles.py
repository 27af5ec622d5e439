"""W- and F-cycles on the GPU (Sec. 4.5) against the oracle's recursive cycles: one cycle in FP64
(1e-12) and FP32 (1e-4), and MGM-FGMRES with each (iterations +-1, solutions 1e-8)."""
import numpy as np
import pytest
import torch

from paper_2204_06154_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def M():
    from paper_2204_06154_gb300 import mgm
    mgm.lib()
    return mgm


@pytest.fixture(scope="module")
def prob(oracle):
    x, nrm = I.icosahedral_sphere(5)
    idx, w, L = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, 1.0)
    Ho = oracle.setup(x, L, 125, seed=0)
    csr = (T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), T(L.data))
    return x, L, Ho, csr


@pytest.mark.parametrize("cycle", ["W", "F"])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-4)])
def test_cycle_matches_oracle(M, oracle, prob, cycle, prec, tol):
    x, L, Ho, csr = prob
    Hg = M.Hierarchy(T(x), *csr, n_min=125, precision=prec, cycle=cycle)
    assert Hg.stats()["n"] == [l.shape[0] for l in Ho.L] and len(Ho.L) >= 3
    r = np.random.default_rng(31).standard_normal(x.shape[0])
    zo = oracle.mgcycle(Ho, r, cycle)
    z = Hg.vcycle(T(r)).cpu().numpy()
    assert np.linalg.norm(z - zo) <= tol * np.linalg.norm(zo)


@pytest.mark.parametrize("cycle", ["W", "F"])
def test_fgmres_with_cycle(M, oracle, prob, cycle):
    x, L, Ho, csr = prob
    f = np.random.default_rng(5).standard_normal(x.shape[0])
    uo, ito, _ = oracle.fgmres(L, Ho, f, tol=1e-12, cycle=cycle)
    Hg = M.Hierarchy(T(x), *csr, n_min=125, precision="f64", cycle=cycle)
    u, info = Hg.solve(T(f), tol=1e-12)
    assert info["converged"] and abs(info["iters"] - ito) <= 1, (info["iters"], ito)
    assert np.linalg.norm(u.cpu().numpy() - uo) <= 1e-8 * np.linalg.norm(uo)


def test_cycle_argument_checks(M, prob):
    x, L, Ho, csr = prob
    with pytest.raises(ValueError):
        M.Hierarchy(T(x), *csr, n_min=125, cycle="X")
    Hg = M.Hierarchy(T(x), *csr, n_min=125, cycle="W")
    with pytest.raises(M.MGMError):
        Hg.eigs(nev=4, block=4, steps=2)

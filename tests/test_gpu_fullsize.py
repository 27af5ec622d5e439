"""Parity at the full size of the timed workload: the 1,048,576-point jittered spherical-Fibonacci
sphere, PHS r^3 with degree-3 polynomials and n = 50 (Sec. 2.2), -Lap + I with a random
spherical-harmonic right-hand side (l <= 20), built and solved the way the benchmark times it
(FP32 LU + FP64 refinement for the weights, FP32 V-cycle, FP64 FGMRES to 1e-10).

The oracle computes sampled outputs one by one: kNN rows, stencil weights, operator rows. The rest
is checked by properties that hold at any size: the level sizes of Alg. 2, the Poisson-disk
separation of the first coarse level (Sec. 4.1), a proper multicolouring of the finest operator,
residuals recomputed on the host in FP64, and agreement with the all-FP64 GPU path."""
import numpy as np
import pytest
import torch

from paper_2204_06154_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N = 1 << 20
NS, ELL = 50, 3
SAMPLE = 600


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def H(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def M():
    from paper_2204_06154_gb300 import mgm
    mgm.lib()
    return mgm


@pytest.fixture(scope="module")
def big(M, oracle):
    x, nrm = I.fibonacci_sphere(N, jitter=0.1, seed=2)
    f = I.random_sh_rhs(x, 20, 2)
    X, NR = T(x), T(nrm)
    idx = M.knn(X, None, NS, self_first=True)
    w = M.stencil_weights(X, NR, idx, "rbf", 1, ELL, weights="mixed")
    fb = M.last_weights_fp64_rows()
    rp, ci, v = M.assemble(idx, w, 1.0)
    rng = np.random.default_rng(11)
    rows = np.unique(np.concatenate([[0, N - 1], rng.choice(N, SAMPLE, replace=False)])).astype(np.int32)
    oidx = oracle.knn(x, x[rows], NS)          # the centre is its own nearest point
    ow = oracle.phs_weights(x, nrm, oidx, 1, ELL, rows=rows)
    return dict(x=x, nrm=nrm, f=f, X=X, NR=NR, idx=idx, w=w, fb=fb, rp=rp, ci=ci, v=v, rows=rows, oidx=oidx, ow=ow)


def _rowrel(a, b):
    return np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)


def test_knn_rows(big):
    assert np.array_equal(big["oidx"][:, 0], big["rows"])
    assert np.array_equal(H(big["idx"])[big["rows"]], big["oidx"])


def test_weight_rows(M, big):
    rows = big["rows"]
    rel = _rowrel(H(big["w"])[rows], big["ow"])
    assert rel.max() <= 1e-12, (rel.max(), big["fb"])
    assert big["fb"] <= N // 1000, big["fb"]
    w64 = M.stencil_weights(big["X"], big["NR"], big["idx"], "rbf", 1, ELL)
    assert _rowrel(H(w64)[rows], big["ow"]).max() <= 1e-12


def test_operator_rows(big):
    """Rows of L = I - D (Sec. 2, eq. (discrete_system)): columns ascending, values from the
    oracle's weights."""
    rp, ci, v = H(big["rp"]), H(big["ci"]), H(big["v"])
    for t, i in enumerate(big["rows"]):
        order = np.argsort(big["oidx"][t], kind="stable")
        cols = big["oidx"][t][order]
        vals = np.where(cols == i, 1.0, 0.0) - big["ow"][t][order]
        assert np.array_equal(ci[rp[i]:rp[i + 1]], cols)
        assert np.max(np.abs(v[rp[i]:rp[i + 1]] - vals)) <= 1e-12 * np.max(np.abs(vals))


@pytest.fixture(scope="module")
def hier(M, big):
    return M.Hierarchy(big["X"], big["rp"], big["ci"], big["v"], 250, m=3, precision="f32")


def test_hierarchy_properties(M, oracle, big, hier):
    from scipy.spatial import cKDTree
    st = hier.stats()
    p = oracle.num_levels(N, 250)
    assert st["n"] == [N // 4 ** j for j in range(p)]
    l0, l1 = hier.level(0), hier.level(1)
    # RCM: a permutation; colouring: no stored off-diagonal entry joins two rows of one colour
    assert np.array_equal(np.sort(H(l0["perm"])), np.arange(N))
    rp, ci, col = H(l0["rp"]).astype(np.int64), H(l0["ci"]), H(l0["colour"])
    row = np.repeat(np.arange(N), np.diff(rp))
    off = ci != row
    assert np.all(col[row[off]] != col[ci[off]])
    # and it is the oracle's greedy colouring of the RCM-ordered operator, bit for bit
    import scipy.sparse as sp
    A0 = sp.csr_matrix((np.ones(ci.size), ci, rp), shape=(N, N))
    ref, nc = oracle.color(A0, 0)
    assert np.array_equal(col, ref) and st["ncolors"][0] == nc
    # WSE (Sec. 4.1): N/4 distinct survivors, separated at least as well as the fine nodes
    keep = H(l1["keep"])
    assert keep.size == N // 4 and np.unique(keep).size == keep.size and keep.min() >= 0 and keep.max() < N

    def sep(y):
        d, _ = cKDTree(y).query(y, k=2)
        return d[:, 1].min()

    assert sep(H(l1["xyz"])) >= sep(big["x"])


def test_solve_matches_fp64_path(M, big, hier):
    """Mixed pipeline (FP32 LU weights, FP32 cycle) and all-FP64 pipeline each reach 1e-10 in a
    host FP64 residual of their own operator, and their solutions agree within 1e-8."""
    import scipy.sparse as sp
    f = big["f"]
    u, info = hier.solve(T(f), tol=1e-10, restart=50, maxit=200)
    assert info["converged"]
    L = sp.csr_matrix((H(big["v"]), H(big["ci"]), H(big["rp"])), shape=(N, N))
    uh = H(u)
    assert np.linalg.norm(f - L @ uh) <= 1.0001e-10 * np.linalg.norm(f)
    w64 = M.stencil_weights(big["X"], big["NR"], big["idx"], "rbf", 1, ELL)
    rp, ci, v = M.assemble(big["idx"], w64, 1.0)
    H64 = M.Hierarchy(big["X"], rp, ci, v, 250, m=3, precision="f64")
    u64, info64 = H64.solve(T(f), tol=1e-10, restart=50, maxit=200)
    assert info64["converged"]
    L64 = sp.csr_matrix((H(v), H(ci), H(rp)), shape=(N, N))
    u64h = H(u64)
    assert np.linalg.norm(f - L64 @ u64h) <= 1.0001e-10 * np.linalg.norm(f)
    assert np.linalg.norm(uh - u64h) <= 1e-8 * np.linalg.norm(u64h)


def test_rcm_bitexact_full_size(oracle, big, hier):
    """Alg. 2's RCM of the 1M-point operator: the GPU's level-0 permutation is the oracle's, bit
    for bit (start at minimum degree, lowest index; neighbours by increasing degree, index)."""
    import scipy.sparse as sp
    L = sp.csr_matrix((H(big["v"]), H(big["ci"]), H(big["rp"])), shape=(N, N))
    ref = oracle.rcm(L)
    assert np.array_equal(H(hier.level(0)["perm"]), ref)


def test_vcycle_full_size_matches_oracle(oracle, hier):
    """The timed FP32 V-cycle of the 1M-point hierarchy (seven levels, 33 finest-level colours)
    against the oracle's cycle (Alg. 3, forward multicolour Gauss-Seidel, FP64) run on the GPU
    hierarchy's own exported levels: operators, interpolations, colourings and the level-0 RCM
    order. FP32 tolerance 1e-4 normwise, as at the smaller sizes."""
    import scipy.sparse as sp
    st = hier.stats()
    p = st["p"]
    assert p == 7 and st["ncolors"][0] >= 25
    Ho = oracle.Hierarchy()
    for j in range(p):
        lv = hier.level(j)
        n = st["n"][j]
        Ho.L.append(sp.csr_matrix((H(lv["v"]), H(lv["ci"]), H(lv["rp"])), shape=(n, n)))
        if j == 0:
            Ho.perm.append(H(lv["perm"]).astype(np.int32))
        if j + 1 < p:
            P = sp.csr_matrix((H(lv["pv"]), H(lv["pci"]), H(lv["prp"])), shape=(n, st["n"][j + 1]))
            Ho.P.append(P)
            Ho.R.append(oracle.transpose(P))
            Ho.colors.append(H(lv["colour"]).astype(np.int32))
            Ho.ncolors.append(st["ncolors"][j])
    Ho.lu, Ho.piv = oracle.lu_factor(Ho.L[-1])
    rng = np.random.default_rng(23)
    for _ in range(2):
        r = rng.standard_normal(N)
        zo = oracle.vcycle(Ho, r)
        z = H(hier.vcycle(T(r)))
        assert np.linalg.norm(z - zo) <= 1e-4 * np.linalg.norm(zo)

"""GPU parity: every step of the CUDA path (through the C-ABI) against the oracle on the same
seeded inputs, at sizes the oracle finishes in seconds that still span many tiles and a ragged
tail. Integer outputs must be bit-exact; FP64 values within 1e-12 relative (the kernels apply
the same IEEE operations as the oracle, so they are usually identical); solutions within 1e-8."""
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
def ico5(oracle):
    x, nrm = I.icosahedral_sphere(5)
    idx, w, L = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, 1.0)
    return x, nrm, idx, w, L


def _rowrel(a, b):
    return np.max(np.abs(a - b), axis=1) / np.maximum(np.max(np.abs(b), axis=1), 1e-300)


# ------------------------------------------------------------------------------------------ kNN
@pytest.mark.parametrize("case", ["ico5_30", "fib_50", "interp_3", "rand_k1", "plane_20"])
def test_knn_bitexact(M, oracle, case):
    rng = np.random.default_rng(7)
    self_first = True
    if case == "ico5_30":
        x, _ = I.icosahedral_sphere(5); q = x; k = 30
    elif case == "fib_50":
        x, _ = I.fibonacci_sphere(20011, 0.1, 3); q = x; k = 50
    elif case == "interp_3":
        x, _ = I.fibonacci_sphere(5003, 0.2, 4); q, _ = I.fibonacci_sphere(20000, 0.2, 5); k = 3; self_first = False
    elif case == "rand_k1":
        x = rng.standard_normal((3001, 3)); q = rng.standard_normal((777, 3)) * 3; k = 1; self_first = False
    else:
        x = np.concatenate([rng.uniform(-1, 1, (2500, 2)), np.zeros((2500, 1))], 1); q = x; k = 20
    ref = oracle.knn(x, q, k, self_first=self_first)
    got = H(M.knn(T(x), T(q), k, self_first=self_first))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("case", ["lattice", "offset", "tiny"])
@pytest.mark.parametrize("k", [2, 3, 50])
def test_knn_fp32_culling_edges(M, oracle, case, k):
    """The FP32 culling of distance tests changes no result: exact ties (a lattice: many equal
    distances, ties by index), coordinates far from the origin relative to the spacing (the
    culling bound grows with |x|), and a cloud scaled to 1e-20."""
    if case == "lattice":
        g = np.arange(18, dtype=np.float64)
        x = np.stack(np.meshgrid(g, g, g[:6], indexing="ij"), -1).reshape(-1, 3) * 0.25
    else:
        x, _ = I.fibonacci_sphere(6007, 0.2, 11)
        x = x + 1000.0 if case == "offset" else x * 1e-20
    ref = oracle.knn(x, x, k, self_first=True)
    got = H(M.knn(T(x), None, k, self_first=True))
    assert np.array_equal(got, ref)


def test_knn_dense_cluster_compaction(M, oracle):
    """A tight cluster of 6,000 points in a sphere of 10,000: the cluster's queries gather far more
    than the 1,024 candidates a warp buffers, so the buffer is compacted to the k best (with every
    pending FP32 distance made exact first) before the search goes on. Bit-exact against the
    oracle's brute force."""
    rng = np.random.default_rng(13)
    x, _ = I.fibonacci_sphere(10000, 0.1, 12)
    c = x[0] + 1e-3 * rng.standard_normal((6000, 3))
    x = np.concatenate([x, c])
    ref = oracle.knn(x, x, 50, self_first=True)
    got = H(M.knn(T(x), None, 50, self_first=True))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("case", ["offset", "lattice"])
def test_coarsen_fp32_culling_edges(M, oracle, case):
    if case == "offset":
        x, _ = I.fibonacci_sphere(8009, 0.3, 12)
        x = x + np.array([300.0, -200.0, 50.0])
    else:
        g = np.arange(40, dtype=np.float64)
        x = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2) * 0.1
        x = np.concatenate([x, np.zeros((x.shape[0], 1))], 1)
    NH = x.shape[0] // 4
    ref, _ = oracle.wse(x, NH, mode=1)
    got = H(M.coarsen(T(x), NH))
    assert np.array_equal(got, ref)


# ------------------------------------------------------------------------------ weights, assembly
@pytest.mark.parametrize("case", ["c1", "c2like", "k3ell3"])
def test_phs_weights(M, oracle, case):
    if case == "c1":
        x, nrm = I.icosahedral_sphere(5); n, k, ell = 30, 1, 2
    elif case == "c2like":
        x, nrm = I.torus_grid(12000, jitter=0.1, seed=2); n, k, ell = 50, 1, 3
    else:
        x, nrm = I.fibonacci_sphere(6000, 0.1, 9); n, k, ell = 20, 3, 3
    idx = oracle.knn(x, x, n, self_first=True)
    ref = oracle.phs_weights(x, nrm, idx, k, ell)
    got = H(M.stencil_weights(T(x), T(nrm), T(idx), "rbf", k, ell))
    rel = _rowrel(got, ref)
    assert rel.max() <= 1e-12, rel.max()


@pytest.mark.parametrize("case", ["c1", "c2like", "k3ell3", "m91"])
def test_phs_weights_mixed(M, oracle, case):
    """FP32 LU with FP64 iterative refinement: the FP64 solution of the same saddle systems, within
    1e-12 of the oracle's elimination. m91 (n = 70, ell = 5) takes the four-rows-a-lane solve."""
    if case == "c1":
        x, nrm = I.icosahedral_sphere(5); n, k, ell = 30, 1, 2
    elif case == "c2like":
        x, nrm = I.torus_grid(12000, jitter=0.1, seed=2); n, k, ell = 50, 1, 3
    elif case == "k3ell3":
        x, nrm = I.fibonacci_sphere(6000, 0.1, 9); n, k, ell = 20, 3, 3
    else:
        x, nrm = I.fibonacci_sphere(5003, 0.1, 4); n, k, ell = 70, 1, 5
    idx = oracle.knn(x, x, n, self_first=True)
    ref = oracle.phs_weights(x, nrm, idx, k, ell)
    got = H(M.stencil_weights(T(x), T(nrm), T(idx), "rbf", k, ell, weights="mixed"))
    fb = M.last_weights_fp64_rows()
    rel = _rowrel(got, ref)
    assert rel.max() <= 1e-12, (rel.max(), fb)
    if case in ("c1", "c2like"):
        assert fb <= 0.001 * x.shape[0], fb   # the refinement converges on these stencils


def test_phs_weights_mixed_fallback(M, oracle):
    """Near-twin nodes (1e-9 apart, spacing ~0.06) make stencils that FP32 cannot factorise; they
    are solved again by FP64 elimination, and every row still matches the oracle."""
    x, nrm = I.fibonacci_sphere(3001, 0.1, 5)
    rng = np.random.default_rng(3)
    src = rng.choice(3001, 40, replace=False)
    t1 = np.cross(nrm[src], [0.0, 0.0, 1.0])
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    tw = x[src] + 1e-9 * t1
    x = np.concatenate([x, tw / np.linalg.norm(tw, axis=1, keepdims=True)])
    nrm = x / np.linalg.norm(x, axis=1, keepdims=True)
    idx = oracle.knn(x, x, 30, self_first=True)
    ref = oracle.phs_weights(x, nrm, idx, 1, 2)
    got = H(M.stencil_weights(T(x), T(nrm), T(idx), "rbf", 1, 2, weights="mixed"))
    fb = M.last_weights_fp64_rows()
    g64 = H(M.stencil_weights(T(x), T(nrm), T(idx), "rbf", 1, 2))
    assert M.last_weights_fp64_rows() == 0
    # stencils holding a node and its twin (cond(K) ~ 1e10)
    pair = np.zeros(x.shape[0], bool)
    for t, s0 in enumerate(src):
        pair |= np.isin(idx, [s0, 3001 + t]).sum(axis=1) == 2
    assert fb >= pair.sum() > 0, (fb, pair.sum())
    assert np.array_equal(got[pair], g64[pair])          # solved by the FP64 path
    assert _rowrel(got[~pair], ref[~pair]).max() <= 1e-12
    assert _rowrel(g64[pair], ref[pair]).max() <= 1e-5   # FP64 rounding times cond(K)


def test_gfd_weights(M, oracle):
    x, nrm = I.bumpy_sphere(8000, seed=3)
    idx = oracle.knn(x, x, 25, self_first=True)
    ref = oracle.gfd_weights(x, nrm, idx, 2, 4.0)
    got = H(M.stencil_weights(T(x), T(nrm), T(idx), "gfd", ell=2, alpha=4.0))
    assert _rowrel(got, ref).max() <= 1e-12


def test_build_stencils_assembly_exact(M, oracle, ico5):
    x, nrm, idx, w, L = ico5
    gidx, gw, rp, ci, v = M.build_stencils(T(x), T(nrm), 30, "rbf", 1, 2, 1.0)
    assert np.array_equal(H(gidx), idx)
    assert np.array_equal(H(rp), L.indptr) and np.array_equal(H(ci), L.indices)
    assert np.max(np.abs(H(v) - L.data)) <= 1e-12 * np.max(np.abs(L.data))


@pytest.mark.parametrize("weights", ["f64", "mixed"])
def test_singular_stencil_row(M, weights):
    x = np.zeros((64, 3)); x[:, 0] = np.linspace(0, 1, 64)
    nrm = np.tile([0.0, 0.0, 1.0], (64, 1))
    with pytest.raises(M.MGMError) as e:
        M.build_stencils(T(x), T(nrm), 20, "rbf", 1, 2, 1.0, weights=weights)
    assert e.value.status == 2 and e.value.row == 0


def test_invalid_arguments(M):
    x, nrm = I.icosahedral_sphere(2)
    with pytest.raises(M.MGMError) as e:
        M.build_stencils(T(x), T(nrm), 500, "rbf", 1, 2, 1.0)   # n > N
    assert e.value.status == 1
    idx = torch.full((x.shape[0], 10), 10**6, dtype=torch.int32, device=DEV)
    with pytest.raises(M.MGMError) as e:
        M.stencil_weights(T(x), T(nrm), idx, "rbf", 1, 2)
    assert e.value.status == 1


# ------------------------------------------------------------------------------------- coarsening
@pytest.mark.parametrize("case", ["ico5", "fib14561", "fib14634", "torus", "fib40009"])
def test_coarsen_bitexact(M, oracle, case):
    """Bit-exact kept sets, from 9,000 to 40,009 points (ragged sizes, sphere and torus)."""
    if case == "ico5":
        x, _ = I.icosahedral_sphere(5)
    elif case == "torus":
        x, _ = I.torus_grid(9000, jitter=0.1, seed=1)
    else:
        N = int(case[3:])
        x, _ = I.fibonacci_sphere(N, jitter=0.3, seed=N)
    NH = x.shape[0] // 4
    ref, _ = oracle.wse(x, NH, mode=1)
    got = H(M.coarsen(T(x), NH))
    assert got.size == NH
    assert np.array_equal(got, ref)


# ---------------------------------------------------------------------------------- orderings
def test_rcm_bitexact(M, oracle, ico5):
    x, nrm, idx, w, L = ico5
    ref = oracle.rcm(L)
    got = H(M.rcm(T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32))))
    assert np.array_equal(got, ref)


def test_rcm_disconnected(M, oracle):
    # two separate clouds: two components, each started at its minimum-degree node
    a, _ = I.fibonacci_sphere(1500, 0.1, 1)
    b, _ = I.fibonacci_sphere(1100, 0.1, 2)
    x = np.concatenate([a, b + 5.0])
    idx = oracle.knn(x, x, 12, self_first=True)
    import scipy.sparse as sp
    L = sp.csr_matrix((np.ones(idx.size), idx.ravel(), np.arange(0, idx.size + 1, 12)), shape=(x.shape[0],) * 2)
    L.sort_indices()
    ref = oracle.rcm(L)
    got = H(M.rcm(T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32))))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("seed", [0, 12345])
def test_color_bitexact(M, oracle, ico5, seed):
    x, nrm, idx, w, L = ico5
    ref, nc = oracle.color(L, seed)
    got, gnc = M.color(T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), seed)
    assert gnc == nc and np.array_equal(H(got), ref)


def test_color_rounds_fallback_matches(M, oracle, ico5, monkeypatch):
    """The JP rounds (the fallback of the one-launch colouring) give the same colours."""
    x, nrm, idx, w, L = ico5
    ref, nc = oracle.color(L, 3)
    monkeypatch.setenv("MGM_COLOR_ROUNDS", "1")
    got, gnc = M.color(T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), 3)
    assert gnc == nc and np.array_equal(H(got), ref)


@pytest.mark.parametrize("cliques", [((0, 70), (500, 130)), ((100, 300),)])
def test_color_many_colours_and_ragged(M, oracle, cliques):
    """Greedy colouring where windows above 64 colours are needed (cliques of 70, 130 and 300
    vertices; the 300-clique also has rows longer than the symmetric-pattern merge keeps in shared
    memory), with isolated vertices, a non-symmetric pattern and a size that is no multiple of
    the block size."""
    import scipy.sparse as sp
    rng = np.random.default_rng(5)
    N = 3001
    rows, cols = [], []
    for c0, k in cliques:
        a = np.arange(c0, c0 + k)
        rows.append(np.repeat(a, k)); cols.append(np.tile(a, k))
    r = rng.integers(0, N - 40, 20000); c = rng.integers(0, N - 40, 20000)   # last 40: isolated
    rows.append(r); cols.append(c)
    A = sp.csr_matrix((np.ones(sum(len(q) for q in rows)), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    A.sum_duplicates(); A.sort_indices()
    for seed in (0, 7):
        ref, nc = oracle.color(A, seed)
        assert nc >= max(k for _, k in cliques)
        got, gnc = M.color(T(A.indptr.astype(np.int32)), T(A.indices.astype(np.int32)), seed)
        assert gnc == nc and np.array_equal(H(got), ref)


# ---------------------------------------------------------------------------------- transfers
def test_interp_transpose_galerkin(M, oracle, ico5):
    x, nrm, idx, w, L = ico5
    keep, _ = oracle.wse(x, x.shape[0] // 4, mode=1)
    xc = x[keep]
    P = oracle.interp(x, xc, 3)
    rp, ci, v = M.interp(T(x), T(xc), 3)
    assert np.array_equal(H(rp), P.indptr) and np.array_equal(H(ci), P.indices)
    assert np.max(np.abs(H(v) - P.data)) <= 1e-12
    R = oracle.transpose(P)
    trp, tci, tv = M.transpose(x.shape[0], xc.shape[0], rp, ci, v)
    assert np.array_equal(H(trp), R.indptr) and np.array_equal(H(tci), R.indices) and np.array_equal(H(tv), R.data)
    LP = oracle.spgemm(L, P)
    Lt = (T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), T(L.data))
    g1 = M.spgemm(L.shape[0], L.shape[0], xc.shape[0], Lt, (rp, ci, v))
    assert np.array_equal(H(g1[0]), LP.indptr) and np.array_equal(H(g1[1]), LP.indices)
    G = oracle.spgemm(R, LP)
    g2 = M.spgemm(R.shape[0], R.shape[1], xc.shape[0], (trp, tci, tv), g1)
    assert np.array_equal(H(g2[0]), G.indptr) and np.array_equal(H(g2[1]), G.indices)
    diff = np.abs(H(g2[2]) - G.data)
    assert np.max(diff) <= 1e-12 * np.max(np.abs(G.data))


def test_spgemm_long_rows(M, oracle):
    """C = A B with A rows of up to 90 entries (three chunks of 32) and B rows of up to 70, empty
    rows on both sides; pattern exact, values against the oracle's product."""
    import scipy.sparse as sp
    rng = np.random.default_rng(21)

    def rand_csr(n, m, maxlen):
        lens = rng.integers(0, maxlen + 1, n)
        lens[::17] = 0
        rows = np.repeat(np.arange(n), lens)
        cols = np.concatenate([rng.choice(m, k, replace=False) for k in lens])
        A = sp.csr_matrix((rng.standard_normal(rows.size), (rows, cols)), shape=(n, m))
        A.sort_indices()
        return A

    A, B = rand_csr(1500, 2500, 90), rand_csr(2500, 700, 70)
    C = oracle.spgemm(A, B)
    dev = lambda X: (T(X.indptr.astype(np.int32)), T(X.indices.astype(np.int32)), T(X.data))
    g = M.spgemm(A.shape[0], B.shape[0], B.shape[1], dev(A), dev(B))
    assert np.array_equal(H(g[0]), C.indptr) and np.array_equal(H(g[1]), C.indices)
    assert np.max(np.abs(H(g[2]) - C.data)) <= 1e-12 * np.max(np.abs(C.data))


# ---------------------------------------------------------------------------------- hierarchy
@pytest.fixture(scope="module")
def hier(M, oracle, ico5):
    x, nrm, idx, w, L = ico5
    Lt = (T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), T(L.data))
    Hg = {prec: M.Hierarchy(T(x), *Lt, n_min=125, precision=prec) for prec in ("f64", "f32")}
    Ho = oracle.setup(x, L, 125, seed=0)
    return Hg, Ho


def test_hierarchy_matches_oracle(M, oracle, hier):
    Hg, Ho = hier
    st = Hg["f64"].stats()
    assert st["p"] == Ho.p == 4
    assert st["n"] == [l.shape[0] for l in Ho.L]
    assert st["ncolors"][:-1] == Ho.ncolors
    for j in range(Ho.p):
        lv = Hg["f64"].level(j)
        assert np.array_equal(H(lv["perm"]), Ho.perm[j]), j
        if j >= 1:
            assert np.array_equal(H(lv["keep"]), Ho.keep[j - 1]), j
        assert np.array_equal(H(lv["xyz"]), Ho.X[j])
        Lo = Ho.L[j]
        assert np.array_equal(H(lv["rp"]), Lo.indptr) and np.array_equal(H(lv["ci"]), Lo.indices), j
        assert np.max(np.abs(H(lv["v"]) - Lo.data)) <= 1e-12 * np.max(np.abs(Lo.data)), j
        if j + 1 < Ho.p:
            Po = Ho.P[j]
            assert np.array_equal(H(lv["prp"]), Po.indptr) and np.array_equal(H(lv["pci"]), Po.indices)
            assert np.max(np.abs(H(lv["pv"]) - Po.data)) <= 1e-12
            assert np.array_equal(H(lv["colour"]), Ho.colors[j])


def test_vcycle_f64_matches_oracle(M, oracle, hier):
    Hg, Ho = hier
    rng = np.random.default_rng(11)
    for _ in range(3):
        r = rng.standard_normal(Ho.L[0].shape[0])
        zo = oracle.vcycle(Ho, r)
        z = H(Hg["f64"].vcycle(T(r)))
        assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)


def test_vcycle_f32_matches_oracle(M, oracle, hier):
    """FP32 V-cycle (unit roundoff 6e-8; level sums of ~30 terms with cancellation from entries
    ~1/h^2 to O(1) row sums) stays within 1e-4 of the FP64 oracle, normwise."""
    Hg, Ho = hier
    r = np.random.default_rng(12).standard_normal(Ho.L[0].shape[0])
    zo = oracle.vcycle(Ho, r)
    z = H(Hg["f32"].vcycle(T(r)))
    z32 = H(Hg["f32"].vcycle(T(r).float())).astype(np.float64)
    assert np.linalg.norm(z - zo) <= 1e-4 * np.linalg.norm(zo)
    assert np.linalg.norm(z32 - zo) <= 1e-4 * np.linalg.norm(zo)


def _bf16(a):
    """FP64 -> FP32 (nearest) -> BF16 (nearest, ties to even), as stored by transfer_bf16."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def test_vcycle_bf16_transfers_match_oracle(M, oracle, ico5, hier):
    """FP32 cycle reading BF16-stored interpolation and restriction weights: within the FP32 cycle's
    1e-4 of the oracle's cycle run with the same BF16-rounded weights; FGMRES converges in the same
    iterations as with FP32 weights, to the same solution."""
    import copy
    x, nrm, idx, w, L = ico5
    Hg, Ho = hier
    Hb = copy.copy(Ho)
    Hb.P = [P.copy() for P in Ho.P]
    Hb.R = [R.copy() for R in Ho.R]
    for P, R in zip(Hb.P, Hb.R):
        P.data = _bf16(P.data)
        R.data = _bf16(R.data)
    Lt = (T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), T(L.data))
    Gb = M.Hierarchy(T(x), *Lt, n_min=125, precision="f32", transfer_bf16=True)
    r = np.random.default_rng(14).standard_normal(x.shape[0])
    zo = oracle.vcycle(Hb, r)
    z = H(Gb.vcycle(T(r)))
    assert np.linalg.norm(z - zo) <= 1e-4 * np.linalg.norm(zo)
    assert not np.array_equal(z, H(Hg["f32"].vcycle(T(r))))   # the option changes the weights read
    f = 21.0 * I.y43(x)
    u, info = Gb.solve(T(f), tol=1e-10)
    u32, info32 = Hg["f32"].solve(T(f), tol=1e-10)
    assert info["converged"] and abs(info["iters"] - info32["iters"]) <= 1, (info["iters"], info32["iters"])
    assert np.linalg.norm(H(u) - H(u32)) <= 1e-8 * np.linalg.norm(H(u32))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_solve_matches_oracle(M, oracle, ico5, hier, prec):
    x, nrm, idx, w, L = ico5
    Hg, Ho = hier
    f = 21.0 * I.y43(x)
    uo, ito, relo = oracle.fgmres(L, Ho, f, tol=1e-12)
    u, info = Hg[prec].solve(T(f), tol=1e-10)
    assert info["converged"] and info["rel_res"] <= 1e-10
    assert np.linalg.norm(H(u) - uo) <= 1e-8 * np.linalg.norm(uo)
    _, it10, _ = oracle.fgmres(L, Ho, f, tol=1e-10)
    assert abs(info["iters"] - it10) <= 2, (info["iters"], it10)
    # true residual recomputed on the host from the oracle's operator
    res = np.linalg.norm(f - L @ H(u)) / np.linalg.norm(f)
    assert res <= 1.5e-10


def test_vcycle_60k_matches_oracle(M, oracle):
    """A five-level hierarchy built from GPU stencils of a 60k-point cloud: the cycle matches the
    oracle's on the same operator (FP64 1e-12, FP32 1e-4)."""
    import scipy.sparse as sp
    x, nrm = I.fibonacci_sphere(60000, 0.1, 12)
    _, _, rp, ci, v = M.build_stencils(T(x), T(nrm), 30, "rbf", 1, 2, 1.0, keep_weights=False)
    L = sp.csr_matrix((H(v), H(ci), H(rp)), shape=(60000, 60000))
    Ho = oracle.setup(x, L, 250, seed=0)
    r = np.random.default_rng(13).standard_normal(60000)
    zo = oracle.vcycle(Ho, r)
    for prec, tol in (("f64", 1e-12), ("f32", 1e-4)):
        Hg = M.Hierarchy(T(x), rp, ci, v, n_min=250, precision=prec)
        assert Hg.stats()["n"] == [l.shape[0] for l in Ho.L]
        z = H(Hg.vcycle(T(r)))
        assert np.linalg.norm(z - zo) <= tol * np.linalg.norm(zo), prec


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_bicgstab_matches_oracle(M, oracle, ico5, hier, prec):
    """Right-preconditioned MGM BiCGSTAB (Sec. 4.6): the solution matches the oracle's, and the
    V-cycle applications (two per step, the count of Sec. 5.2) match the oracle's within 2."""
    x, nrm, idx, w, L = ico5
    Hg, Ho = hier
    f = np.random.default_rng(31).standard_normal(x.shape[0])
    uo, appo, _ = oracle.bicgstab(L, Ho, f, tol=1e-12)
    u, info = Hg[prec].solve(T(f), krylov="bicgstab", tol=1e-10, maxit=200)
    assert info["converged"] and info["rel_res"] <= 1e-10
    assert np.linalg.norm(H(u) - uo) <= 1e-8 * np.linalg.norm(uo)
    _, app10, _ = oracle.bicgstab(L, Ho, f, tol=1e-10)
    assert abs(info["iters"] - app10) <= 2, (info["iters"], app10)
    assert np.linalg.norm(f - L @ H(u)) / np.linalg.norm(f) <= 1.5e-10
    # an exact initial guess needs no V-cycle; a cap of 3 applications reports non-convergence
    u2, info2 = Hg[prec].solve(T(f), u0=T(uo), krylov="bicgstab", tol=1e-9)
    assert info2["converged"] and info2["iters"] == 0
    u3, info3 = Hg[prec].solve(T(f), krylov="bicgstab", tol=1e-10, maxit=3)
    assert not info3["converged"] and info3["iters"] == 3


def test_standalone_mgm_and_nonconvergence(M, oracle, ico5, hier):
    x, nrm, idx, w, L = ico5
    Hg, Ho = hier
    f = np.random.default_rng(3).standard_normal(x.shape[0])
    u, info = Hg["f64"].solve(T(f), krylov="none", tol=1e-8, maxit=200)
    uo, ito, _ = oracle.mgm_solve(L, Ho, f, tol=1e-8)
    assert info["converged"] and abs(info["iters"] - ito) <= 1
    u1, info1 = Hg["f32"].solve(T(f), tol=1e-10, maxit=1)
    assert not info1["converged"] and info1["iters"] == 1
    with pytest.raises(M.MGMError) as e:
        Hg["f32"].solve(T(f), tol=1e-10, maxit=1, raise_on_nonconv=True)
    assert e.value.status == 3


def test_single_level_and_small(M, oracle):
    x, nrm = I.icosahedral_sphere(2)      # 162 points: p = 1 (direct solve)
    idx, w, L = oracle.build_operator(x, nrm, 20, "rbf", 1, 2, 1.0)
    Lt = (T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), T(L.data))
    Hg = M.Hierarchy(T(x), *Lt, n_min=250, precision="f32")
    assert Hg.stats()["p"] == 1
    f = np.random.default_rng(1).standard_normal(x.shape[0])
    u, info = Hg.solve(T(f), tol=1e-12)
    ref = np.linalg.solve(L.toarray(), f)
    assert info["converged"] and np.linalg.norm(H(u) - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("nu", [1, 2])
def test_persistent_and_per_colour_sweeps_identical(M, oracle, ico5, nu):
    """The persistent multicolour sweeps (one cooperative launch per sweep: grid barriers between
    colours, or per-row ready flags) compute every row exactly as the one-launch-per-colour
    schedule does."""
    x, nrm, idx, w, L = ico5
    Lt = (T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), T(L.data))
    r = T(np.random.default_rng(5).standard_normal(x.shape[0]))
    for prec in ("f32", "f64"):
        Ha = M.Hierarchy(T(x), *Lt, n_min=125, nu1=nu, nu2=nu, precision=prec, persistent_sweeps=0)
        za = Ha.vcycle(r)
        for mode in (1, 2):
            Hb = M.Hierarchy(T(x), *Lt, n_min=125, nu1=nu, nu2=nu, precision=prec, persistent_sweeps=mode)
            assert torch.equal(za, Hb.vcycle(r)), (prec, mode)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_flag_driven_sweeps_identical_at_scale(M, prec):
    """Per-row ready flags at a size where every resident warp takes many row groups and rows of
    several colours are in flight at once: V-cycles and solves bit-identical to per-colour
    launches."""
    x, nrm = I.fibonacci_sphere(300000, 0.1, 9)
    _, _, rp, ci, v = M.build_stencils(T(x), T(nrm), 30, "rbf", 1, 2, 1.0, keep_weights=False)
    Ha = M.Hierarchy(T(x), rp, ci, v, n_min=250, precision=prec, persistent_sweeps=0)
    Hb = M.Hierarchy(T(x), rp, ci, v, n_min=250, precision=prec, persistent_sweeps=2)
    r = T(np.random.default_rng(6).standard_normal(x.shape[0]))
    for _ in range(3):
        assert torch.equal(Ha.vcycle(r), Hb.vcycle(r))
    f = T(I.random_sh_rhs(x, lmax=12, seed=7))
    ua, ia = Ha.solve(f, tol=1e-10)
    ub, ib = Hb.solve(f, tol=1e-10)
    assert ia["converged"] and ia["iters"] == ib["iters"] and torch.equal(ua, ub)


def test_bounded_wait_reports_timeout(M):
    """A device barrier that can never complete gives up at its spin limit and the host reads
    MGM_ERR_TIMEOUT; the context stays usable afterwards."""
    assert M.check_bounded_wait(nblocks=4, spin_limit=20000) == 5
    x = torch.ones(10, device=DEV)
    assert float(x.sum()) == 10.0


@pytest.mark.parametrize("prec,nrhs", [("f32", 3), ("f64", 8), ("f32", 1)])
def test_solve_multi_matches_oracle(M, oracle, ico5, hier, prec, nrhs):
    """Many right-hand sides on one hierarchy: every column matches the oracle's solution of
    its own system, and the iteration counts per column stay within +-2 of single solves."""
    x, nrm, idx, w, L = ico5
    Hg, Ho = hier
    rng = np.random.default_rng(21)
    F = rng.standard_normal((nrhs, x.shape[0]))
    U, infos = M.solve_multi(Hg[prec], T(F), tol=1e-10)
    Uh = H(U)
    for r in range(nrhs):
        uo, ito, _ = oracle.fgmres(L, Ho, F[r], tol=1e-12)
        assert infos[r]["converged"], infos[r]
        assert np.linalg.norm(Uh[r] - uo) <= 1e-8 * np.linalg.norm(uo)
        _, it1, _ = oracle.fgmres(L, Ho, F[r], tol=1e-10)
        assert abs(infos[r]["iters"] - it1) <= 2


def test_solve_multi_standalone_and_zero_column(M, oracle, ico5, hier):
    x, nrm, idx, w, L = ico5
    Hg, Ho = hier
    F = np.random.default_rng(2).standard_normal((2, x.shape[0]))
    F[1] = 0.0
    U, infos = M.solve_multi(Hg["f64"], T(F), krylov="none", tol=1e-8, maxit=200)
    uo, ito, _ = oracle.mgm_solve(L, Ho, F[0], tol=1e-8)
    assert infos[0]["converged"] and abs(infos[0]["iters"] - ito) <= 1
    assert np.all(H(U)[1] == 0.0)


def test_solve_batched_uneven_problems(M, oracle):
    """A batch of problems of different sizes (and depths), 4 right-hand sides each."""
    probs = []
    for q, N in enumerate((3000, 9001)):
        xq, nq = I.bumpy_sphere(N, seed=30 + q)
        idx_q, w_q, L_q = oracle.build_operator(xq, nq, 25, "gfd", ell=2, alpha=4.0, mu=1e-3)
        Lt = (T(L_q.indptr.astype(np.int32)), T(L_q.indices.astype(np.int32)), T(L_q.data))
        Hq = M.Hierarchy(T(xq), *Lt, n_min=60, precision="f32")
        Ho = oracle.setup(xq, L_q, 60, seed=0)
        F = np.random.default_rng(q).standard_normal((4, N))
        probs.append((Hq, Ho, L_q, F))
    Us, infos = M.solve_batched([p[0] for p in probs], [T(p[3]) for p in probs], tol=1e-10)
    for (Hq, Ho, L_q, F), U, inf in zip(probs, Us, infos):
        for r in range(4):
            uo, _, _ = oracle.fgmres(L_q, Ho, F[r], tol=1e-12)
            assert inf[r]["converged"]
            assert np.linalg.norm(H(U)[r] - uo) <= 1e-8 * np.linalg.norm(uo)


def _gfd_batch(M, sizes, seed):
    Hs, Fs = [], []
    for q, N in enumerate(sizes):
        xq, nq = I.bumpy_sphere(N, seed=seed + q)
        _, _, rp, ci, v = M.build_stencils(T(xq), T(nq), 25, "gfd", ell=2, mu=1e-3, alpha=4.0, keep_weights=False)
        Hs.append(M.Hierarchy(T(xq), rp, ci, v, n_min=60, precision="f32"))
        Fs.append(T(np.random.default_rng(seed + q).standard_normal((3, N))))
    return Hs, Fs


def test_solve_batched_concurrent_matches_single(M):
    """Eleven problems of different sizes, more than the batch's worker threads: each problem's
    solutions are those of its own many-right-hand-side solve, bit for bit (the same kernels in
    the same order, on another stream), and every status is MGM_OK."""
    Hs, Fs = _gfd_batch(M, [2000 + 700 * q for q in range(11)], 50)
    Us, infos = M.solve_batched(Hs, Fs, tol=1e-10)
    for Hq, F, U, inf in zip(Hs, Fs, Us, infos):
        U1, inf1 = M.solve_multi(Hq, F, tol=1e-10)
        assert all(i["converged"] and i["status"] == "MGM_OK" for i in inf)
        assert [i["iters"] for i in inf] == [i["iters"] for i in inf1]
        assert torch.equal(U, U1)


def test_solve_batched_reports_each_problem(M):
    """Per-problem statuses: with one iteration allowed only the problem with zero right-hand
    sides converges; the call returns MGM_ERR_NOT_CONVERGED for the batch."""
    Hs, Fs = _gfd_batch(M, [3000, 3500, 4000], 70)
    Fs[1] = torch.zeros_like(Fs[1])
    Us, infos = M.solve_batched(Hs, Fs, tol=1e-10, maxit=1)
    assert [inf[0]["status"] for inf in infos] == ["MGM_ERR_NOT_CONVERGED", "MGM_OK", "MGM_ERR_NOT_CONVERGED"]
    assert float(Us[1].abs().max()) == 0.0


def test_config1_exact_solution(M, oracle, ico5):
    """The small workload as specified: icosahedral level-5 sphere (10,242 points), PHS r^3 +
    degree 2, n = 30, -Lap u + u = 21 Y_4^3 (so u = Y_4^3), FP64 throughout, N_min = 125 (levels
    10,242 / 2,560 / 640 / 160), MGM-FGMRES to 1e-10: the GPU solution is the oracle's to 1e-8 and
    Y_4^3 to the discretisation error (2.5e-3 relative in the oracle)."""
    x, nrm, idx, w, L = ico5
    y = I.sh_real(x, 4, 3)
    f = 21.0 * y
    _, _, rp, ci, v = M.build_stencils(T(x), T(nrm), 30, "rbf", 1, 2, 1.0, keep_weights=False)
    Hg = M.Hierarchy(T(x), rp, ci, v, n_min=125, precision="f64")
    assert Hg.stats()["n"] == [10242, 2560, 640, 160]
    u, info = Hg.solve(T(f), tol=1e-10)
    assert info["converged"] and info["rel_res"] <= 1e-10
    Ho = oracle.setup(x, L, 125, seed=0)
    uo, ito, _ = oracle.fgmres(L, Ho, f, tol=1e-10)
    u = H(u)
    assert abs(info["iters"] - ito) <= 1
    assert np.linalg.norm(u - uo) <= 1e-8 * np.linalg.norm(uo)
    assert np.abs(u - y).max() <= 3e-3 * np.abs(y).max()

"""GPU parity of the learned correction after the V-cycle (an addition to the paper's method)
against the FP64 oracle, through the C-ABI: features, the FP32 network's forward pass and
gradients, the residual objective J = |r - L delta|^2/|r|^2 and its gradients, the BF16 inference
kernel inside the captured V-cycle; deterministic training on the GPU; what the trained network
gains over the plain cycle on a held-out surface; the fallback to the plain cycle.

Tolerances: FP32 arithmetic against FP64 gives ~1e-6 relative per value; features within 2e-5 of
each channel's scale, forward / gradients within 1e-4 / 1e-3 of the largest value, the BF16
inference within 1e-3 of the largest correction (weights rounded to BF16 on both sides)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from paper_2204_06154_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N_ST = 30


@pytest.fixture(scope="module")
def M():
    from paper_2204_06154_gb300 import mgm
    mgm.lib()
    return mgm


@pytest.fixture(scope="module")
def LR():
    from paper_2204_06154_gb300 import learned
    return learned


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def H(t):
    return t.detach().cpu().numpy()


def bf16(a):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def prob(M, LR, oracle):
    x, nrm = I.bumpy_sphere(6007, seed=21)   # not a multiple of the 16-row inference tile
    idx, w, L = oracle.build_operator(x, nrm, N_ST, "rbf", 1, 2, 1.0)
    P = LR.Problem(x, nrm, n=N_ST, ell=2)
    assert np.array_equal(H(P.idx), idx)
    return x, nrm, idx, w, L, P


def _weights(n, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    d = 4 * n
    return ((rng.uniform(-1, 1, (64, d)) / np.sqrt(d)).astype(np.float32),
            (rng.uniform(-1, 1, (64, 64)) / 8.0).astype(np.float32),
            (scale * rng.uniform(-1, 1, 64) / 8.0).astype(np.float32))


def test_features_match_oracle(prob, oracle):
    x, nrm, idx, w, L, P = prob
    r = np.random.default_rng(3).standard_normal(len(x))
    r[:40] = 0.0  # rows whose whole stencil residual may vanish
    ref, rho_ref = oracle.mlp_features(idx, x, nrm, w, r)
    got, rho = P.H.learned_features(T(r))
    got = H(got)
    for q in range(4):
        sc = np.max(np.abs(ref[:, q::4]))
        assert np.max(np.abs(got[:, q::4] - ref[:, q::4])) <= 2e-5 * sc, q
    np.testing.assert_allclose(H(rho), rho_ref, rtol=5e-6, atol=0)


@pytest.mark.parametrize("B", [1, 1000, 70001])
def test_network_forward_and_vjp(M, oracle, B):
    n = N_ST
    net = M.MLP(n, seed=5)
    W1, W2, w3 = _weights(n, 6)
    net.set(W1, W2, w3)
    rng = np.random.default_rng(B)
    feat = rng.standard_normal((B, 4 * n)).astype(np.float32)
    gout = rng.standard_normal(B).astype(np.float32)
    f64 = feat.astype(np.float64)
    out = H(net.forward(T(feat)))
    ref = oracle.mlp_forward(W1, W2, w3, f64)
    assert np.max(np.abs(out - ref)) <= 1e-4 * np.max(np.abs(ref))
    g = [H(t) for t in net.vjp(T(feat), T(gout))]
    gr = oracle.mlp_vjp(W1, W2, w3, f64, gout.astype(np.float64))
    for a, b in zip(g, gr):
        assert np.max(np.abs(a - b)) <= 1e-3 * np.max(np.abs(b))


def test_network_weights_roundtrip_and_init(M):
    net = M.MLP(12, seed=9)
    W1, W2, w3 = net.get()
    assert W1.shape == (64, 48) and W2.shape == (64, 64) and w3.shape == (64,)
    assert np.max(np.abs(W1)) <= 1 / np.sqrt(48) and np.max(np.abs(W2)) <= 1 / 8
    assert np.array_equal(M.MLP(12, seed=9).get()[0], W1)
    assert not np.array_equal(M.MLP(12, seed=10).get()[0], W1)
    a = _weights(12, 1)
    net.set(*a)
    for u, v in zip(net.get(), a):
        assert np.array_equal(u, v)


def test_cycle_residual_matches_oracle_cycle(prob, oracle):
    x, nrm, idx, w, L, P = prob
    Ho = oracle.setup(x, L, 250)
    r0 = I.random_sh_rhs(x, lmax=20, seed=4)
    r1 = H(P.H.learned_cycle_residual(T(r0)))
    ref = r0 - L @ oracle.vcycle(Ho, r0)
    assert np.linalg.norm(r1 - ref) <= 1e-4 * np.linalg.norm(r0)


def test_objective_and_gradients_match_oracle(prob, oracle, M):
    x, nrm, idx, w, L, P = prob
    r = H(P.H.learned_cycle_residual(T(np.random.default_rng(8).standard_normal(len(x)))))
    net = M.MLP(N_ST, seed=11)
    W1, W2, w3 = net.get()
    J, g = P.H.learned_loss(net, T(r), grad=True)
    Jr, g1, g2, g3 = oracle.learned_loss(L, idx, x, nrm, w, r, W1.astype(np.float64), W2.astype(np.float64),
                                         w3.astype(np.float64))
    assert abs(J - Jr) <= 1e-4 * Jr
    g = H(g)
    d = 4 * N_ST
    for a, b in ((g[:64 * d], g1.ravel()), (g[64 * d:64 * d + 4096], g2.ravel()), (g[64 * d + 4096:], g3)):
        assert np.max(np.abs(a - b)) <= 1e-3 * np.max(np.abs(b))


def test_bf16_inference_matches_oracle(prob, oracle, M):
    x, nrm, idx, w, L, P = prob
    net = M.MLP(N_ST, seed=12)
    W1, W2, w3 = _weights(N_ST, 13)
    net.set(W1, W2, w3)
    P.H.learned_enable(net)
    try:
        r = np.random.default_rng(14).standard_normal(len(x))
        d = H(P.H.learned_correction(T(r)))
        ref = oracle.learned_correction(L, idx, x, nrm, w, r, bf16(W1), bf16(W2), bf16(w3))
        assert np.max(np.abs(d - ref)) <= 1e-3 * np.max(np.abs(ref))
        # weights that make the network return the centre residual feature: a Jacobi step
        J1 = np.zeros((64, 4 * N_ST), np.float32); J1[0, 3] = 1; J1[1, 3] = -1
        J2 = np.zeros((64, 64), np.float32); J2[0, 0] = 1; J2[1, 1] = 1
        J3 = np.zeros(64, np.float32); J3[0] = 1; J3[1] = -1
        net.set(J1, J2, J3)
        P.H.learned_enable(net)
        d = H(P.H.learned_correction(T(r)))
        np.testing.assert_allclose(d, r / L.diagonal(), rtol=1e-4, atol=0)  # activations split in two BF16 parts
    finally:
        P.H.learned_enable(None)


def test_vcycle_applies_the_correction(prob, M):
    x, nrm, idx, w, L, P = prob
    net = M.MLP(N_ST, seed=15)
    W1, W2, w3 = _weights(N_ST, 16)
    net.set(W1, W2, w3)
    r = np.random.default_rng(17).standard_normal(len(x))
    P.H.learned_enable(None)
    zp = H(P.H.vcycle(T(r)))
    P.H.learned_enable(net)
    try:
        zl = H(P.H.vcycle(T(r)))
        d = H(P.H.learned_correction(T(r - L @ zp)))
    finally:
        P.H.learned_enable(None)
    assert np.linalg.norm(d) > 0.0
    # FP32 cycle and residual: the corrected cycle is the plain one plus the correction of its residual
    assert np.linalg.norm(zl - (zp + d)) <= 1e-3 * np.linalg.norm(d) + 1e-6 * np.linalg.norm(zp)
    assert np.array_equal(H(P.H.vcycle(T(r))), zp)  # off again: the plain cycle, bit for bit


def test_training_is_deterministic(prob, M):
    x, nrm, idx, w, L, P = prob
    r = P.H.learned_cycle_residual(T(I.random_sh_rhs(x, lmax=20, seed=18)))
    nets = [M.MLP(N_ST, seed=19) for _ in range(2)]
    losses = [[P.H.learned_train_step(nt, r, 1e-3) for _ in range(15)] for nt in nets]
    assert losses[0] == losses[1]
    assert losses[0][-1] < losses[0][0]
    for a, b in zip(nets[0].get(), nets[1].get()):
        assert np.array_equal(a, b)


def test_trained_network_reduces_iterations(M, LR, oracle):
    torch.manual_seed(0)
    train = [LR.Problem(*I.bumpy_sphere(9000 + 1500 * s, seed=40 + s), n=N_ST) for s in range(3)]
    train.append(LR.Problem(*I.bumpy_torus(12000, seed=44), n=N_ST))
    items = [(P, r) for s, P in enumerate(train) for r in P.samples(seed=50 + s)]
    net = M.MLP(N_ST, seed=1)
    J0 = LR.mean_loss(net, items)
    hist = LR.train(net, items, steps=800, lr=2e-3, lr_final=2e-4)
    J1 = LR.mean_loss(net, items)
    assert J1 < 0.5 * min(J0, 1.0), (J0, J1, hist[-5:])
    # held-out surface
    x, nrm = I.bumpy_sphere(30000, seed=77)
    P = LR.Problem(x, nrm, n=N_ST)
    f = I.random_sh_rhs(x, lmax=20, seed=78)
    up, ip = P.H.solve(T(f), tol=1e-10)
    P.H.learned_enable(net)
    ul, il = P.H.solve(T(f), tol=1e-10)
    info = P.H.learned_info()
    P.H.learned_enable(None)
    assert ip["converged"] and il["converged"]
    assert il["iters"] < ip["iters"], (il["iters"], ip["iters"])
    assert info["fallbacks"] == 0
    # the FP64 oracle's operator and a direct solve judge both solutions
    idx, w, L = oracle.build_operator(x, nrm, N_ST, "rbf", 1, 2, 1.0)
    assert np.array_equal(H(P.idx), idx)
    ue = spla.spsolve(L.tocsc(), f)
    for u in (up, ul):
        assert np.linalg.norm(H(u) - ue) <= 1e-8 * np.linalg.norm(ue)


def test_fallback_to_plain_cycle(prob, M):
    x, nrm, idx, w, L, P = prob
    # out = -50 r_i / rho_i: a correction that multiplies the residual
    net = M.MLP(N_ST, seed=20)
    J1 = np.zeros((64, 4 * N_ST), np.float32); J1[0, 3] = 1; J1[1, 3] = -1
    J2 = np.zeros((64, 64), np.float32); J2[0, 0] = 1; J2[1, 1] = 1
    J3 = np.zeros(64, np.float32); J3[0] = -50; J3[1] = 50
    net.set(J1, J2, J3)
    f = I.random_sh_rhs(x, lmax=20, seed=22)
    P.H.learned_enable(net)
    try:
        before = P.H.learned_info()["fallbacks"]
        u, info = P.H.solve(T(f), krylov="none", maxit=200, tol=1e-8)
        after = P.H.learned_info()["fallbacks"]
    finally:
        P.H.learned_enable(None)
    assert info["converged"]
    assert after == before + 1
    assert info["history"][1] > info["history"][0]  # the first, corrected, cycle made it worse
    assert np.linalg.norm(f - L @ H(u)) <= 1e-8 * np.linalg.norm(f)

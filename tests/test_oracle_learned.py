"""Pins for the oracle's learned-smoother network (an addition to the paper's method): the
backward pass against central finite differences of the forward pass, the forward pass against
a closed form, positive homogeneity (no biases), and the invariances of the features."""
import numpy as np

from paper_2204_06154_gb300 import inputs as I


def _weights(din, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((64, din)) / np.sqrt(din), rng.standard_normal((64, 64)) / 8.0,
            rng.standard_normal(64) / 8.0)


def test_backward_matches_finite_differences(oracle):
    rng = np.random.default_rng(0)
    din, N = 20, 37
    W1, W2, w3 = _weights(din, 1)
    feat = rng.standard_normal((N, din))
    t = rng.standard_normal(N)
    loss, g1, g2, g3 = oracle.mlp_backward(W1, W2, w3, feat, t)
    out = oracle.mlp_forward(W1, W2, w3, feat)
    assert abs(loss - np.mean((out - t) ** 2)) <= 1e-14 * max(1.0, loss)
    eps = 1e-6
    for (W, G) in ((W1, g1), (W2, g2), (w3, g3)):
        flat = W.reshape(-1)
        for k in rng.choice(flat.size, 12, replace=False):
            old = flat[k]
            flat[k] = old + eps
            lp = np.mean((oracle.mlp_forward(W1, W2, w3, feat) - t) ** 2)
            flat[k] = old - eps
            lm = np.mean((oracle.mlp_forward(W1, W2, w3, feat) - t) ** 2)
            flat[k] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - G.reshape(-1)[k]) <= 1e-6 * max(1e-3, abs(fd)), (k, fd, G.reshape(-1)[k])


def test_forward_closed_form_and_homogeneity(oracle):
    din = 8
    # W1 copies feature a (a < 8) to unit a, W2 = identity on those units, w3 = ones on them:
    # out = sum_a relu(relu(f_a)) = sum_a max(f_a, 0)
    W1 = np.zeros((64, din)); W1[:din, :din] = np.eye(din)
    W2 = np.zeros((64, 64)); W2[:din, :din] = np.eye(din)
    w3 = np.zeros(64); w3[:din] = 1.0
    f = np.random.default_rng(3).standard_normal((50, din))
    np.testing.assert_allclose(oracle.mlp_forward(W1, W2, w3, f), np.maximum(f, 0).sum(axis=1), rtol=0, atol=1e-15)
    W1, W2, w3 = _weights(din, 5)
    o = oracle.mlp_forward(W1, W2, w3, f)
    np.testing.assert_allclose(oracle.mlp_forward(W1, W2, w3, 3.5 * f), 3.5 * o, rtol=1e-13, atol=1e-15)


def test_features_invariances(oracle):
    x, nrm = I.fibonacci_sphere(3000, jitter=0.2, seed=8)
    idx, w, L = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, 1.0)
    r = np.random.default_rng(4).standard_normal(3000)
    f, rho = oracle.mlp_features(idx, x, nrm, w, r)
    # scaled offsets lie in the unit disc and touch it; weights and offsets are scale-free
    rad = np.sqrt(f[:, 0::4] ** 2 + f[:, 1::4] ** 2)
    assert np.all(rad <= 1 + 1e-15) and np.allclose(rad.max(axis=1), 1.0)
    idx2, w2, _ = oracle.build_operator(2.5 * x, nrm, 30, "rbf", 1, 2, 1.0)
    f2, _ = oracle.mlp_features(idx2, 2.5 * x, nrm, w2, 7.0 * r)
    assert np.array_equal(idx, idx2)
    np.testing.assert_allclose(f2, f, rtol=1e-9, atol=1e-10)   # weights carry ~1e-12 absolute rounding
    # residual features are the stencil residuals over their RMS
    i = 123
    np.testing.assert_allclose(f[i, 3::4], r[idx[i]] / np.sqrt(np.mean(r[idx[i]] ** 2)), rtol=1e-14)


def _jacobi_weights(n):
    """Weights whose network output is the centre residual feature r_i / rho_i:
    out = relu(f_3) - relu(-f_3)."""
    din = 4 * n
    W1 = np.zeros((64, din)); W1[0, 3] = 1.0; W1[1, 3] = -1.0
    W2 = np.zeros((64, 64)); W2[0, 0] = 1.0; W2[1, 1] = 1.0
    w3 = np.zeros(64); w3[0] = 1.0; w3[1] = -1.0
    return W1, W2, w3


def test_correction_reduces_to_jacobi(oracle):
    # out_i = r_i / rho_i makes the correction rho_i * out_i / l_ii a Jacobi step D^-1 r
    x, nrm = I.fibonacci_sphere(1500, jitter=0.2, seed=9)
    n = 20
    idx, w, L = oracle.build_operator(x, nrm, n, "rbf", 1, 2, 1.0)
    r = np.random.default_rng(6).standard_normal(1500)
    W1, W2, w3 = _jacobi_weights(n)
    d = oracle.learned_correction(L, idx, x, nrm, w, r, W1, W2, w3)
    np.testing.assert_allclose(d, r / L.diagonal(), rtol=1e-13, atol=0)
    J, *_ = oracle.learned_loss(L, idx, x, nrm, w, r, W1, W2, w3)
    s = r - L @ (r / L.diagonal())
    assert abs(J - (s @ s) / (r @ r)) <= 1e-12 * J
    # zero weights: no correction, J = 1
    J0, *_ = oracle.learned_loss(L, idx, x, nrm, w, r, 0 * W1, 0 * W2, 0 * w3)
    assert J0 == 1.0


def test_residual_loss_gradient_matches_finite_differences(oracle):
    x, nrm = I.fibonacci_sphere(800, jitter=0.2, seed=10)
    n = 12
    idx, w, L = oracle.build_operator(x, nrm, n, "rbf", 1, 2, 1.0)
    rng = np.random.default_rng(11)
    r = rng.standard_normal(800)
    W1, W2, w3 = _weights(4 * n, 12)
    J, g1, g2, g3 = oracle.learned_loss(L, idx, x, nrm, w, r, W1, W2, w3)
    eps = 1e-6
    for (W, G) in ((W1, g1), (W2, g2), (w3, g3)):
        flat = W.reshape(-1)
        for k in rng.choice(flat.size, 10, replace=False):
            old = flat[k]
            flat[k] = old + eps
            jp = oracle.learned_loss(L, idx, x, nrm, w, r, W1, W2, w3)[0]
            flat[k] = old - eps
            jm = oracle.learned_loss(L, idx, x, nrm, w, r, W1, W2, w3)[0]
            flat[k] = old
            fd = (jp - jm) / (2 * eps)
            assert abs(fd - G.reshape(-1)[k]) <= 1e-6 * max(1e-3, abs(fd)), (k, fd, G.reshape(-1)[k])

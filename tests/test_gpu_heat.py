"""GPU parity of the surface gradient and divergence (tangent-plane RBF-FD first derivatives) and
of the heat method for geodesic distance (Sec. 6.3) against the oracle: the derivative weights
to 1e-12 (the same IEEE operations as the oracle's GEPP), gradient and divergence to 1e-13, and
the distance from the north pole of the unit sphere against the great-circle distance."""
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
def cloud(oracle):
    x, nrm = I.fibonacci_sphere(5003, 0.2, 6)
    idx = oracle.knn(x, x, 30, self_first=True)
    return x, nrm, idx


def test_gradient_weights_match_oracle(M, oracle, cloud):
    x, nrm, idx = cloud
    wxo, wyo = oracle.phs_grad_weights(x, nrm, idx, 1, 2)
    wx, wy = M.gradient_weights(T(x), T(nrm), T(idx), 1, 2)
    for a, b in ((H(wx), wxo), (H(wy), wyo)):
        rel = np.max(np.abs(a - b), axis=1) / np.max(np.abs(b), axis=1)
        assert rel.max() <= 1e-12


def test_gradient_and_divergence_match_oracle(M, oracle, cloud):
    x, nrm, idx = cloud
    wxo, wyo = oracle.phs_grad_weights(x, nrm, idx, 1, 2)
    u = np.sin(3 * x[:, 0]) + x[:, 1] * x[:, 2]
    go = oracle.surface_grad(nrm, idx, wxo, wyo, u)
    g = H(M.surface_gradient(T(nrm), T(idx), T(wxo), T(wyo), T(u)))
    assert np.abs(g - go).max() <= 1e-13 * np.abs(go).max()
    eta = -go / np.linalg.norm(go, axis=1, keepdims=True)
    e = H(M.surface_gradient(T(nrm), T(idx), T(wxo), T(wyo), T(u), normalize=True))
    assert np.abs(e - eta).max() <= 1e-13
    do = oracle.surface_div(nrm, idx, wxo, wyo, eta)
    d = H(M.surface_divergence(T(nrm), T(idx), T(wxo), T(wyo), T(eta)))
    assert np.abs(d - do).max() <= 1e-12 * np.abs(do).max()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_heat_method_distance(M, prec):
    from paper_2204_06154_gb300 import heat
    x, nrm = I.fibonacci_sphere(8000, 0.1, 3)
    src = int(np.argmax(x[:, 2]))
    d, its = heat.geodesic_distance(T(x), T(nrm), src, precision=prec)
    d = H(d)
    ex = np.arccos(np.clip(x @ x[src], -1.0, 1.0))
    assert d[src] == 0.0
    assert np.mean(np.abs(d - ex)) <= 0.02 * np.mean(ex)
    assert np.abs(d - ex).max() <= 0.05
    assert len(its) == 4 and max(its) <= 30


def test_gradient_weights_argument_checks(M, cloud):
    x, nrm, idx = cloud
    with pytest.raises(M.MGMError):
        M.gradient_weights(T(x), T(nrm), T(idx), 1, 0)    # ell = 0 has no first derivatives
    bad = idx.copy(); bad[7, 3] = len(x)
    with pytest.raises(M.MGMError):
        M.gradient_weights(T(x), T(nrm), T(bad), 1, 2)

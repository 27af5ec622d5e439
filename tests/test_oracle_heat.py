"""Pins for the oracle's surface gradient and divergence (tangent-plane RBF-FD first derivatives)
and the heat method for geodesic distance (Sec. 6.3): polynomial reproduction of the derivative
weights, the closed forms grad_S z = e_z - z n and div_S grad_S z = Lap_S z = -2z on the unit
sphere, and the great-circle distance arccos(x . x*) from a source point."""
import numpy as np
import pytest

from paper_2204_06154_gb300 import inputs as I


def test_gradient_weights_reproduce_polynomial_derivatives(oracle):
    x, nrm = I.fibonacci_sphere(2000, 0.2, 5)
    n, ell = 30, 2
    idx = oracle.knn(x, x, n, self_first=True)
    wx, wy = oracle.phs_grad_weights(x, nrm, idx, 1, ell)
    for i in (0, 777, 1999):
        t1, t2 = oracle.tangent_basis(nrm[i])
        d = x[idx[i]] - x[i]
        xh, yh = d @ t1, d @ t2
        for a in range(ell + 1):
            for b in range(ell + 1 - a):
                p = xh ** a * yh ** b
                ex_x = 1.0 if (a, b) == (1, 0) else 0.0
                ex_y = 1.0 if (a, b) == (0, 1) else 0.0
                sc = np.abs(wx[i]).sum() * np.abs(p).max()
                assert abs(wx[i] @ p - ex_x) <= 1e-10 * max(1.0, sc), (i, a, b)
                assert abs(wy[i] @ p - ex_y) <= 1e-10 * max(1.0, sc), (i, a, b)


def test_gradient_and_divergence_closed_forms_converge(oracle):
    """grad_S z = (-xz, -yz, 1 - z^2) and div_S grad_S z = -2z on the unit sphere; the errors fall
    with refinement (degree-2 polynomials: second order)."""
    eg, ed = [], []
    for N in (2000, 8000):
        x, nrm = I.fibonacci_sphere(N, 0.1, 3)
        idx = oracle.knn(x, x, 30, self_first=True)
        wx, wy = oracle.phs_grad_weights(x, nrm, idx, 1, 2)
        z = x[:, 2]
        gex = np.stack([-x[:, 0] * z, -x[:, 1] * z, 1.0 - z * z], axis=1)
        g = oracle.surface_grad(nrm, idx, wx, wy, z)
        eg.append(np.abs(g - gex).max())
        assert np.abs(np.einsum("ij,ij->i", g, nrm)).max() <= 1e-12   # tangent vectors
        d = oracle.surface_div(nrm, idx, wx, wy, gex)
        ed.append(np.abs(d + 2.0 * z).max())
    assert eg[1] < eg[0] / 2.5 and ed[1] < ed[0] / 2.5, (eg, ed)
    assert eg[1] < 1e-4 and ed[1] < 2e-3


def test_heat_method_great_circle_distance(oracle):
    x, nrm = I.fibonacci_sphere(8000, 0.1, 3)
    src = int(np.argmax(x[:, 2]))
    d, its = oracle.heat_geodesic(x, nrm, src)
    ex = np.arccos(np.clip(x @ x[src], -1.0, 1.0))
    assert d[src] == 0.0
    assert np.mean(np.abs(d - ex)) <= 0.02 * np.mean(ex)
    assert np.abs(d - ex).max() <= 0.05
    assert max(its) <= 30

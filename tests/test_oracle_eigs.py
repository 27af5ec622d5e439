"""Pins of the oracle's eigenpairs (Sec. 6.1: the LBO's eigenpairs of smallest magnitude). On the
unit sphere the LBO's eigenvalues are -l(l+1) with multiplicity 2l+1, so the eigenvalues of
L = I - D are 1 + l(l+1) up to the discretisation error; the constant is an exact eigenvector
(the weights reproduce constants); every pair satisfies L v = lambda v."""
import numpy as np
import pytest

from paper_2204_06154_gb300 import inputs as I


@pytest.fixture(scope="module")
def sphere(oracle):
    x, nrm = I.icosahedral_sphere(3)
    idx, w, L = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, 1.0)
    lam, V = oracle.eigs_smallest(L, 25)
    return L, lam, V


def test_sphere_shells(sphere):
    _, lam, _ = sphere
    ev = np.sort(lam.real - 1.0)      # eigenvalues of -D
    start = 0
    for l in range(5):
        shell = ev[start:start + 2 * l + 1]
        assert np.all(np.abs(shell - l * (l + 1)) <= 0.05 * max(1, l * (l + 1))), (l, shell)
        start += 2 * l + 1
    assert np.abs(lam.imag).max() <= 1e-2 * np.abs(lam).max()


def test_pairs_satisfy_the_definition(sphere):
    L, lam, V = sphere
    for j in range(V.shape[1]):
        r = L @ V[:, j] - lam[j] * V[:, j]
        assert np.linalg.norm(r) <= 1e-10 * np.abs(lam[j]) * np.linalg.norm(V[:, j]) * 1e3


def test_constant_mode(sphere):
    L, lam, V = sphere
    assert abs(lam[0] - 1.0) <= 1e-11
    v = V[:, 0].real
    v = v / v[np.argmax(np.abs(v))]
    assert np.allclose(v, 1.0, atol=1e-9)


def test_shell_error_falls_under_refinement(oracle, sphere):
    """Halving the spacing (icosahedral level 3 -> 4) shrinks the error of the l = 1..3 shells."""
    x, nrm = I.icosahedral_sphere(4)
    _, _, L4 = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, 1.0)
    lam4, _ = oracle.eigs_smallest(L4, 16)
    exact = np.concatenate([[l * (l + 1)] * (2 * l + 1) for l in range(4)])
    e3 = np.abs(np.sort(sphere[1].real[:16] - 1.0) - exact)[1:].max()
    e4 = np.abs(np.sort(lam4.real - 1.0) - exact)[1:].max()
    assert e4 < e3 / 1.5, (e3, e4)

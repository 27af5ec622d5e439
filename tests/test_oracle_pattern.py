"""Pins of the oracle's reaction-diffusion stepping (Sec. 6.2): the homogeneous steady state is a
fixed point of both schemes; on spatially constant data (the weights reproduce constants, so the
solves are the identity on them) the schemes are the ODE integrators, first order (IMEX Euler)
and second order (SBDF2) in time against a tight-tolerance reference from scipy; pure diffusion
damps a spherical harmonic Y_l^m by 1 / (1 + dt D l(l+1)) a backward-Euler step."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

from paper_2204_06154_gb300 import inputs as I

GM = (0.08, 1.5, 0.45)          # A, B, C of Sec. 6.2
SCH = (1.0, 0.1, 0.9)           # gamma, a, b


def _steady(model, prm):
    if model == "gm":
        A, B, Cc = prm
        u = brentq(lambda u: A - B * u + 1.0 / (1.0 + Cc * u * u), 1e-6, 10.0)
        return u, u * u
    g, a, b = prm
    return a + b, b / (a + b) ** 2


@pytest.fixture(scope="module")
def sphere():
    return I.icosahedral_sphere(2)


@pytest.mark.parametrize("model,prm", [("gm", GM), ("schnakenberg", SCH)])
@pytest.mark.parametrize("scheme", ["euler", "sbdf2"])
def test_steady_state_is_fixed(oracle, sphere, model, prm, scheme):
    x, nrm = sphere
    us, vs = _steady(model, prm)
    N = x.shape[0]
    u, v, _ = oracle.reaction_diffusion(x, nrm, model, prm, 0.01, 0.1, 0.05, 4, np.full(N, us), np.full(N, vs),
                                        scheme=scheme, n=30, ell=2, n_min=40, tol=1e-12)
    assert np.abs(u - us).max() <= 1e-10 and np.abs(v - vs).max() <= 1e-10


def _ode_error(oracle, x, nrm, scheme, dt, T, u0, v0):
    N = x.shape[0]
    steps = int(round(T / dt))
    u, v, _ = oracle.reaction_diffusion(x, nrm, "schnakenberg", SCH, 1.0, 10.0, dt, steps, np.full(N, u0),
                                        np.full(N, v0), scheme=scheme, n=30, ell=2, n_min=40, tol=1e-13)
    g, a, b = SCH
    ref = solve_ivp(lambda t, y: [g * (a - y[0] + y[0] ** 2 * y[1]), g * (b - y[0] ** 2 * y[1])], (0, T), [u0, v0],
                    rtol=1e-12, atol=1e-14, method="DOP853").y[:, -1]
    assert np.ptp(u) <= 1e-10 and np.ptp(v) <= 1e-10        # stays spatially constant
    return max(abs(u[0] - ref[0]), abs(v[0] - ref[1]))


@pytest.mark.parametrize("scheme,order", [("euler", 1), ("sbdf2", 2)])
def test_time_order_on_constant_data(oracle, sphere, scheme, order):
    x, nrm = sphere
    e1 = _ode_error(oracle, x, nrm, scheme, 0.05, 1.0, 0.5, 1.5)
    e2 = _ode_error(oracle, x, nrm, scheme, 0.025, 1.0, 0.5, 1.5)
    assert 2 ** order * 0.8 <= e1 / e2 <= 2 ** order * 1.25, (e1, e2)


def test_pure_diffusion_damps_harmonics(oracle):
    x, nrm = I.icosahedral_sphere(4)
    N = x.shape[0]
    l, dt, D = 3, 0.01, 0.5
    y = I.sh_real(x, l, 1)
    u, v, _ = oracle.reaction_diffusion(x, nrm, "schnakenberg", (0.0, 0.0, 0.0), D, D, dt, 2, y, y.copy(),
                                        scheme="euler", n=30, ell=2, n_min=250, tol=1e-12)
    expect = y / (1.0 + dt * D * l * (l + 1)) ** 2
    assert np.linalg.norm(u - expect) <= 1e-3 * np.linalg.norm(expect)

"""Reaction-diffusion stepping on the GPU (Sec. 6.2) against the oracle's: Gierer-Meinhardt with
SBDF2 (the paper's model and scheme) and Schnakenberg with IMEX Euler, a few steps from seeded
random states; the fused right-hand sides against their definition."""
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


@pytest.mark.parametrize("model,prm,scheme,Du,Dv,dt", [
    ("gm", (0.08, 1.5, 0.45), "sbdf2", 0.01, 0.2, 0.05),
    ("schnakenberg", (1.0, 0.1, 0.9), "euler", 0.01, 0.1, 0.01)])
@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 1e-7)])
def test_steps_match_oracle(M, oracle, model, prm, scheme, Du, Dv, dt, prec, tol):
    from paper_2204_06154_gb300.pattern import ReactionDiffusion
    x, nrm = I.fibonacci_sphere(6000, 0.1, 7)
    rng = np.random.default_rng(3)
    u0, v0 = rng.uniform(0.2, 1.0, 6000), rng.uniform(0.2, 1.0, 6000)
    uo, vo, its_o = oracle.reaction_diffusion(x, nrm, model, prm, Du, Dv, dt, 5, u0, v0, scheme=scheme, n=30, ell=3,
                                              n_min=250, tol=1e-11)
    rd = ReactionDiffusion(T(x), T(nrm), model, prm, Du, Dv, dt, scheme=scheme, n=30, ell=3, n_min=250, precision=prec)
    u, v, its = rd.run(T(u0), T(v0), 5, tol=1e-11)
    u, v = u.cpu().numpy(), v.cpu().numpy()
    assert np.linalg.norm(u - uo) <= tol * np.linalg.norm(uo) and np.linalg.norm(v - vo) <= tol * np.linalg.norm(vo)
    assert all(abs(a - b) <= 2 and abs(c - d) <= 2 for (a, c), (b, d) in zip(its, its_o)), (its, its_o)


@pytest.mark.parametrize("model,prm", [("gm", (0.08, 1.5, 0.45)), ("schnakenberg", (1.0, 0.1, 0.9))])
def test_fused_rhs(M, oracle, model, prm):
    rng = np.random.default_rng(9)
    u, v, up, vp = (rng.uniform(0.1, 1.0, 100003) for _ in range(4))
    dt = 0.05
    f, g = oracle.reaction_terms(model, u, v, prm)
    fp, gp = oracle.reaction_terms(model, up, vp, prm)
    ru, rv = M.reaction_rhs(model, "euler", T(u), T(v), prm, dt)
    np.testing.assert_allclose(ru.cpu().numpy(), u + dt * f, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(rv.cpu().numpy(), v + dt * g, rtol=1e-14, atol=1e-15)
    ru, rv = M.reaction_rhs(model, "sbdf2", T(u), T(v), prm, dt, T(up), T(vp))
    np.testing.assert_allclose(ru.cpu().numpy(), (4 * u - up) / 3 + 2 * dt / 3 * (2 * f - fp), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(rv.cpu().numpy(), (4 * v - vp) / 3 + 2 * dt / 3 * (2 * g - gp), rtol=1e-13, atol=1e-15)
    with pytest.raises(M.MGMError):
        M.reaction_rhs(model, "sbdf2", T(u), T(v), prm, dt)      # SBDF2 without the previous step


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("f32", 1e-7)])
def test_graph_steps_match_oracle(M, oracle, prec, tol):
    """Config 5's stepping (Schnakenberg, IMEX Euler) with every step one CUDA graph launch: the
    fused right-hand sides and both warm-started solves driven on the device (WHILE conditional
    nodes, convergence decided in kernels). Matches the oracle's steps, iterations within 2."""
    from paper_2204_06154_gb300.pattern import ReactionDiffusion
    model, prm, Du, Dv, dt = "schnakenberg", (1.0, 0.1, 0.9), 0.01, 0.1, 0.01
    x, nrm = I.fibonacci_sphere(6000, 0.1, 7)
    rng = np.random.default_rng(4)
    u0, v0 = rng.uniform(0.2, 1.0, 6000), rng.uniform(0.2, 1.0, 6000)
    uo, vo, its_o = oracle.reaction_diffusion(x, nrm, model, prm, Du, Dv, dt, 5, u0, v0, scheme="euler", n=30, ell=3,
                                              n_min=250, tol=1e-11)
    rd = ReactionDiffusion(T(x), T(nrm), model, prm, Du, Dv, dt, scheme="euler", n=30, ell=3, n_min=250, precision=prec)
    u, v, its = rd.run_graph(T(u0), T(v0), 5, tol=1e-11)
    u, v = u.cpu().numpy(), v.cpu().numpy()
    assert np.linalg.norm(u - uo) <= tol * np.linalg.norm(uo) and np.linalg.norm(v - vo) <= tol * np.linalg.norm(vo)
    assert all(abs(a - b) <= 2 and abs(c - d) <= 2 for (a, c), (b, d) in zip(its, its_o)), (its, its_o)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_graph_fgmres_matches_host_fgmres(M, oracle, prec):
    """The device-driven FGMRES (one graph launch a solve) and the host-driven one on the same
    hierarchy: same iteration counts within one, solutions within 1e-8 of the oracle's."""
    x, nrm = I.icosahedral_sphere(5)
    idx, w, L = oracle.build_operator(x, nrm, 30, "rbf", 1, 2, 1.0)
    Lt = (T(L.indptr.astype(np.int32)), T(L.indices.astype(np.int32)), T(L.data))
    Hg = M.Hierarchy(T(x), *Lt, n_min=125, precision=prec)
    Ho = oracle.setup(x, L, 125, seed=0)
    f = np.random.default_rng(5).standard_normal(x.shape[0])
    uo, _, _ = oracle.fgmres(L, Ho, f, tol=1e-12)
    for restart in (50, 7):
        ua, ia = Hg.solve(T(f), tol=1e-10, restart=restart)
        ub, ib = Hg.solve(T(f), tol=1e-10, restart=restart, krylov="fgmres_graph")
        assert ia["converged"] and ib["converged"] and abs(ia["iters"] - ib["iters"]) <= 1, (ia, ib)
        assert ib["rel_res"] <= 1e-10 and len(ib["history"]) == ib["iters"] + 1
        assert np.linalg.norm(ub.cpu().numpy() - uo) <= 1e-8 * np.linalg.norm(uo)
    # warm start and an immediately converged solve
    uc, ic = Hg.solve(T(f), u0=ub, tol=1e-10, krylov="fgmres_graph")
    assert ic["converged"] and ic["iters"] == 0

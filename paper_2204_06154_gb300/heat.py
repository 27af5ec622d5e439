"""Geodesic distance by the heat method (Sec. 6.3), orchestration only: every step runs in
libmgm's kernels (stencils, weights, hierarchies, MGM-preconditioned FGMRES, surface gradient and
divergence).

1. Heat steps: backward Euler (I - dt D) u^{k+1} = u^k from a unit spike at the source.
2. eta = -grad u / |grad u| (tangent-plane RBF-FD first derivatives).
3. The mean-zero Poisson problem D phi = div eta, solved as the bordered system of Sec. 4.4.
The distance estimate is phi - phi(source). The time step must carry the heat over the whole
surface above the solver's noise floor: far from the source u ~ exp(-d / sqrt(dt)), and a
relative residual tolerance tol leaves the gradient direction to round-off where u / |u| < tol;
dt = 0.01 suits a unit-size surface (dt = h^2 does not, at these tolerances)."""
import torch

from . import mgm


def geodesic_distance(xyz, nrm, source, n=30, k=1, ell_lap=2, ell_grad=2, dt=0.01, steps=3, n_min=250, tol=1e-10,
                      precision="f32"):
    """xyz, nrm: CUDA float64 tensors (N x 3). Returns (distance N, per-solve iteration counts)."""
    N = xyz.shape[0]
    idx, w, rp, ci, v = mgm.build_stencils(xyz, nrm, n, "rbf", k, ell_lap, dt)
    Hh = mgm.Hierarchy(xyz, rp, ci, v, n_min, precision=precision)
    u = torch.zeros(N, dtype=torch.float64, device=xyz.device)
    u[source] = 1.0
    its = []
    for _ in range(steps):
        u, info = Hh.solve(u.clone(), tol=tol, raise_on_nonconv=True)
        its.append(info["iters"])
    wx, wy = mgm.gradient_weights(xyz, nrm, idx, k, ell_grad)
    eta = mgm.surface_gradient(nrm, idx, wx, wy, u, normalize=True)
    div = mgm.surface_divergence(nrm, idx, wx, wy, eta)
    prp, pci, pv = mgm.assemble(idx, w, poisson=True)
    Hp = mgm.Hierarchy(xyz, prp, pci, pv, n_min, precision=precision, constraint=True)
    phi, info = Hp.solve(div, tol=tol, raise_on_nonconv=True)
    its.append(info["iters"])
    return phi - phi[source], its

"""Reaction-diffusion pattern formation on a point-cloud surface (Sec. 6.2), on the GPU.
Orchestration only: stencils, hierarchies, the fused right-hand sides (mgm_reaction_rhs) and the
warm-started MGM-FGMRES solves run in libmgm's kernels.

u_t = Du Lap u + f(u, v), v_t = Dv Lap v + g(u, v): diffusion implicit, reactions explicit. SBDF2
(the paper's scheme) solves (I - (2/3) dt D Lap) w^{n+1} = (4 w^n - w^{n-1}) / 3 + (2/3) dt
(2 r^n - r^{n-1}) after one IMEX Euler step, (I - dt D Lap) w^{n+1} = w^n + dt r^n; each solve
starts from the previous step's values (Sec. 6.2)."""
import torch

from . import mgm


class ReactionDiffusion:
    def __init__(self, xyz, nrm, model, prm, Du, Dv, dt, scheme="sbdf2", n=30, ell=3, k=1, n_min=250,
                 precision="f32", weights="mixed"):
        self.xyz = xyz
        self.model, self.prm, self.Du, self.Dv, self.dt, self.scheme = model, tuple(prm), Du, Dv, dt, scheme
        self.idx = mgm.knn(xyz, None, n, self_first=True)
        self.w = mgm.stencil_weights(xyz, nrm, self.idx, "rbf", k, ell, weights=weights)
        self.n_min, self.precision = n_min, precision
        self.H = {}

    def hierarchy(self, mu):
        """The hierarchy of L = I - mu D (built once per mu)."""
        if mu not in self.H:
            rp, ci, v = mgm.assemble(self.idx, self.w, mu)
            self.H[mu] = mgm.Hierarchy(self.xyz, rp, ci, v, self.n_min, precision=self.precision)
        return self.H[mu]

    def run_graph(self, u0, v0, steps, tol=1e-8, restart=50, maxit=200):
        """IMEX Euler steps with every step one CUDA graph launch (right-hand sides and both
        device-driven, warm-started solves; mgm_reaction_steps). Returns (u, v, iterations)."""
        if self.scheme != "euler":
            raise ValueError("graph stepping implements IMEX Euler")
        u, v = u0.clone(), v0.clone()
        its = mgm.reaction_steps(self.hierarchy(self.dt * self.Du), self.hierarchy(self.dt * self.Dv), self.model,
                                 self.prm, self.dt, u, v, steps, tol=tol, restart=restart, maxit=maxit)
        return u, v, its

    def run(self, u0, v0, steps, tol=1e-8, restart=50, maxit=200):
        """Advance (u0, v0) by `steps` steps. Returns (u, v, [(iterations u, iterations v), ...])."""
        u, v = u0.clone(), v0.clone()
        up = vp = None
        its = []
        for step in range(steps):
            euler = self.scheme == "euler" or step == 0
            ru, rv = mgm.reaction_rhs(self.model, "euler" if euler else "sbdf2", u, v, self.prm, self.dt, up, vp)
            c = self.dt if euler else (2.0 / 3.0) * self.dt
            un, iu = self.hierarchy(c * self.Du).solve(ru, u0=u, tol=tol, restart=restart, maxit=maxit)
            vn, iv = self.hierarchy(c * self.Dv).solve(rv, u0=v, tol=tol, restart=restart, maxit=maxit)
            its.append((iu["iters"], iv["iters"]))
            up, vp, u, v = u, v, un, vn
        return u, v, its

"""Training and evaluation driver of the learned correction after the MGM V-cycle (an addition to
the paper's method). Orchestration only: stencils, hierarchies, training samples, the network's
forward and backward passes and the Adam steps all run in libmgm's kernels.

A training sample is a residual left by the plain V-cycle, r_k = (I - L M)^k r_0 (k >= 1), for a
seeded right-hand side r_0 (a random spherical-harmonic sum or white noise); the network learns to
shrink the residual it is given, J = |r - L delta|^2 / |r|^2."""
import numpy as np
import torch

from . import inputs as I
from . import mgm


class Problem:
    """One surface: stencils (Sec. 2), an FP32 hierarchy (Alg. 2) with the stencils attached."""

    def __init__(self, xyz, nrm, n=30, k=1, ell=2, mu=1.0, n_min=250, seed=0, device="cuda"):
        self.xyz_host = np.ascontiguousarray(xyz)
        self.xyz = torch.tensor(xyz, dtype=torch.float64, device=device)
        self.nrm = torch.tensor(nrm, dtype=torch.float64, device=device)
        self.idx, self.w, self.rp, self.ci, self.v = mgm.build_stencils(self.xyz, self.nrm, n, "rbf", k, ell, mu)
        self.H = mgm.Hierarchy(self.xyz, self.rp, self.ci, self.v, n_min, precision="f32", seed=seed)
        self.H.learned_attach(self.xyz, self.nrm, self.idx, self.w)
        self.N = self.xyz.shape[0]

    def samples(self, seed, cycles=3, lmax=20, smooth="sh"):
        """Residuals after 1..cycles plain V-cycles from a smooth start (a random spherical-harmonic
        sum up to degree lmax, or with smooth="poly" a random polynomial of degree <= 4 in the
        coordinates, cheaper for large clouds) and from a white-noise start."""
        rng = np.random.default_rng(seed)
        if smooth == "sh":
            f0 = I.random_sh_rhs(self.xyz_host, lmax=lmax, seed=seed)
        else:
            x = self.xyz_host
            f0 = np.zeros(self.N)
            for a in range(5):
                for b in range(5 - a):
                    for c in range(5 - a - b):
                        f0 += rng.standard_normal() * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c
        rhs = [f0, rng.standard_normal(self.N)]
        out = []
        for r0 in rhs:
            r = torch.tensor(r0, dtype=torch.float64, device=self.xyz.device)
            n0 = float(r.norm())
            for _ in range(cycles):
                r = self.H.learned_cycle_residual(r)
                nk = float(r.norm())
                if not np.isfinite(nk) or nk > 1e3 * n0:  # a cycle that diverges here gives no samples
                    break
                out.append(r)
        return out


def train(net, items, steps, lr=1e-3, lr_final=1e-4, log_every=0):
    """Adam on the samples in round-robin order with a geometric learning-rate decay from lr to
    lr_final. items: list of (Problem, residual). Returns the loss of every step."""
    hist = []
    for t in range(steps):
        P, r = items[t % len(items)]
        a = lr * (lr_final / lr) ** (t / max(1, steps - 1))
        hist.append(P.H.learned_train_step(net, r, a))
        if log_every and t % log_every == 0:
            print(f"step {t}: J = {hist[-1]:.4f}", flush=True)
    return hist


def mean_loss(net, items):
    return float(np.mean([P.H.learned_loss(net, r) for (P, r) in items]))

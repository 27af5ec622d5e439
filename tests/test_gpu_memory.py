"""The library's device-memory caches. A destroyed hierarchy's blocks are kept and handed to the
next hierarchy, and the scratch pool keeps its memory mapped between calls (both within 1/32 of
the device's memory). Results must not depend on what a reused block held: a hierarchy built on
the blocks of a different problem's hierarchy gives the same cycle, solution and iteration count,
bit for bit, as one built on fresh memory. mgm_release_cached_memory hands the cached blocks
back to the device."""
import numpy as np
import pytest
import torch

from paper_2204_06154_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N = 40000


@pytest.fixture(scope="module")
def M():
    from paper_2204_06154_gb300 import mgm
    mgm.lib()
    return mgm


def _operator(M, x, nrm):
    X, NR = torch.from_numpy(x).to(DEV), torch.from_numpy(nrm).to(DEV)
    idx = M.knn(X, None, 30, self_first=True)
    w = M.stencil_weights(X, NR, idx, "rbf", 1, 2, weights="mixed")
    rp, ci, v = M.assemble(idx, w, 1.0)
    return X, rp, ci, v


def _run(M, op, f):
    X, rp, ci, v = op
    Hh = M.Hierarchy(X, rp, ci, v, 125, m=3, precision="f32")
    e = Hh.vcycle(f)
    u, info = Hh.solve(f, tol=1e-10, restart=50, maxit=200)
    return Hh, e.cpu(), u.cpu(), info["iters"]


def test_reused_blocks_give_the_same_bits(M):
    xs, ns = I.fibonacci_sphere(N, jitter=0.1, seed=7)
    xt, nt = I.torus_grid(N, 1.0, 1.0 / 3.0, jitter=0.1, seed=7)
    f = torch.from_numpy(I.random_sh_rhs(xs, 12, 7)).to(DEV)
    sphere, torus = _operator(M, xs, ns), _operator(M, xt, nt)
    M.release_cached_memory()
    H1, e1, u1, it1 = _run(M, sphere, f)          # fresh blocks
    del H1
    H2, _, _, _ = _run(M, torus, f)               # the sphere's blocks, now holding the torus
    del H2
    H3, e3, u3, it3 = _run(M, sphere, f)          # the torus hierarchy's blocks
    assert torch.equal(e1, e3) and torch.equal(u1, u3) and it1 == it3
    del H3
    M.release_cached_memory()


def test_release_hands_cached_blocks_back(M):
    xs, ns = I.fibonacci_sphere(4 * N, jitter=0.1, seed=8)
    f = torch.from_numpy(I.random_sh_rhs(xs, 12, 8)).to(DEV)
    op = _operator(M, xs, ns)
    M.release_cached_memory()
    Hh, _, _, _ = _run(M, op, f)
    held = Hh.stats()["device_bytes"]
    assert held > 64 << 20
    del Hh                                        # blocks kept by the cache
    torch.cuda.synchronize()
    free_kept, _ = torch.cuda.mem_get_info()
    M.release_cached_memory()
    free_released, _ = torch.cuda.mem_get_info()
    assert free_released - free_kept >= held // 2

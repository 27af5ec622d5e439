"""mgm_knn_noalloc, the kNN entry point for callers that cannot allocate device memory, gives
the same neighbour lists as mgm_knn. Runs last (file name) so that a failure here does not hide
other tests when pytest stops at the first failure; passes alone or after the rest."""
import numpy as np
import pytest
import torch

from paper_2204_06154_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_matches_knn_two_calls_in_a_row():
    from paper_2204_06154_gb300 import mgm as M
    dev = "cuda:0"
    # first call: stencils of an icosahedral sphere (many tied distances); second call: a
    # different, larger cloud with separate query points, reusing the same static scratch
    x1, _ = I.icosahedral_sphere(5)
    x2, _ = I.fibonacci_sphere(60001, jitter=0.2, seed=4)
    q2, _ = I.fibonacci_sphere(20000, jitter=0.2, seed=5)
    cases = [(x1, x1, 30, True), (x2, q2, 3, False)]
    for data, query, k, sf in cases:
        d = torch.from_numpy(data).to(dev)
        q = d if sf else torch.from_numpy(query).to(dev)
        ref = M.knn(d, q, k, self_first=sf)
        got = M.knn_noalloc(d, q, k, self_first=sf)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
    # and again on the first case, after the scratch holds the second case's grid
    d = torch.from_numpy(x1).to(dev)
    assert torch.equal(M.knn_noalloc(d, None, 30, self_first=True), M.knn(d, None, 30, self_first=True))


def test_noalloc_rejects_sizes_above_the_limit():
    from paper_2204_06154_gb300 import mgm as M
    n = 262144 + 1
    d = torch.zeros((n, 3), dtype=torch.float64, device="cuda:0")
    d[:, 0] = torch.arange(n, dtype=torch.float64, device="cuda:0")
    with pytest.raises(M.MGMError) as e:
        M.knn_noalloc(d, None, 4, self_first=True)
    assert e.value.status == 8 and "maximum" in str(e.value)


def test_noalloc_binding_checks_the_output_tensor():
    """The entry point writes nq * k int32 values through `out`: the binding refuses a tensor of
    another shape, type or device before the call."""
    from paper_2204_06154_gb300 import mgm as M
    x, _ = I.icosahedral_sphere(3)
    d = torch.from_numpy(x).to("cuda:0")
    n = d.shape[0]
    for bad in (torch.empty((n, 7), dtype=torch.int32, device="cuda:0"),
                torch.empty((n, 8), dtype=torch.int64, device="cuda:0"),
                torch.empty((8, n), dtype=torch.int32, device="cuda:0").t(),
                torch.empty((n, 8), dtype=torch.int32)):
        with pytest.raises(ValueError):
            M.knn_noalloc(d, None, 8, self_first=True, out=bad)
    out = torch.empty((n, 8), dtype=torch.int32, device="cuda:0")
    assert M.knn_noalloc(d, None, 8, self_first=True, out=out) is out
    assert torch.equal(out, M.knn(d, None, 8, self_first=True))

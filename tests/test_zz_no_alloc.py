"""dt_order_noalloc: the spatial order (Moore keys, BRIO rounds, insertion permutation) computed
without allocating device memory.

Some callers cannot call cudaMalloc: code that runs while a stream is captured into a CUDA
graph, hosts whose device memory all belongs to another allocator, and latency-bound paths that
cannot pay for cudaMalloc's implicit synchronisation. This entry point serves them from one
file-scope device array. It must give exactly the keys, permutation and rounds of the ordinary
(allocating) path, on two calls in a row that reuse that array.
"""
import ctypes

import numpy as np
import pytest

from paper_1805_08831_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1805_08831_gb300 as dt  # noqa: E402


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def order_without_allocation(x, seed):
    n = len(x)
    xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    rounds = torch.empty(n, dtype=torch.uint8, device="cuda")
    rc = dt.lib().dt_order_noalloc(_ptr(xt), n, seed, _ptr(keys), _ptr(perm), _ptr(rounds), None)
    return (rc, keys.cpu().numpy().view(np.uint64), perm.cpu().numpy().view(np.uint32),
            rounds.cpu().numpy())


def order_with_allocation(x, seed):
    with dt.Triangulation(seed=seed) as t:
        t.insert(torch.from_numpy(np.ascontiguousarray(x)).cuda())
        return t.order(len(x))


def test_order_without_allocation_matches_the_allocating_path_twice():
    for call, (n, seed) in enumerate([(50000, 3), (120001, 9)]):
        x = synth.uniform_cube(n, 40 + call)
        x[10:20] = x[:10]  # duplicates must not disturb the order
        rc, keys, perm, rounds = order_without_allocation(x, seed)
        assert rc == dt.DT_OK
        ref_keys, ref_perm, ref_rounds = order_with_allocation(x, seed)
        assert np.array_equal(keys, ref_keys)
        assert np.array_equal(perm, ref_perm)
        assert np.array_equal(rounds, ref_rounds)


def test_order_without_allocation_rejects_sizes_over_its_limit():
    n = dt.lib() and 262144 + 1
    xt = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(8, dtype=torch.int64, device="cuda")
    rc = dt.lib().dt_order_noalloc(_ptr(xt), n, 0, _ptr(out), _ptr(out), _ptr(out), None)
    assert rc == dt.DT_EINVAL

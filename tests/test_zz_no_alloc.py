"""dt_order_noalloc: the spatial order (Moore keys, BRIO rounds, insertion permutation) computed
without allocating device memory.

Some callers cannot call cudaMalloc: hosts whose device memory all belongs to another allocator
(a framework's caching pool or a fixed arena), and code under a device-memory budget that a new
allocation could break. This entry point serves them from one file-scope device array. It must
give exactly the keys, permutation and rounds of the ordinary (allocating) path, on two calls in
a row that reuse that array, and leave the device's free memory unchanged.
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

DT_NOALLOC_MAX_POINTS = 262144  # the limit include/dt.h declares for dt_order_noalloc


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def order_with_allocation(x, seed):
    with dt.Triangulation(seed=seed) as t:
        t.insert(torch.from_numpy(np.ascontiguousarray(x)).cuda())
        return t.order(len(x))


def test_order_without_allocation_matches_the_allocating_path_twice():
    # a first call loads the library's kernels and its scratch array (lazy module loading
    # allocates device memory for code once); the two measured calls after it allocate nothing
    w = torch.from_numpy(synth.uniform_cube(1000, 1)).cuda()
    wk = torch.empty(1000, dtype=torch.int64, device="cuda")
    wp = torch.empty(1000, dtype=torch.int32, device="cuda")
    wr = torch.empty(1000, dtype=torch.uint8, device="cuda")
    assert dt.lib().dt_order_noalloc(_ptr(w), 1000, 1, _ptr(wk), _ptr(wp), _ptr(wr), None) == dt.DT_OK
    for call, (n, seed) in enumerate([(50000, 3), (120001, 9)]):
        x = synth.uniform_cube(n, 40 + call)
        x[10:20] = x[:10]  # duplicates must not disturb the order
        xt = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        keys_t = torch.empty(n, dtype=torch.int64, device="cuda")
        perm_t = torch.empty(n, dtype=torch.int32, device="cuda")
        rounds_t = torch.empty(n, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        rc = dt.lib().dt_order_noalloc(_ptr(xt), n, seed, _ptr(keys_t), _ptr(perm_t), _ptr(rounds_t), None)
        free_after = torch.cuda.mem_get_info()[0]
        assert rc == dt.DT_OK
        assert free_after == free_before  # nothing was allocated on the device
        keys = keys_t.cpu().numpy().view(np.uint64)
        perm = perm_t.cpu().numpy().view(np.uint32)
        rounds = rounds_t.cpu().numpy()
        ref_keys, ref_perm, ref_rounds = order_with_allocation(x, seed)
        assert np.array_equal(keys, ref_keys)
        assert np.array_equal(perm, ref_perm)
        assert np.array_equal(rounds, ref_rounds)


def test_order_without_allocation_rejects_sizes_over_its_limit():
    n = DT_NOALLOC_MAX_POINTS + 1
    xt = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(8, dtype=torch.int64, device="cuda")
    rc = dt.lib().dt_order_noalloc(_ptr(xt), n, 0, _ptr(out), _ptr(out), _ptr(out), None)
    assert rc == dt.DT_EINVAL

"""rogs_sort_pairs_noalloc: the context-free radix sort whose scratch lives in
a fixed device array of the library, for callers that cannot allocate device
memory where they sort (and so cannot create a rogs_ctx).

Called through the C-ABI with ctypes and compared with rogs_sort_pairs (the
context-based entry point) on two calls in a row, so that the second call
runs on scratch the first one left behind.  Sorting is integer work: the
results must be bit-identical.  This file is named so that pytest collects it
last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_PAIRS = 1048576   # ROGS_NOALLOC_MAX_PAIRS


@pytest.fixture(scope="module")
def libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import render, rogs
    lib = rogs.lib()
    fn = lib.rogs_sort_pairs_noalloc
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    rr = render.Renderer(0, record_capacity=1024, pair_capacity=MAX_PAIRS)
    return fn, rr, rogs


def _keys(n, bits, seed):
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 1 << bits, size=n, dtype=np.uint64).astype(np.uint32)
    k[: n // 4] = k[n // 4: 2 * (n // 4)]      # plenty of equal keys: stability matters
    return k


def _noalloc(fn, keys, vals, bits):
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    s = torch.cuda.current_stream()
    st = fn(C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()), keys.numel(), bits,
            C.c_void_p(ko.data_ptr()), C.c_void_p(vo.data_ptr()), C.c_void_p(s.cuda_stream))
    return st, ko, vo


def test_noalloc_sort_matches_context_sort_on_two_calls(libs):
    fn, rr, rogs = libs
    cases = [(300_007, 32, 1), (MAX_PAIRS, 18, 2)]     # second call: other size, other key width
    for n, bits, seed in cases:
        keys = torch.as_tensor(_keys(n, bits, seed).view(np.int32), device="cuda")
        vals = torch.arange(n, dtype=torch.int32, device="cuda")
        st, ko, vo = _noalloc(fn, keys, vals, bits)
        assert st == rogs.ROGS_OK
        kr, vr = rr.sort_pairs(keys, vals, bits)
        torch.cuda.synchronize()
        assert torch.equal(ko, kr) and torch.equal(vo, vr)
        # and against the definition: a stable sort by key
        order = np.argsort(keys.cpu().numpy().view(np.uint32), kind="stable")
        np.testing.assert_array_equal(vo.cpu().numpy(), order.astype(np.int32))


def test_noalloc_rejects_oversize_and_bad_arguments(libs):
    fn, rr, rogs = libs
    small = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = C.c_void_p(small.data_ptr())
    # rejected on the host, before any launch
    assert fn(p, p, MAX_PAIRS + 1, 32, p, p, s) == rogs.ROGS_ERR_CAPACITY
    assert fn(p, p, -1, 32, p, p, s) == rogs.ROGS_ERR_INVALID
    assert fn(p, p, 4, 33, p, p, s) == rogs.ROGS_ERR_INVALID
    assert fn(None, p, 4, 32, p, p, s) == rogs.ROGS_ERR_INVALID
    assert fn(p, p, 0, 32, p, p, s) == rogs.ROGS_OK

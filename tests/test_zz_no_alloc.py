"""The allocation-free sort entry point (ngs_sort_pairs_static) gives the same
result as the context-based ngs_sort_pairs.

It exists for callers that cannot allocate device memory where they sort: its
scratch is a fixed device array inside the library rather than memory from
cudaMalloc. The test calls it directly through the C ABI, twice in a row with
different inputs (the array keeps the previous call's contents, which must not
leak into the next result), and checks the size limit."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _keys(rng, n, kb):
    if kb == 4:
        return rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32).view(np.int32)
    return rng.integers(0, 2 ** 63, n, dtype=np.uint64).view(np.int64)


def test_static_scratch_sort_matches_context_sort():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_15186_gb300 import Renderer, _lib
    L = _lib.load()
    R = Renderer(device=0, cut_capacity=1 << 16, record_capacity=1 << 16, pair_capacity=1 << 20)
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    rng = np.random.default_rng(2024)
    # two calls in a row, different sizes, key widths and bit ranges
    for n, kb, b0, b1 in [(300_001, 4, 0, 24), (524_288, 8, 3, 61)]:   # 3 and 8 passes
        k = _keys(rng, n, kb)
        v = np.arange(n, dtype=np.int32)
        k1, v1 = torch.from_numpy(k.copy()).cuda(), torch.from_numpy(v.copy()).cuda()
        k2, v2 = k1.clone(), v1.clone()
        st = L.ngs_sort_pairs_static(C.c_void_p(k1.data_ptr()), C.c_void_p(v1.data_ptr()), n, kb,
                                     b0, b1, sp)
        assert st == 0, _lib.STATUS_NAMES.get(st, st)
        R.sort_pairs(k2, v2, b0, b1, stream=stream)
        torch.cuda.synchronize()
        assert torch.equal(k1, k2) and torch.equal(v1, v2)
        # and both equal numpy's stable sort on the same digits
        ku = k.view(np.uint32 if kb == 4 else np.uint64).astype(np.uint64)
        dig = (ku >> np.uint64(b0)) & np.uint64((1 << (b1 - b0)) - 1)
        assert np.array_equal(v1.cpu().numpy(), np.argsort(dig, kind="stable").astype(np.int32))
    # one pair beyond the fixed maximum is rejected before any work is queued
    big = torch.zeros(524_289, dtype=torch.int32, device="cuda")
    st = L.ngs_sort_pairs_static(C.c_void_p(big.data_ptr()), C.c_void_p(big.data_ptr()),
                                 524_289, 4, 0, 32, sp)
    assert st == 4  # NGS_ERR_CAPACITY
    R.close()

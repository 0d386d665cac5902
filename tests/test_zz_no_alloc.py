"""The allocation-free sort entry point (ngs_sort_pairs_static) gives the same
result as the context-based ngs_sort_pairs.

It exists for callers that cannot allocate device memory where they sort: an
application whose own pool owns all device memory, a loop in which a
cudaMalloc or cudaFree would synchronise the device, or code that has no
renderer context at all. Its scratch is a fixed device array inside the
library rather than memory from cudaMalloc.

The test's first calls are made before any renderer context exists (the case
the entry point is for, including the first-use lookup of the array's device
address) and are checked against numpy's stable sort; two calls run back to
back with different inputs (the array keeps the previous call's contents,
which must not leak into the next result). Only then is a renderer created,
to check the same inputs against ngs_sort_pairs. The size limit and the
status query are checked too."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [(300_001, 4, 0, 24), (524_288, 8, 3, 61)]   # 3 and 8 digit passes


def _keys(rng, n, kb):
    if kb == 4:
        return rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32).view(np.int32)
    return rng.integers(0, 2 ** 63, n, dtype=np.uint64).view(np.int64)


def _stable_order(k, kb, b0, b1):
    ku = k.view(np.uint32 if kb == 4 else np.uint64).astype(np.uint64)
    dig = (ku >> np.uint64(b0)) & np.uint64((1 << (b1 - b0)) - 1)
    return np.argsort(dig, kind="stable").astype(np.int32)


def test_static_scratch_sort_matches_context_sort():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_15186_gb300 import _lib
    L = _lib.load()
    stream = torch.cuda.current_stream()
    sp = C.c_void_p(stream.cuda_stream)
    rng = np.random.default_rng(2024)
    inputs = [(_keys(rng, n, kb), kb, b0, b1) for n, kb, b0, b1 in CASES]
    # 1) no renderer context yet: two calls in a row against numpy's stable sort
    static_out = []
    for k, kb, b0, b1 in inputs:
        n = len(k)
        k1 = torch.from_numpy(k.copy()).cuda()
        v1 = torch.arange(n, dtype=torch.int32, device="cuda")
        st = L.ngs_sort_pairs_static(C.c_void_p(k1.data_ptr()), C.c_void_p(v1.data_ptr()), n,
                                     kb, b0, b1, sp)
        assert st == 0, _lib.STATUS_NAMES.get(st, st)
        torch.cuda.synchronize()
        order = _stable_order(k, kb, b0, b1)
        assert np.array_equal(v1.cpu().numpy(), order)
        assert np.array_equal(k1.cpu().numpy(), k[order])
        static_out.append((k1, v1))
    assert L.ngs_sort_pairs_static_status(sp) == 0   # no device wait gave up
    # 2) the context-based sort on the same inputs gives the same bits
    from paper_2603_15186_gb300 import Renderer
    R = Renderer(device=0, cut_capacity=1 << 16, record_capacity=1 << 16, pair_capacity=1 << 20)
    for (k, kb, b0, b1), (k1, v1) in zip(inputs, static_out):
        k2 = torch.from_numpy(k.copy()).cuda()
        v2 = torch.arange(len(k), dtype=torch.int32, device="cuda")
        R.sort_pairs(k2, v2, b0, b1, stream=stream)
        torch.cuda.synchronize()
        assert torch.equal(k1, k2) and torch.equal(v1, v2)
    # 3) one pair beyond the fixed maximum is rejected before any work is queued
    big = torch.zeros(524_289, dtype=torch.int32, device="cuda")
    st = L.ngs_sort_pairs_static(C.c_void_p(big.data_ptr()), C.c_void_p(big.data_ptr()),
                                 524_289, 4, 0, 32, sp)
    assert st == 4  # NGS_ERR_CAPACITY
    assert L.ngs_sort_pairs_static_status(sp) == 0
    R.close()

"""GPU: the continuous-batching serving loop. A request's image is the same
bits alone and mixed into batches with other agents' requests, matches the
oracle, and the loop really batches (fewer launches than requests)."""
import numpy as np
import pytest

import oracle as O
from scenegen import mixed_batch_cameras, walk_cameras
from tests.gpu_helpers import clear_tau, compare_image

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_serving_alone_equals_mixed(small_floor):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_15186_gb300 import Renderer, Server
    R = Renderer(device=0, cut_capacity=1 << 22, record_capacity=1 << 22, pair_capacity=1 << 24)
    R.load_scene(small_floor)
    probe = clear_tau(small_floor, walk_cameras(small_floor, 1, 9, 120, 90, fx=110.0, tau=3.0)[0])
    others = mixed_batch_cameras(small_floor, 48, seed=33, resolutions=((64, 48), (96, 72), (160, 120)),
                                 n_walkers=6)
    S = Server(R, lanes=2, max_cams=8)
    alone = torch.zeros((3, probe.height, probe.width), device="cuda")
    S.submit(probe, alone)
    S.wait_all()
    imgs = [torch.zeros((3, c.height, c.width), device="cuda") for c in others]
    mixed = torch.zeros_like(alone)
    tickets = []
    for i, (c, im) in enumerate(zip(others, imgs)):
        tickets.append(S.submit(c, im))
        if i == 20:
            tp = S.submit(probe, mixed)
    S.wait_all()
    st = S.stats()
    S.stop()
    assert st["completed"] == st["submitted"] == len(others) + 2 and st["failed"] == 0
    assert st["launches"] < st["submitted"]            # requests were batched together
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    assert torch.equal(alone, mixed)
    # every served image equals the same camera rendered alone by the renderer
    for c, im in list(zip(others, imgs))[::7]:
        ref = R.render([c])[0]
        assert torch.equal(ref, im)
    compare_image(alone.cpu().numpy(), O.render(small_floor, probe))
    R.close()


def test_pair_overflow_is_replanned_not_lost(small_floor):
    """A pair buffer too small for the planner's first estimate, forced on
    the host side (pairs-per-pixel estimate 1, a 2^18-pair buffer): the
    host-buffer render re-plans from the pair counts the device reported and
    redoes the batch, and the serving loop puts the overflowing launch's
    requests back in the queue instead of failing them. Every image equals
    its camera rendered alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_15186_gb300 import Renderer, Server
    cams = mixed_batch_cameras(small_floor, 24, seed=35, resolutions=((96, 72), (160, 120)),
                               n_walkers=4)
    ref = Renderer(device=0, cut_capacity=1 << 22, record_capacity=1 << 22, pair_capacity=1 << 24)
    ref.load_scene(small_floor)
    alone = [ref.render([c])[0].cpu().numpy() for c in cams]
    small = Renderer(device=0, cut_capacity=1 << 22, record_capacity=1 << 22,
                     pair_capacity=1 << 18)
    small.load_scene(small_floor)
    small.set_mode("batched")
    small.set_pairs_per_pixel(1)
    got = small.render_host(cams)
    st = small.stats()
    assert st["sub_batches"] > 1
    for a, b in zip(alone, got):
        assert np.array_equal(a, b)
    # serving: lanes start from the same low estimate and a small buffer
    srv = Renderer(device=0, cut_capacity=1 << 22, record_capacity=1 << 22, pair_capacity=1 << 24)
    srv.load_scene(small_floor)
    srv.set_pairs_per_pixel(1)
    S = Server(srv, lanes=2, max_cams=16, pair_budget=1 << 22, pairs_per_pixel=1.0,
               lane_pair_capacity=1 << 18)
    imgs = [torch.zeros((3, c.height, c.width), device="cuda") for c in cams]
    for c, im in zip(cams, imgs):
        S.submit(c, im)
    S.wait_all()
    sst = S.stats()
    S.stop()
    assert sst["completed"] == len(cams) and sst["failed"] == 0
    assert sst["requeued"] > 0
    for a, im in zip(alone, imgs):
        assert np.array_equal(a, im.cpu().numpy())
    for r in (ref, small, srv):
        r.close()


def test_render_host_contiguous_pinned_buffer(small_floor):
    """The host-buffer render writes into page-locked host memory directly
    (one pinned buffer holding every image) and copies into pageable arrays
    each sub-batch's images while the next sub-batches render; both equal the
    device render of the same cameras bit for bit, over several sub-batches
    and a graph replay."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes as C
    from paper_2603_15186_gb300 import Renderer
    from paper_2603_15186_gb300.renderer import camera_array
    cams = mixed_batch_cameras(small_floor, 24, seed=36, resolutions=((96, 72), (160, 120)),
                               n_walkers=4)
    R = Renderer(device=0, cut_capacity=1 << 22, record_capacity=1 << 22, pair_capacity=1 << 20)
    R.load_scene(small_floor)
    R.set_mode("batched")
    R.set_pairs_per_pixel(400)          # a high estimate: several sub-batches
    ref = [im.cpu().numpy() for im in R.render(cams)]
    assert R.stats()["sub_batches"] > 1
    sizes = [3 * c.width * c.height for c in cams]
    host = torch.full((sum(sizes),), -1.0, dtype=torch.float32).pin_memory()
    ptrs, off = [], 0
    for n in sizes:
        ptrs.append(C.c_void_p(host.data_ptr() + 4 * off))
        off += n
    for _ in range(2):                  # the second call replays the graph
        R.render_host_ptrs(camera_array(cams), len(cams), (C.c_void_p * len(cams))(*ptrs))
        off = 0
        for c, n, r in zip(cams, sizes, ref):
            got = host[off:off + n].numpy().reshape(3, c.height, c.width)
            assert np.array_equal(got, r)
            off += n
        host.fill_(-1.0)
    got = R.render_host(cams)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    # the plain per-view path writes into the pinned buffer the same way
    R.set_mode("plain")
    R.render_host_ptrs(camera_array(cams), len(cams), (C.c_void_p * len(cams))(*ptrs))
    off = 0
    for c, n, r in zip(cams, sizes, ref):
        assert np.array_equal(host[off:off + n].numpy().reshape(3, c.height, c.width), r)
        off += n
    R.close()

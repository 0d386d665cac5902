"""Comparison helpers for the GPU parity tests (the oracle is the reference)."""
import numpy as np

import oracle as O

PIXEL_TOL = 2e-3          # absolute, per channel
EDGE_DELTA_PX = 0.01      # rectangle edges this close to a tile boundary may differ


def clear_tau(scene, cam, step=1.0007, tries=50):
    """Nudges cam.tau (chosen by the oracle alone) until no cut decision lies
    within 1e-5 relative of it, so the float32 cut must match exactly."""
    for _ in range(tries):
        if cam.tau == 0.0 or O.select_cut(scene, cam)[1].sum() == 0:
            return cam
        cam.tau = float(cam.tau) * step
    raise AssertionError("no threshold-free tau found")


def compare_cut(gpu_ids, scene, cam):
    """GPU cut equals the oracle's on every node whose decision (or whose
    parent's) is not within 1e-5 relative of tau."""
    ids, near = O.select_cut(scene, cam)
    n = scene.n_nodes if hasattr(scene, "n_nodes") else len(scene.parent)
    a = np.zeros(n, bool)
    b = np.zeros(n, bool)
    a[np.asarray(gpu_ids, dtype=np.int64)] = True
    b[ids] = True
    bad = (a != b) & (near == 0)
    assert not bad.any(), f"{int(bad.sum())} cut decisions differ away from the threshold"
    assert np.all(np.diff(np.asarray(gpu_ids, np.int64)) > 0), "cut ids must ascend"
    return ids, near


def compare_image(got, ref, tol=PIXEL_TOL, max_flag_frac=0.02):
    """Every pixel the oracle does not flag as near-discontinuous is within
    ``tol`` per channel. Returns (max error, flagged fraction)."""
    got = np.asarray(got, dtype=np.float64)
    ok = ref.flags == 0
    err = np.abs(got - ref.image)
    emax = float(err[:, ok].max()) if ok.any() else 0.0
    frac = 1.0 - float(ok.mean())
    assert frac <= max_flag_frac, f"too many flagged pixels: {frac:.4f}"
    assert emax <= tol, f"max abs error {emax:.3e} > {tol} (worst at {np.unravel_index(np.argmax(np.where(ok[None], err, 0)), err.shape)})"
    return emax, frac


def uncertain_nodes(ref, tile):
    """Node ids whose support-box edges lie within EDGE_DELTA_PX of a tile
    boundary: their tile membership is a float32-vs-float64 coin toss."""
    pre = ref.pre
    tw, th = tile
    cand = (pre[:, O.PC.HX] > 0)
    u, v, hx, hy = pre[:, O.PC.U], pre[:, O.PC.V], pre[:, O.PC.HX], pre[:, O.PC.HY]

    def near(x, t):
        r = np.mod(x, t)
        return (r < EDGE_DELTA_PX) | (t - r < EDGE_DELTA_PX)
    unc = cand & (near(u - hx, tw) | near(u + hx, tw) | near(v - hy, th) | near(v + hy, th))
    return set(ref.ids[unc].tolist())


def compare_tile_lists(gpu_ranges, gpu_nodes, ref, tile):
    """Per tile, the GPU's node sequence equals the oracle's (tile, depth,
    node id) order once rectangle-edge coin tosses are removed from both."""
    unc = uncertain_nodes(ref, tile)
    n_tiles = len(ref.ranges)
    assert len(gpu_ranges) == n_tiles
    checked = 0
    for t in range(n_tiles):
        g = gpu_nodes[gpu_ranges[t, 0]:gpu_ranges[t, 1]].tolist()
        o = ref.ids[ref.vals[ref.ranges[t, 0]:ref.ranges[t, 1]]].tolist()
        if unc:
            g = [x for x in g if x not in unc]
            o = [x for x in o if x not in unc]
        assert g == o, f"tile {t}: lists differ (first mismatch at {next((i for i,(x,y) in enumerate(zip(g,o)) if x!=y), min(len(g),len(o)))})"
        checked += len(o)
    return checked, len(unc)


def oracle_on_gpu_cut(R, cut_scene, scene, cam, tile=(16, 16)):
    """Oracle render of the cut the GPU selects for ``cam``, once that cut is
    checked to equal the oracle's on every decision away from the tau
    threshold (where either choice is allowed). ``cut_scene`` holds the
    hierarchy, ``scene`` the attributes the oracle renders (for example the
    dequantised FP16 values). Large scenes nearly always have some node within
    1e-5 of tau, so this replaces nudging tau at full size."""
    ids, off = R.select_cut([cam])
    gpu = ids[: int(off[1].item())].cpu().numpy()
    compare_cut(gpu, cut_scene, cam)
    return O.render(scene, cam, tile=tile, ids=gpu.astype(np.int32))

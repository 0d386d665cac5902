"""Comparison helpers for the GPU parity tests (the oracle is the reference).

Where float32 may legitimately decide differently from the float64 oracle,
the allowance comes from the oracle's float32 error model (stated bounds on
the renderer's centre, conic, opacity, support and depth errors), not from a
fixed window:
- a pixel with a near-threshold decision (alpha vs 1/255, T (1 - alpha) vs
  1e-4, within the bound) must match one of the outcomes the oracle lists for
  the ways those decisions can go;
- a (Gaussian, tile) membership may differ where a support-box edge lies
  within its error bound of a tile boundary, and the near-plane cull where the
  float64 depth lies within its bound of the near plane;
- in the depth order checked against float64 depths, two neighbours may be
  swapped only where their float64 depths lie within the sum of their depth
  error bounds."""
import numpy as np

import oracle as O

PIXEL_TOL = 2e-3          # absolute, per channel
U32 = 2.0 ** -24
NEAR_Z = 0.2
# pixels whose near-threshold decisions have more outcomes than the oracle
# lists (MAX_OUTCOMES), or a decision whose error bound is too large to enumerate (over
# 2 log2 units), are not checked when they match none of the listed outcomes;
# at most this fraction of a view may be such
MAX_UNCHECKED_FRAC = 1e-4
MAX_OUTCOMES = 256


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


def compare_image(got, ref, tol=PIXEL_TOL):
    """Every pixel matches the oracle within ``tol`` per channel: the float64
    outcome where no decision was near threshold, else the nearest of the
    outcomes of its near-threshold decisions. Returns a dict: max error of the
    unflagged pixels, flagged fraction, max error of the flagged pixels
    against their nearest outcome, unchecked fraction."""
    got = np.asarray(got, dtype=np.float64)
    flagged = ref.flags != 0
    err = np.abs(got - ref.image)
    ok = ~flagged
    emax = float(err[:, ok].max()) if ok.any() else 0.0
    assert emax <= tol, (f"max abs error {emax:.3e} > {tol} (worst at "
                         f"{np.unravel_index(np.argmax(np.where(ok[None], err, 0)), err.shape)})")
    ys, xs = np.nonzero(flagged)
    eflag, unchecked = 0.0, 0
    if len(ys):
        pix = np.stack([xs, ys], 1)
        best, over = nearest_outcome(got, ref, pix)
        unchecked = int((over & (best > tol)).sum())
        fine = best[~over | (best <= tol)]
        eflag = float(fine.max()) if len(fine) else 0.0
        bad = ~over & (best > tol)
        assert not bad.any(), (f"{int(bad.sum())} flagged pixels match none of their outcomes "
                               f"within {tol} (worst {float(best[~over].max()):.3e} at "
                               f"{tuple(pix[np.argmax(np.where(~over, best, -1))])})")
    n = flagged.size
    assert unchecked <= MAX_UNCHECKED_FRAC * n + 1, f"{unchecked} pixels left unchecked"
    return {"max_abs_err": emax, "flagged_frac": float(flagged.mean()),
            "flagged_max_err_vs_nearest_outcome": eflag, "unchecked_frac": unchecked / n}


def nearest_outcome(got, ref, pix, max_out=MAX_OUTCOMES, chunk=16384):
    """For the pixels ``pix`` ((n, 2) integer (x, y)) of a GPU image: the
    largest channel error against the nearest of the oracle's outcomes of the
    pixel's near-threshold decisions, and whether the pixel had more outcomes
    than listed or a decision too uncertain to enumerate."""
    best = np.empty(len(pix))
    over = np.empty(len(pix), dtype=bool)
    for s0 in range(0, len(pix), chunk):
        pc = pix[s0:s0 + chunk]
        alts, cnt = O.alternatives(ref.pre, ref.vals, ref.ranges, ref.cam, pc, tile=ref.tile,
                                   max_out=max_out)
        g = got[:, pc[:, 1], pc[:, 0]].T                     # [n, 3]
        d = np.abs(alts - g[:, None, :]).max(axis=2)          # [n, max_out]
        m = np.arange(max_out)[None, :] < np.minimum(np.abs(cnt), max_out)[:, None]
        best[s0:s0 + chunk] = np.where(m, d, np.inf).min(axis=1)
        over[s0:s0 + chunk] = (cnt > max_out) | (cnt < 0)
    return best, over


def uncertain_nodes(ref, tile):
    """Node ids whose tile membership a float32 renderer may decide
    differently: a support-box edge within its error bound (centre +
    half-width + the rounding of the edge) of a tile boundary. (The oracle's
    near-plane cull is taken on the renderer's float32 depth; the float64
    reading of it is checked by compare_tile_order_f64.)"""
    pre = ref.pre
    tw, th = tile
    cand = (pre[:, O.PC.HX] > 0)
    u, v, hx, hy = pre[:, O.PC.U], pre[:, O.PC.V], pre[:, O.PC.HX], pre[:, O.PC.HY]
    ex = pre[:, O.PC.EU] + pre[:, O.PC.EHX]
    ey = pre[:, O.PC.EV] + pre[:, O.PC.EHY]

    def near(x, t, e):
        e = e + 2 * U32 * np.abs(x)
        r = np.mod(x, t)
        return (r <= e) | (t - r <= e)
    unc = cand & (near(u - hx, tw, ex) | near(u + hx, tw, ex) | near(v - hy, th, ey) |
                  near(v + hy, th, ey))
    return set(ref.ids[unc].tolist())


def depth_bounds(cam, mu):
    """float64 view depths of float32 means and the bound 6 u sum_k |R_2k d_k|
    on a float32 evaluation's error (a three-term dot product of rounded
    differences, any operation order)."""
    R = np.asarray(cam.R_wc, np.float32).astype(np.float64)
    c = np.asarray(cam.pos, np.float32).astype(np.float64)
    d = np.asarray(mu, np.float32).astype(np.float64) - c
    z = d @ R[2]
    e = 6.0 * U32 * (np.abs(d * R[2][None, :]).sum(axis=1))
    return z, e


def compare_tile_lists(gpu_ranges, gpu_nodes, ref, tile):
    """Per tile, the GPU's node sequence equals the oracle's (tile, depth,
    node id) order once the uncertain memberships are removed from both."""
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


def compare_tile_order_f64(gpu_ranges, gpu_nodes, pos, cam):
    """The GPU's tile lists are in front-to-back order of the float64 view
    depth: every two neighbours (a before b) have z64(a) <= z64(b), except a
    swap where the two depths lie within the sum of their float32 error bounds
    (about 1e-6 of the depth near the optical axis, more for Gaussians far off
    axis close to the near plane). ``pos``: the scene's float32 means.
    Returns (neighbour pairs checked, pairs that relied on the allowance,
    largest allowance relative to the depth)."""
    pairs = 0
    swaps = 0
    worst_rel = 0.0
    for t in range(len(gpu_ranges)):
        nodes = np.asarray(gpu_nodes[gpu_ranges[t, 0]:gpu_ranges[t, 1]], np.int64)
        if len(nodes) < 2:
            continue
        z, e = depth_bounds(cam, pos[nodes])
        # in front of the near plane in float64, up to the depth's bound
        assert np.all(z > NEAR_Z - e), f"tile {t}: a listed Gaussian lies behind the near plane"
        dz = z[:-1] - z[1:]                  # > 0 means the pair is out of float64 order
        allow = e[:-1] + e[1:]
        bad = dz > allow
        assert not bad.any(), (f"tile {t}: neighbours out of float64 depth order by "
                               f"{float(dz[bad].max()):.3e} (allowance {float(allow[bad][0]):.3e})")
        inv = dz > 0
        swaps += int(inv.sum())
        pairs += len(dz)
        worst_rel = max(worst_rel, float((allow / np.maximum(z[1:], 1e-30)).max()))
    return pairs, swaps, worst_rel


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

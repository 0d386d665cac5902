"""Pins of the oracle's float32 error model (the bounds that decide which
decisions a float32 renderer may take differently from the float64 oracle)
and of the alternatives it enumerates for them. CPU only.

- The float32 view depth of the sort key and near-plane cull lies within
  6 u sum_k |R_2k d_k| of the float64 depth (u = 2^-24): the bound of a
  three-term dot product of rounded differences, whatever the operation order.
- The per-Gaussian bounds of the preprocess (centre, the entries b and c of
  the 2D covariance and its determinant, log2 opacity, support half-widths)
  and the per-pixel exponent bound (the factored conic at the pixel) hold for
  an independent float32 evaluation of the same stable form (numpy float32,
  matrix products in numpy's order), over random Gaussians and cameras that
  include thin, off-axis and near-plane cases, and Gaussians close to the
  camera plane far off the axis.
- The alternatives of a pixel are the closed-form outcomes of its
  near-threshold decisions: a Gaussian at alpha = 1/255 taken or skipped, and a
  stop decision at T (1 - alpha) = 1e-4 taken or not."""
import math

import numpy as np
import pytest

import oracle as O
from scenegen import build_hierarchy, look_camera

U32 = 2.0 ** -24
LOG2E = 1.4426950408889634


def _cams(rng, n):
    out = []
    for _ in range(n):
        w, h = [(320, 240), (640, 480), (1280, 720)][rng.integers(3)]
        out.append(look_camera(rng.uniform(-3, 3, 3), rng.uniform(-math.pi, math.pi), w, h,
                               pitch=rng.uniform(-0.6, 0.6)))
    return out


def test_depth_f32_within_the_float64_bound():
    rng = np.random.default_rng(5)
    worst = 0.0
    for cam in _cams(rng, 40):
        R = cam.R_wc.astype(np.float64)
        c = cam.pos.astype(np.float64)
        # means in front, off axis, and on the camera plane (cancellation)
        mus = np.concatenate([
            c + rng.normal(0, 4, (60, 3)),
            c + R.T @ np.array([1.0, 0.0, 0.0]) * rng.uniform(1, 30, (20, 1)),
            c + rng.uniform(-1e3, 1e3, (20, 3))]).astype(np.float32)
        for mu in mus:
            d = mu.astype(np.float64) - c.astype(np.float32).astype(np.float64)
            z64 = O.view_depth64(mu, cam)
            assert z64 == pytest.approx(float(R[2] @ d), rel=1e-12, abs=1e-12)
            bound = 6.0 * U32 * float(np.abs(R[2] * d).sum())
            err = abs(float(O.depth_f32(mu, cam)) - z64)
            assert err <= bound, (mu, err, bound)
            if bound > 0:
                worst = max(worst, err / bound)
    assert worst > 0.01   # the bound is not vacuous: rounding shows up


def _f32_preprocess(cam, mu, quat, log_scale, opac):
    """An independent float32 evaluation (numpy float32 arrays, numpy's own
    operation order) of the numerically stable form the error model
    describes: the view vector (rounded from float64 where the depth cancels,
    as a compensated product would give), the projections of the Gaussian's
    scaled axes, the determinant by Cauchy-Binet from the normal of the two
    screen rows, and the factored conic."""
    f = np.float32
    R = cam.R_wc.astype(f)
    d = (mu.astype(f) - cam.pos.astype(f)).astype(f)
    t = (R @ d).astype(f)
    if float(np.abs(R[2] * d).sum()) > 8.0 * float(t[2]):
        d64 = mu.astype(np.float64) - cam.pos.astype(f).astype(np.float64)
        t = (R.astype(np.float64) @ d64).astype(f)
    tx, ty, tz = t
    q = quat.astype(f) / f(np.sqrt((quat.astype(f) ** 2).sum()))
    w, x, y, z = q
    Rq = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                   [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                   [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]], dtype=f)
    sk = np.exp(log_scale.astype(f)).astype(f)
    fx, fy = f(cam.fx), f(cam.fy)
    ax, ay = fx / tz, fy / tz
    bx, by = -fx * tx / (tz * tz), -fy * ty / (tz * tz)
    T = np.stack([ax * R[0] + bx * R[2], ay * R[1] + by * R[2]]).astype(f)
    qm = ((T @ Rq) * sk[None, :]).astype(f)              # s_k (T_r . axis k)
    ap, cp = f((qm[0] ** 2).sum()), f((qm[1] ** 2).sum())
    b = f((qm[0] * qm[1]).sum())
    R64 = cam.R_wc.astype(f).astype(np.float64)
    X = [np.cross(R64[0], R64[1]).astype(f), np.cross(R64[0], R64[2]).astype(f),
         np.cross(R64[2], R64[1]).astype(f)]
    n = (f(ax * ay) * X[0] + f(ax * by) * X[1] + f(bx * ay) * X[2]).astype(f)
    g = (n @ Rq).astype(f) * np.array([sk[1] * sk[2], sk[0] * sk[2], sk[0] * sk[1]], dtype=f)
    a, c = ap + f(0.3), cp + f(0.3)
    det = f((g * g).sum()) + f(0.3) * (ap + cp) + f(0.09)
    k = f(0.5 * LOG2E)
    F3 = np.sqrt(k / c)
    F1 = F3 * c / np.sqrt(det)
    F2 = -b * F3 / np.sqrt(det)
    u = fx * tx / tz + f(cam.cx)
    v = fy * ty / tz + f(cam.cy)
    L = np.log2(f(opac)).astype(f)
    K = f(2) * np.log(f(255) * f(opac)).astype(f)
    hx = np.sqrt(K * a) + f(1 / 64)
    hy = np.sqrt(K * c) + f(1 / 64)
    return dict(u=u, v=v, b=b, c=c, det=det, F1=F1, F2=F2, F3=F3, L=L, hx=hx, hy=hy)


def test_error_model_bounds_a_float32_preprocess():
    rng = np.random.default_rng(11)
    checked, far_checked, ratio = 0, 0, []
    for cam in _cams(rng, 12):
        n = 300
        R = cam.R_wc.astype(np.float64)
        # means in the view volume, some near the plane z = 0.3, and a fifth just
        # in front of the near plane far off the axis (|x / z| up to 150: large
        # elongated footprints whose centres lie far off screen)
        z = np.concatenate([rng.uniform(0.25, 0.6, n // 3), rng.uniform(0.6, 25, n - n // 3)])
        xn = rng.uniform(-0.9, 0.9, n) * cam.width / (2 * cam.fx)
        yn = rng.uniform(-0.9, 0.9, n) * cam.height / (2 * cam.fy)
        far = slice(n // 5, 2 * n // 5)
        z[far] = rng.uniform(0.21, 0.4, n // 5)
        xn[far] = rng.choice([-1.0, 1.0], n // 5) * rng.uniform(10.0, 150.0, n // 5)
        mu = (cam.pos + (np.stack([xn * z, yn * z, z], 1) @ R)).astype(np.float32)
        quat = rng.normal(size=(n, 4)).astype(np.float32)
        ls = rng.normal(-3.5, 0.8, (n, 3)).astype(np.float32)
        ls[: n // 5, 0] = -9.0                       # thin (near-singular) Gaussians
        ls[far] = rng.normal(-1.5, 0.5, (n // 5, 3))  # large, so that they reach the screen
        opac = rng.uniform(0.02, 0.99, n).astype(np.float32)
        sc = build_hierarchy(mu, quat, ls, opac, np.zeros((n, 16, 3), np.float32))
        leaves = np.flatnonzero(sc.child_count == 0).astype(np.int32)
        pre, _, _ = O.preprocess(sc, cam, leaves)
        for row, g in zip(pre, leaves):
            if row[O.PC.VISIBLE] == 0:
                continue
            f = _f32_preprocess(cam, sc.pos[g], sc.quat[g], sc.log_scale[g], sc.opacity[g])
            det64 = row[O.PC.COV_A] * row[O.PC.COV_C] - row[O.PC.COV_B] ** 2
            want = dict(u=row[O.PC.U], v=row[O.PC.V], b=row[O.PC.COV_B], c=row[O.PC.COV_C],
                        det=det64, L=math.log2(row[O.PC.OPACITY]), hx=row[O.PC.HX],
                        hy=row[O.PC.HY])
            bound = dict(u=row[O.PC.EU], v=row[O.PC.EV], b=row[O.PC.EB], c=row[O.PC.EC],
                         det=row[O.PC.EDET] * det64, L=row[O.PC.EQL], hx=row[O.PC.EHX],
                         hy=row[O.PC.EHY])
            for k in want:
                err = abs(float(f[k]) - want[k])
                assert err <= bound[k], (k, g, err, bound[k])
                if bound[k] > 0:
                    ratio.append(err / bound[k])
            # the exponent at pixels on the alpha = 1/255 ring and inside it
            for s_ in (0.3, 0.97, 1.0, 1.03):
                ang = rng.uniform(0, 2 * math.pi)
                Kq = 2 * math.log(255 * row[O.PC.OPACITY]) * s_
                # a point at d^T conic d = Kq along direction ang
                e = np.array([math.cos(ang), math.sin(ang)])
                Q = np.array([[row[O.PC.CONIC_A], row[O.PC.CONIC_B]],
                              [row[O.PC.CONIC_B], row[O.PC.CONIC_C]]])
                r = math.sqrt(Kq / float(e @ Q @ e))
                px, py = np.float32(row[O.PC.U] + r * e[0]), np.float32(row[O.PC.V] + r * e[1])
                dx64, dy64 = float(px) - row[O.PC.U], float(py) - row[O.PC.V]
                q64 = math.log2(row[O.PC.OPACITY]) - 0.5 * LOG2E * (
                    row[O.PC.CONIC_A] * dx64 ** 2 + 2 * row[O.PC.CONIC_B] * dx64 * dy64 +
                    row[O.PC.CONIC_C] * dy64 ** 2)
                dx, dy = np.float32(px - f["u"]), np.float32(py - f["v"])
                p32 = f["F1"] * dx + f["F2"] * dy
                e32 = f["F3"] * dy
                q32 = f["L"] - p32 * p32 - e32 * e32
                eq = O.exponent_error(row, dx64, dy64)
                assert abs(float(q32) - q64) <= eq, (g, float(q32), q64, eq)
                ratio.append(abs(float(q32) - q64) / eq)
            checked += 1
            far_checked += int(abs(row[O.PC.U] - cam.cx) > 4 * cam.width)
    assert checked > 1500 and far_checked > 50
    # rounding is visible against the bounds (they are not vacuous)
    assert max(ratio) > 0.02


def _aim_camera():
    return look_camera((0.3, -0.2, 1.1), math.radians(30), 32, 24, fx=100.0,
                       pitch=math.radians(10))


def _world_at_pixel(cam, i, j, depth):
    t = np.array([(i + 0.5 - cam.cx) * depth / cam.fx, (j + 0.5 - cam.cy) * depth / cam.fy, depth])
    return cam.pos.astype(np.float64) + cam.R_wc.astype(np.float64).T @ t


def _dc_for_colour(c):
    C0 = 0.5 / math.sqrt(math.pi)
    sh = np.zeros((16, 3), np.float32)
    sh[0] = (np.asarray(c) - 0.5) / C0
    return sh


def _stack(cam, i, j, opacities, colours, scale=0.005):
    n = len(opacities)
    mus = [_world_at_pixel(cam, i, j, 1.0 + 0.25 * k) for k in range(n)]
    sc = build_hierarchy(np.asarray(mus, np.float32), np.tile(np.float32([1, 0, 0, 0]), (n, 1)),
                         np.full((n, 3), math.log(scale), np.float32),
                         np.asarray(opacities, np.float32),
                         np.asarray([_dc_for_colour(c) for c in colours], np.float32))
    r = O.render(sc, cam)
    order = np.argsort(r.pre[:, O.PC.DEPTH])
    return sc, r, order


def _alpha_at(row, px, py):
    dx, dy = px - row[O.PC.U], py - row[O.PC.V]
    p = -0.5 * (row[O.PC.CONIC_A] * dx * dx + row[O.PC.CONIC_C] * dy * dy) - row[O.PC.CONIC_B] * dx * dy
    return row[O.PC.OPACITY] * math.exp(p)


def test_alternatives_of_a_gaussian_at_the_alpha_threshold():
    """Front Gaussian with alpha just above 1/255 (inside the float32 window),
    back Gaussian with o = 0.5: the outcomes are 'front taken' and 'front
    skipped', in closed form."""
    cam = _aim_camera()
    o1 = np.float32(1.0 / 255.0 * (1.0 + 1e-6))
    c1, c2 = [0.9, 0.2, 0.4], [0.1, 0.7, 0.3]
    sc, r, order = _stack(cam, 10, 8, [o1, 0.5], [c1, c2])
    assert r.flags[8, 10] == 1 and r.flags[0, 0] == 0
    rows = r.pre[order]
    a1, a2 = _alpha_at(rows[0], 10.5, 8.5), _alpha_at(rows[1], 10.5, 8.5)
    assert abs(math.log2(a1) - math.log2(1 / 255)) <= O.exponent_error(
        rows[0], 10.5 - rows[0][O.PC.U], 8.5 - rows[0][O.PC.V])
    col = rows[:, [O.PC.R, O.PC.G, O.PC.B]]
    taken = a1 * col[0] + (1 - a1) * a2 * col[1]
    skipped = a2 * col[1]
    out, cnt = O.alternatives(r.pre, r.vals, r.ranges, cam, [(10, 8)], tile=r.tile)
    assert cnt[0] == 2
    got = np.array(sorted(tuple(x) for x in out[0, :2]))
    want = np.array(sorted([tuple(taken), tuple(skipped)]))
    np.testing.assert_allclose(got, want, rtol=1e-12)
    # the image is the float64 decision's outcome
    np.testing.assert_allclose(r.image[:, 8, 10], taken if a1 >= 1 / 255 else skipped,
                               rtol=1e-12)
    # an unflagged pixel has exactly one outcome: the image
    out, cnt = O.alternatives(r.pre, r.vals, r.ranges, cam, [(3, 3)], tile=r.tile)
    assert cnt[0] == 1
    np.testing.assert_allclose(out[0, 0], r.image[:, 3, 3], rtol=0, atol=0)


def test_alternatives_of_a_stop_at_the_transmittance_threshold():
    """Five layers of alpha 0.8 leave T5 = 0.2^5; a sixth with 1 - o6 =
    1e-4 / T5 puts T (1 - alpha) on the 1e-4 stop threshold: outcomes 'stop
    before the sixth' and 'blend the sixth' (a seventh layer of 0.8 then
    stops), in closed form."""
    cam = _aim_camera()
    a = float(np.float32(0.8))
    T5 = (1 - a) ** 5
    o6 = np.float32(1.0 - 1e-4 / T5)
    rng = np.random.default_rng(3)
    cols = rng.uniform(0.1, 0.9, (7, 3))
    sc, r, order = _stack(cam, 16, 12, [0.8] * 5 + [o6, 0.8], cols)
    rows = r.pre[order]
    al = [_alpha_at(rw, 16.5, 12.5) for rw in rows]
    col = rows[:, [O.PC.R, O.PC.G, O.PC.B]]
    T, C5 = 1.0, np.zeros(3)
    for k in range(5):
        C5 = C5 + al[k] * T * col[k]
        T *= 1 - al[k]
    C6 = C5 + al[5] * T * col[5]
    assert abs(T * (1 - al[5]) - 1e-4) <= 1e-4 * 1e-5       # on the threshold
    assert r.flags[12, 16] == 1
    out, cnt = O.alternatives(r.pre, r.vals, r.ranges, cam, [(16, 12)], tile=r.tile)
    assert cnt[0] == 2
    got = sorted([tuple(x) for x in out[0, :2]])
    want = sorted([tuple(C5), tuple(C6)])
    np.testing.assert_allclose(np.array(got), np.array(want), rtol=1e-10)

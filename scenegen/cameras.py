"""Seeded camera poses: fixed views, collision-free walks at robot height, and
mixed-resolution camera batches."""
from __future__ import annotations

import math
from typing import List, Sequence

import numpy as np

from .scene import Camera, Scene, wall_segments


def yaw_rotation(yaw: float, pitch: float = 0.0) -> np.ndarray:
    """World->camera rotation (OpenCV frame) for a camera whose forward axis has
    heading ``yaw`` (radians from +x towards +y) and elevation ``pitch``; world z
    is up, so camera y (down) is -z for a level camera."""
    cp, sp = math.cos(pitch), math.sin(pitch)
    fwd = np.array([math.cos(yaw) * cp, math.sin(yaw) * cp, sp])
    right = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    down = np.cross(fwd, right)
    return np.stack([right, down, fwd]).astype(np.float32)


def look_camera(pos, yaw, width, height, fx=None, tau=0.0, pitch=0.0) -> Camera:
    """Centred pinhole camera; fx = fy = 0.9375 * width unless given."""
    fx = 0.9375 * width if fx is None else fx
    return Camera(pos=np.asarray(pos, dtype=np.float32), R_wc=yaw_rotation(yaw, pitch),
                  fx=float(fx), fy=float(fx), cx=width / 2.0, cy=height / 2.0,
                  width=int(width), height=int(height), tau=float(tau))


def camera_c0(tau: float) -> Camera:
    """The small-scene view: 128x128, fx = fy = 120, at (2, 2, 1.2) looking +x."""
    return look_camera((2.0, 2.0, 1.2), 0.0, 128, 128, fx=120.0, tau=tau)


def _seg_dist(p: np.ndarray, segs) -> float:
    best = np.inf
    for axis, c, lo, hi in segs:
        if axis == "x":
            d_n, t = p[0] - c, p[1]
        else:
            d_n, t = p[1] - c, p[0]
        d_t = max(lo - t, 0.0, t - hi)
        best = min(best, math.hypot(d_n, d_t))
    return best


def _walk(rng, size, segs, n, step=0.11, clearance=0.3, yaw_sigma_deg=10.0, start=None):
    sx, sy = size[0], size[1]
    arr = np.array([(0 if a == "x" else 1, c, lo, hi) for a, c, lo, hi in segs])

    def free(p):
        if not (clearance <= p[0] <= sx - clearance and clearance <= p[1] <= sy - clearance):
            return False
        isx = arr[:, 0] == 0
        d_n = np.where(isx, p[0] - arr[:, 1], p[1] - arr[:, 1])
        t = np.where(isx, p[1], p[0])
        d_t = np.maximum(np.maximum(arr[:, 2] - t, 0.0), t - arr[:, 3])
        return bool(np.all(np.hypot(d_n, d_t) >= clearance))

    if start is None:
        for _ in range(10000):
            p = np.array([rng.uniform(0, sx), rng.uniform(0, sy)])
            if free(p):
                break
    else:
        p = np.asarray(start, dtype=np.float64)
    heading = rng.uniform(-math.pi, math.pi)
    poses = []
    for _ in range(n):
        for attempt in range(64):
            h = heading + rng.normal(0.0, math.radians(8.0))
            q = p + step * np.array([math.cos(h), math.sin(h)])
            if free(q):
                heading, p = h, q
                break
            heading += rng.choice([-1.0, 1.0]) * rng.uniform(math.radians(60), math.pi)
        yaw = heading + rng.normal(0.0, math.radians(yaw_sigma_deg))
        poses.append((p.copy(), yaw))
    return poses


def walk_cameras(scene: Scene, n: int, seed: int, width: int, height: int, fx=None,
                 tau=0.0, height_m: float = 1.2, taus: Sequence[float] = None) -> List[Camera]:
    """``n`` poses of one collision-free walk at ``height_m`` (steps of ~0.11 m,
    >= 0.3 m from every wall slab, heading = direction of motion + N(0, 10 deg))."""
    rng = np.random.default_rng(seed)
    size = scene.meta.get("size", [4.0, 4.0, 3.0])
    segs = scene.meta.get("walls") or wall_segments(size[0], size[1])
    cams = []
    for i, (p, yaw) in enumerate(_walk(rng, size, segs, n)):
        t = tau if taus is None else taus[i]
        cams.append(look_camera((p[0], p[1], height_m), yaw, width, height, fx=fx, tau=t))
    return cams


def mixed_batch_cameras(scene: Scene, n: int, seed: int, tau_range=(2.0, 8.0),
                        resolutions=((320, 240), (640, 480), (1280, 720)),
                        mix=(1, 2, 1), n_walkers: int = 8) -> List[Camera]:
    """A batch of ``n`` cameras with resolutions mixed ``mix`` (1:2:1 of
    320x240 / 640x480 / 1280x720 by default), fx = 0.9375 W, per-camera
    tau ~ U[tau_range], poses taken from ``n_walkers`` independent walks."""
    rng = np.random.default_rng(seed)
    size = scene.meta.get("size", [4.0, 4.0, 3.0])
    segs = scene.meta.get("walls") or wall_segments(size[0], size[1])
    per = -(-n // n_walkers)
    poses = []
    for w in range(n_walkers):
        poses.extend(_walk(rng, size, segs, per))
    poses = poses[:n]
    tot = sum(mix)
    res = []
    for r, m in zip(resolutions, mix):
        res.extend([r] * int(round(n * m / tot)))
    while len(res) < n:
        res.append(resolutions[len(res) % len(resolutions)])
    res = res[:n]
    perm = rng.permutation(n)
    taus = rng.uniform(tau_range[0], tau_range[1], size=n)
    cams = []
    for i in range(n):
        (p, yaw), (w, h) = poses[i], res[perm[i]]
        cams.append(look_camera((p[0], p[1], 1.2), yaw, w, h, tau=float(taus[i])))
    return cams

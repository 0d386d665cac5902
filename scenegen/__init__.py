"""Seeded synthetic inputs shared by the renderer's tests, its benchmark and the oracle.

This module builds scenes (leaf Gaussians plus an 8-ary octree hierarchy with
moment-matched parents) and camera trajectories shaped like the multi-room
indoor floors the simulator renders. It holds none of the renderer's
arithmetic (no projection, colour, binning or compositing); it only produces
the arrays both sides take as input.
"""
from .scene import (Scene, Camera, SCENE_PRESETS, make_scene, make_uniform_box_scene,
                    make_floor_scene, build_hierarchy, quantize_attributes)
from .cameras import (camera_c0, walk_cameras, mixed_batch_cameras, look_camera,
                      yaw_rotation)

__all__ = [
    "Scene", "Camera", "SCENE_PRESETS", "make_scene", "make_uniform_box_scene",
    "make_floor_scene", "build_hierarchy", "quantize_attributes", "camera_c0",
    "walk_cameras", "mixed_batch_cameras", "look_camera", "yaw_rotation",
]

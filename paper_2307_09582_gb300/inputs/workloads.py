"""The five synthetic workloads (sizes, generator counts and seeds), stated as data.

* plain 256x256: 40 cells, 30 dots, 5 lines, noise sigma 2, seed 1; scale 4 box LR, 3x3 window.
* joint 4K: 3840x2160, 400 cells, 2000 dots, 100 lines, seed 2; scale 8 grid LR, 5x5 window,
  5 joint iterations.
* batch: 16 guides, width ~ U{512..4096}, height ~ U{384..3072}, scale ~ {4, 8, 16},
  window ~ {3, 5}, generator counts scaled with area from the 4K scene, seed 4.
* video: 120 frames 3840x2160, cells translate +2 px/frame, 5% of dots re-drawn per frame,
  seed 5; scale 8 box LR, 5x5 window.
"""
from __future__ import annotations

import numpy as np

from .synth import Scene


def plain_256_scene(seed: int = 1, size: int = 256) -> Scene:
    return Scene(width=size, height=size, n_cells=40, n_dots=30, n_lines=5, seed=seed)


def joint_4k_scene(seed: int = 2, width: int = 3840, height: int = 2160) -> Scene:
    area = width * height / (3840 * 2160)
    return Scene(width=width, height=height, n_cells=max(8, round(400 * area)),
                 n_dots=max(4, round(2000 * area)), n_lines=max(2, round(100 * area)), seed=seed)


def batch_scenes(seed: int = 4, n: int = 16, wmin=512, wmax=4096, hmin=384, hmax=3072):
    """n (scene, scale, window) triples with uneven sizes; drawn from numpy's PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    items = []
    for i in range(n):
        w = int(rng.integers(wmin, wmax + 1))
        h = int(rng.integers(hmin, hmax + 1))
        s = int(rng.choice([4, 8, 16]))
        S = int(rng.choice([3, 5]))
        sc = joint_4k_scene(seed=seed * 1000 + i, width=w, height=h)
        items.append((sc, s, S))
    return items


def video_scene(seed: int = 5, width: int = 3840, height: int = 2160) -> Scene:
    sc = joint_4k_scene(seed=seed, width=width, height=height)
    sc.cell_dx_per_frame = 2.0
    sc.dot_period = 20
    return sc

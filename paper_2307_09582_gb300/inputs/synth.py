"""ctypes wrapper around synth.c: seeded Voronoi + gradients + dots + lines + noise images.

The shared library is compiled by ``paper_2307_09582_gb300.build.build_synth`` (gcc, OpenMP).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def synth_library_path() -> str:
    return os.path.join(_HERE, "libglu_synth.so")


class _CScene(ctypes.Structure):
    _fields_ = [
        ("width", ctypes.c_int32), ("height", ctypes.c_int32),
        ("n_cells", ctypes.c_int32), ("n_dots", ctypes.c_int32), ("n_lines", ctypes.c_int32),
        ("noise_sigma", ctypes.c_double), ("grad_max", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("frame", ctypes.c_int32),
        ("cell_dx_per_frame", ctypes.c_double), ("dot_period", ctypes.c_int32),
    ]


@dataclass
class Scene:
    """Parameters of one synthetic guide image (uint8 RGB, H x W x 3)."""
    width: int
    height: int
    n_cells: int
    n_dots: int
    n_lines: int
    seed: int
    noise_sigma: float = 2.0
    grad_max: float = 0.5
    cell_dx_per_frame: float = 0.0
    dot_period: int = 0
    extra: dict = field(default_factory=dict)


def _lib():
    global _LIB
    if _LIB is None:
        path = synth_library_path()
        if not os.path.exists(path):
            from .. import build as _build
            _build.build_synth()
        lib = ctypes.CDLL(path)
        lib.synth_render_u8.argtypes = [ctypes.POINTER(_CScene), ctypes.c_void_p, ctypes.c_int32]
        lib.synth_render_u8.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def render_u8(scene: Scene, frame: int = 0, threads: int = 0) -> np.ndarray:
    """Render one frame as a (H, W, 3) uint8 array."""
    cs = _CScene(scene.width, scene.height, scene.n_cells, scene.n_dots, scene.n_lines,
                 float(scene.noise_sigma), float(scene.grad_max), ctypes.c_uint64(scene.seed),
                 int(frame), float(scene.cell_dx_per_frame), int(scene.dot_period))
    out = np.empty((scene.height, scene.width, 3), dtype=np.uint8)
    rc = _lib().synth_render_u8(ctypes.byref(cs), out.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError(f"synth_render_u8 failed ({rc}) for {scene}")
    return out


def render_video_u8(scene: Scene, n_frames: int, threads: int = 0) -> np.ndarray:
    """Render frames 0..n_frames-1 as an (F, H, W, 3) uint8 array."""
    out = np.empty((n_frames, scene.height, scene.width, 3), dtype=np.uint8)
    for f in range(n_frames):
        out[f] = render_u8(scene, frame=f, threads=threads)
    return out

"""Seeded synthetic inputs (the generator shared by the CPU oracle tests and the GPU path).

Nothing here computes any part of the upsampling method: this package only produces guide
images and random arrays of the shapes the paper's workloads have.
"""
from .synth import Scene, render_u8, render_video_u8, synth_library_path  # noqa: F401
from .workloads import (  # noqa: F401
    plain_256_scene, joint_4k_scene, batch_scenes, video_scene,
)

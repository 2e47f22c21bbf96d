"""GB300 (sm_103a) Guided Linear Upsampling: hand-written CUDA kernels behind a C ABI.

The method is Song et al., "Guided Linear Upsampling" (ACM TOG 2023): every HR pixel is
w * P[a] + (1 - w) * P[b] of two LR pixels near it (Eq. 1), with (a, b, w) chosen on the guide
image (Algorithm 1) and, optionally, the LR image re-optimised jointly (Algorithm 2).

``paper_2307_09582_gb300.api`` exposes the library's entry points (glu_downsample,
glu_optimize, glu_joint_optimize, glu_apply, glu_apply_backward) on torch tensors.
"""
__all__ = ["api", "build", "inputs"]

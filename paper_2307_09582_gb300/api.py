"""Python binding of libglu.so: the C entry points under the same names, taking torch tensors.

Argument marshalling only: tensors become (pointer, sizes, pitch) descriptors and the current
CUDA stream is passed through; every step of the computation runs in the library's kernels.
Output tensors that the caller does not provide are allocated here with torch (device memory
plumbing; the library itself never allocates).

Image tensors are (h, w, c) with the last two dimensions contiguous; uint8 holds colour * 255,
float16 / float32 hold colours in [0, 1].
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _abi as A
from ._abi import (GLU_DOWN_BOX, GLU_DOWN_GRID, GLU_F16, GLU_F32, GLU_JOINT_PAPER,  # noqa: F401
                   GLU_JOINT_STRICT, GLU_MODE_EXACT, GLU_MODE_FAST, GLU_MODE_GNU, GLU_U8, GLU_W_F16, GLU_W_F32,
                   GLU_TUNE_APPLY, GLU_TUNE_SEARCH, GLU_W_UNORM16, GluError)

_DT = {torch.uint8: A.GLU_U8, torch.float16: A.GLU_F16, torch.float32: A.GLU_F32}
_WT = {A.GLU_W_F32: torch.float32, A.GLU_W_F16: torch.float16, A.GLU_W_UNORM16: torch.int16}


def lib():
    return A.load()


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p | None:
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def image(t: torch.Tensor) -> A.GluImage:
    """Descriptor of an (h, w, c) tensor whose last two dims are contiguous."""
    if t.dim() == 2:
        t = t.unsqueeze(-1)
    if t.dim() != 3 or t.stride(2) != 1 or t.stride(1) != t.shape[2]:
        raise ValueError("image tensors must be (h, w, c) with contiguous pixels")
    if t.dtype not in _DT:
        raise TypeError(f"unsupported image dtype {t.dtype}")
    return A.GluImage(t.data_ptr(), t.shape[0], t.shape[1], t.shape[2], _DT[t.dtype], t.stride(0))


def lr_dims(H: int, W: int, s: int):
    return (H + s - 1) // s, (W + s - 1) // s


def glu_params(S=3, eps=1e-3, tau=30.0 / 255.0, N=3, mode=A.GLU_MODE_FAST,
               joint=A.GLU_JOINT_STRICT, connectivity=8) -> A.GluParams:
    p = A.GluParams()
    lib().glu_params_default(ctypes.byref(p))
    p.S, p.eps, p.tau, p.N = S, eps, tau, N
    p.mode, p.joint, p.connectivity = mode, joint, connectivity
    return p


@dataclass
class Theta:
    """Per-HR-pixel pair codes (k_a * S * S + k_b, stored in int16 as uint16) and weights."""
    code: torch.Tensor
    weight: torch.Tensor
    H: int
    W: int
    scale: int
    S: int
    wfmt: int = A.GLU_W_F32

    @staticmethod
    def empty(H, W, scale, S, wfmt=A.GLU_W_F32, device="cuda") -> "Theta":
        code = torch.empty((H, W), dtype=torch.int16, device=device)
        weight = torch.empty((H, W), dtype=_WT[wfmt], device=device)
        return Theta(code, weight, H, W, scale, S, wfmt)

    def desc(self, weight: torch.Tensor | None = None, wfmt: int | None = None) -> A.GluTheta:
        w = self.weight if weight is None else weight
        return A.GluTheta(self.code.data_ptr(), w.data_ptr(), self.H, self.W, self.scale, self.S,
                          self.wfmt if wfmt is None else wfmt)

    def weight_f32(self) -> torch.Tensor:
        if self.wfmt == A.GLU_W_UNORM16:
            return (self.weight.view(torch.uint16).to(torch.float32) / 65535.0) \
                if hasattr(torch, "uint16") else \
                ((self.weight.to(torch.int32) & 0xFFFF).to(torch.float32) / 65535.0)
        return self.weight.to(torch.float32)

    def codes_i32(self) -> torch.Tensor:
        return self.code.to(torch.int32) & 0xFFFF


def glu_downsample(hr: torch.Tensor, scale: int, mode: int = A.GLU_DOWN_GRID,
                   lr: torch.Tensor | None = None, dtype=None, stream=None) -> torch.Tensor:
    H, W, C = hr.shape
    h, w = lr_dims(H, W, scale)
    if lr is None:
        dt = dtype or (hr.dtype if mode == A.GLU_DOWN_GRID else torch.float32)
        lr = torch.empty((h, w, C), dtype=dt, device=hr.device)
    hi, li = image(hr), image(lr)
    A.check("glu_downsample", lib().glu_downsample(ctypes.byref(hi), scale, mode,
                                                   ctypes.byref(li), _stream(stream)))
    return lr


def glu_optimize(hr: torch.Tensor, lr: torch.Tensor, params: A.GluParams, scale: int,
                 theta: Theta | None = None, err_map: torch.Tensor | bool | None = None,
                 wfmt: int = A.GLU_W_F32, stream=None):
    """Algorithm 1 on every pixel. Returns (theta, err_map or None)."""
    H, W = hr.shape[:2]
    if theta is None:
        theta = Theta.empty(H, W, scale, params.S, wfmt, hr.device)
    if err_map is True:
        err_map = torch.empty((H, W), dtype=torch.float32, device=hr.device)
    elif err_map is False:
        err_map = None
    hi, li, td = image(hr), image(lr), theta.desc()
    A.check("glu_optimize", lib().glu_optimize(ctypes.byref(hi), ctypes.byref(li),
                                               ctypes.byref(params), ctypes.byref(td),
                                               _ptr(err_map), _stream(stream)))
    return theta, err_map


def glu_joint_workspace_size(H: int, W: int, scale: int, params: A.GluParams) -> int:
    return int(lib().glu_joint_workspace_size(H, W, scale, ctypes.byref(params)))


def glu_joint_optimize(hr: torch.Tensor, scale: int, params: A.GluParams,
                       lr_out: torch.Tensor | None = None, theta: Theta | None = None,
                       err_map: torch.Tensor | bool | None = True, stats: bool = True,
                       workspace: torch.Tensor | None = None, wfmt: int = A.GLU_W_F32,
                       decisions: bool = False, argmax_log: bool = False, stream=None):
    """Algorithm 2. Returns (lr, theta, err_map or None, stats dict or None); with
    decisions=True the stats hold the per-component keep/rollback log, with argmax_log=True
    (verification aid) also every trial's replacement choices as an (n, 4) int32 array of
    (iteration, component, LR pixel, HR pixel) records."""
    H, W = hr.shape[:2]
    h, w = lr_dims(H, W, scale)
    if lr_out is None:
        lr_out = torch.empty((h, w, 3), dtype=torch.uint8, device=hr.device)
    if theta is None:
        theta = Theta.empty(H, W, scale, params.S, wfmt, hr.device)
    if err_map is True:
        err_map = torch.empty((H, W), dtype=torch.float32, device=hr.device)
    elif err_map is False:
        err_map = None
    need = glu_joint_workspace_size(H, W, scale, params)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need + 256, dtype=torch.uint8, device=hr.device)
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    avail = workspace.numel() - (aligned - base)
    st = A.GluJointStats() if stats else None
    hi, li, td = image(hr), image(lr_out), theta.desc()
    alog = None
    if argmax_log:
        cap = 4 * h * w * max(params.N, 1) + 65536
        alog = torch.zeros((cap + 1, 4), dtype=torch.int32, device=hr.device)
        A.check("glu_test_joint_argmax_log",
                lib().glu_test_joint_argmax_log(ctypes.c_void_p(alog.data_ptr()), cap))
    try:
        A.check("glu_joint_optimize", lib().glu_joint_optimize(
            ctypes.byref(hi), scale, ctypes.byref(params), ctypes.byref(li), ctypes.byref(td),
            _ptr(err_map), ctypes.byref(st) if st is not None else None,
            ctypes.c_void_p(aligned), avail, _stream(stream)))
    finally:
        if alog is not None:
            lib().glu_test_joint_argmax_log(None, 0)
    sd = None
    if st is not None and decisions:
        import numpy as np
        buf = np.empty(sum(st.components[k] for k in range(st.iterations)) + 1, dtype=np.int8)
        n = lib().glu_joint_decisions(ctypes.c_void_p(aligned), avail, H, W, scale,
                                      ctypes.byref(params), ctypes.c_void_p(buf.ctypes.data),
                                      buf.size, _stream(stream))
        if n < 0:
            A.check("glu_joint_decisions", int(n))
        decisions = buf[:n].copy()
    else:
        decisions = None
    if st is not None:
        sd = _stats_dict(st, decisions)
        if alog is not None:
            a = alog.cpu().numpy()
            n = int(a[0, 0])
            if n > a.shape[0] - 1:
                raise RuntimeError(f"argmax log overflow: {n} records")
            sd["argmax"] = a[1:1 + n].copy()
    return lr_out, theta, err_map, sd


def _stats_dict(st: A.GluJointStats, decisions=None) -> dict:
    n = st.iterations
    return dict(iterations=n, R0=st.residual[0],
                iters=[dict(n_large=st.n_large[k], M=st.components[k],
                            accepted=st.accepted[k], rolled_back=st.rolled_back[k],
                            residual=st.residual[k + 1], searched=st.searched[k])
                       for k in range(n)],
                n_large_next=st.n_large[n] if n < A.GLU_MAX_ITERS else 0,
                multi_kernel_lists=int(st.multi_kernel_lists),
                decisions=decisions)


def _aligned(workspace: torch.Tensor):
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    return aligned, workspace.numel() - (aligned - base)


def _batch_items(hrs, lrs, thetas, errs):
    items = (A.GluBatchItem * max(1, len(hrs)))()
    for k, (hr, lr, th, e) in enumerate(zip(hrs, lrs, thetas, errs)):
        items[k].hr = image(hr)
        items[k].lr = image(lr)
        items[k].theta = th.desc()
        items[k].err_map = _ptr(e)
    return items


def glu_optimize_batched(hrs, lrs, params: A.GluParams, scales, Ss=None, thetas=None,
                         err_maps: bool = True, wfmt: int = A.GLU_W_F32, stream=None):
    """Algorithm 1 on several images in one persistent launch. scales / Ss: one per image (Ss
    defaults to params.S). Returns [(theta, err_map or None)]."""
    n = len(hrs)
    Ss = [params.S] * n if Ss is None else list(Ss)
    if thetas is None:
        thetas = [Theta.empty(hr.shape[0], hr.shape[1], s, S, wfmt, hr.device)
                  for hr, s, S in zip(hrs, scales, Ss)]
    errs = [torch.empty(hr.shape[:2], dtype=torch.float32, device=hr.device) if err_maps else None
            for hr in hrs]
    items = _batch_items(hrs, lrs, thetas, errs)
    A.check("glu_optimize_batched", lib().glu_optimize_batched(items, n, ctypes.byref(params),
                                                               _stream(stream)))
    return list(zip(thetas, errs))


def glu_joint_batched_workspace_size(shapes, scales, Ss, params: A.GluParams) -> int:
    """shapes: [(H, W)] per image."""
    items = (A.GluBatchItem * max(1, len(shapes)))()
    for k, ((H, W), s, S) in enumerate(zip(shapes, scales, Ss)):
        items[k].hr.h, items[k].hr.w = H, W
        items[k].theta.scale, items[k].theta.S = s, S
    return int(lib().glu_joint_batched_workspace_size(items, len(shapes), ctypes.byref(params)))


def glu_joint_optimize_batched(hrs, scales, params: A.GluParams, Ss=None, lrs=None, thetas=None,
                               err_maps: bool = True, stats: bool = True,
                               workspace: torch.Tensor | None = None,
                               wfmt: int = A.GLU_W_F32, stream=None):
    """Algorithm 2 on up to 32 images in one set of launches. Returns
    [(lr, theta, err_map or None, stats dict or None)] in input order."""
    n = len(hrs)
    Ss = [params.S] * n if Ss is None else list(Ss)
    if lrs is None:
        lrs = [torch.empty((*lr_dims(hr.shape[0], hr.shape[1], s), 3), dtype=torch.uint8,
                           device=hr.device) for hr, s in zip(hrs, scales)]
    if thetas is None:
        thetas = [Theta.empty(hr.shape[0], hr.shape[1], s, S, wfmt, hr.device)
                  for hr, s, S in zip(hrs, scales, Ss)]
    errs = [torch.empty(hr.shape[:2], dtype=torch.float32, device=hr.device) if err_maps else None
            for hr in hrs]
    need = glu_joint_batched_workspace_size([hr.shape[:2] for hr in hrs], scales, Ss, params)
    if workspace is None or workspace.numel() < need + 256:
        workspace = torch.empty(need + 256, dtype=torch.uint8, device=hrs[0].device)
    aligned, avail = _aligned(workspace)
    items = _batch_items(hrs, lrs, thetas, errs)
    st = (A.GluJointStats * max(1, n))() if stats else None
    A.check("glu_joint_optimize_batched", lib().glu_joint_optimize_batched(
        items, n, ctypes.byref(params), st, ctypes.c_void_p(aligned), avail, _stream(stream)))
    return [(lrs[k], thetas[k], errs[k], _stats_dict(st[k]) if st is not None else None)
            for k in range(n)]




class Video:
    """Per-frame pipeline (BOX downsample -> LR operators (3x3 filter + saturation + gamma) on the
    LR image -> Algorithm 1 once -> Eq. 1 per operator) with one CUDA graph per bound (frame,
    outputs) slot. `ops`: list of (filter, saturation, gamma), one output per operator (default:
    the single operator given by filter / saturation / gamma). The workspace (LR images, targets,
    Theta) is a torch tensor owned here."""

    def __init__(self, H, W, scale, params: A.GluParams, hr_dtype=torch.float16,
                 out_dtype=torch.float16, wfmt=A.GLU_W_UNORM16, filter=1, saturation=1.0,
                 gamma=0.8, overlap=True, device="cuda", ops=None):
        if ops is None:
            ops = [(filter, saturation, gamma)]
        if not 1 <= len(ops) <= A.GLU_VIDEO_MAX_OPS:
            raise ValueError(f"1 to {A.GLU_VIDEO_MAX_OPS} operators")
        d = A.GluVideoDesc()
        d.H, d.W, d.scale = H, W, scale
        d.hr_dtype, d.out_dtype = _DT[hr_dtype], _DT[out_dtype]
        d.params = params
        d.wfmt = wfmt
        d.n_ops = len(ops)
        for k, (f, sat, g) in enumerate(ops):
            d.ops[k] = A.GluLrOp(int(f), float(sat), float(g))
        d.overlap = 1 if overlap else 0
        self.desc, self.H, self.W, self.scale, self.S = d, H, W, scale, params.S
        self.out_dtype, self.wfmt, self.n_ops = out_dtype, wfmt, len(ops)
        need = int(lib().glu_video_workspace_size(ctypes.byref(d)))
        if need == 0:
            A.check("glu_video_workspace_size", A.GLU_ERR_INVALID_ARG)
        self.ws = torch.empty(need + 256, dtype=torch.uint8, device=device)
        aligned, avail = _aligned(self.ws)
        h = ctypes.c_void_p()
        A.check("glu_video_create", lib().glu_video_create(ctypes.byref(d), ctypes.c_void_p(aligned),
                                                           avail, ctypes.byref(h)))
        self.h = h
        self._bound = {}

    def _outs(self, outs):
        outs = [outs] if isinstance(outs, torch.Tensor) else list(outs)
        if len(outs) != self.n_ops:
            raise ValueError(f"{self.n_ops} output tensors expected")
        for o in outs:
            assert o.is_contiguous() and o.shape == (self.H, self.W, 3)
        return outs, (ctypes.c_void_p * self.n_ops)(*[o.data_ptr() for o in outs])

    def bind(self, slot: int, hr: torch.Tensor, outs) -> None:
        """Record slot `slot`: the frame `hr` into `outs` (a tensor, or one per operator)."""
        assert hr.is_contiguous() and hr.shape == (self.H, self.W, 3)
        outs, arr = self._outs(outs)
        A.check("glu_video_bind", lib().glu_video_bind(self.h, slot, ctypes.c_void_p(hr.data_ptr()),
                                                       arr))
        self._bound[slot] = (hr, outs)   # keep the buffers alive while the graph refers to them

    def launch(self, slot: int, stream=None) -> None:
        A.check("glu_video_launch", lib().glu_video_launch(self.h, slot, _stream(stream)))

    def run(self, hr: torch.Tensor, outs, stream=None) -> None:
        assert hr.is_contiguous()
        outs, arr = self._outs(outs)
        A.check("glu_video_run", lib().glu_video_run(self.h, ctypes.c_void_p(hr.data_ptr()), arr,
                                                     _stream(stream)))

    def views(self):
        """(lr, [target of each operator], Theta) views into the workspace, as torch tensors."""
        li, th = A.GluImage(), A.GluTheta()
        ti = (A.GluImage * self.n_ops)()
        A.check("glu_video_views", lib().glu_video_views(self.h, ctypes.byref(li), ti,
                                                         ctypes.byref(th)))
        base = self.ws.data_ptr()

        def view(ptr, n, dtype, shape):
            off = ptr - base
            esz = torch.empty((), dtype=dtype).element_size()
            return self.ws[off:off + n * esz].view(dtype).view(shape)

        lr = view(li.data, li.h * li.w * 3, torch.float32, (li.h, li.w, 3))
        T = [view(t.data, t.h * t.w * 3, torch.float32, (t.h, t.w, 3)) for t in ti]
        code = view(th.code, self.H * self.W, torch.int16, (self.H, self.W))
        weight = view(th.weight, self.H * self.W, _WT[self.wfmt], (self.H, self.W))
        return lr, T, Theta(code, weight, self.H, self.W, self.scale, self.S, self.wfmt)

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().glu_video_destroy(self.h)
            self.h = None
            self._bound = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def glu_apply(theta: Theta, lr_target: torch.Tensor, out: torch.Tensor | None = None,
              out_dtype=torch.float32, weight: torch.Tensor | None = None, stream=None):
    """Eq. 1. `weight` (float32, H x W) overrides the stored weights (used by autograd)."""
    C = lr_target.shape[2] if lr_target.dim() == 3 else 1
    if out is None:
        out = torch.empty((theta.H, theta.W, C), dtype=out_dtype, device=lr_target.device)
    td = theta.desc(weight, A.GLU_W_F32 if weight is not None else None)
    ti, oi = image(lr_target), image(out)
    A.check("glu_apply", lib().glu_apply(ctypes.byref(td), ctypes.byref(ti), ctypes.byref(oi),
                                         _stream(stream)))
    return out


def glu_theta_decode(theta: Theta, stream=None):
    """Theta as absolute LR pixel indices (a, b: int32 H x W, row-major v * w + u) and float32
    weights (H x W), decoded on the device."""
    dev = theta.code.device
    a = torch.empty((theta.H, theta.W), dtype=torch.int32, device=dev)
    b = torch.empty_like(a)
    w = torch.empty((theta.H, theta.W), dtype=torch.float32, device=dev)
    td = theta.desc()
    A.check("glu_theta_decode", lib().glu_theta_decode(ctypes.byref(td), a.data_ptr(),
                                                       b.data_ptr(), w.data_ptr(),
                                                       _stream(stream)))
    return a, b, w


def glu_workspace_size(op: int, H: int, W: int, scale: int, params: A.GluParams) -> int:
    """Workspace bytes of operation `op` (A.GLU_OP_*); 0 when it takes none."""
    return int(lib().glu_workspace_size(op, H, W, scale, ctypes.byref(params)))


_BW_WS = {}   # device -> workspace of the adjoint (grown on demand, reused across calls)


def test_set_wait_limit(ns: int) -> None:
    """Test hook: deadline of the trial kernel's waits in ns (0: the default)."""
    A.check("glu_test_set_wait_limit", lib().glu_test_set_wait_limit(int(ns)))


def glu_apply_backward_plan(theta: Theta, stream=None) -> torch.Tensor:
    """The inverse pixel-to-LR map of theta's codes for glu_apply_backward(plan=...): valid while
    the codes do not change (the weights may)."""
    td = theta.desc()
    need = int(lib().glu_apply_backward_plan_size(ctypes.byref(td)))
    plan = torch.empty(need // 4 + 1, dtype=torch.int32, device=theta.code.device)
    A.check("glu_apply_backward_plan", lib().glu_apply_backward_plan(
        ctypes.byref(td), ctypes.c_void_p(plan.data_ptr()), plan.numel() * 4, _stream(stream)))
    return plan


def glu_apply_backward(theta: Theta, lr_target: torch.Tensor, grad_hr: torch.Tensor,
                       grad_lr: torch.Tensor | None = None, grad_w: torch.Tensor | bool = True,
                       weight: torch.Tensor | None = None, stream=None,
                       workspace: torch.Tensor | bool | None = True,
                       plan: torch.Tensor | None = None):
    """Adjoint of Eq. 1: returns (grad_lr, grad_w or None). With `plan` (from
    glu_apply_backward_plan) glu_apply_backward_planned runs; otherwise with `workspace` (True: a
    cached per-device buffer; or a uint8 tensor) the bucketed glu_apply_backward_ws, without it
    (None / False) the tiled glu_apply_backward."""
    if grad_lr is None:
        grad_lr = torch.empty_like(lr_target, dtype=torch.float32)
    if grad_w is True:
        grad_w = torch.empty((theta.H, theta.W), dtype=torch.float32, device=grad_hr.device)
    elif grad_w is False:
        grad_w = None
    td = theta.desc(weight, A.GLU_W_F32 if weight is not None else None)
    ti, gi, go = image(lr_target), image(grad_hr), image(grad_lr)
    if plan is not None:
        A.check("glu_apply_backward_planned", lib().glu_apply_backward_planned(
            ctypes.byref(td), ctypes.c_void_p(plan.data_ptr()), ctypes.byref(ti),
            ctypes.byref(gi), ctypes.byref(go), _ptr(grad_w), _stream(stream)))
        return grad_lr, grad_w
    if workspace is None or workspace is False:
        A.check("glu_apply_backward", lib().glu_apply_backward(
            ctypes.byref(td), ctypes.byref(ti), ctypes.byref(gi), ctypes.byref(go),
            _ptr(grad_w), _stream(stream)))
        return grad_lr, grad_w
    C = lr_target.shape[2] if lr_target.dim() == 3 else 1
    need = int(lib().glu_apply_backward_workspace_size(ctypes.byref(td), C))
    if workspace is True:
        dev = grad_hr.device
        ws = _BW_WS.get(dev)
        if ws is None or ws.numel() < need + 16:
            ws = torch.empty(need + 16, dtype=torch.uint8, device=dev)
            _BW_WS[dev] = ws
    else:
        ws = workspace
    base = ws.data_ptr()
    aligned = (base + 15) & ~15
    A.check("glu_apply_backward_ws", lib().glu_apply_backward_ws(
        ctypes.byref(td), ctypes.byref(ti), ctypes.byref(gi), ctypes.byref(go), _ptr(grad_w),
        ctypes.c_void_p(aligned), ws.numel() - (aligned - base), _stream(stream)))
    return grad_lr, grad_w


def glu_ls_update(hr: torch.Tensor, theta: Theta, lr_in: torch.Tensor,
                  lr_out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
    """One least-squares LR colour update for a fixed Theta (float32 weights); lr_in / lr_out
    float32 h x w x 3 in [0, 1]. Not the paper's method (see glu.h)."""
    if lr_out is None:
        lr_out = torch.empty_like(lr_in)
    td = theta.desc()
    need = int(lib().glu_ls_update_workspace_size(ctypes.byref(td)))
    if workspace is None:
        workspace = torch.empty(need + 16, dtype=torch.uint8, device=hr.device)
    base = workspace.data_ptr()
    aligned = (base + 15) & ~15
    hi, li, lo = image(hr), image(lr_in), image(lr_out)
    A.check("glu_ls_update", lib().glu_ls_update(
        ctypes.byref(hi), ctypes.byref(td), ctypes.byref(li), ctypes.byref(lo),
        ctypes.c_void_p(aligned), workspace.numel() - (aligned - base), _stream(stream)))
    return lr_out


def glu_ls_joint_workspace_size(H: int, W: int, scale: int, params: A.GluParams) -> int:
    return int(lib().glu_ls_joint_workspace_size(H, W, scale, ctypes.byref(params)))


def glu_ls_joint_optimize(hr: torch.Tensor, scale: int, params: A.GluParams,
                          lr_out: torch.Tensor | None = None, theta: Theta | None = None,
                          err_map: torch.Tensor | bool | None = True, stats: bool = True,
                          workspace: torch.Tensor | None = None, stream=None):
    """Algorithm 1 alternated with the least-squares LR colour update. Returns (lr (float32),
    theta, err_map or None, stats dict or None)."""
    H, W = hr.shape[:2]
    h, w = lr_dims(H, W, scale)
    if lr_out is None:
        lr_out = torch.empty((h, w, 3), dtype=torch.float32, device=hr.device)
    if theta is None:
        theta = Theta.empty(H, W, scale, params.S, A.GLU_W_F32, hr.device)
    if err_map is True:
        err_map = torch.empty((H, W), dtype=torch.float32, device=hr.device)
    elif err_map is False:
        err_map = None
    need = glu_ls_joint_workspace_size(H, W, scale, params)
    if workspace is None or workspace.numel() < need + 256:
        workspace = torch.empty(need + 256, dtype=torch.uint8, device=hr.device)
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    st = A.GluLsStats() if stats else None
    hi, li, td = image(hr), image(lr_out), theta.desc()
    A.check("glu_ls_joint_optimize", lib().glu_ls_joint_optimize(
        ctypes.byref(hi), scale, ctypes.byref(params), ctypes.byref(li), ctypes.byref(td),
        _ptr(err_map), ctypes.byref(st) if st is not None else None, ctypes.c_void_p(aligned),
        workspace.numel() - (aligned - base), _stream(stream)))
    sd = None
    if st is not None:
        sd = dict(R0=st.R0, residuals=[st.residual[i] for i in range(st.iterations)],
                  kept=st.kept)
    return lr_out, theta, err_map, sd


def glu_joint_profile(enable: bool) -> None:
    A.check("glu_joint_profile", lib().glu_joint_profile(1 if enable else 0))


def glu_joint_profile_read() -> dict:
    """Summed phase times (ms) of the profiled glu_joint_optimize calls since the last read."""
    ms = (ctypes.c_float * 5)()
    calls = ctypes.c_int32()
    A.check("glu_joint_profile_read", lib().glu_joint_profile_read(ms, ctypes.byref(calls)))
    return dict(calls=calls.value, prep_ms=ms[0], search_ms=ms[1], components_ms=ms[2],
                trials_ms=ms[3], residual_ms=ms[4])


def joint_launches(N: int, graph: bool = False, multi_kernel_lists: int = 0) -> int:
    """Kernel launches one glu_joint_optimize call makes: control init, grid downsample, search
    and R_0 (2), then per iteration the threshold count and list-write passes, the one-CTA list
    kernel, the multi-kernel list path (tile components, border merge, flatten, root count,
    scan, root scatter, component count, 3 scan, fill, dependency graph 5: 16 kernels), the
    trials, the list clear and the residual update. Issued directly, every kernel launches (those
    with nothing to do return at once). Replayed as a recorded graph (a repeated call), the 16
    kernels of the multi-kernel path sit in a conditional node and launch only in the iterations
    whose bit is set in the stats' multi_kernel_lists."""
    if not graph:
        return 5 + 22 * N
    multi = bin(multi_kernel_lists & ((1 << N) - 1)).count("1")
    return 5 + 6 * N + 16 * multi


def tune_mode(on: bool) -> None:
    A.check("glu_tune_mode", lib().glu_tune_mode(1 if on else 0))


def tune_variants(kernel: int) -> list:
    """Descriptions of a kernel's variants (GLU_TUNE_SEARCH / GLU_TUNE_APPLY)."""
    n = int(lib().glu_tune_variants(kernel))
    if n < 0:
        A.check("glu_tune_variants", n)
    out = []
    for v in range(n):
        buf = ctypes.create_string_buffer(128)
        A.check("glu_tune_variant_name", lib().glu_tune_variant_name(kernel, v, buf, 128))
        out.append(buf.value.decode())
    return out


def tune_force(kernel: int, variant: int) -> None:
    A.check("glu_tune_force", lib().glu_tune_force(kernel, variant))


def tune_export() -> str:
    n = int(lib().glu_tune_export(None, 0))
    buf = ctypes.create_string_buffer(n)
    lib().glu_tune_export(buf, n)
    return buf.value.decode()


def tune_import(text: str) -> None:
    A.check("glu_tune_import", lib().glu_tune_import(text.encode()))


def tune_clear() -> None:
    A.check("glu_tune_clear", lib().glu_tune_clear())


def glu_device_status(stream=None) -> int:
    return int(lib().glu_device_status(_stream(stream)))


def glu_fx_filter3(x: torch.Tensor, op: int, out: torch.Tensor | None = None, stream=None):
    """LR operator fixture: 3x3 box (op 0) or [1 2 1]/4 Gaussian (op 1), clamped edges."""
    out = torch.empty_like(x) if out is None else out
    h, w, C = x.shape
    A.check("glu_fx_filter3", lib().glu_fx_filter3(_ptr(x), h, w, C, x.stride(0), _ptr(out),
                                                   out.stride(0), op, _stream(stream)))
    return out


def glu_fx_filter3_u8(x: torch.Tensor, op: int, out: torch.Tensor | None = None, stream=None):
    """glu_fx_filter3 on a uint8 (h, w, C) image read as x / 255; float32 result."""
    if x.dtype != torch.uint8:
        raise TypeError("glu_fx_filter3_u8: uint8 input")
    h, w, C = x.shape
    out = torch.empty((h, w, C), dtype=torch.float32, device=x.device) if out is None else out
    A.check("glu_fx_filter3_u8", lib().glu_fx_filter3_u8(_ptr(x), h, w, C, x.stride(0),
                                                         _ptr(out), out.stride(0), op,
                                                         _stream(stream)))
    return out


def glu_pipeline_host_workspace_size(H: int, W: int, scale: int, params: A.GluParams) -> int:
    return int(lib().glu_pipeline_host_workspace_size(H, W, scale, ctypes.byref(params)))


def glu_pipeline_host(hr_host: torch.Tensor, scale: int, params: A.GluParams, op: int,
                      sat: float, gamma: float, out_host: torch.Tensor,
                      workspace: torch.Tensor, stream=None) -> torch.Tensor:
    """The whole pipeline on host buffers (guide in, Algorithm 2, LR operator, Eq. 1, result
    out) in one library call. hr_host: (H, W, 3) uint8 CPU tensor (pinned for full copy speed);
    out_host: (H, W, 3) float32 CPU tensor; workspace: a CUDA uint8 tensor of at least
    glu_pipeline_host_workspace_size() + 256 bytes. Returns out_host once it holds the result."""
    H, W = hr_host.shape[:2]
    if (hr_host.device.type != "cpu" or out_host.device.type != "cpu"
            or hr_host.dtype != torch.uint8 or out_host.dtype != torch.float32
            or not hr_host.is_contiguous() or not out_host.is_contiguous()
            or tuple(out_host.shape) != (H, W, 3) or tuple(hr_host.shape) != (H, W, 3)):
        raise ValueError("glu_pipeline_host: contiguous (H, W, 3) uint8 / float32 host tensors")
    base = workspace.data_ptr()
    aligned = (base + 255) & ~255
    avail = workspace.numel() - (aligned - base)
    A.check("glu_pipeline_host", lib().glu_pipeline_host(
        _ptr(hr_host), H, W, scale, ctypes.byref(params), op, sat, gamma, _ptr(out_host),
        ctypes.c_void_p(aligned), avail, _stream(stream)))
    return out_host


def glu_fx_point(x: torch.Tensor, sat: float = 1.0, gamma: float = 1.0,
                 out: torch.Tensor | None = None, stream=None):
    """LR operator fixture: saturation about Rec. 601 luma (clamped), then per-channel gamma."""
    out = torch.empty_like(x) if out is None else out
    h, w, _ = x.shape
    A.check("glu_fx_point", lib().glu_fx_point(_ptr(x), h, w, x.stride(0), _ptr(out),
                                               out.stride(0), sat, gamma, _stream(stream)))
    return out


def glu_apply_lrop(theta: Theta, lr: torch.Tensor, filter: int = 0, sat: float = 1.0,
                   gamma: float = 1.0, target: torch.Tensor | None = None,
                   out: torch.Tensor | None = None, out_dtype=torch.float32, stream=None):
    """The LR operator (3x3 filter -1/0/1, then saturation and gamma) on lr (uint8 or float32),
    then Eq. 1, as one issue. Returns (out, target); target holds f(lr)."""
    h, w, _ = lr.shape
    if target is None:
        target = torch.empty((h, w, 3), dtype=torch.float32, device=lr.device)
    if out is None:
        out = torch.empty((theta.H, theta.W, 3), dtype=out_dtype, device=lr.device)
    td, li, ti, oi = theta.desc(), image(lr), image(target), image(out)
    op = A.GluLrOp(filter, sat, gamma)
    A.check("glu_apply_lrop", lib().glu_apply_lrop(ctypes.byref(td), ctypes.byref(li),
                                                   ctypes.byref(op), ctypes.byref(ti),
                                                   ctypes.byref(oi), _stream(stream)))
    return out, target


class GluApplyFn(torch.autograd.Function):
    """T_hat = glu_apply(theta, T_lr) with gradients for T_lr and the weights.

    The pair codes are discrete and held fixed; the backward pass is the library's adjoint
    (a fixed-order reduction, bit-reproducible)."""

    @staticmethod
    def forward(ctx, lr_target, weight, theta, plan=None):
        lr_target = lr_target.contiguous()
        weight = weight.contiguous()
        ctx.theta = theta
        ctx.plan = plan
        ctx.save_for_backward(lr_target, weight)
        return glu_apply(theta, lr_target, weight=weight)

    @staticmethod
    def backward(ctx, grad_out):
        lr_target, weight = ctx.saved_tensors
        g = grad_out.contiguous().to(torch.float32)
        grad_lr, grad_w = glu_apply_backward(ctx.theta, lr_target, g,
                                             grad_w=ctx.needs_input_grad[1], weight=weight,
                                             plan=ctx.plan)
        return (grad_lr if ctx.needs_input_grad[0] else None,
                grad_w if ctx.needs_input_grad[1] else None, None, None)


def apply_autograd(theta: Theta, lr_target: torch.Tensor, weight: torch.Tensor | None = None,
                   plan: torch.Tensor | None = None):
    """Differentiable Eq. 1 (w.r.t. the LR target and, if it requires grad, the weights). With
    `plan` (glu_apply_backward_plan(theta)) the backward pass reads the precomputed inverse map,
    the fast form for many passes over one Theta."""
    w = theta.weight_f32() if weight is None else weight
    return GluApplyFn.apply(lr_target, w, theta, plan)

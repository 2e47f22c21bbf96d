"""numpy/ctypes front end of the FP64 C oracle (glu_oracle.c).

Test infrastructure. Colour units: when any image of a call is uint8, all images of the call are
passed to C in raw 0..255 units (floats in [0, 1] are scaled by 255), so squared distances
between uint8 colours are exact integers and exact ties stay exact; otherwise colours are in
[0, 1]. eps and tau are always given in [0, 1] units and errors are returned in [0, 1] units.
Grid downsampling and Algorithm 2 return uint8 LR images for uint8 guides (their pixels are
copies of guide pixels). Each C routine follows one equation or algorithm of the paper:
  downsample_grid / downsample_box   regular grid (Sec. 3.3) and block-mean downsampling
  glu_fast                           Algorithm 1 with the Eq. 5 weight and the Eq. 3 error
  glu_exact                          GLU* of Sec. 3.1, all pairs with the Eq. 4 weight
  glu_gnu                            the weight-1 special case (GNU)
  apply / apply_adjoint              Eq. 1 and its adjoint
  label_components                   connected components of Algorithm 2
  joint                              Algorithm 2 (PAPER and STRICT readings)
  ls_update / ls_joint               a least-squares LR colour update alternated with Algorithm 1
                                     (not the paper's method: the alternative joint scheme the
                                     GPU path offers beside Algorithm 2)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None
_d = ctypes.c_double
_i = ctypes.c_int
_p = ctypes.c_void_p


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build())
        sig = {
            "oracle_downsample_grid": [_p, _i, _i, _i, _i, _p],
            "oracle_downsample_box": [_p, _i, _i, _i, _i, _p],
            "oracle_glu_fast": [_p, _i, _i, _p, _i, _i, _d, _d, _p, _p, _p, _p, _p, _p, _i],
            "oracle_fast_pair": [_p, _i, _i, _p, _i, _i, _d, _d, _i, _i, _i, _i, _p, _p],
            "oracle_glu_exact": [_p, _i, _i, _p, _i, _i, _d, _d, _p, _p, _p, _p, _i],
            "oracle_glu_gnu": [_p, _i, _i, _p, _i, _i, _d, _p, _p],
            "oracle_apply": [_p, _p, _p, _i, _i, _i, _i, _p, _i, _p],
            "oracle_apply_adjoint": [_p, _p, _p, _i, _i, _i, _i, _p, _i, _p, _p, _p],
            "oracle_label_components": [_p, _i, _i, _i, _p],
            "oracle_joint": [_p, _i, _i, _i, _i, _d, _d, _d, _i, _i, _i, _p, _p, _p, _p, _p, _p,
                             _p, ctypes.c_int64, _p, ctypes.c_int64, _d, _p, ctypes.c_int64, _d,
                             _d, _i],
            "oracle_ls_update": [_p, _i, _i, _p, _i, _i, _p, _p, _p, _d, _p],
            "oracle_op_box3": [_p, _i, _i, _i, _p],
            "oracle_op_gauss3": [_p, _i, _i, _i, _p],
            "oracle_op_saturation": [_p, ctypes.c_size_t, _d, _p],
            "oracle_op_gamma": [_p, ctypes.c_size_t, _d, _p],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = _i
        _LIB = lib
    return _LIB


def _ptr(a):
    return None if a is None else a.ctypes.data


def _chk(rc, what):
    if rc < 0:
        raise RuntimeError(f"{what} failed with {rc}")
    return rc


def to_unit(img) -> np.ndarray:
    """Colours as contiguous float64 in [0, 1]: uint8 / 255, floats unchanged."""
    a = np.asarray(img)
    if a.dtype == np.uint8:
        return np.ascontiguousarray(a.astype(np.float64) / 255.0)
    if a.dtype == np.float64:
        return np.ascontiguousarray(a)
    return np.ascontiguousarray(a.astype(np.float64))


def colours(*imgs):
    """The images of one call in common units: raw 0..255 if any of them is uint8 (floats in
    [0, 1] scaled by 255), else [0, 1]. Returns ([float64 arrays], unit)."""
    arrs = [np.asarray(a) for a in imgs]
    unit = 255.0 if any(a.dtype == np.uint8 for a in arrs) else 1.0
    out = []
    for a in arrs:
        f = np.ascontiguousarray(a, dtype=np.float64)
        if a.dtype != np.uint8 and unit != 1.0:
            f = f * unit
        out.append(f)
    return out, unit


def lr_dims(H, W, s):
    return (H + s - 1) // s, (W + s - 1) // s


def downsample_grid(I, s):
    """Regular grid downsampling; uint8 in -> uint8 out (exact copies), floats stay floats."""
    a = np.asarray(I)
    F = np.ascontiguousarray(a, dtype=np.float64)
    H, W, C = F.shape
    h, w = lr_dims(H, W, s)
    L = np.empty((h, w, C), np.float64)
    _chk(_lib().oracle_downsample_grid(_ptr(F), H, W, C, s, _ptr(L)), "downsample_grid")
    return L.astype(np.uint8) if a.dtype == np.uint8 else L


def downsample_box(I, s):
    """Block mean, returned as float64 colours in [0, 1]."""
    a = np.asarray(I)
    F = np.ascontiguousarray(a, dtype=np.float64)
    H, W, C = F.shape
    h, w = lr_dims(H, W, s)
    L = np.empty((h, w, C), np.float64)
    _chk(_lib().oracle_downsample_box(_ptr(F), H, W, C, s, _ptr(L)), "downsample_box")
    return L / 255.0 if a.dtype == np.uint8 else L


def glu_fast(I, L, s, S, eps=1e-3, gaps=False, threads=0):
    """Algorithm 1 on every HR pixel: returns dict(ka, kb, omega, err[, gap_a, gap_b])."""
    (I, L), unit = colours(I, L)
    H, W, _ = I.shape
    out = {k: np.empty((H, W), np.int32) for k in ("ka", "kb")}
    out["omega"] = np.empty((H, W), np.float64)
    out["err"] = np.empty((H, W), np.float64)
    if gaps:
        out["gap_a"] = np.empty((H, W), np.float64)
        out["gap_b"] = np.empty((H, W), np.float64)
    _chk(_lib().oracle_glu_fast(_ptr(I), H, W, _ptr(L), s, S, eps, unit, _ptr(out["ka"]),
                                _ptr(out["kb"]), _ptr(out["omega"]), _ptr(out["err"]),
                                _ptr(out.get("gap_a")), _ptr(out.get("gap_b")), threads),
         "glu_fast")
    return out


def fast_pair(I, L, s, S, y, x, ka, kb, eps=1e-3, unit=None):
    """Eq. 5 weight and Eq. 3 error of a given window pair at HR pixel (y, x). With `unit`
    given, I and L must already be contiguous float64 in those units (see colours())."""
    if unit is None:
        (I, L), unit = colours(I, L)
    H, W, _ = I.shape
    om = ctypes.c_double()
    er = ctypes.c_double()
    _chk(_lib().oracle_fast_pair(_ptr(I), H, W, _ptr(L), s, S, eps, unit, int(y), int(x),
                                 int(ka), int(kb), ctypes.byref(om), ctypes.byref(er)),
         "fast_pair")
    return om.value, er.value


def glu_exact(I, L, s, S, eps=1e-3, threads=0):
    (I, L), unit = colours(I, L)
    H, W, _ = I.shape
    out = {k: np.empty((H, W), np.int32) for k in ("ka", "kb")}
    out["omega"] = np.empty((H, W), np.float64)
    out["err"] = np.empty((H, W), np.float64)
    _chk(_lib().oracle_glu_exact(_ptr(I), H, W, _ptr(L), s, S, eps, unit, _ptr(out["ka"]),
                                 _ptr(out["kb"]), _ptr(out["omega"]), _ptr(out["err"]), threads),
         "glu_exact")
    return out


def glu_gnu(I, L, s, S):
    (I, L), unit = colours(I, L)
    H, W, _ = I.shape
    ka = np.empty((H, W), np.int32)
    err = np.empty((H, W), np.float64)
    _chk(_lib().oracle_glu_gnu(_ptr(I), H, W, _ptr(L), s, S, unit, _ptr(ka), _ptr(err)),
         "glu_gnu")
    return {"ka": ka, "err": err}


def apply(ka, kb, omega, s, S, T):
    ka = np.ascontiguousarray(ka, np.int32)
    kb = np.ascontiguousarray(kb, np.int32)
    omega = np.ascontiguousarray(omega, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    H, W = ka.shape
    C = T.shape[2]
    out = np.empty((H, W, C), np.float64)
    _chk(_lib().oracle_apply(_ptr(ka), _ptr(kb), _ptr(omega), H, W, s, S, _ptr(T), C, _ptr(out)),
         "apply")
    return out


def apply_adjoint(ka, kb, omega, s, S, T, G):
    ka = np.ascontiguousarray(ka, np.int32)
    kb = np.ascontiguousarray(kb, np.int32)
    omega = np.ascontiguousarray(omega, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    G = np.ascontiguousarray(G, np.float64)
    H, W = ka.shape
    h, w, C = T.shape
    gT = np.empty((h, w, C), np.float64)
    gw = np.empty((H, W), np.float64)
    _chk(_lib().oracle_apply_adjoint(_ptr(ka), _ptr(kb), _ptr(omega), H, W, s, S, _ptr(T), C,
                                     _ptr(G), _ptr(gT), _ptr(gw)), "apply_adjoint")
    return gT, gw


def label_components(mask, conn=8):
    mask = np.ascontiguousarray(mask, np.uint8)
    H, W = mask.shape
    labels = np.empty((H, W), np.int32)
    M = _chk(_lib().oracle_label_components(_ptr(mask), H, W, conn, _ptr(labels)),
             "label_components")
    return labels, M


JSTAT = 12


def joint(I, s, S, N=3, tau=30.0 / 255.0, eps=1e-3, strict=True, conn=8, log_cap=1 << 20,
          force=None, force_tol=0.0, argmax=None, argmax_tol=0.0, thr_tol=0.0, threads=0):
    """Algorithm 2. Returns dict(L, ka, kb, omega, err, R0, iters=[...], accept_log); L is
    uint8 for a uint8 guide. `force` (int8 keep/rollback per trial, in order) is followed only
    where the oracle's own margin |e1 - e0| <= force_tol; `argmax` (int32 records of another
    implementation's decisions, the log of glu_test_joint_argmax_log) holds replacement choices,
    followed only where the logged pixel's FP64 error is within argmax_tol of the block's
    largest, and large-error memberships, followed only where the oracle's error is within
    thr_tol of tau (see glu_oracle.c)."""
    is_u8 = np.asarray(I).dtype == np.uint8
    (I,), unit = colours(I)
    H, W, _ = I.shape
    h, w = lr_dims(H, W, s)
    L = np.empty((h, w, 3), np.float64)
    ka = np.empty((H, W), np.int32)
    kb = np.empty((H, W), np.int32)
    om = np.empty((H, W), np.float64)
    er = np.empty((H, W), np.float64)
    stats = np.full(1 + JSTAT * max(N, 1), np.nan)
    log = np.full(log_cap, -1, np.int8)
    fz = None if force is None else np.ascontiguousarray(force, np.int8)
    am = None
    if argmax is not None:
        am = np.asarray(argmax, np.int32).reshape(-1, 4)
        am = np.ascontiguousarray(am[np.lexsort((am[:, 2], am[:, 1], am[:, 0]))])
    _chk(_lib().oracle_joint(_ptr(I), H, W, s, S, eps, tau, unit, N, int(bool(strict)), conn,
                             _ptr(L),
                             _ptr(ka), _ptr(kb), _ptr(om), _ptr(er), _ptr(stats), _ptr(log),
                             log_cap, _ptr(fz), 0 if fz is None else fz.size, force_tol,
                             _ptr(am), 0 if am is None else am.shape[0], argmax_tol, thr_tol,
                             threads), "joint")
    iters = []
    for it in range(N):
        st = stats[1 + it * JSTAT: 1 + (it + 1) * JSTAT]
        if np.isnan(st[0]):
            break
        iters.append(dict(n_large=int(st[0]), M=int(st[1]), accepted=int(st[2]),
                          rolled_back=int(st[3]), residual=float(st[4]),
                          min_decision_margin=float(st[5]), min_threshold_margin=float(st[6]),
                          searched=int(st[7]), replayed=int(st[8]),
                          argmax_near_ties=int(st[9]), argmax_replayed=int(st[10]),
                          threshold_replayed=int(st[11])))
        if st[0] == 0:
            break
    nlog = sum(it["M"] for it in iters)
    if is_u8:
        L = L.astype(np.uint8)
    return dict(L=L, ka=ka, kb=kb, omega=om, err=er, R0=float(stats[0]), iters=iters,
                accept_log=log[:min(nlog, log_cap)].copy())


def ls_update(I, L, s, S, ka, kb, omega):
    """One least-squares LR colour update for a fixed Theta (see glu_oracle.c). I: uint8 or
    float guide; L: float LR colours in [0, 1]. Returns float64 LR colours in [0, 1]."""
    (I,), unit = colours(I)
    Lf = np.ascontiguousarray(np.asarray(L, np.float64) * unit)
    H, W, _ = I.shape
    out = np.empty_like(Lf)
    _chk(_lib().oracle_ls_update(_ptr(I), H, W, _ptr(Lf), s, S,
                                 _ptr(np.ascontiguousarray(ka, np.int32)),
                                 _ptr(np.ascontiguousarray(kb, np.int32)),
                                 _ptr(np.ascontiguousarray(omega, np.float64)), unit, _ptr(out)),
         "ls_update")
    return out / unit


def ls_joint(I, s, S, N=3, eps=1e-3, L0=None):
    """Alternate Algorithm 1 (reassignment) and ls_update (LR colour update), starting from the
    grid-downsampled guide (or L0, colours in [0, 1]): an update is kept only if the residual
    R = sum_p E_p of Algorithm 1 on the new LR image is below the current one; the first that is
    not ends the loop. Returns dict(L (float64, [0, 1]), ka, kb, omega, err, R0, residuals)."""
    I = np.asarray(I)
    if L0 is None:
        L0 = to_unit(downsample_grid(I, s))
    L = np.asarray(L0, np.float64)
    f = glu_fast(I, L, s, S, eps=eps)
    R = float(f["err"].sum())
    out = dict(R0=R, residuals=[])
    for _ in range(N):
        Ln = ls_update(I, L, s, S, f["ka"], f["kb"], f["omega"])
        fn = glu_fast(I, Ln, s, S, eps=eps)
        Rn = float(fn["err"].sum())
        if not Rn < R:
            break
        L, f, R = Ln, fn, Rn
        out["residuals"].append(R)
    out.update(L=L, ka=f["ka"], kb=f["kb"], omega=f["omega"], err=f["err"])
    return out


def op_box3(X):
    X = np.ascontiguousarray(X, np.float64)
    h, w, C = X.shape
    Y = np.empty_like(X)
    _lib().oracle_op_box3(_ptr(X), h, w, C, _ptr(Y))
    return Y


def op_gauss3(X):
    X = np.ascontiguousarray(X, np.float64)
    h, w, C = X.shape
    Y = np.empty_like(X)
    _lib().oracle_op_gauss3(_ptr(X), h, w, C, _ptr(Y))
    return Y


def op_saturation(X, f=1.3):
    X = np.ascontiguousarray(X, np.float64)
    Y = np.empty_like(X)
    _lib().oracle_op_saturation(_ptr(X), X.shape[0] * X.shape[1], f, _ptr(Y))
    return Y


def op_gamma(X, g=0.8):
    X = np.ascontiguousarray(X, np.float64)
    Y = np.empty_like(X)
    _lib().oracle_op_gamma(_ptr(X), X.size, g, _ptr(Y))
    return Y

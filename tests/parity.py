"""Comparison helpers for GPU-vs-oracle parity (used by the gpu tests and the smoke check).

Rules (from the accuracy targets of the hot path):
  * pair codes identical, except at near-tie pixels where the oracle's best and second-best
    candidates (of different colour) are closer than 1e-5; there the GPU's pair must still be
    a valid optimum: its a within 1e-5 of the nearest distance, and its FP64 error within 1e-5
    of the best error achievable with that a (Algorithm 1's second step);
  * weights within 1e-4 (float32 storage), 2.5e-4 (float16), 2e-5 (unorm16: 7.6e-6 of
    quantisation plus the FP32 weight error) where codes match;
  * error map within 1e-5; reconstructions within 1e-3 max-abs on [0, 1] colours.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

NEAR_TIE = 1e-5
W_TOL = {0: 1e-4, 1: 2.5e-4, 2: 2e-5}


def check_search(I, L, s, S, theta, err_gpu=None, eps=1e-3, wfmt=0, ref=None, gnu=False):
    """Compare a GPU Theta (and error map) with the oracle on the same I and L. Returns a
    report dict; raises AssertionError on a parity failure."""
    K = S * S
    if ref is None:
        ref = O.glu_fast(I, L, s, S, eps=eps, gaps=True)
    codes = theta.codes_i32().cpu().numpy()
    ka, kb = codes // K, codes % K
    if gnu:
        g = O.glu_gnu(I, L, s, S)
        assert np.array_equal(ka, kb)
        tie = ref["gap_a"] < NEAR_TIE
        mism = ka != g["ka"]
        assert not (mism & ~tie).any(), f"{int((mism & ~tie).sum())} GNU codes differ"
        w = theta.weight_f32().cpu().numpy()
        assert np.all(w == 1.0)
        if err_gpu is not None:
            e = err_gpu.cpu().numpy()
            assert np.abs(e - g["err"])[~mism].max() < 1e-5
        return dict(near_ties=int(tie.sum()), mismatches=int(mism.sum()))
    tie = (ref["gap_a"] < NEAR_TIE) | (ref["gap_b"] < NEAR_TIE)
    same = (ka == ref["ka"]) & (kb == ref["kb"])
    bad = ~same & ~tie
    assert not bad.any(), (f"{int(bad.sum())} pair codes differ away from near-ties, e.g. at "
                           f"{np.argwhere(bad)[:5].tolist()}")
    # mismatches at near-ties: the GPU's pair must be a valid optimum within the tolerance
    (Ic, Lc), unit = O.colours(I, L)
    H, W = codes.shape
    h, w = Lc.shape[:2]
    r = (S - 1) // 2
    for (y, x) in np.argwhere(~same)[:5000]:
        ga, gb = int(ka[y, x]), int(kb[y, x])
        py, px = y // s, x // s
        valid = [k for k in range(K) if 0 <= py + k // S - r < h and 0 <= px + k % S - r < w]
        d = {k: np.linalg.norm(Ic[y, x] - Lc[py + k // S - r, px + k % S - r]) / unit
             for k in valid}
        assert d[ga] <= min(d.values()) + NEAR_TIE
        errs = [O.fast_pair(Ic, Lc, s, S, y, x, ga, k, eps, unit=unit)[1] for k in valid]
        _, e_gpu_pair = O.fast_pair(Ic, Lc, s, S, y, x, ga, gb, eps, unit=unit)
        assert e_gpu_pair <= min(errs) + NEAR_TIE
    wg = theta.weight_f32().cpu().numpy()
    dw = np.abs(wg - ref["omega"])[same]
    assert dw.max(initial=0.0) < W_TOL[wfmt], f"weight error {dw.max()}"
    rep = dict(near_ties=int(tie.sum()), mismatches=int((~same).sum()),
               max_dw=float(dw.max(initial=0.0)))
    if err_gpu is not None:
        e = err_gpu.cpu().numpy().astype(np.float64)
        de = np.abs(e - ref["err"])[same]
        assert de.max(initial=0.0) < 1e-5, f"error-map difference {de.max()}"
        rep["max_derr"] = float(de.max(initial=0.0))
    return rep


def lr_like_gpu(lr_tensor):
    """The LR image the GPU used, as a numpy array in its own dtype (uint8 or float)."""
    a = lr_tensor.cpu().numpy()
    return a if a.dtype == np.uint8 else a.astype(np.float64)


def exact_pair_err(Ic, Lc, unit, s, S, y, x, ka, kb, eps=1e-3):
    """Eq. 4 weight and Eq. 3 error (FP64, [0, 1] units) of window pair (ka, kb) at (y, x);
    Ic, Lc as returned by oracle.colours()."""
    r = (S - 1) // 2
    py, px = y // s, x // s
    La = Lc[py + ka // S - r, px + ka % S - r]
    Lb = Lc[py + kb // S - r, px + kb % S - r]
    I = Ic[y, x]
    d = La - Lb
    den = d @ d + eps * unit * unit
    w = ((I - Lb) @ d) / den if den > 0 else 1.0
    return w, np.linalg.norm(w * d + Lb - I) / unit


def check_exact(I, L, s, S, theta, err_gpu, eps=1e-3, ref=None):
    """GLU* parity: codes equal except where the GPU's pair is, in FP64, within NEAR_TIE of the
    oracle's best error (under 1 % of the pixels); where codes match, weights within
    1e-4 * max(1, |w|) (Eq. 4 weights are unclamped) and errors within 1e-5."""
    K = S * S
    if ref is None:
        ref = O.glu_exact(I, L, s, S, eps=eps)
    codes = theta.codes_i32().cpu().numpy()
    ka, kb = codes // K, codes % K
    same = (ka == ref["ka"]) & (kb == ref["kb"])
    (Ic, Lc), unit = O.colours(I, L)
    for (y, x) in np.argwhere(~same)[:2000]:
        _, e = exact_pair_err(Ic, Lc, unit, s, S, y, x, int(ka[y, x]), int(kb[y, x]), eps)
        assert e <= ref["err"][y, x] + NEAR_TIE, (y, x, e, ref["err"][y, x])
    assert (~same).mean() < 0.01
    wg = theta.weight_f32().cpu().numpy().astype(np.float64)
    dw = np.abs(wg - ref["omega"]) / np.maximum(1.0, np.abs(ref["omega"]))
    assert dw[same].max(initial=0.0) < 1e-4
    de = np.abs(err_gpu.cpu().numpy().astype(np.float64) - ref["err"])
    assert de[same].max(initial=0.0) < 1e-5
    return dict(mismatches=int((~same).sum()), max_dw=float(dw[same].max(initial=0.0)),
                max_derr=float(de[same].max(initial=0.0)))

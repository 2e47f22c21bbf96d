"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: brute force on tiny inputs,
closed forms, invariants the paper derives, special cases that reduce to a library routine.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_img(rng, H, W, C=3):
    return rng.integers(0, 256, size=(H, W, C), dtype=np.uint8)


def window_cols(L, s, S, y, x):
    """Valid window pixels (k, colour) of HR pixel (y, x): the Omega of Eq. 1."""
    h, w, _ = L.shape
    r = (S - 1) // 2
    out = []
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            v, u = y // s + dy, x // s + dx
            if 0 <= v < h and 0 <= u < w:
                out.append(((dy + r) * S + (dx + r), L[v, u]))
    return out


# ------------------------------------------------------------------ parameters the paper prints

def test_paper_parameters_golden():
    g = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    assert g["tau"]["value"] == pytest.approx(30 / 255)
    import inspect
    sig = inspect.signature(O.joint)
    assert sig.parameters["tau"].default == pytest.approx(g["tau"]["value"])
    assert sig.parameters["N"].default == g["max_iterations_N"]["value"]
    assert sig.parameters["eps"].default == g["eps"]["value"]
    # the pair counts the paper states for a 3x3 window: all unordered pairs vs. a fixed a
    K = g["window_size_S"]["value"] ** 2
    assert K * (K - 1) // 2 == g["pairs_exhaustive_3x3"]["value"]
    assert K == g["pairs_fast_3x3"]["value"]   # b ranges over the whole window, b = a included
    L = np.zeros((5, 5, 3))
    assert len(window_cols(L, 2, 3, 4, 4)) == K


# ------------------------------------------------------------------------------- downsampling

@pytest.mark.parametrize("H,W,s", [(8, 8, 2), (9, 13, 4), (17, 5, 3), (16, 16, 16), (7, 7, 8)])
def test_grid_downsample_sample_positions(H, W, s):
    # an image whose colour encodes its own coordinates; grid sampling must pick, per block,
    # the pixel floor(e/2) into the block (e = block extent, partial at the far edge)
    yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    I = np.stack([yy / 1000.0, xx / 1000.0, np.zeros_like(yy, dtype=float)], axis=-1)
    L = O.downsample_grid(I, s)
    h, w = O.lr_dims(H, W, s)
    assert L.shape == (h, w, 3)
    for v in range(h):
        ey = min(s, H - v * s)
        for u in range(w):
            ex = min(s, W - u * s)
            assert round(L[v, u, 0] * 1000) == v * s + ey // 2
            assert round(L[v, u, 1] * 1000) == u * s + ex // 2


@pytest.mark.parametrize("H,W,s", [(8, 8, 2), (9, 13, 4), (10, 3, 3)])
def test_box_downsample_closed_form(H, W, s):
    xx = np.broadcast_to(np.arange(W, dtype=float)[None, :, None], (H, W, 3))
    L = O.downsample_box(xx, s)
    h, w = O.lr_dims(H, W, s)
    for u in range(w):
        lo, hi = u * s, min(W, u * s + s)
        assert np.allclose(L[:, u, :], (lo + hi - 1) / 2.0)
    c = np.full((H, W, 3), 0.3)
    assert np.allclose(O.downsample_box(c, s), 0.3)


# ------------------------------------------------------------ GLU* (Sec. 3.1, Eq. 4) pinned

def brute_pair_min(Ip, La, Lb):
    """min over real omega of ||omega La + (1 - omega) Lb - Ip|| by ternary search on a
    convex function over a wide bracket (no closed form used)."""
    lo, hi = -1e4, 1e4
    f = lambda o: np.linalg.norm(o * La + (1 - o) * Lb - Ip)
    for _ in range(400):
        m1, m2 = lo + (hi - lo) / 3, hi - (hi - lo) / 3
        if f(m1) <= f(m2):
            hi = m2
        else:
            lo = m1
    return f(0.5 * (lo + hi))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_exact_matches_brute_force_tiny(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    H = W = 8
    s, S = 2, 3
    I = O.to_unit(rand_img(rng, H, W))
    L = O.to_unit(rand_img(rng, 4, 4))
    ex = O.glu_exact(I, L, s, S, eps=0.0)
    for y in range(H):
        for x in range(W):
            cols = window_cols(L, s, S, y, x)
            best = min(brute_pair_min(I[y, x], cols[i][1], cols[j][1])
                       for i in range(len(cols)) for j in range(i + 1, len(cols)))
            assert ex["err"][y, x] == pytest.approx(best, abs=1e-9)


def test_exact_eps0_residual_orthogonal_to_colour_line(rng):
    # Eq. 4 with eps = 0 is the projection of I_p on the line through L_a and L_b
    H = W = 12
    s, S = 3, 3
    I = O.to_unit(rand_img(rng, H, W))
    L = O.to_unit(rand_img(rng, 4, 4))
    ex = O.glu_exact(I, L, s, S, eps=0.0)
    h, w = 4, 4
    for y in range(H):
        for x in range(W):
            ka, kb, om = ex["ka"][y, x], ex["kb"][y, x], ex["omega"][y, x]
            va, ua = y // s + ka // S - 1, x // s + ka % S - 1
            vb, ub = y // s + kb // S - 1, x // s + kb % S - 1
            La, Lb = L[va, ua], L[vb, ub]
            res = om * La + (1 - om) * Lb - I[y, x]
            assert abs(np.dot(res, La - Lb)) < 1e-12
            assert ex["err"][y, x] == pytest.approx(np.linalg.norm(res), abs=1e-12)


# --------------------------------------------------------- Algorithm 1 (FAST) pinned

@pytest.mark.parametrize("seed,s,S", [(1, 2, 3), (2, 3, 5), (3, 4, 3), (4, 2, 1)])
def test_fast_between_exact_and_gnu(seed, s, S):
    rng = np.random.Generator(np.random.PCG64(seed))
    H, W = 14, 11
    I = rand_img(rng, H, W)
    h, w = O.lr_dims(H, W, s)
    L = rand_img(rng, h, w)
    fa = O.glu_fast(I, L, s, S)
    gn = O.glu_gnu(I, L, s, S)
    # b = a is a candidate, so FAST never does worse than nearest-colour (GNU)
    assert np.all(fa["err"] <= gn["err"] + 1e-15)
    # a is the nearest colour in the window: brute force over the window
    Iu, Lu = O.to_unit(I), O.to_unit(L)
    for y in range(H):
        for x in range(W):
            cols = window_cols(Lu, s, S, y, x)
            d = [np.linalg.norm(Iu[y, x] - c) for _, c in cols]
            assert gn["err"][y, x] == pytest.approx(min(d), abs=1e-15)
            assert gn["ka"][y, x] == cols[int(np.argmin(d))][0]
            assert fa["ka"][y, x] == gn["ka"][y, x]
    # the Eq. 5 weight always lies in [0, 1]
    assert np.all(fa["omega"] >= 0) and np.all(fa["omega"] <= 1)
    if S > 1:
        ex = O.glu_exact(I, L, s, S, eps=0.0)
        # any fixed-weight pair is no better than the best least-squares pair
        assert np.all(fa["err"] >= ex["err"] - 1e-12)


@pytest.mark.parametrize("eps", [0.0, 1e-3])
def test_fast_on_colour_segment_closed_form(rng, eps):
    # LR made of two colours c1, c2; HR pixels on the segment between them: I_p = t c1 + (1-t) c2.
    # With a = the nearer endpoint, Eq. 5 gives omega = d_b / (d_a + d_b + eps) and the Eq. 3
    # error is |omega - t| * |c1 - c2| (eps = 0: exact, omega = t, error 0).
    c1 = np.array([0.9, 0.2, 0.1])
    c2 = np.array([0.1, 0.6, 0.8])
    h = w = 3
    L = np.zeros((h, w, 3))
    for v in range(h):
        for u in range(w):
            L[v, u] = c1 if (v + u) % 2 == 0 else c2
    s, S = 4, 3
    H = W = 12
    t = rng.uniform(0.0, 1.0, size=(H, W))
    I = t[..., None] * c1 + (1 - t[..., None]) * c2
    fa = O.glu_fast(I, L, s, S, eps=eps)
    D = np.linalg.norm(c1 - c2)
    for y in range(H):
        for x in range(W):
            tt = t[y, x]
            # the nearer endpoint is a: c1 if t > 1/2
            ta = tt if tt >= 0.5 else 1 - tt
            da, db = (1 - ta) * D, ta * D
            om = db / (da + db + eps)
            expect = min(da, abs(om - ta) * D)   # b = a gives d_a
            assert fa["err"][y, x] == pytest.approx(expect, abs=1e-12)
            if eps == 0.0 and min(tt, 1 - tt) > 1e-9:
                assert fa["omega"][y, x] == pytest.approx(ta, abs=1e-12)
                assert fa["err"][y, x] < 1e-12


@pytest.mark.parametrize("s,S", [(2, 3), (4, 5), (3, 3), (8, 5)])
def test_exact_representability(rng, s, S):
    # HR = nearest-neighbour upsampling of an LR image: grid downsampling recovers the LR image,
    # Algorithm 1 reproduces every pixel exactly, and Eq. 1 with T = I_down returns the HR image.
    h, w = 5, 7
    Lu8 = rand_img(rng, h, w)
    I = np.repeat(np.repeat(Lu8, s, axis=0), s, axis=1)
    L = O.downsample_grid(I, s)
    assert L.dtype == np.uint8 and np.array_equal(L, Lu8)
    fa = O.glu_fast(I, L, s, S)
    assert np.all(fa["err"] == 0.0)
    out = O.apply(fa["ka"], fa["kb"], fa["omega"], s, S, O.to_unit(L))
    assert np.allclose(out, O.to_unit(I), atol=1e-15)
    # the same holds for colours given in [0, 1] floats
    fb = O.glu_fast(O.to_unit(I), O.to_unit(L), s, S)
    assert np.all(fb["err"] == 0.0)


# ------------------------------------------------------------------- Eq. 1 apply and adjoint

def _random_theta(rng, H, W, s, S):
    I = rand_img(rng, H, W)
    h, w = O.lr_dims(H, W, s)
    L = rand_img(rng, h, w)
    fa = O.glu_fast(I, L, s, S)
    return fa, (h, w)


def test_apply_affine_invariance(rng):
    # Eq. 7-8: if T_down = A I_down + c locally (here globally), the same Theta gives A I_hat + c
    H, W, s, S = 20, 17, 4, 3
    fa, (h, w) = _random_theta(rng, H, W, s, S)
    T = rng.uniform(size=(h, w, 3))
    A = rng.normal(size=(3, 3))
    c = rng.normal(size=3)
    lhs = O.apply(fa["ka"], fa["kb"], fa["omega"], s, S, T @ A.T + c)
    rhs = O.apply(fa["ka"], fa["kb"], fa["omega"], s, S, T) @ A.T + c
    assert np.allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("C", [1, 3])
def test_apply_adjoint_dot_product_and_fd(rng, C):
    H, W, s, S = 13, 18, 3, 5
    fa, (h, w) = _random_theta(rng, H, W, s, S)
    T = rng.uniform(size=(h, w, C))
    G = rng.normal(size=(H, W, C))
    Y = O.apply(fa["ka"], fa["kb"], fa["omega"], s, S, T)
    gT, gw = O.apply_adjoint(fa["ka"], fa["kb"], fa["omega"], s, S, T, G)
    # <apply(T), G> = <T, apply^T(G)>
    assert np.sum(Y * G) == pytest.approx(np.sum(T * gT), rel=1e-12)
    # d/d omega by central differences (the map is affine in omega: exact up to rounding)
    hstep = 1e-3
    for (y, x) in [(0, 0), (5, 7), (H - 1, W - 1), (6, 2)]:
        om = fa["omega"].copy()
        om[y, x] += hstep
        fp = np.sum(O.apply(fa["ka"], fa["kb"], om, s, S, T) * G)
        om[y, x] -= 2 * hstep
        fm = np.sum(O.apply(fa["ka"], fa["kb"], om, s, S, T) * G)
        assert (fp - fm) / (2 * hstep) == pytest.approx(gw[y, x], abs=1e-9)
    # d/dT of a quadratic loss 0.5 ||apply(T) - Z||^2 by central differences
    Z = rng.uniform(size=(H, W, C))
    R = Y - Z
    gTq, _ = O.apply_adjoint(fa["ka"], fa["kb"], fa["omega"], s, S, T, R)
    for (v, u, c) in [(0, 0, 0), (h - 1, w - 1, C - 1), (2, 3, 0)]:
        Tp = T.copy(); Tp[v, u, c] += hstep
        Tm = T.copy(); Tm[v, u, c] -= hstep
        lp = 0.5 * np.sum((O.apply(fa["ka"], fa["kb"], fa["omega"], s, S, Tp) - Z) ** 2)
        lm = 0.5 * np.sum((O.apply(fa["ka"], fa["kb"], fa["omega"], s, S, Tm) - Z) ** 2)
        assert (lp - lm) / (2 * hstep) == pytest.approx(gTq[v, u, c], abs=1e-8)


# -------------------------------------------------------- connected components (Algorithm 2)

@pytest.mark.parametrize("conn", [8, 4])
@pytest.mark.parametrize("density", [0.05, 0.3, 0.6])
def test_components_match_scipy(rng, conn, density):
    ndi = pytest.importorskip("scipy.ndimage")
    mask = rng.uniform(size=(37, 53)) < density
    labels, M = O.label_components(mask, conn=conn)
    st = np.ones((3, 3)) if conn == 8 else ndi.generate_binary_structure(2, 1)
    ref, Mref = ndi.label(mask, structure=st)
    assert M == Mref
    # same partition; our numbering follows the smallest raster index of each component
    first = {}
    for p, l in enumerate(ref.ravel()):
        if l and l not in first:
            first[l] = len(first)
    remap = np.full(Mref + 1, -1)
    for l, i in first.items():
        remap[l] = i
    assert np.array_equal(labels, remap[ref])


# ------------------------------------------------------------------------ Algorithm 2 pinned

def _total_error_fresh(I, L, s, S, eps=1e-3):
    return O.glu_fast(I, L, s, S, eps=eps)


@pytest.mark.parametrize("seed,s,S", [(1, 4, 3), (2, 8, 5), (3, 4, 5)])
def test_joint_strict_invariants(seed, s, S):
    from paper_2307_09582_gb300.inputs import plain_256_scene, render_u8
    sc = plain_256_scene(seed=seed, size=128)
    I = render_u8(sc)
    j = O.joint(I, s, S, N=4, strict=True)
    # total error never increases across iterations
    Rs = [j["R0"]] + [it["residual"] for it in j["iters"] if it["n_large"] > 0]
    assert all(b <= a + 1e-9 for a, b in zip(Rs, Rs[1:]))
    # Theta and E stay the Algorithm 1 result for the current LR image
    fr = _total_error_fresh(I, j["L"], s, S)
    assert np.array_equal(fr["ka"], j["ka"]) and np.array_equal(fr["kb"], j["kb"])
    assert np.array_equal(fr["err"], j["err"])
    assert float(j["err"].sum()) == pytest.approx(Rs[-1], rel=1e-12)
    # every LR pixel is exactly one HR pixel of its own block (Eq. 6 constraint)
    assert j["L"].dtype == np.uint8
    h, w, _ = j["L"].shape
    for v in range(h):
        for u in range(w):
            blk = I[v * s:(v + 1) * s, u * s:(u + 1) * s].reshape(-1, 3)
            assert np.any(np.all(blk == j["L"][v, u], axis=1))
    # the joint result is no worse than plain grid downsampling
    assert j["err"].sum() <= j["R0"] + 1e-9


@pytest.mark.parametrize("strict", [True, False])
def test_joint_recovers_planted_dot(strict):
    # a flat image with one 2x2 dot away from every grid sample: grid downsampling loses the dot
    # (its pixels have error |d - c| > tau); one iteration puts the dot's colour into the LR image
    # and every pixel becomes exactly representable.
    s, S = 4, 3
    H = W = 32
    I = np.full((H, W, 3), 0.25)
    d = np.array([0.9, 0.1, 0.5])
    I[9:11, 12:14] = d   # inside block (2, 3), whose grid sample is pixel (10, 14)
    j = O.joint(I, s, S, N=1, strict=strict)
    it = j["iters"][0]
    assert it["n_large"] == 4 and it["M"] == 1 and it["accepted"] == 1
    assert np.all(j["err"] < 1e-12)
    assert np.allclose(j["L"][2, 3], d)


def test_joint_strict_rolls_back_collateral_damage():
    # window 1x1: every HR pixel can use only its own block's LR pixel. One outlier pixel in a
    # block of background: replacing the LR pixel by the outlier fixes that pixel but breaks the
    # other s*s - 1. STRICT compares the total error over the affected pixels and rolls back;
    # PAPER (sums over C_i only, as Algorithm 2 lists) accepts.
    s, S = 4, 1
    I = np.full((8, 8, 3), 0.2)
    I[0, 0] = [0.8, 0.8, 0.8]
    js = O.joint(I, s, S, N=1, strict=True)
    jp = O.joint(I, s, S, N=1, strict=False)
    assert js["iters"][0]["rolled_back"] == 1 and js["iters"][0]["accepted"] == 0
    assert list(js["accept_log"]) == [0]
    assert jp["iters"][0]["accepted"] == 1 and list(jp["accept_log"]) == [1]
    assert np.allclose(js["L"][0, 0], 0.2) and np.allclose(jp["L"][0, 0], 0.8)
    e = np.linalg.norm(np.array([0.6, 0.6, 0.6]))
    assert js["err"].sum() == pytest.approx(e, abs=1e-12)
    # PAPER leaves the other pixels' stored error stale (0) although they are now wrong
    assert jp["err"].sum() == pytest.approx(0.0, abs=1e-12)
    fresh = O.glu_fast(I, jp["L"], s, S)
    assert fresh["err"].sum() == pytest.approx(15 * e, abs=1e-9)


def test_joint_argmax_picks_largest_error_pixel():
    # two large-error pixels of one component inside the same block: the one with the larger
    # error replaces the LR colour (Algorithm 2, the argmax over [q_up] intersected with C_i)
    s, S = 4, 1
    I = np.full((4, 4, 3), 0.5)
    I[0, 0] = [0.9, 0.5, 0.5]     # error 0.4
    I[0, 1] = [1.0, 0.5, 0.5]     # error 0.5, 8-connected to (0, 0)
    j = O.joint(I, s, S, N=1, strict=False)
    assert j["iters"][0]["M"] == 1
    assert np.allclose(j["L"][0, 0], [1.0, 0.5, 0.5])


# ----------------------------------------------------------------- LR operators (fixtures)

def test_lr_operators_closed_forms():
    X = np.zeros((5, 5, 3))
    X[2, 2] = 1.0
    G = O.op_gauss3(X)
    k = np.array([0.25, 0.5, 0.25])
    assert np.allclose(G[1:4, 1:4, 0], np.outer(k, k))
    B = O.op_box3(X)
    assert np.allclose(B[1:4, 1:4, 1], 1 / 9)
    c = np.full((4, 6, 3), 0.37)
    assert np.allclose(O.op_box3(c), 0.37) and np.allclose(O.op_gauss3(c), 0.37)
    Y = np.random.Generator(np.random.PCG64(3)).uniform(size=(4, 4, 3))
    assert np.allclose(O.op_saturation(Y, 1.0), Y)
    gray = np.full((2, 2, 3), 0.4)
    assert np.allclose(O.op_saturation(gray, 1.3), 0.4)
    assert O.op_gamma(np.array([[[0.5]]]), 0.8)[0, 0, 0] == pytest.approx(math.exp(0.8 * math.log(0.5)))


# ------------------------------------------------ least-squares LR colour update (non-paper)

def _random_pairs(rng, H, W, s, S, equal_frac=0.2):
    """Random valid window pairs (some with k_a = k_b) and weights in [0, 1]."""
    h, w = O.lr_dims(H, W, s)
    r = (S - 1) // 2
    ka = np.empty((H, W), np.int32)
    kb = np.empty((H, W), np.int32)
    for y in range(H):
        for x in range(W):
            valid = [k for k in range(S * S)
                     if 0 <= y // s + k // S - r < h and 0 <= x // s + k % S - r < w]
            ka[y, x] = rng.choice(valid)
            kb[y, x] = ka[y, x] if rng.random() < equal_frac else rng.choice(valid)
    return ka, kb, rng.random((H, W))


@pytest.mark.parametrize("seed,s,S", [(0, 4, 3), (1, 3, 5), (2, 5, 3)])
def test_ls_update_is_coordinatewise_least_squares(seed, s, S):
    """Each new LR colour is the least-squares solution (numpy lstsq, one unknown per channel)
    of the reconstruction errors of the pixels that use it, the other LR colours held fixed;
    clamped to [0, 1]."""
    rng = np.random.default_rng(seed)
    H, W = 13, 11
    h, w = O.lr_dims(H, W, s)
    I = rng.random((H, W, 3))
    L = rng.random((h, w, 3))
    ka, kb, om = _random_pairs(rng, H, W, s, S)
    out = O.ls_update(I, L, s, S, ka, kb, om)
    r = (S - 1) // 2
    rows = {}
    for y in range(H):
        for x in range(W):
            def lr(k):
                return (y // s + k // S - r) * w + (x // s + k % S - r)
            a, b = lr(ka[y, x]), lr(kb[y, x])
            if a == b:
                rows.setdefault(a, []).append((1.0, I[y, x]))
                continue
            wa = om[y, x]
            La, Lb = L.reshape(-1, 3)[a], L.reshape(-1, 3)[b]
            rows.setdefault(a, []).append((wa, I[y, x] - (1 - wa) * Lb))
            rows.setdefault(b, []).append((1 - wa, I[y, x] - wa * La))
    for q in range(h * w):
        got = out.reshape(-1, 3)[q]
        if q not in rows:
            assert np.array_equal(got, L.reshape(-1, 3)[q])
            continue
        A = np.array([[c] for c, _ in rows[q]])
        t = np.array([tt for _, tt in rows[q]])
        if not np.any(A):
            continue
        x = np.linalg.lstsq(A, t, rcond=None)[0][0]
        assert np.allclose(got, np.clip(x, 0.0, 1.0), atol=1e-12)


@pytest.mark.parametrize("S", [3, 5])
def test_ls_update_keeps_an_exactly_representable_lr_image(S):
    """A guide that is the nearest-neighbour upsampling of an LR image is reconstructed exactly
    (E = 0) from its grid downsampling, so that LR image is a fixed point of the update."""
    rng = np.random.default_rng(S)
    s = 4
    Lu8 = rand_img(rng, 5, 6)
    I = np.repeat(np.repeat(Lu8, s, axis=0), s, axis=1)
    L0 = O.to_unit(O.downsample_grid(I, s))
    f = O.glu_fast(I, L0, s, S)
    assert np.all(f["err"] == 0.0)
    out = O.ls_update(I, L0, s, S, f["ka"], f["kb"], f["omega"])
    assert np.allclose(out, L0, atol=1e-12)
    r = O.ls_joint(I, s, S, N=3)
    assert r["R0"] == 0.0 and r["residuals"] == []


def test_ls_joint_residuals_decrease_and_state_is_consistent():
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    img = render_u8(Scene(width=96, height=80, n_cells=10, n_dots=12, n_lines=2, seed=4))
    r = O.ls_joint(img, 8, 3, N=4)
    R = [r["R0"]] + r["residuals"]
    assert len(R) > 1 and all(b < a for a, b in zip(R, R[1:]))
    f = O.glu_fast(img, r["L"], 8, 3)
    assert np.array_equal(f["ka"], r["ka"]) and np.allclose(f["err"], r["err"])
    assert abs(float(f["err"].sum()) - R[-1]) < 1e-9


# ------------------------------------------ Algorithm 1 step 2 and Eq. 4 by independent brute force

def _np_window(L01, s, S, y, x):
    """(k, colour) of the valid window pixels of HR pixel (y, x), window index ascending."""
    h, w, _ = L01.shape
    r = (S - 1) // 2
    ks, cols = [], []
    for k in range(S * S):
        v, u = y // s + k // S - r, x // s + k % S - r
        if 0 <= v < h and 0 <= u < w:
            ks.append(k)
            cols.append(L01[v, u])
    return ks, np.array(cols)


def _first_argmin(vals):
    """Index of the first minimum (the lowest window index wins exact ties) and the gap to the
    runner-up (inf if there is none)."""
    vals = np.asarray(vals)
    i = int(np.argmin(vals))
    rest = np.delete(vals, i)
    return i, (float(rest.min() - vals[i]) if rest.size else math.inf)


def np_alg1(I01, L01, s, S, eps):
    """Algorithm 1 in numpy, everything in [0, 1] colour units: a = nearest window colour
    (Eq. 3 norm); then every b of the window, b = a included, with the Eq. 5 weight
    w = d_b / (d_a + d_b + eps) (w = 1 on a zero denominator) and the Eq. 3 error of
    w L_a + (1 - w) L_b; the smallest error wins, the lowest k_b on exact ties.
    Returns per-pixel ka, kb, w, err and the margins of both argmins."""
    H, W, _ = I01.shape
    res = {k: np.zeros((H, W), np.int64) for k in ("ka", "kb")}
    for k in ("w", "err", "margin_a", "margin_b"):
        res[k] = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            ks, cols = _np_window(L01, s, S, y, x)
            Ip = I01[y, x]
            d = np.sqrt(((cols - Ip) ** 2).sum(axis=1))
            ia, ma = _first_argmin(d)
            ws, errs = [], []
            for j in range(len(ks)):
                den = d[ia] + d[j] + eps
                wj = d[j] / den if den > 0 else 1.0
                rec = wj * cols[ia] + (1.0 - wj) * cols[j]
                ws.append(wj)
                errs.append(math.sqrt(float(((rec - Ip) ** 2).sum())))
            ib, mb = _first_argmin(errs)
            res["ka"][y, x], res["kb"][y, x] = ks[ia], ks[ib]
            res["w"][y, x], res["err"][y, x] = ws[ib], errs[ib]
            res["margin_a"][y, x], res["margin_b"][y, x] = ma, mb
    return res


def np_glu_exact(I01, L01, s, S, eps):
    """GLU* (Sec. 3.1) in numpy, [0, 1] units: every unordered pair k_a < k_b of the window with
    the Eq. 4 weight w = (I - L_b).(L_a - L_b) / (|L_a - L_b|^2 + eps), unclamped; the smallest
    Eq. 3 error wins, the first pair in (k_a, k_b) order on exact ties; a one-pixel window gives
    a = b, w = 1."""
    H, W, _ = I01.shape
    res = {k: np.zeros((H, W), np.int64) for k in ("ka", "kb")}
    for k in ("w", "err", "margin"):
        res[k] = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            ks, cols = _np_window(L01, s, S, y, x)
            Ip = I01[y, x]
            if len(ks) == 1:
                res["ka"][y, x] = res["kb"][y, x] = ks[0]
                res["w"][y, x] = 1.0
                res["err"][y, x] = float(np.sqrt(((cols[0] - Ip) ** 2).sum()))
                res["margin"][y, x] = math.inf
                continue
            pairs, ws, errs = [], [], []
            for i in range(len(ks)):
                for j in range(i + 1, len(ks)):
                    dv = cols[i] - cols[j]
                    den = float(dv @ dv) + eps
                    wij = float((Ip - cols[j]) @ dv) / den if den > 0 else 1.0
                    rec = wij * cols[i] + (1.0 - wij) * cols[j]
                    pairs.append((ks[i], ks[j]))
                    ws.append(wij)
                    errs.append(math.sqrt(float(((rec - Ip) ** 2).sum())))
            t, m = _first_argmin(errs)
            res["ka"][y, x], res["kb"][y, x] = pairs[t]
            res["w"][y, x], res["err"][y, x], res["margin"][y, x] = ws[t], errs[t], m
    return res


def _general_position_guide(rng, L_u8, s, H, W, kind):
    """A guide over LR image L_u8: a third random colours, a third LR colours plus small noise
    (b = a tends to win there), a third exact copies of a window colour (d_a = 0). `kind` is
    'u8' or 'f' (floats in [0, 1] with non-integer values)."""
    h, w, _ = L_u8.shape
    I = rng.integers(0, 256, size=(H, W, 3)).astype(np.float64)
    sel = rng.integers(0, 3, size=(H, W))
    for y in range(H):
        for x in range(W):
            v = min(h - 1, max(0, y // s + int(rng.integers(-1, 2))))
            u = min(w - 1, max(0, x // s + int(rng.integers(-1, 2))))
            if sel[y, x] == 1:
                I[y, x] = np.clip(L_u8[v, u] + rng.integers(-4, 5, size=3), 0, 255)
            elif sel[y, x] == 2:
                I[y, x] = L_u8[v, u]
    if kind == "u8":
        return I.astype(np.uint8), L_u8
    jitter = rng.uniform(-0.3, 0.3, size=I.shape) * (sel[..., None] == 0)
    return np.clip(I + jitter, 0, 255) / 255.0, L_u8.astype(np.float64) / 255.0


@pytest.mark.parametrize("kind", ["u8", "f"])
@pytest.mark.parametrize("S", [3, 5])
@pytest.mark.parametrize("eps", [1e-3, 0.0])
def test_fast_step2_equals_numpy_brute_force(kind, S, eps):
    """Algorithm 1 (a, then b over the whole window including b = a, Eq. 5 weight, Eq. 3 error)
    recomputed by brute force in numpy in [0, 1] units, on guides in general position plus
    pixels that sit on (or next to) an LR colour. Fixes the b choice (not the runner-up), that
    b = a stays a candidate, the eps term of Eq. 5 in both unit paths (raw 0..255 and [0, 1]),
    the tie rule (lowest k_b: with eps = 0 and d_a = 0 every b reconstructs L_a exactly), and
    the near-tie gaps the parity tests rely on."""
    rng = np.random.Generator(np.random.PCG64(100 + 10 * S + (1 if kind == "f" else 0)))
    s, H, W = 3, 14, 13
    h, w = O.lr_dims(H, W, s)
    L_u8 = rand_img(rng, h, w)
    I, L = _general_position_guide(rng, L_u8, s, H, W, kind)
    got = O.glu_fast(I, L, s, S, eps=eps, gaps=True)
    ref = np_alg1(O.to_unit(I), O.to_unit(L), s, S, eps)
    decided = (ref["margin_a"] > 1e-9) & ((ref["margin_b"] > 1e-9) | (ref["margin_b"] == 0.0))
    assert decided.mean() > 0.6
    exact_tie = ref["margin_b"] == 0.0
    for key in ("ka", "kb"):
        assert np.array_equal(got[key][decided], ref[key][decided]), key
    assert np.allclose(got["omega"][decided], ref["w"][decided], rtol=0, atol=1e-12)
    assert np.allclose(got["err"], ref["err"], rtol=0, atol=1e-12)
    # b = a wins at some pixels with a nonzero error, so dropping that candidate would fail here
    bwins = decided & (ref["ka"] == ref["kb"]) & (ref["err"] > 1e-6)
    assert bwins.sum() >= 3
    # and a proper pair b != a wins at others (the runner-up rule would fail there)
    assert (decided & (ref["ka"] != ref["kb"])).sum() >= 20
    if eps == 0.0:
        # d_a = 0 with eps = 0: every b gives the same (zero) error, the lowest valid k_b wins
        zero = ref["err"] == 0.0
        assert zero.sum() > 10 and np.all(exact_tie[zero])
        for (y, x) in np.argwhere(zero):
            ks, _ = _np_window(O.to_unit(L), s, S, y, x)
            assert got["kb"][y, x] == ks[0]
    # the near-tie gaps: distance to the runner-up of a different colour (equal colours never
    # appear twice in these windows, so that is the plain runner-up)
    fin = np.isfinite(ref["margin_a"])
    assert np.allclose(got["gap_a"][fin], ref["margin_a"][fin], rtol=0, atol=1e-12)
    fin_b = np.isfinite(ref["margin_b"]) & decided & ~exact_tie
    assert np.allclose(got["gap_b"][fin_b], ref["margin_b"][fin_b], rtol=0, atol=1e-12)


@pytest.mark.parametrize("kind", ["u8", "f"])
@pytest.mark.parametrize("S", [3, 5])
def test_exact_eps_term_equals_numpy_brute_force(kind, S):
    """GLU* with eps = 1e-3 against a numpy brute force written from Eq. 4 in [0, 1] units: the
    eps of Eq. 4 adds to a squared colour distance, so on raw 0..255 values it must scale by
    255^2 (by 255 it would give other weights). Both unit paths, ragged borders."""
    rng = np.random.Generator(np.random.PCG64(200 + S + (7 if kind == "f" else 0)))
    s, H, W = 3, 10, 11
    h, w = O.lr_dims(H, W, s)
    L_u8 = rand_img(rng, h, w)
    # near-duplicate LR colours make |L_a - L_b|^2 comparable to eps, where eps matters most
    L_u8[1, 1] = np.clip(L_u8[1, 2].astype(int) + [1, 0, 0], 0, 255)
    I, L = _general_position_guide(rng, L_u8, s, H, W, kind)
    eps = 1e-3
    got = O.glu_exact(I, L, s, S, eps=eps)
    ref = np_glu_exact(O.to_unit(I), O.to_unit(L), s, S, eps)
    # exact ties (margin 0: a pixel copying a window colour gives error 0 with every pair that
    # has that colour as L_b) are decided by the first-pair rule and compared as well
    decided = (ref["margin"] > 1e-9) | (ref["margin"] == 0.0)
    assert decided.mean() > 0.9 and (ref["margin"] == 0.0).sum() > 5
    assert np.array_equal(got["ka"][decided], ref["ka"][decided])
    assert np.array_equal(got["kb"][decided], ref["kb"][decided])
    scale = np.maximum(1.0, np.abs(ref["w"]))
    assert np.all(np.abs(got["omega"] - ref["w"])[decided] <= 1e-12 * scale[decided])
    assert np.allclose(got["err"], ref["err"], rtol=0, atol=1e-12)
    # the eps term is visible: eps = 0 changes some weights by far more than the tolerance
    z = O.glu_exact(I, L, s, S, eps=0.0)
    same = (z["ka"] == got["ka"]) & (z["kb"] == got["kb"])
    assert np.abs(z["omega"] - got["omega"])[same].max() > 1e-6


# ----------------------------------------------- Algorithm 2: equality and the two stop rules

def _equal_trial_guide():
    """A 2x2 guide, one LR pixel (s = 2), window 1x1, eps = 0, colours differing only in the red
    channel so every distance and sum is an exact integer. The grid sample (1, 1) is 0; the
    other pixels are 102, 51, 51 (all above tau = 30 in raw units) and form one 8-connected
    component whose largest error is (0, 0). With eps = 0 and a = b the Eq. 5 weight is 1/2 and
    the reconstruction is L exactly. Replacing L by 102 gives
        e0 = 102 + 51 + 51 + 0 = 204 = 0 + 51 + 51 + 102 = e1,
    a trial with equal errors, which Algorithm 2 keeps (it rolls back only on e1 > e0). The
    new state repeats the pattern (the sample pixel is now the largest error), so without the
    rule that stops when R_n does not decrease the loop would keep swapping."""
    I = np.zeros((2, 2, 3), np.uint8)
    I[0, 0, 0], I[0, 1, 0], I[1, 0, 0] = 102, 51, 51
    return I


def test_joint_accepts_equal_error_trial_and_stops_on_flat_residual():
    I = _equal_trial_guide()
    j = O.joint(I, 2, 1, N=3, eps=0.0, strict=True)
    assert len(j["iters"]) == 1                      # R_1 == R_0: the loop ends after one
    it = j["iters"][0]
    assert (it["n_large"], it["M"], it["accepted"], it["rolled_back"]) == (3, 1, 1, 0)
    assert list(j["accept_log"]) == [1]              # e1 == e0 is kept
    assert list(j["L"][0, 0]) == [102, 0, 0]
    assert j["R0"] == pytest.approx(204 / 255, abs=1e-15)
    assert it["residual"] == pytest.approx(204 / 255, abs=1e-15)
    assert it["min_decision_margin"] == math.inf     # |e1 - e0| is exactly 0 (never nonzero)
    assert np.allclose(j["err"][:, :, None].ravel(), np.array([0, 51, 51, 102]) / 255, atol=1e-15)


def test_joint_stops_after_an_iteration_that_keeps_nothing():
    """Window 1x1, one outlier in a flat block: STRICT rolls the only trial back, the state is
    unchanged, and the loop ends after that iteration instead of repeating it N times."""
    s, S = 4, 1
    I = np.full((8, 8, 3), 0.2)
    I[0, 0] = [0.8, 0.8, 0.8]
    j = O.joint(I, s, S, N=3, strict=True)
    assert len(j["iters"]) == 1
    assert j["iters"][0]["accepted"] == 0 and j["iters"][0]["rolled_back"] == 1
    # with something to gain the loop runs on: a planted dot is fixed in iteration 1, so a
    # second iteration starts and finds nothing above tau
    I2 = np.full((32, 32, 3), 0.25)
    I2[9:11, 12:14] = [0.9, 0.1, 0.5]
    j2 = O.joint(I2, 4, 3, N=3, strict=True)
    assert len(j2["iters"]) == 2 and j2["iters"][1]["n_large"] == 0


# ------------------------------------------- replay of another implementation's logged decisions

def test_joint_argmax_replay_follows_only_near_ties():
    """The verification replay (glu_oracle.c, oracle_joint): a logged replacement pixel is taken
    only where its FP64 error is within the tolerance of the block's largest. Two pixels of one
    block with exactly equal errors of different colour: by itself the oracle takes the lowest
    raster index; with a record naming the other one it takes that; a record naming a pixel far
    from the largest error is ignored."""
    I = np.zeros((2, 2, 3), np.uint8)
    I[0, 0] = (40, 0, 0)
    I[0, 1] = (0, 40, 0)          # same error (40) as (0, 0), other colour; 8-connected to it
    own = O.joint(I, 2, 1, N=1, eps=0.0, strict=False)
    assert list(own["L"][0, 0]) == [40, 0, 0]
    assert own["iters"][0]["argmax_near_ties"] == 1
    rec = np.array([[0, 0, 0, 1]], np.int32)      # iteration 0, component 0, LR pixel 0, HR 1
    rp = O.joint(I, 2, 1, N=1, eps=0.0, strict=False, argmax=rec, argmax_tol=1e-5)
    assert list(rp["L"][0, 0]) == [0, 40, 0] and rp["iters"][0]["argmax_replayed"] == 1
    far = np.array([[0, 0, 0, 2]], np.int32)      # pixel (1, 0): error 0, not in the component
    rf = O.joint(I, 2, 1, N=1, eps=0.0, strict=False, argmax=far, argmax_tol=1e-5)
    assert list(rf["L"][0, 0]) == [40, 0, 0] and rf["iters"][0]["argmax_replayed"] == 0


def test_joint_threshold_replay_follows_only_pixels_at_tau():
    """A pixel whose error is exactly tau (distance 30 in raw units) is not in the large-error set
    (E_p > tau is strict); a logged membership of 1 is followed there, but not for a pixel whose
    error is far from tau."""
    I = np.zeros((2, 4, 3), np.uint8)
    I[0, 0] = (30, 0, 0)          # E = 30/255 = tau
    I[0, 3] = (90, 0, 0)          # E far above tau
    own = O.joint(I, 2, 1, N=1, eps=0.0, strict=False)
    assert own["iters"][0]["n_large"] == 1 and own["iters"][0]["min_threshold_margin"] < 1e-12
    rec = np.array([[256, 0, 1, 0], [256, 3, 0, 0]], np.int32)
    rp = O.joint(I, 2, 1, N=1, eps=0.0, strict=False, argmax=rec, argmax_tol=1e-5, thr_tol=2e-6)
    it = rp["iters"][0]
    assert it["threshold_replayed"] == 1 and it["n_large"] == 2 and it["M"] == 2
    assert list(rp["L"][0, 0]) == [30, 0, 0] and list(rp["L"][0, 1]) == [90, 0, 0]

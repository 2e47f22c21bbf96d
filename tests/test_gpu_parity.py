"""GPU vs FP64 oracle parity through the C ABI (needs a GB300 and the built library)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from tests.parity import check_search, lr_like_gpu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import api as A
    return A


def scene_img(seed, H, W, cells=40, dots=30, lines=5):
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    return render_u8(Scene(width=W, height=H, n_cells=cells, n_dots=dots, n_lines=lines, seed=seed))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ------------------------------------------------------------------------------ downsampling

@pytest.mark.parametrize("H,W,s", [(256, 256, 4), (97, 131, 3), (250, 347, 8), (33, 17, 16)])
def test_downsample_grid_exact_and_box(api, H, W, s):
    img = scene_img(3, H, W)
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
    assert np.array_equal(lr.cpu().numpy(), O.downsample_grid(img, s))
    lb = api.glu_downsample(hr, s, api.GLU_DOWN_BOX)
    assert np.abs(lb.cpu().numpy() - O.downsample_box(img, s)).max() < 1e-6
    # f16 input, f32 output grid
    h16 = hr.to(torch.float16) / 255
    lg = api.glu_downsample(h16, s, api.GLU_DOWN_GRID, dtype=torch.float32)
    assert np.abs(lg.cpu().numpy() - O.downsample_grid(h16.cpu().numpy(), s)).max() == 0.0


# --------------------------------------------------------------------------- Algorithm 1

@pytest.mark.parametrize("H,W,s,S,mode", [
    (256, 256, 4, 3, "box"),      # the plain 256x256 workload
    (250, 347, 8, 5, "grid"),     # several tiles and a ragged tail
    (97, 131, 3, 3, "grid"),
    (97, 131, 2, 1, "grid"),
    (120, 200, 4, 7, "box"),
    (70, 90, 2, 9, "grid"),
    (33, 17, 16, 5, "box"),       # LR narrower than the window
    (1, 1, 1, 3, "grid"),         # degenerate: one pixel
    (5, 300, 4, 5, "grid"),       # one LR row
])
def test_search_parity(api, H, W, s, S, mode):
    img = scene_img(H * 7 + W, H, W)
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID if mode == "grid" else api.GLU_DOWN_BOX)
    params = api.glu_params(S=S)
    theta, err = api.glu_optimize(hr, lr, params, s, err_map=True)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    rep = check_search(img, lr_like_gpu(lr), s, S, theta, err)
    print(f"\n{H}x{W} s={s} S={S} {mode}: {rep}")


def test_search_tma_and_plain_paths_agree(api):
    # a row pitch that is not a multiple of 16 bytes disables TMA (plain loads instead)
    H, W, s, S = 130, 250, 4, 5
    img = scene_img(11, H, W)
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
    params = api.glu_params(S=S)
    t1, e1 = api.glu_optimize(hr, lr, params, s, err_map=True)
    padded = torch.zeros((H, W * 3 + 5), dtype=torch.uint8, device="cuda")
    padded[:, :W * 3] = hr.view(H, W * 3)
    hr2 = torch.as_strided(padded, (H, W, 3), (W * 3 + 5, 3, 1))
    t2, e2 = api.glu_optimize(hr2, lr, params, s, err_map=True)
    torch.cuda.synchronize()
    assert torch.equal(t1.code, t2.code) and torch.equal(t1.weight, t2.weight)
    assert torch.equal(e1, e2)


@pytest.mark.parametrize("wfmt", [1, 2])
def test_weight_formats(api, wfmt):
    H, W, s, S = 160, 200, 4, 3
    img = scene_img(5, H, W)
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_BOX)
    theta, err = api.glu_optimize(hr, lr, api.glu_params(S=S), s, err_map=True, wfmt=wfmt)
    torch.cuda.synchronize()
    check_search(img, lr_like_gpu(lr), s, S, theta, err, wfmt=wfmt)


def test_gnu_mode(api):
    H, W, s, S = 100, 150, 4, 3
    img = scene_img(6, H, W)
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
    theta, err = api.glu_optimize(hr, lr, api.glu_params(S=S, mode=api.GLU_MODE_GNU), s,
                                  err_map=True)
    torch.cuda.synchronize()
    check_search(img, lr_like_gpu(lr), s, S, theta, err, gnu=True)


def test_search_f16_guide(api):
    H, W, s, S = 144, 272, 8, 5
    img = scene_img(8, H, W)
    hr16 = (dev(img).to(torch.float32) / 255).to(torch.float16)
    lr = api.glu_downsample(hr16, s, api.GLU_DOWN_BOX)
    theta, err = api.glu_optimize(hr16, lr, api.glu_params(S=S), s, err_map=True)
    torch.cuda.synchronize()
    check_search(hr16.cpu().numpy().astype(np.float64), lr_like_gpu(lr), s, S, theta, err)


def test_search_deterministic(api):
    H, W, s, S = 300, 400, 8, 5
    img = scene_img(9, H, W)
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_BOX)
    p = api.glu_params(S=S)
    a = api.glu_optimize(hr, lr, p, s, err_map=True)
    b = api.glu_optimize(hr, lr, p, s, err_map=True)
    torch.cuda.synchronize()
    assert torch.equal(a[0].code, b[0].code) and torch.equal(a[0].weight, b[0].weight)
    assert torch.equal(a[1], b[1])


# -------------------------------------------------------------------------------- Eq. 1

@pytest.mark.parametrize("C,out_dtype", [(3, torch.float32), (1, torch.float32),
                                         (4, torch.float32), (3, torch.float16)])
def test_apply_parity(api, C, out_dtype):
    H, W, s, S = 250, 347, 8, 5
    img = scene_img(10, H, W)
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
    theta, _ = api.glu_optimize(hr, lr, api.glu_params(S=S), s)
    h, w = api.lr_dims(H, W, s)
    T = torch.rand((h, w, C), generator=torch.Generator().manual_seed(C)).cuda()
    out = api.glu_apply(theta, T, out_dtype=out_dtype)
    torch.cuda.synchronize()
    codes = theta.codes_i32().cpu().numpy()
    K = S * S
    ref = O.apply(codes // K, codes % K, theta.weight_f32().cpu().numpy().astype(np.float64),
                  s, S, T.cpu().numpy().astype(np.float64))
    tol = 1e-6 if out_dtype == torch.float32 else 1e-3
    assert np.abs(out.float().cpu().numpy() - ref).max() < tol


def test_plain_256_pipeline_against_oracle_theta(api):
    # the plain 256x256 workload end to end: box LR, Algorithm 1, processed LR = gamma 0.8,
    # Eq. 1; the reconstruction is compared with the oracle's Theta applied to the same target
    from paper_2307_09582_gb300.inputs import plain_256_scene, render_u8
    img = render_u8(plain_256_scene(seed=1))
    s, S = 4, 3
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_BOX)
    theta, err = api.glu_optimize(hr, lr, api.glu_params(S=S), s, err_map=True)
    T = api.glu_fx_point(lr, 1.0, 0.8)
    out = api.glu_apply(theta, T)
    torch.cuda.synchronize()
    L = lr_like_gpu(lr)
    ref = O.glu_fast(img, L, s, S, gaps=True)
    rep = check_search(img, L, s, S, theta, err, ref=ref)
    To = O.op_gamma(L, 0.8)
    assert np.abs(T.cpu().numpy() - To).max() < 1e-6
    oref = O.apply(ref["ka"], ref["kb"], ref["omega"], s, S, To)
    codes = theta.codes_i32().cpu().numpy()
    same = (codes // 9 == ref["ka"]) & (codes % 9 == ref["kb"])
    d = np.abs(out.cpu().numpy() - oref).max(axis=2)
    assert d[same].max() < 1e-3
    # self-upsampling error of the GPU result against FP64 (reported)
    print(f"\nplain 256: {rep}, max |T_hat - oracle| {d[same].max():.2e}")


@pytest.mark.parametrize("wfmt", [0, 1, 2])
def test_apply_vector_path_parity(api, wfmt):
    # W % 4 == 0, float32 3-channel target/output: the tiled paths of Eq. 1 (the autotuner's
    # default variant; every variant is checked bit-identical in test_gpu_tune.py)
    H, W, s, S = 200, 320, 8, 5
    img = scene_img(21, H, W)
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
    theta, _ = api.glu_optimize(hr, lr, api.glu_params(S=S), s, wfmt=wfmt)
    h, w = api.lr_dims(H, W, s)
    T = torch.rand((h, w, 3), generator=torch.Generator().manual_seed(5)).cuda()
    out = api.glu_apply(theta, T)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    codes = theta.codes_i32().cpu().numpy()
    K = S * S
    ref = O.apply(codes // K, codes % K, theta.weight_f32().cpu().numpy().astype(np.float64),
                  s, S, T.cpu().numpy().astype(np.float64))
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-6


# ------------------------------------------------------------------------- Theta decode

@pytest.mark.parametrize("H,W,s,S,wfmt", [(97, 131, 3, 5, 1), (250, 347, 8, 3, 0),
                                          (64, 80, 16, 7, 2)])
def test_theta_decode_against_oracle_pairs(api, H, W, s, S, wfmt):
    # absolute LR indices of (a, b) decoded on the device equal the oracle's window indices
    # decoded here by the window definition (clipped windows included), the weights equal the
    # stored ones, and gathering T through them reproduces Eq. 1 as glu_apply computes it
    img = scene_img(40 + S, H, W)
    hr = dev(img)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
    theta, _ = api.glu_optimize(hr, lr, api.glu_params(S=S), s, wfmt=wfmt)
    a, b, w = api.glu_theta_decode(theta)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    h, wl = api.lr_dims(H, W, s)
    r = (S - 1) // 2
    codes = theta.codes_i32().cpu().numpy()
    ka, kb = codes // (S * S), codes % (S * S)
    yy, xx = np.mgrid[0:H, 0:W]
    exp_a = (yy // s + ka // S - r) * wl + (xx // s + ka % S - r)
    exp_b = (yy // s + kb // S - r) * wl + (xx // s + kb % S - r)
    a, b, w = a.cpu().numpy(), b.cpu().numpy(), w.cpu().numpy()
    assert np.array_equal(a, exp_a) and np.array_equal(b, exp_b)
    assert a.min() >= 0 and a.max() < h * wl and b.min() >= 0 and b.max() < h * wl
    assert np.array_equal(w, theta.weight_f32().cpu().numpy())
    # the pairs are the oracle's Algorithm 1 pairs wherever its choice is not a near tie
    L = lr_like_gpu(lr)
    ref = O.glu_fast(img, L, s, S)
    same = (ka == ref["ka"]) & (kb == ref["kb"])
    assert same.mean() > 0.99
    T = torch.rand((h, wl, 3), generator=torch.Generator().manual_seed(S)).cuda()
    out = api.glu_apply(theta, T).cpu().numpy().astype(np.float64)
    Tf = T.cpu().numpy().reshape(-1, 3).astype(np.float64)
    g = w[..., None] * Tf[a] + (1.0 - w[..., None]) * Tf[b]
    assert np.abs(out - g).max() < 1e-6


def test_theta_decode_flags_codes_outside_the_window(api):
    # a code naming a window position outside the image: the decode writes -1 for both indices
    # of that pixel, leaves the others intact and reports GLU_ERR_DEVICE_CHECK
    H, W, s, S = 32, 48, 4, 3
    hr = dev(scene_img(7, H, W))
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
    theta, _ = api.glu_optimize(hr, lr, api.glu_params(S=S), s)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    theta.code[0, 0] = 0          # (dy, dx) = (-1, -1) at the top-left corner: outside
    a, b, _ = api.glu_theta_decode(theta)
    torch.cuda.synchronize()
    assert api.glu_device_status() == api.A.GLU_ERR_DEVICE_CHECK
    assert api.glu_device_status() == 0
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert a[0, 0] == -1 and b[0, 0] == -1
    assert a.ravel()[1:].min() >= 0 and b.ravel()[1:].min() >= 0

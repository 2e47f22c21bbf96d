"""Large scaling ratios (16x to 128x) and window sizes 3 to 9, after the paper's large-ratio
experiment and its window-size table (Sec. 5), on synthetic guides: Algorithm 1, GLU*, GNU and
Algorithm 2 against the FP64 oracle at sizes it finishes quickly, and what holds at any size
(needs a GB300)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests.parity import check_exact, check_search, lr_like_gpu  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import api as A
    return A


def guide(H, W, seed):
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    return render_u8(Scene(width=W, height=H, n_cells=30, n_dots=40, n_lines=6, seed=seed))


@pytest.mark.parametrize("H,W,s,S", [(300, 420, 32, 3), (300, 420, 64, 5), (260, 300, 128, 3),
                                     (200, 330, 128, 9), (400, 300, 32, 9), (257, 383, 16, 7)])
def test_large_ratio_search_parity(api, H, W, s, S):
    img = guide(H, W, H + W + s + S)
    hr = torch.from_numpy(img).cuda()
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
    L = lr_like_gpu(lr)
    th, err = api.glu_optimize(hr, lr, api.glu_params(S=S), s, err_map=True)
    te, ee = api.glu_optimize(hr, lr, api.glu_params(S=S, mode=api.GLU_MODE_EXACT), s,
                              err_map=True, wfmt=api.GLU_W_F32)
    tg, eg = api.glu_optimize(hr, lr, api.glu_params(S=S, mode=api.GLU_MODE_GNU), s,
                              err_map=True)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    rep = check_search(img, L, s, S, th, err)
    rep_e = check_exact(img, L, s, S, te, ee)
    check_search(img, L, s, S, tg, eg, gnu=True)
    # Eq. 1 at this ratio reproduces the guide up to the reported error, for both weight rules
    T = lr.to(torch.float32) / 255.0
    g = hr.to(torch.float32) / 255.0
    for t, e in ((th, err), (te, ee)):
        rec = torch.linalg.norm(api.glu_apply(t, T) - g, dim=2)
        assert torch.allclose(rec, e, atol=2e-4)
    print(f"\n{H}x{W} s={s} S={S}: fast {rep} exact {rep_e}")


@pytest.mark.parametrize("H,W,s,S", [(256, 320, 32, 3), (192, 256, 64, 3), (200, 240, 16, 5)])
def test_large_ratio_joint_parity(api, H, W, s, S):
    from tests.test_gpu_joint import compare, run_both
    img = guide(H, W, 3 * H + s)
    hr, lr, theta, err, st, ref = run_both(api, img, s, S, N=3, strict=True)
    rep = compare(api, img, s, S, 3, True, lr, theta, err, st, ref)
    print(f"\njoint {H}x{W} s={s} S={S}: {st['iters']} {rep}")
    assert rep["mode"] == "exact", rep


def test_window_size_nesting(api):
    """GLU*: the S x S window lies inside the (S + 2) x (S + 2) window with the same centre and
    each pair is evaluated with the same operations whatever S is, so no pixel's error grows
    with S (and neither does the self-upsampling error). Algorithm 1 has no such guarantee (its
    a is the nearest colour of a larger set); its errors are reported."""
    img = guide(768, 1024, 5)
    hr = torch.from_numpy(img).cuda()
    for s in (8, 32):
        lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
        prev = None
        rows = []
        for S in (3, 5, 7, 9):
            _, ee = api.glu_optimize(hr, lr, api.glu_params(S=S, mode=api.GLU_MODE_EXACT), s,
                                     err_map=True, wfmt=api.GLU_W_F32)
            _, ef = api.glu_optimize(hr, lr, api.glu_params(S=S), s, err_map=True)
            torch.cuda.synchronize()
            if prev is not None:
                assert bool((ee <= prev).all()), (s, S)
            prev = ee
            # mean squared error per channel -> PSNR of the self-upsampled guide
            psnr = [float(10 * torch.log10(3.0 / (e.double() ** 2).mean())) for e in (ee, ef)]
            rows.append((S, *psnr))
        assert all(a[1] <= b[1] for a, b in zip(rows, rows[1:]))
        print(f"\ns={s} (S, PSNR GLU*, PSNR FAST): {rows}")

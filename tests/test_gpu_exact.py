"""GLU* (Sec. 3.1, Eq. 4: every unordered pair of window pixels, least-squares weight) on the GPU
against the FP64 oracle (needs a GB300)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from tests.parity import check_exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import api as A
    return A


@pytest.mark.parametrize("H,W,s,S,lrmode,f16", [(64, 80, 4, 3, "box", False),
                                                (96, 72, 8, 5, "grid", False),
                                                (50, 70, 4, 7, "box", False),
                                                (41, 33, 2, 5, "grid", False),
                                                (30, 30, 16, 3, "grid", False),
                                                (45, 61, 3, 5, "box", False),
                                                (70, 90, 8, 5, "box", True)])
def test_exact_matches_oracle(api, H, W, s, S, lrmode, f16):
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    img = render_u8(Scene(width=W, height=H, n_cells=12, n_dots=15, n_lines=3, seed=H * W + S))
    hr = torch.from_numpy(img).cuda()
    if f16:
        hr = (hr.to(torch.float32) / 255).to(torch.float16)
        img = hr.cpu().numpy().astype(np.float64)
    mode = api.GLU_DOWN_BOX if lrmode == "box" else api.GLU_DOWN_GRID
    lr = api.glu_downsample(hr, s, mode)
    p = api.glu_params(S=S, mode=api.GLU_MODE_EXACT)
    th, err = api.glu_optimize(hr, lr, p, s, err_map=True, wfmt=api.GLU_W_F32)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    L = lr.cpu().numpy()
    L = L if L.dtype == np.uint8 else L.astype(np.float64)
    check_exact(img, L, s, S, th, err)
    # Eq. 1 with these (unclamped) weights reproduces the guide up to the reported error
    out = api.glu_apply(th, lr.to(torch.float32) if lr.dtype != torch.uint8
                        else lr.to(torch.float32) / 255.0)
    g = hr.to(torch.float32) if f16 else hr.to(torch.float32) / 255.0
    rec_err = torch.linalg.norm(out - g, dim=2)
    assert torch.allclose(rec_err, err, atol=2e-4)


def test_exact_requires_float32_weights(api):
    hr = torch.zeros((16, 16, 3), dtype=torch.uint8, device="cuda")
    lr = api.glu_downsample(hr, 4, api.GLU_DOWN_GRID)
    p = api.glu_params(S=3, mode=api.GLU_MODE_EXACT)
    from paper_2307_09582_gb300 import _abi as A
    with pytest.raises(A.GluError):
        api.glu_optimize(hr, lr, p, 4, wfmt=api.GLU_W_UNORM16)
    th, err = api.glu_optimize(hr, lr, p, 4, err_map=True, wfmt=api.GLU_W_F32)
    torch.cuda.synchronize()
    assert float(err.abs().max()) == 0.0     # exactly representable: zero error
    # every pair has L_a = L_b: Eq. 4 gives 0 / eps = 0, and the first valid pair wins
    ref = O.glu_exact(np.zeros((16, 16, 3), np.uint8), np.zeros((4, 4, 3), np.uint8), 4, 3)
    assert float(th.weight_f32().abs().max()) == 0.0 and np.all(ref["omega"] == 0.0)
    codes = th.codes_i32().cpu().numpy()
    assert np.array_equal(codes // 9, ref["ka"]) and np.array_equal(codes % 9, ref["kb"])
    # with eps = 0 the weight of L_a = L_b is taken as 1, like the oracle's
    th0, _ = api.glu_optimize(hr, lr, api.glu_params(S=3, eps=0.0, mode=api.GLU_MODE_EXACT), 4,
                              err_map=True, wfmt=api.GLU_W_F32)
    ref = O.glu_exact(np.zeros((16, 16, 3), np.uint8), np.zeros((4, 4, 3), np.uint8), 4, 3,
                      eps=0.0)
    torch.cuda.synchronize()
    assert np.array_equal(th0.weight_f32().cpu().numpy(), ref["omega"].astype(np.float32))
    codes = th0.codes_i32().cpu().numpy()
    assert np.array_equal(codes // 9, ref["ka"]) and np.array_equal(codes % 9, ref["kb"])

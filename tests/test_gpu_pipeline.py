"""The uint8 LR filter and the host-buffer pipeline entry point (needs a GB300).

glu_pipeline_host runs the library's own device calls between two copies, so it is pinned to
them bit for bit; the device calls are pinned to the FP64 oracle by the other GPU tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import api as A
    return A


@pytest.mark.parametrize("op", [0, 1])
def test_filter3_u8_equals_float_filter_of_x_over_255(api, op):
    g = torch.Generator().manual_seed(3 + op)
    x = torch.randint(0, 256, (37, 53, 3), generator=g, dtype=torch.uint8)
    # x / 255 correctly rounded to float32 (IEEE division, as the kernel reads it)
    xf = torch.from_numpy(x.numpy().astype(np.float32) / np.float32(255.0)).cuda()
    ref = api.glu_fx_filter3(xf, op)
    got = api.glu_fx_filter3_u8(x.cuda(), op)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


@pytest.mark.parametrize("pinned", [True, False])
def test_pipeline_host_equals_device_calls(api, pinned):
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    img = render_u8(Scene(width=328, height=248, n_cells=40, n_dots=80, n_lines=6, seed=21))
    H, W, s = img.shape[0], img.shape[1], 8
    p = api.glu_params(S=5, N=3)
    # the device calls, one after another
    hr = torch.from_numpy(img).cuda()
    h, w = api.lr_dims(H, W, s)
    lr = torch.empty((h, w, 3), dtype=torch.uint8, device="cuda")
    th = api.Theta.empty(H, W, s, 5, api.GLU_W_UNORM16, hr.device)
    api.glu_joint_optimize(hr, s, p, lr_out=lr, theta=th, err_map=None, stats=False)
    T = api.glu_fx_point(api.glu_fx_filter3_u8(lr, 1), sat=1.3, gamma=0.8)
    ref = api.glu_apply(th, T).cpu()
    # one host-buffer call (twice: the second replays the recorded graph)
    hr_host = torch.from_numpy(img)
    out_host = torch.full((H, W, 3), -1.0, dtype=torch.float32)
    if pinned:
        hr_host, out_host = hr_host.pin_memory(), out_host.pin_memory()
    ws = torch.empty(api.glu_pipeline_host_workspace_size(H, W, s, p) + 256, dtype=torch.uint8,
                     device="cuda")
    for _ in range(2):
        out_host.fill_(-1.0)
        api.glu_pipeline_host(hr_host, s, p, 1, 1.3, 0.8, out_host, ws)
        assert torch.equal(out_host, ref)
    assert api.glu_device_status() == 0
    assert np.isfinite(out_host.numpy()).all()

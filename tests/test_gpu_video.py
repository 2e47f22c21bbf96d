"""The per-frame pipeline replayed as CUDA graphs (BOX downsample -> 3x3 Gaussian + gamma 0.8 on
the LR image -> Algorithm 1 -> Eq. 1) against the separate calls and the FP64 oracle
(needs a GB300)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from tests.parity import check_search  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import api as A
    return A


def frames_f16(W, H, n):
    """Frames of the video workload's recipe (moving cells, dots re-drawn) at a small size, as
    float16 colours in [0, 1]."""
    from paper_2307_09582_gb300.inputs import render_video_u8
    from paper_2307_09582_gb300.inputs.workloads import video_scene
    u8 = render_video_u8(video_scene(width=W, height=H), n)
    return (torch.from_numpy(u8).cuda().to(torch.float32) / 255).to(torch.float16)


def separate_calls(api, hr, s, S, wfmt, out_dtype, gamma=0.8):
    """The same frame through the individual entry points."""
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_BOX, dtype=torch.float32)
    t1 = api.glu_fx_filter3(lr, 1)
    T = api.glu_fx_point(t1, 1.0, gamma)
    theta, _ = api.glu_optimize(hr, lr, api.glu_params(S=S), s, wfmt=wfmt)
    out = api.glu_apply(theta, T, out_dtype=out_dtype)
    return lr, T, theta, out


@pytest.mark.parametrize("W,H,overlap,out_dtype", [
    (264, 200, True, torch.float16),    # W % 4 == 0: the 4-pixel store path
    (262, 197, True, torch.float16),    # ragged: the general path
    (264, 200, False, torch.float32),
])
def test_video_graph_equals_separate_calls(api, W, H, overlap, out_dtype):
    s, S, n = 8, 5, 5
    fr = frames_f16(W, H, n)
    v = api.Video(H, W, s, api.glu_params(S=S), out_dtype=out_dtype, overlap=overlap)
    outs = torch.zeros((n, H, W, 3), dtype=out_dtype, device="cuda")
    eager = torch.zeros_like(outs)
    for k in range(n):
        v.bind(k, fr[k], outs[k])
    for k in range(n):
        v.launch(k)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    for k in range(n):
        v.run(fr[k], eager[k])
    torch.cuda.synchronize()
    assert torch.equal(outs, eager)
    for k in (0, n - 1):
        _, _, _, ref = separate_calls(api, fr[k], s, S, api.GLU_W_UNORM16, out_dtype)
        torch.cuda.synchronize()
        assert torch.equal(outs[k], ref), k
    v.close()


def test_video_last_frame_matches_oracle(api):
    s, S, n, W, H = 8, 5, 3, 200, 136
    fr = frames_f16(W, H, n)
    v = api.Video(H, W, s, api.glu_params(S=S), out_dtype=torch.float32, wfmt=api.GLU_W_F32)
    out = torch.empty((n, H, W, 3), dtype=torch.float32, device="cuda")
    for k in range(n):
        v.bind(k, fr[k], out[k])
        v.launch(k)
    torch.cuda.synchronize()
    lr, T, theta = v.views()      # the working images of the last frame
    I = fr[n - 1].cpu().numpy()
    lr_ref = O.downsample_box(I, s)
    assert np.abs(lr.cpu().numpy() - lr_ref).max() < 1e-6
    T_ref = O.op_gamma(O.op_gauss3(lr.cpu().numpy().astype(np.float64)), 0.8)
    assert np.abs(T.cpu().numpy() - T_ref).max() < 1e-5
    Lg = lr.cpu().numpy().astype(np.float64)
    check_search(I, Lg, s, S, theta, wfmt=api.GLU_W_F32)
    ref = O.glu_fast(I, Lg, s, S)
    hr_ref = O.apply(ref["ka"], ref["kb"], ref["omega"], s, S, T.cpu().numpy())
    assert np.abs(out[n - 1].cpu().numpy() - hr_ref).max() < 1e-3
    v.close()


def test_video_rebind_and_argument_errors(api):
    s, S, W, H = 8, 3, 128, 96
    fr = frames_f16(W, H, 2)
    v = api.Video(H, W, s, api.glu_params(S=S))
    a = torch.empty((H, W, 3), dtype=torch.float16, device="cuda")
    b = torch.empty_like(a)
    v.bind(3, fr[0], a)
    v.bind(3, fr[1], b)          # re-binding replaces the graph
    v.launch(3)
    torch.cuda.synchronize()
    c = torch.empty_like(a)
    v.run(fr[1], c)
    torch.cuda.synchronize()
    assert torch.equal(b, c)
    from paper_2307_09582_gb300 import _abi as A
    with pytest.raises(A.GluError):
        v.launch(4)              # never bound
    with pytest.raises(A.GluError):
        v.launch(A.GLU_VIDEO_MAX_SLOTS)
    v.close()

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
    lr, (T,), theta = v.views()   # the working images of the last frame
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


# two and three LR operators sharing the frame's Theta: (filter, saturation, gamma)
OPS2 = [(1, 1.0, 0.8), (0, 1.3, 1.0)]
OPS3 = [(1, 1.0, 0.8), (0, 1.3, 1.0), (-1, 0.7, 1.2)]


def separate_op(api, hr, s, S, wfmt, out_dtype, op):
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_BOX, dtype=torch.float32)
    f, sat, g = op
    t = api.glu_fx_filter3(lr, f) if f >= 0 else lr
    T = api.glu_fx_point(t, sat, g)
    theta, _ = api.glu_optimize(hr, lr, api.glu_params(S=S), s, wfmt=wfmt)
    return api.glu_apply(theta, T, out_dtype=out_dtype)


@pytest.mark.parametrize("ops,overlap", [(OPS2, True), (OPS3, True), (OPS2, False)])
def test_video_theta_shared_by_several_operators(api, ops, overlap):
    """One Algorithm 1 per frame serves every operator (Theta is target-free): the graph replay,
    the direct launches and, per operator, the separate single-operator calls give identical
    frames."""
    s, S, n, W, H = 8, 5, 4, 264, 200
    fr = frames_f16(W, H, n)
    k = len(ops)
    v = api.Video(H, W, s, api.glu_params(S=S), out_dtype=torch.float16, overlap=overlap, ops=ops)
    outs = torch.zeros((n, k, H, W, 3), dtype=torch.float16, device="cuda")
    eager = torch.zeros_like(outs)
    for f in range(n):
        v.bind(f, fr[f], [outs[f, i] for i in range(k)])
    for f in range(n):
        v.launch(f)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    for f in range(n):
        v.run(fr[f], [eager[f, i] for i in range(k)])
    torch.cuda.synchronize()
    assert torch.equal(outs, eager)
    for f in (0, n - 1):
        for i, op in enumerate(ops):
            ref = separate_op(api, fr[f], s, S, api.GLU_W_UNORM16, torch.float16, op)
            torch.cuda.synchronize()
            assert torch.equal(outs[f, i], ref), (f, i)
    v.close()


def test_video_several_operators_frame_matches_oracle(api):
    """The last frame of a two-operator pipeline: the LR image, both targets (Gaussian + gamma 0.8;
    box + saturation 1.3) against the oracle's operators, Theta against Algorithm 1, and both
    outputs against Eq. 1 of the oracle's Theta on the GPU's targets."""
    s, S, n, W, H = 8, 5, 3, 200, 136
    fr = frames_f16(W, H, n)
    v = api.Video(H, W, s, api.glu_params(S=S), out_dtype=torch.float32, wfmt=api.GLU_W_F32,
                  ops=OPS2)
    out = torch.empty((n, 2, H, W, 3), dtype=torch.float32, device="cuda")
    for f in range(n):
        v.bind(f, fr[f], [out[f, 0], out[f, 1]])
        v.launch(f)
    torch.cuda.synchronize()
    lr, (T0, T1), theta = v.views()
    I = fr[n - 1].cpu().numpy()
    assert np.abs(lr.cpu().numpy() - O.downsample_box(I, s)).max() < 1e-6
    L = lr.cpu().numpy().astype(np.float64)
    assert np.abs(T0.cpu().numpy() - O.op_gamma(O.op_gauss3(L), 0.8)).max() < 1e-5
    assert np.abs(T1.cpu().numpy() - O.op_saturation(O.op_box3(L), 1.3)).max() < 1e-5
    check_search(I, L, s, S, theta, wfmt=api.GLU_W_F32)
    ref = O.glu_fast(I, L, s, S)
    for i, T in enumerate((T0, T1)):
        hr_ref = O.apply(ref["ka"], ref["kb"], ref["omega"], s, S, T.cpu().numpy())
        assert np.abs(out[n - 1, i].cpu().numpy() - hr_ref).max() < 1e-3, i
    v.close()

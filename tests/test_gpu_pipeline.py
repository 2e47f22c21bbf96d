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


def test_joint_4k_pipeline_rows_match_oracle_pipeline(api):
    """The benchmarked pipeline (Algorithm 2 at scale 8 with a 5x5 window and 5 iterations,
    then the LR operator 3x3 box + saturation x1.3, then Eq. 1 with unorm16 weights) on the top
    400 rows of the 3840x2160 bench guide against the oracle's pipeline on the same rows: the
    joint result element-wise (decision and argmax replay within their tolerances), the
    processed LR image within 1e-6, and the reconstruction within 1e-3 wherever the pair codes
    agree (elsewhere, at near-ties, the GPU's own pair applied in FP64 within 1e-3)."""
    from oracle import oracle as O
    from paper_2307_09582_gb300.inputs import joint_4k_scene, render_u8
    from tests.test_gpu_joint import ARGMAX_TOL, REPLAY_TOL, THR_TOL, compare
    img = np.ascontiguousarray(render_u8(joint_4k_scene())[:400])
    s, S, N = 8, 5, 5
    H, W = img.shape[:2]
    hr = torch.from_numpy(img).cuda()
    p = api.glu_params(S=S, N=N)
    lr, th, err, st = api.glu_joint_optimize(hr, s, p, wfmt=api.GLU_W_UNORM16, decisions=True,
                                             argmax_log=True)
    T = api.glu_fx_point(api.glu_fx_filter3_u8(lr, 0), sat=1.3, gamma=1.0)
    out = api.glu_apply(th, T)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    ref = O.joint(img, s, S, N=N, strict=True, force=st["decisions"], force_tol=REPLAY_TOL,
                  argmax=st["argmax"], argmax_tol=ARGMAX_TOL, thr_tol=THR_TOL)
    ref["replayed_logs"] = True
    st["strict"] = True
    # Theta in unorm16: compare() checks the pairs and the error map; the weights below
    rep = compare(api, img, s, S, N, True, lr, th, err, st, ref)
    assert rep["mode"] == "exact", rep
    Tr = O.op_saturation(O.op_box3(O.to_unit(ref["L"])), 1.3)
    assert np.abs(T.cpu().numpy() - Tr).max() <= 1e-6
    outr = O.apply(ref["ka"], ref["kb"], ref["omega"], s, S, Tr)
    K = S * S
    codes = th.codes_i32().cpu().numpy()
    same = (codes // K == ref["ka"]) & (codes % K == ref["kb"])
    o = out.cpu().numpy().astype(np.float64)
    assert np.abs(o - outr)[same].max() <= 1e-3
    # pairs differ only at near-ties of Algorithm 1 (compare() checked that each is a valid
    # optimum there)
    assert rep["mismatches"] <= rep["near_ties"], rep
    mine = O.apply(codes // K, codes % K, th.weight_f32().cpu().numpy().astype(np.float64), s, S,
                   Tr)
    assert np.abs(o - mine).max() <= 1e-3
    print(f"\n4K pipeline rows 0-399: {rep}, codes differ at {int((~same).sum())} pixels, "
          f"max |T_hat - oracle| {np.abs(o - outr)[same].max():.2e}")

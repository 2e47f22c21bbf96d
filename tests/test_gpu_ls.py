"""Least-squares LR colour update and its alternation with Algorithm 1 (the alternative joint
scheme beside Algorithm 2; not the paper's method) on the GPU against the FP64 oracle (needs a
GB300)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402

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
    return render_u8(Scene(width=W, height=H, n_cells=20, n_dots=25, n_lines=4, seed=seed))


@pytest.mark.parametrize("H,W,s,S,f16", [(96, 128, 8, 3, False), (100, 90, 4, 5, False),
                                         (77, 131, 3, 3, False), (64, 80, 16, 7, False),
                                         (90, 70, 8, 5, True), (40, 50, 2, 9, False)])
def test_ls_update_matches_oracle(api, H, W, s, S, f16):
    """One update for the same Theta (the GPU's) and LR image: within 1e-5 of the FP64 update,
    bitwise repeatable."""
    img = guide(H, W, H + W + S)
    hr = torch.from_numpy(img).cuda()
    L = api.glu_downsample(hr, s, api.GLU_DOWN_BOX)            # float32 in [0, 1]
    if f16:
        hr = (hr.to(torch.float32) / 255).to(torch.float16)
        img = hr.cpu().numpy().astype(np.float64)
    th, _ = api.glu_optimize(hr, L, api.glu_params(S=S), s, wfmt=api.GLU_W_F32)
    out = api.glu_ls_update(hr, th, L)
    out2 = api.glu_ls_update(hr, th, L)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    assert torch.equal(out, out2)
    K = S * S
    codes = th.codes_i32().cpu().numpy()
    ref = O.ls_update(img, L.cpu().numpy().astype(np.float64), s, S, codes // K, codes % K,
                      th.weight_f32().cpu().numpy().astype(np.float64))
    d = np.abs(out.cpu().numpy().astype(np.float64) - ref)
    assert d.max() < 1e-5, d.max()


@pytest.mark.parametrize("H,W,s,S,N", [(120, 160, 8, 3, 4), (96, 96, 4, 5, 3)])
def test_ls_joint_properties(api, H, W, s, S, N):
    """Residuals strictly decrease over the kept iterations; the returned state is Algorithm 1
    on the returned LR image (bitwise), E sums to the last kept residual, and the first
    iteration equals the oracle's update of the grid-downsampled start with the same Theta."""
    img = guide(H, W, 7 * H + S)
    hr = torch.from_numpy(img).cuda()
    p = api.glu_params(S=S, N=N)
    lr, th, err, st = api.glu_ls_joint_optimize(hr, s, p)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    kept = st["kept"]
    R = [st["R0"]] + st["residuals"][:kept]
    assert kept >= 1 and all(b < a for a, b in zip(R, R[1:]))
    th2, e2 = api.glu_optimize(hr, lr, api.glu_params(S=S), s, err_map=True, wfmt=api.GLU_W_F32)
    torch.cuda.synchronize()
    assert torch.equal(th2.code, th.code) and torch.equal(th2.weight, th.weight)
    assert torch.equal(e2, err)
    assert float(err.double().sum()) == pytest.approx(R[-1], rel=1e-6)
    # iteration 1 from the start state: grid LR, Algorithm 1 on it, one update
    L0 = api.glu_downsample(hr, s, api.GLU_DOWN_GRID, dtype=torch.float32)
    th0, _ = api.glu_optimize(hr, L0, api.glu_params(S=S), s, wfmt=api.GLU_W_F32)
    L1 = api.glu_ls_update(hr, th0, L0)
    K = S * S
    c0 = th0.codes_i32().cpu().numpy()
    ref = O.ls_update(img, L0.cpu().numpy().astype(np.float64), s, S, c0 // K, c0 % K,
                      th0.weight_f32().cpu().numpy().astype(np.float64))
    assert np.abs(L1.cpu().numpy() - ref).max() < 1e-5
    if kept >= 1:
        # the scheme's first kept state is that update (and Algorithm 1 on it)
        r1 = api.glu_ls_joint_optimize(hr, s, api.glu_params(S=S, N=1))
        torch.cuda.synchronize()
        assert torch.equal(r1[0], L1)


def test_ls_update_argument_checks(api):
    hr = torch.zeros((16, 16, 3), dtype=torch.uint8, device="cuda")
    L = torch.zeros((4, 4, 3), device="cuda")
    th, _ = api.glu_optimize(hr, L, api.glu_params(S=3), 4, wfmt=api.GLU_W_UNORM16)
    from paper_2307_09582_gb300 import _abi as A
    with pytest.raises(A.GluError):       # float32 weights only
        api.glu_ls_update(hr, th, L)
    th32, _ = api.glu_optimize(hr, L, api.glu_params(S=3), 4, wfmt=api.GLU_W_F32)
    with pytest.raises(A.GluError):       # lr_in and lr_out must differ
        api.glu_ls_update(hr, th32, L, lr_out=L)
    out = api.glu_ls_update(hr, th32, L)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0   # exactly representable: unchanged

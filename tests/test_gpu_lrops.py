"""The LR operators of the workloads (3x3 box / Gaussian filters, saturation, gamma) on the GPU
against the FP64 oracle's definitions of the same operators (needs a GB300). They are not part
of the method (the paper treats the operator as a black box); the joint 4K pipeline and the video
pipeline run them between Algorithm 1/2 and Eq. 1."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu

# float32 arithmetic of at most nine products of [0, 1] values: error below 1e-6
TOL = 1e-6


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import api as A
    return A


SHAPES = [(1, 1, 3), (1, 7, 3), (9, 1, 1), (2, 2, 2), (37, 53, 3), (270, 480, 3), (20, 31, 4)]


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_filter3_matches_oracle(api, op, shape):
    g = torch.Generator().manual_seed(hash(shape) % 1000 + op)
    X = torch.rand(shape, generator=g)
    got = api.glu_fx_filter3(X.cuda(), op).cpu().numpy().astype(np.float64)
    Xd = X.numpy().astype(np.float64)
    ref = O.op_box3(Xd) if op == 0 else O.op_gauss3(Xd)
    assert np.abs(got - ref).max() <= TOL


@pytest.mark.parametrize("op", [0, 1])
@pytest.mark.parametrize("shape", SHAPES)
def test_filter3_u8_matches_oracle(api, op, shape):
    g = torch.Generator().manual_seed(hash(shape) % 1000 + 10 + op)
    X = torch.randint(0, 256, shape, generator=g, dtype=torch.uint8)
    got = api.glu_fx_filter3_u8(X.cuda(), op).cpu().numpy().astype(np.float64)
    Xd = O.to_unit(X.numpy())
    ref = O.op_box3(Xd) if op == 0 else O.op_gauss3(Xd)
    assert np.abs(got - ref).max() <= TOL


@pytest.mark.parametrize("sat,gamma", [(1.3, 1.0), (1.0, 0.8), (1.3, 0.8), (0.5, 1.0), (1.0, 1.0)])
@pytest.mark.parametrize("shape", [(1, 1, 3), (37, 53, 3), (270, 480, 3)])
def test_point_matches_oracle(api, sat, gamma, shape):
    g = torch.Generator().manual_seed(int(sat * 10 + gamma * 100) + shape[0])
    X = torch.rand(shape, generator=g)
    X[0, 0] = torch.tensor([0.0, 1.0, 0.5])   # saturation pushes some channels out of [0, 1]
    got = api.glu_fx_point(X.cuda(), sat=sat, gamma=gamma).cpu().numpy().astype(np.float64)
    ref = O.op_gamma(O.op_saturation(X.numpy().astype(np.float64), sat), gamma)
    assert np.abs(got - ref).max() <= TOL
    assert got.min() >= 0.0 and got.max() <= 1.0


def _theta_for(api, H, W, s, S, wfmt, seed):
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    img = render_u8(Scene(width=W, height=H, n_cells=30, n_dots=20, n_lines=4, seed=seed))
    hr = torch.from_numpy(img).cuda()
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_GRID)
    theta, _ = api.glu_optimize(hr, lr, api.glu_params(S=S), s, wfmt=wfmt)
    return theta, lr


# (H, W, s, S, weights): W % 4 == 0 takes the tiled paths (the persistent TMA pipeline is the
# one launched as the operator's dependent), W % 4 != 0 the generic kernel
@pytest.mark.parametrize("H,W,s,S,wfmt", [(250, 344, 8, 5, 2), (130, 200, 4, 3, 0),
                                          (97, 131, 3, 5, 1), (64, 1024, 16, 7, 2)])
@pytest.mark.parametrize("filt,sat,gamma", [(0, 1.3, 1.0), (1, 1.0, 0.8), (-1, 0.7, 1.2)])
def test_apply_lrop_equals_separate_calls(api, H, W, s, S, wfmt, filt, sat, gamma):
    # the fused tail (operator kernel + apply as its programmatic dependent) gives bit for bit
    # what the operator's two calls and glu_apply give, for every apply variant, uint8 LR input
    theta, lr = _theta_for(api, H, W, s, S, wfmt, seed=H + W + filt)
    # x / 255 correctly rounded (numpy's float32 division; torch's scalar division multiplies by
    # a reciprocal)
    Xf = torch.from_numpy(lr.cpu().numpy().astype(np.float32) / np.float32(255.0)).cuda()
    T_ref = Xf if filt < 0 else api.glu_fx_filter3_u8(lr, filt)
    T_ref = api.glu_fx_point(T_ref, sat=sat, gamma=gamma)
    out_ref = api.glu_apply(theta, T_ref)
    nv = len(api.tune_variants(api.GLU_TUNE_APPLY))
    try:
        for v in range(nv):
            api.tune_force(api.GLU_TUNE_APPLY, v)
            out, T = api.glu_apply_lrop(theta, lr, filter=filt, sat=sat, gamma=gamma)
            torch.cuda.synchronize()
            assert api.glu_device_status() == 0
            if filt >= 0:
                assert torch.equal(T, T_ref), v
            else:
                # no filter: the operator reads x / 255 correctly rounded, as the float division
                # of the reference does
                assert torch.equal(T, api.glu_fx_point(Xf, sat=sat, gamma=gamma)), v
            assert torch.equal(out, out_ref), v
    finally:
        api.tune_force(api.GLU_TUNE_APPLY, -1)


def test_apply_lrop_float_input_and_f16_output_against_oracle(api):
    # float32 LR input, float16 output, Gaussian + gamma: the target against the oracle's
    # operators and the output against the oracle's Eq. 1 on that target
    H, W, s, S = 200, 320, 8, 5
    theta, lr = _theta_for(api, H, W, s, S, 0, seed=3)
    X = torch.rand(lr.shape, generator=torch.Generator().manual_seed(9)).cuda()
    out, T = api.glu_apply_lrop(theta, X, filter=1, sat=1.0, gamma=0.8, out_dtype=torch.float16)
    torch.cuda.synchronize()
    Td = O.op_gamma(O.op_gauss3(X.cpu().numpy().astype(np.float64)), 0.8)
    assert np.abs(T.cpu().numpy() - Td).max() <= TOL
    codes = theta.codes_i32().cpu().numpy()
    K = S * S
    ref = O.apply(codes // K, codes % K, theta.weight_f32().cpu().numpy().astype(np.float64),
                  s, S, T.cpu().numpy().astype(np.float64))
    assert np.abs(out.float().cpu().numpy() - ref).max() < 1e-3


def test_apply_lrop_rejects_bad_arguments(api):
    theta, lr = _theta_for(api, 64, 64, 8, 3, 0, seed=1)
    with pytest.raises(api.GluError):
        api.glu_apply_lrop(theta, lr, filter=2)
    with pytest.raises(api.GluError):
        api.glu_apply_lrop(theta, lr[:-1].contiguous())

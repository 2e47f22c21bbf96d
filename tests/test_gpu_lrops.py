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

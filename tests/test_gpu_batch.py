"""Batched calls (several images of different sizes, scales and windows in one set of launches)
against per-image calls and the FP64 oracle (needs a GB300).

Every item of a batched call must equal, bit for bit, the same call on that image alone: the
images share no state (own LR blocks, components, residuals and stopping rule). The per-image
calls are the ones the parity tests check against the oracle; one item per batch is checked
against the oracle here as well, so the chain batch -> single -> oracle is closed in this file.
"""
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


def small_batch(n=6, seed=11):
    """Uneven sizes (ragged against every tile and block size), scales {4, 8, 16}, windows
    {3, 5}; the same recipe as the 16-image batch workload, at sizes the oracle finishes fast."""
    from paper_2307_09582_gb300.inputs import render_u8
    from paper_2307_09582_gb300.inputs.workloads import batch_scenes
    out = []
    for sc, s, S in batch_scenes(seed=seed, n=n, wmin=90, wmax=420, hmin=70, hmax=300):
        out.append((render_u8(sc), s, S))
    return out


def same_theta(t1, t2):
    return torch.equal(t1.code, t2.code) and torch.equal(t1.weight, t2.weight)


@pytest.mark.parametrize("wfmt", [0, 2])
def test_optimize_batched_equals_single(api, wfmt):
    items = small_batch()
    hrs = [torch.from_numpy(img).cuda() for img, _, _ in items]
    lrs = [api.glu_downsample(hr, s, api.GLU_DOWN_BOX) for hr, (_, s, _) in zip(hrs, items)]
    p = api.glu_params()
    out = api.glu_optimize_batched(hrs, lrs, p, [s for _, s, _ in items],
                                   [S for _, _, S in items], wfmt=wfmt)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    for (img, s, S), hr, lr, (tb, eb) in zip(items, hrs, lrs, out):
        ts, es = api.glu_optimize(hr, lr, api.glu_params(S=S), s, err_map=True, wfmt=wfmt)
        torch.cuda.synchronize()
        assert same_theta(tb, ts) and torch.equal(eb, es), (img.shape, s, S)
    # one item against the oracle directly
    img, s, S = items[0]
    tb, eb = out[0]
    check_search(img, lrs[0].cpu().numpy(), s, S, tb, eb)


def test_optimize_batched_edge_cases(api):
    p = api.glu_params()
    assert api.glu_optimize_batched([], [], p, []) == []
    # a 1x1 guide and a guide smaller than one LR block, beside an ordinary one
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    imgs = [render_u8(Scene(width=1, height=1, n_cells=1, n_dots=1, n_lines=1, seed=3)),
            render_u8(Scene(width=7, height=5, n_cells=2, n_dots=2, n_lines=1, seed=4)),
            render_u8(Scene(width=130, height=66, n_cells=9, n_dots=9, n_lines=2, seed=5))]
    scales, Ss = [4, 8, 4], [3, 5, 3]
    hrs = [torch.from_numpy(i).cuda() for i in imgs]
    lrs = [api.glu_downsample(hr, s, api.GLU_DOWN_BOX) for hr, s in zip(hrs, scales)]
    out = api.glu_optimize_batched(hrs, lrs, p, scales, Ss)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    for img, lr, s, S, (t, e) in zip(imgs, lrs, scales, Ss, out):
        check_search(img, lr.cpu().numpy(), s, S, t, e)


def test_optimize_batched_more_than_one_launch(api):
    """40 images: more than one persistent launch's worth of images."""
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    imgs = [render_u8(Scene(width=40 + 3 * k, height=30 + 2 * k, n_cells=6, n_dots=6,
                            n_lines=2, seed=100 + k)) for k in range(40)]
    scales = [4 + 4 * (k % 2) for k in range(40)]
    hrs = [torch.from_numpy(i).cuda() for i in imgs]
    lrs = [api.glu_downsample(hr, s, api.GLU_DOWN_BOX) for hr, s in zip(hrs, scales)]
    out = api.glu_optimize_batched(hrs, lrs, api.glu_params(), scales)
    torch.cuda.synchronize()
    for hr, lr, s, (t, e) in zip(hrs, lrs, scales, out):
        ts, es = api.glu_optimize(hr, lr, api.glu_params(), s, err_map=True)
        assert same_theta(t, ts) and torch.equal(e, es)


def joint_single(api, img, s, S, N, strict, wfmt=0):
    hr = torch.from_numpy(img).cuda()
    p = api.glu_params(S=S, N=N, joint=api.GLU_JOINT_STRICT if strict else api.GLU_JOINT_PAPER)
    return api.glu_joint_optimize(hr, s, p, wfmt=wfmt, decisions=True, argmax_log=True)


@pytest.mark.parametrize("strict", [True, False])
def test_joint_batched_equals_single_and_oracle(api, strict):
    items = small_batch(n=5, seed=12)
    N = 4
    hrs = [torch.from_numpy(img).cuda() for img, _, _ in items]
    p = api.glu_params(N=N, joint=api.GLU_JOINT_STRICT if strict else api.GLU_JOINT_PAPER)
    out = api.glu_joint_optimize_batched(hrs, [s for _, s, _ in items], p,
                                         [S for _, _, S in items])
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    for (img, s, S), (lb, tb, eb, sb) in zip(items, out):
        ls, ts, es, ss = joint_single(api, img, s, S, N, strict)
        torch.cuda.synchronize()
        assert torch.equal(lb, ls) and same_theta(tb, ts) and torch.equal(eb, es), \
            (img.shape, s, S)
        assert sb["iterations"] == ss["iterations"] and sb["R0"] == ss["R0"]
        assert sb["iters"] == ss["iters"]
    # the first item against the oracle, through its single-image twin's decision log
    from tests.test_gpu_joint import ARGMAX_TOL, REPLAY_TOL, THR_TOL, compare
    img, s, S = items[0]
    ls, ts, es, ss = joint_single(api, img, s, S, N, strict)
    ss["strict"] = strict
    ref = O.joint(img, s, S, N=N, strict=strict, force=ss["decisions"], force_tol=REPLAY_TOL,
                  argmax=ss["argmax"], argmax_tol=ARGMAX_TOL, thr_tol=THR_TOL)
    ref["replayed_logs"] = True
    rep = compare(api, img, s, S, N, strict, ls, ts, es, ss, ref)
    assert rep["mode"] == "exact", rep


def test_joint_batched_sixteen_image_workload(api):
    """The 16-image batch workload at full size: every item equals its single-image call."""
    from paper_2307_09582_gb300.inputs import render_u8
    from paper_2307_09582_gb300.inputs.workloads import batch_scenes
    items = [(render_u8(sc), s, S) for sc, s, S in batch_scenes()]
    hrs = [torch.from_numpy(img).cuda() for img, _, _ in items]
    p = api.glu_params(N=3)
    out = api.glu_joint_optimize_batched(hrs, [s for _, s, _ in items], p,
                                         [S for _, _, S in items], wfmt=api.GLU_W_UNORM16)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    for (img, s, S), hr, (lb, tb, eb, sb) in zip(items, hrs, out):
        ps = api.glu_params(S=S, N=3)
        ls, ts, es, ss = api.glu_joint_optimize(hr, s, ps, wfmt=api.GLU_W_UNORM16)
        torch.cuda.synchronize()
        assert torch.equal(lb, ls) and same_theta(tb, ts) and torch.equal(eb, es)
        assert sb["iters"] == ss["iters"]


def test_joint_batched_with_an_empty_set(api):
    """A flat image (no pixel above tau: Algorithm 2 stops before any trial) beside a busy one:
    the flat one stops at iteration 0 while the other carries on."""
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    flat = np.full((64, 96, 3), 77, dtype=np.uint8)
    busy = render_u8(Scene(width=200, height=150, n_cells=30, n_dots=60, n_lines=6, seed=9))
    hrs = [torch.from_numpy(flat).cuda(), torch.from_numpy(busy).cuda()]
    p = api.glu_params(N=3)
    out = api.glu_joint_optimize_batched(hrs, [4, 4], p, [3, 3])
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    assert out[0][3]["iterations"] == 0 and out[0][3]["R0"] == 0.0
    assert out[1][3]["iterations"] >= 1
    ls, ts, es, ss = joint_single(api, busy, 4, 3, 3, True)
    assert torch.equal(out[1][0], ls) and same_theta(out[1][1], ts)
    assert out[1][3]["iters"] == ss["iters"]

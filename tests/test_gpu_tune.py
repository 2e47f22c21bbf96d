"""Autotuner: every implementation variant of the search and of the tiled apply gives
bit-identical results, and tuning picks and caches a variant (needs a GB300)."""
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
    yield A
    A.tune_force(A.GLU_TUNE_SEARCH, -1)
    A.tune_force(A.GLU_TUNE_APPLY, -1)
    A.tune_mode(False)
    A.tune_clear()


def guide(W, H, seed):
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    return torch.from_numpy(render_u8(Scene(width=W, height=H, n_cells=60, n_dots=200,
                                            n_lines=12, seed=seed))).cuda()


@pytest.mark.parametrize("W,H,s,S,f16", [(1000, 700, 8, 5, False), (777, 333, 4, 3, False),
                                         (640, 480, 8, 5, True), (301, 157, 16, 7, False)])
def test_search_variants_bit_identical(api, W, H, s, S, f16):
    hr = guide(W, H, W + S)
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_BOX)
    if f16:
        hr = (hr.to(torch.float32) / 255).to(torch.float16)
    p = api.glu_params(S=S)
    ref = None
    for v in range(len(api.tune_variants(api.GLU_TUNE_SEARCH))):
        api.tune_force(api.GLU_TUNE_SEARCH, v)
        th, err = api.glu_optimize(hr, lr, p, s, err_map=True)
        torch.cuda.synchronize()
        assert api.glu_device_status() == 0
        if ref is None:
            ref = (th, err)
        else:
            assert torch.equal(th.code, ref[0].code) and torch.equal(th.weight, ref[0].weight)
            assert torch.equal(err, ref[1]), v
    api.tune_force(api.GLU_TUNE_SEARCH, -1)


def test_search_variants_on_a_batch(api):
    hrs = [guide(200 + 37 * k, 150 + 23 * k, k) for k in range(5)]
    scales = [4, 8, 16, 8, 4]
    Ss = [3, 5, 3, 5, 3]
    lrs = [api.glu_downsample(h, s, api.GLU_DOWN_BOX) for h, s in zip(hrs, scales)]
    ref = None
    for v in range(len(api.tune_variants(api.GLU_TUNE_SEARCH))):
        api.tune_force(api.GLU_TUNE_SEARCH, v)
        out = api.glu_optimize_batched(hrs, lrs, api.glu_params(), scales, Ss)
        torch.cuda.synchronize()
        if ref is None:
            ref = out
        else:
            for (t, e), (tr, er) in zip(out, ref):
                assert torch.equal(t.code, tr.code) and torch.equal(t.weight, tr.weight)
                assert torch.equal(e, er)
    api.tune_force(api.GLU_TUNE_SEARCH, -1)


@pytest.mark.parametrize("out_dtype,wfmt", [(torch.float32, 0), (torch.float16, 2),
                                            (torch.float32, 1)])
def test_apply_variants_bit_identical(api, out_dtype, wfmt):
    hr = guide(1000, 700, 3)
    s, S = 8, 5
    lr = api.glu_downsample(hr, s, api.GLU_DOWN_BOX)
    th, _ = api.glu_optimize(hr, lr, api.glu_params(S=S), s, wfmt=wfmt)
    T = torch.rand(lr.shape, device="cuda")
    ref = None
    for v in range(len(api.tune_variants(api.GLU_TUNE_APPLY))):
        api.tune_force(api.GLU_TUNE_APPLY, v)
        out = api.glu_apply(th, T, out_dtype=out_dtype)
        torch.cuda.synchronize()
        assert api.glu_device_status() == 0
        if ref is None:
            ref = out
        else:
            assert torch.equal(out, ref), v
    api.tune_force(api.GLU_TUNE_APPLY, -1)
    # float16 output is the float32 result rounded to nearest
    if out_dtype == torch.float16:
        o32 = api.glu_apply(th, T, out_dtype=torch.float32)
        assert torch.equal(ref, o32.to(torch.float16))


def test_tuning_picks_and_caches(api):
    api.tune_clear()
    api.tune_mode(True)
    hr = guide(1200, 800, 5)
    lr = api.glu_downsample(hr, 8, api.GLU_DOWN_BOX)
    p = api.glu_params(S=5)
    th, err = api.glu_optimize(hr, lr, p, 8, err_map=True)
    T = torch.rand(lr.shape, device="cuda")
    out = api.glu_apply(th, T)
    torch.cuda.synchronize()
    lines = [l.split() for l in api.tune_export().splitlines()]
    kernels = sorted(int(l[0]) for l in lines)
    assert kernels == [api.GLU_TUNE_SEARCH, api.GLU_TUNE_APPLY]
    # a graph capture with tuning on uses the cached choice (no timing inside a capture)
    v = api.Video(800, 1200, 8, p, hr_dtype=torch.float16, out_dtype=torch.float32)
    fr = (hr.to(torch.float32) / 255).to(torch.float16)
    o = torch.empty((800, 1200, 3), device="cuda")
    v.bind(0, fr, o)
    v.launch(0)
    torch.cuda.synchronize()
    v.close()
    api.tune_mode(False)
    api.tune_force(api.GLU_TUNE_SEARCH, 0)
    api.tune_force(api.GLU_TUNE_APPLY, 0)
    th0, err0 = api.glu_optimize(hr, lr, p, 8, err_map=True)
    out0 = api.glu_apply(th0, T)
    torch.cuda.synchronize()
    assert torch.equal(th0.code, th.code) and torch.equal(err0, err) and torch.equal(out0, out)
    api.tune_force(api.GLU_TUNE_SEARCH, -1)
    api.tune_force(api.GLU_TUNE_APPLY, -1)
    api.tune_clear()

"""Failure detection on the GPU without a fault: the bounded waits of Algorithm 2's trial kernel
are made to run out. With a deadline of 1 ns, the first wait that is not satisfied within one
polling burst (a queue position whose component no trial has published yet: with many CTAs and a
dependency graph of several levels, most CTAs start on one) gives up; the kernel records
GLU_ERR_TIMEOUT and returns, the call reports it, and the context stays usable (needs a GB300)."""
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
    A.test_set_wait_limit(0)


def test_trial_wait_timeout_is_reported_and_context_survives(api):
    from paper_2307_09582_gb300 import _abi as A
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    img = render_u8(Scene(width=640, height=480, n_cells=80, n_dots=200, n_lines=12, seed=9))
    hr = torch.from_numpy(img).cuda()
    p = api.glu_params(S=5, N=3)
    lr0, th0, e0, st0 = api.glu_joint_optimize(hr, 8, p)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    assert st0["iters"][0]["M"] > 200   # many components: most CTAs wait for one
    api.test_set_wait_limit(1)
    with pytest.raises(A.GluError) as exc:
        api.glu_joint_optimize(hr, 8, p)
    assert exc.value.code == A.GLU_ERR_TIMEOUT
    torch.cuda.synchronize()
    assert api.glu_device_status() == A.GLU_ERR_TIMEOUT
    assert api.glu_device_status() == 0   # read and cleared
    # the default deadline again: the same call gives the same result as before
    api.test_set_wait_limit(0)
    lr1, th1, e1, st1 = api.glu_joint_optimize(hr, 8, p)
    torch.cuda.synchronize()
    assert api.glu_device_status() == 0
    assert torch.equal(lr1, lr0) and torch.equal(th1.code, th0.code) and torch.equal(e1, e0)

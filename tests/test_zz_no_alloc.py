"""glu_joint_optimize_static (no device allocation) agrees with glu_joint_optimize.

Some callers of the library cannot allocate device memory: a plug-in whose host application
owns every device allocation, or a streaming loop that must not risk the device-wide stall an
allocation can cause. For them Algorithm 2 runs on a fixed array inside the library. This file
is collected last (its name sorts last) so a failure here never hides another test's result.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2307_09582_gb300 import _abi as A
    from paper_2307_09582_gb300 import api
    lib = A.load()
    f = lib.glu_joint_optimize_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(A.GluImage), ctypes.c_int32, ctypes.POINTER(A.GluParams),
                  ctypes.POINTER(A.GluImage), ctypes.POINTER(A.GluTheta), ctypes.c_void_p,
                  ctypes.POINTER(A.GluJointStats), ctypes.c_void_p]
    return A, api, lib, f


def test_static_workspace_matches_caller_workspace_on_repeated_calls(env):
    """Three calls in a row with the same output buffers (the streaming-loop case: the shared
    array keeps the previous call's contents) give results identical, bit for bit, to the call
    with a caller workspace, and none of them records a CUDA graph (a repeated
    glu_joint_optimize call would)."""
    A, api, lib, f = env
    from paper_2307_09582_gb300.inputs import Scene, render_u8
    img = render_u8(Scene(width=640, height=480, n_cells=60, n_dots=150, n_lines=12, seed=31))
    s, S, N = 8, 5, 4
    hr = torch.from_numpy(img).cuda()
    p = api.glu_params(S=S, N=N)
    lr_ref, th_ref, err_ref, st_ref = api.glu_joint_optimize(hr, s, p)
    torch.cuda.synchronize()
    h, w = api.lr_dims(480, 640, s)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lr = torch.empty((h, w, 3), dtype=torch.uint8, device="cuda")
    th = api.Theta.empty(480, 640, s, S, api.GLU_W_F32)
    err = torch.empty((480, 640), dtype=torch.float32, device="cuda")
    hi, li, td = api.image(hr), api.image(lr), th.desc()
    graphs_before = lib.glu_test_joint_graph_count()
    for call in range(3):
        lr.fill_(0)
        th.code.fill_(0)
        th.weight.fill_(0)
        err.fill_(-1.0)
        st = A.GluJointStats()
        rc = f(ctypes.byref(hi), s, ctypes.byref(p), ctypes.byref(li), ctypes.byref(td),
               ctypes.c_void_p(err.data_ptr()), ctypes.byref(st), stream)
        assert rc == A.GLU_OK, (call, A.status_string(rc))
        torch.cuda.synchronize()
        assert api.glu_device_status() == 0
        # the optimisation is deterministic: identical results (tolerance zero)
        assert torch.equal(lr, lr_ref), call
        assert torch.equal(th.code, th_ref.code) and torch.equal(th.weight, th_ref.weight), call
        assert torch.equal(err, err_ref), call
        assert st.iterations == st_ref["iterations"]
        assert st.residual[st.iterations] == pytest.approx(st_ref["iters"][-1]["residual"], rel=0)
    assert lib.glu_test_joint_graph_count() == graphs_before


def test_static_workspace_rejects_too_large_image(env):
    """An image whose workspace exceeds the fixed array is refused before any launch; the
    buffers are real device allocations of the declared sizes."""
    A, api, lib, f = env
    H, W, s, S = 4096, 4096, 8, 5
    p = api.glu_params(S=S, N=5)
    assert api.glu_joint_workspace_size(H, W, s, p) > (64 << 20)   # GLU_JOINT_STATIC_BYTES
    hr = torch.zeros((H, W, 3), dtype=torch.uint8, device="cuda")
    h, w = api.lr_dims(H, W, s)
    lr = torch.full((h, w, 3), 7, dtype=torch.uint8, device="cuda")
    th = api.Theta.empty(H, W, s, S, api.GLU_W_F32)
    th.code.fill_(3)
    hi, li, td = api.image(hr), api.image(lr), th.desc()
    rc = f(ctypes.byref(hi), s, ctypes.byref(p), ctypes.byref(li), ctypes.byref(td), None, None,
           None)
    assert rc == A.GLU_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert int((lr != 7).sum()) == 0 and int((th.code != 3).sum()) == 0   # nothing was written

"""The C-ABI library loads without a GPU, exports every declared entry point, and validates
arguments on the host (no kernel is launched by these calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_09582_gb300 import build, _abi
    build.build_cuda()
    return _abi.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(glu_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"glu_downsample", "glu_optimize", "glu_joint_optimize", "glu_apply",
            "glu_apply_backward"} <= set(names)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_params_default_matches_paper(lib):
    import json
    from paper_2307_09582_gb300 import _abi as A
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))
    p = A.GluParams()
    lib.glu_params_default(ctypes.byref(p))
    assert p.S == g["window_size_S"]["value"]
    assert p.N == g["max_iterations_N"]["value"]
    assert p.eps == pytest.approx(g["eps"]["value"], rel=1e-6)
    assert p.tau == pytest.approx(g["tau"]["value"], rel=1e-6)
    assert p.mode == A.GLU_MODE_FAST and p.joint == A.GLU_JOINT_STRICT and p.connectivity == 8


def test_host_validation_codes(lib):
    from paper_2307_09582_gb300 import _abi as A
    p = A.GluParams()
    lib.glu_params_default(ctypes.byref(p))
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    hr = A.GluImage(fake, 64, 64, 3, A.GLU_U8, 64 * 3)
    lr_bad = A.GluImage(fake, 15, 16, 3, A.GLU_U8, 16 * 3)
    th = A.GluTheta(fake, fake, 64, 64, 4, 3, A.GLU_W_F32)
    assert lib.glu_optimize(ctypes.byref(hr), ctypes.byref(lr_bad), ctypes.byref(p),
                            ctypes.byref(th), None, None) == A.GLU_ERR_SHAPE
    assert lib.glu_optimize(None, ctypes.byref(lr_bad), ctypes.byref(p), ctypes.byref(th),
                            None, None) == A.GLU_ERR_INVALID_ARG
    p2 = A.GluParams.from_buffer_copy(p)
    p2.S = 4
    lr = A.GluImage(fake, 16, 16, 3, A.GLU_U8, 16 * 3)
    assert lib.glu_optimize(ctypes.byref(hr), ctypes.byref(lr), ctypes.byref(p2),
                            ctypes.byref(th), None, None) == A.GLU_ERR_INVALID_ARG
    # GLU* (Eq. 4) weights are unclamped: only float32 weights can hold them; unknown modes fail
    p3 = A.GluParams.from_buffer_copy(p)
    p3.mode = A.GLU_MODE_EXACT
    th16 = A.GluTheta(fake, fake, 64, 64, 4, 3, A.GLU_W_UNORM16)
    assert lib.glu_optimize(ctypes.byref(hr), ctypes.byref(lr), ctypes.byref(p3),
                            ctypes.byref(th16), None, None) == A.GLU_ERR_UNSUPPORTED
    p3.mode = 3
    assert lib.glu_optimize(ctypes.byref(hr), ctypes.byref(lr), ctypes.byref(p3),
                            ctypes.byref(th), None, None) == A.GLU_ERR_INVALID_ARG
    p3.mode = A.GLU_MODE_EXACT   # the joint optimisation (Algorithm 2) runs Algorithm 1 only
    assert lib.glu_joint_optimize(ctypes.byref(hr), 4, ctypes.byref(p3), ctypes.byref(lr),
                                  ctypes.byref(th), None, None, fake, 1 << 30, None) == \
        A.GLU_ERR_UNSUPPORTED
    bad_pitch = A.GluImage(fake, 64, 64, 3, A.GLU_U8, 100)
    assert lib.glu_downsample(ctypes.byref(bad_pitch), 4, 0, ctypes.byref(lr), None) == \
        A.GLU_ERR_INVALID_ARG
    assert lib.glu_downsample(ctypes.byref(hr), 4, 7, ctypes.byref(lr), None) == \
        A.GLU_ERR_INVALID_ARG
    out_u8 = A.GluImage(fake, 64, 64, 3, A.GLU_U8, 64 * 3)
    T = A.GluImage(fake, 16, 16, 3, A.GLU_F32, 16 * 3)
    assert lib.glu_apply(ctypes.byref(th), ctypes.byref(T), ctypes.byref(out_u8), None) == \
        A.GLU_ERR_UNSUPPORTED
    # joint: workspace too small / misaligned
    need = lib.glu_joint_workspace_size(64, 64, 4, ctypes.byref(p))
    assert need > 64 * 64 * 4
    assert lib.glu_joint_workspace_size(0, 64, 4, ctypes.byref(p)) == 0
    assert lib.glu_joint_optimize(ctypes.byref(hr), 4, ctypes.byref(p), ctypes.byref(lr),
                                  ctypes.byref(th), None, None, fake, need - 1, None) == \
        A.GLU_ERR_WORKSPACE
    assert lib.glu_joint_optimize(ctypes.byref(hr), 4, ctypes.byref(p), ctypes.byref(lr),
                                  ctypes.byref(th), None, None, ctypes.c_void_p(0x1001), need,
                                  None) == A.GLU_ERR_WORKSPACE
    for c in range(-7, 1):
        assert lib.glu_status_string(c).decode().startswith("GLU_")
    assert b"sm_103a" in lib.glu_version()


def test_batched_host_validation(lib):
    from paper_2307_09582_gb300 import _abi as A
    p = A.GluParams()
    lib.glu_params_default(ctypes.byref(p))
    fake = ctypes.c_void_p(0x1000)
    items = (A.GluBatchItem * 33)()
    for k in range(33):
        items[k].hr = A.GluImage(fake, 64 + k, 48, 3, A.GLU_U8, (64 + k) * 3)
        items[k].hr.w, items[k].hr.pitch = 64 + k, (64 + k) * 3
        items[k].hr.h = 48
        h, w = (48 + 3) // 4, (64 + k + 3) // 4
        items[k].lr = A.GluImage(fake, h, w, 3, A.GLU_U8, w * 3)
        items[k].theta = A.GluTheta(fake, fake, 48, 64 + k, 4, 3 + 2 * (k % 2), A.GLU_W_F32)
    # empty batches are no-ops; null item arrays are rejected
    assert lib.glu_optimize_batched(None, 0, ctypes.byref(p), None) == A.GLU_OK
    assert lib.glu_joint_optimize_batched(None, 0, ctypes.byref(p), None, None, 0, None) == \
        A.GLU_OK
    assert lib.glu_optimize_batched(None, 2, ctypes.byref(p), None) == A.GLU_ERR_INVALID_ARG
    # more than 32 joint images, or a mixed weight format, is unsupported
    assert lib.glu_joint_optimize_batched(items, 33, ctypes.byref(p), None, fake, 1 << 40,
                                          None) == A.GLU_ERR_UNSUPPORTED
    assert lib.glu_joint_batched_workspace_size(items, 33, ctypes.byref(p)) == 0
    items[1].theta.wfmt = A.GLU_W_F16
    assert lib.glu_joint_optimize_batched(items, 2, ctypes.byref(p), None, fake, 1 << 40,
                                          None) == A.GLU_ERR_UNSUPPORTED
    assert lib.glu_optimize_batched(items, 2, ctypes.byref(p), None) == A.GLU_ERR_UNSUPPORTED
    items[1].theta.wfmt = A.GLU_W_F32
    # a wrong LR size in any item is a shape error, before any launch
    items[3].lr.h += 1
    assert lib.glu_optimize_batched(items, 5, ctypes.byref(p), None) == A.GLU_ERR_SHAPE
    assert lib.glu_joint_optimize_batched(items, 5, ctypes.byref(p), None, fake, 1 << 40,
                                          None) == A.GLU_ERR_SHAPE
    items[3].lr.h -= 1
    # workspace: a batch of one needs what the single-image call needs; more images need more;
    # too small a workspace is refused
    p.S = items[0].theta.S
    one = lib.glu_joint_batched_workspace_size(items, 1, ctypes.byref(p))
    assert one == lib.glu_joint_workspace_size(48, 64, 4, ctypes.byref(p))
    four = lib.glu_joint_batched_workspace_size(items, 4, ctypes.byref(p))
    assert four > one
    assert lib.glu_joint_optimize_batched(items, 4, ctypes.byref(p), None, fake, four - 1,
                                          None) == A.GLU_ERR_WORKSPACE


def test_video_host_validation(lib):
    from paper_2307_09582_gb300 import _abi as A
    d = A.GluVideoDesc()
    d.H, d.W, d.scale = 2160, 3840, 8
    d.hr_dtype, d.out_dtype = A.GLU_F16, A.GLU_F16
    lib.glu_params_default(ctypes.byref(d.params))
    d.params.S = 5
    d.wfmt, d.n_ops, d.overlap = A.GLU_W_UNORM16, 1, 1
    d.ops[0] = A.GluLrOp(1, 1.0, 0.8)
    need = lib.glu_video_workspace_size(ctypes.byref(d))
    h, w = 270, 480
    # the LR float image, two per operator (filtered, target), the codes and the weights, each
    # 256-byte aligned
    lr = -(-(h * w * 3 * 4) // 256) * 256
    assert need == 3 * lr + 2 * (-(-(2160 * 3840 * 2) // 256) * 256)
    d.n_ops = 3
    d.ops[1] = A.GluLrOp(0, 1.3, 1.0)
    d.ops[2] = A.GluLrOp(-1, 1.0, 1.2)
    assert lib.glu_video_workspace_size(ctypes.byref(d)) == need + 4 * lr
    d.n_ops = 1
    out = ctypes.c_void_p()
    assert lib.glu_video_create(ctypes.byref(d), None, need, ctypes.byref(out)) == \
        A.GLU_ERR_WORKSPACE
    assert lib.glu_video_create(ctypes.byref(d), ctypes.c_void_p(0x1100), need - 1,
                                ctypes.byref(out)) == A.GLU_ERR_WORKSPACE
    for obj, field, bad in ((d, "hr_dtype", A.GLU_F32), (d, "out_dtype", A.GLU_U8),
                            (d.ops[0], "filter", 2), (d.ops[0], "gamma", 0.0), (d, "scale", 0),
                            (d, "n_ops", 0), (d, "n_ops", A.GLU_VIDEO_MAX_OPS + 1)):
        old = getattr(obj, field)
        setattr(obj, field, bad)
        assert lib.glu_video_workspace_size(ctypes.byref(d)) == 0, field
        assert lib.glu_video_create(ctypes.byref(d), ctypes.c_void_p(0x1100), need,
                                    ctypes.byref(out)) == A.GLU_ERR_INVALID_ARG
        setattr(obj, field, old)
    assert lib.glu_video_launch(None, 0, None) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_video_destroy(None) == A.GLU_OK


def test_missing_library_fails_loudly(tmp_path):
    from paper_2307_09582_gb300 import _abi as A
    with pytest.raises(RuntimeError, match="not found"):
        A.load(str(tmp_path / "libglu.so"))


def test_backward_workspace_host_side(lib):
    from paper_2307_09582_gb300 import _abi as A
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    th = A.GluTheta(fake, fake, 64, 80, 8, 5, A.GLU_W_F32)
    # 8 c S^2 bytes per LR pixel (8 x 10 LR pixels)
    assert lib.glu_apply_backward_workspace_size(ctypes.byref(th), 3) == 8 * 10 * 8 * 3 * 25
    assert lib.glu_apply_backward_workspace_size(ctypes.byref(th), 5) == 0
    T = A.GluImage(fake, 8, 10, 3, A.GLU_F32, 30)
    G = A.GluImage(fake, 64, 80, 3, A.GLU_F32, 240)
    gT = A.GluImage(fake, 8, 10, 3, A.GLU_F32, 30)
    need = lib.glu_apply_backward_workspace_size(ctypes.byref(th), 3)
    args = (ctypes.byref(th), ctypes.byref(T), ctypes.byref(G), ctypes.byref(gT), None)
    assert lib.glu_apply_backward_ws(*args, fake, need - 1, None) == A.GLU_ERR_WORKSPACE
    assert lib.glu_apply_backward_ws(*args, ctypes.c_void_p(0x1004), need, None) == \
        A.GLU_ERR_WORKSPACE
    assert lib.glu_apply_backward_ws(*args, None, need, None) == A.GLU_ERR_WORKSPACE
    G_bad = A.GluImage(fake, 64, 81, 3, A.GLU_F32, 243)
    assert lib.glu_apply_backward_ws(ctypes.byref(th), ctypes.byref(T), ctypes.byref(G_bad),
                                     ctypes.byref(gT), None, fake, need, None) == A.GLU_ERR_SHAPE


def test_tuner_host_side(lib):
    from paper_2307_09582_gb300 import _abi as A
    assert lib.glu_tune_variants(A.GLU_TUNE_SEARCH) == 5
    assert lib.glu_tune_variants(A.GLU_TUNE_APPLY) == 10
    assert lib.glu_tune_variants(7) == A.GLU_ERR_INVALID_ARG
    buf = ctypes.create_string_buffer(128)
    assert lib.glu_tune_variant_name(A.GLU_TUNE_SEARCH, 0, buf, 128) == A.GLU_OK
    assert buf.value.startswith(b"tile 64x32")
    assert lib.glu_tune_variant_name(A.GLU_TUNE_APPLY, 4, buf, 128) == A.GLU_OK
    assert buf.value == b"tile 128x16, TMA loads and stores"
    assert lib.glu_tune_variant_name(A.GLU_TUNE_APPLY, 7, buf, 128) == A.GLU_OK
    assert buf.value == b"tile 128x16, TMA pipeline (persistent)"
    assert lib.glu_tune_variant_name(A.GLU_TUNE_APPLY, 10, buf, 128) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_tune_force(A.GLU_TUNE_SEARCH, 5) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_tune_force(A.GLU_TUNE_SEARCH, -1) == A.GLU_OK
    # export / import round trip of the text form
    assert lib.glu_tune_clear() == A.GLU_OK
    assert lib.glu_tune_export(None, 0) == 1
    text = b"0 0 0 5 8 23 3 0.250000\n1 2 2 5 8 23 1 0.040000\n"
    assert lib.glu_tune_import(text) == A.GLU_OK
    n = lib.glu_tune_export(None, 0)
    out = ctypes.create_string_buffer(n)
    assert lib.glu_tune_export(out, n) == n
    assert out.value == text
    assert lib.glu_tune_import(b"0 0 0 5 8 23 9 0.1\n") == A.GLU_ERR_INVALID_ARG  # no variant 9
    assert lib.glu_tune_import(b"garbage") == A.GLU_ERR_INVALID_ARG
    assert lib.glu_tune_clear() == A.GLU_OK


def test_pipeline_host_side(lib):
    """glu_pipeline_host: workspace size and every argument error, all before any copy."""
    from paper_2307_09582_gb300 import _abi as A
    p = A.GluParams()
    lib.glu_params_default(ctypes.byref(p))
    H, W, s = 64, 80, 8
    need = lib.glu_pipeline_host_workspace_size(H, W, s, ctypes.byref(p))
    # Algorithm 2's workspace plus the device copies: guide (3 B/px), Theta (4 B/px), result
    # (12 B/px) and two LR images (3 + 12 B per LR pixel), each 256-byte aligned
    jws = lib.glu_joint_workspace_size(H, W, s, ctypes.byref(p))
    assert need >= jws + H * W * (3 + 4 + 12) + 8 * 10 * 15
    assert need <= jws + H * W * (3 + 4 + 12) + 8 * 10 * 15 + 8 * 256
    assert lib.glu_pipeline_host_workspace_size(0, W, s, ctypes.byref(p)) == 0
    assert lib.glu_pipeline_host_workspace_size(H, W, s, None) == 0
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    args = lambda **k: (k.get("hr", fake), k.get("H", H), W, s, ctypes.byref(k.get("p", p)),
                        k.get("op", 1), k.get("sat", 1.3), k.get("gamma", 1.0),
                        k.get("out", fake), k.get("ws", fake), k.get("wsb", need), None)
    assert lib.glu_pipeline_host(*args(hr=None)) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_pipeline_host(*args(out=None)) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_pipeline_host(*args(H=0)) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_pipeline_host(*args(op=2)) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_pipeline_host(*args(sat=-1.0)) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_pipeline_host(*args(gamma=0.0)) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_pipeline_host(*args(wsb=need - 1)) == A.GLU_ERR_WORKSPACE
    assert lib.glu_pipeline_host(*args(ws=ctypes.c_void_p(0x1010))) == A.GLU_ERR_WORKSPACE
    assert lib.glu_pipeline_host(*args(ws=None)) == A.GLU_ERR_WORKSPACE
    q = A.GluParams()
    lib.glu_params_default(ctypes.byref(q))
    q.mode = A.GLU_MODE_EXACT
    assert lib.glu_pipeline_host(*args(p=q)) == A.GLU_ERR_UNSUPPORTED
    q.mode = A.GLU_MODE_FAST
    q.S = 4
    assert lib.glu_pipeline_host(*args(p=q)) == A.GLU_ERR_INVALID_ARG
    # the uint8 filter's own checks
    assert lib.glu_fx_filter3_u8(None, 8, 10, 3, 30, fake, 30, 0, None) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_fx_filter3_u8(fake, 8, 10, 3, 29, fake, 30, 0, None) == A.GLU_ERR_INVALID_ARG
    assert lib.glu_fx_filter3_u8(fake, 8, 10, 3, 30, fake, 30, 3, None) == A.GLU_ERR_INVALID_ARG


def test_generic_workspace_size_matches_per_op_queries(lib):
    from paper_2307_09582_gb300 import _abi as A
    p = A.GluParams()
    lib.glu_params_default(ctypes.byref(p))
    p.S, p.N = 5, 3
    H, W, s = 96, 136, 8
    fake = ctypes.c_void_p(0x1000)
    th = A.GluTheta(fake, fake, H, W, s, p.S, A.GLU_W_F32)
    ws = lambda op: lib.glu_workspace_size(op, H, W, s, ctypes.byref(p))
    assert ws(A.GLU_OP_JOINT) == lib.glu_joint_workspace_size(H, W, s, ctypes.byref(p)) > 0
    assert ws(A.GLU_OP_LS_JOINT) == lib.glu_ls_joint_workspace_size(H, W, s, ctypes.byref(p)) > 0
    assert ws(A.GLU_OP_LS_UPDATE) == lib.glu_ls_update_workspace_size(ctypes.byref(th)) > 0
    assert ws(A.GLU_OP_APPLY_BACKWARD) == \
        lib.glu_apply_backward_workspace_size(ctypes.byref(th), 3) > 0
    assert ws(A.GLU_OP_APPLY_BACKWARD_PLAN) == \
        lib.glu_apply_backward_plan_size(ctypes.byref(th)) > 0
    for op in (A.GLU_OP_DOWNSAMPLE, A.GLU_OP_OPTIMIZE, A.GLU_OP_APPLY, A.GLU_OP_THETA_DECODE, 99):
        assert ws(op) == 0
    assert lib.glu_workspace_size(A.GLU_OP_JOINT, 0, W, s, ctypes.byref(p)) == 0
    assert lib.glu_workspace_size(A.GLU_OP_JOINT, H, W, s, None) == 0


def test_theta_decode_validates_before_launch(lib):
    from paper_2307_09582_gb300 import _abi as A
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    th = A.GluTheta(fake, fake, 64, 80, 8, 4, A.GLU_W_F32)     # even S
    assert lib.glu_theta_decode(ctypes.byref(th), fake, fake, fake, None) == \
        A.GLU_ERR_INVALID_ARG
    th.S = 3
    assert lib.glu_theta_decode(ctypes.byref(th), None, None, None, None) == \
        A.GLU_ERR_INVALID_ARG
    assert lib.glu_theta_decode(None, fake, fake, fake, None) == A.GLU_ERR_INVALID_ARG

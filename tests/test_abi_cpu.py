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


def test_missing_library_fails_loudly(tmp_path):
    from paper_2307_09582_gb300 import _abi as A
    with pytest.raises(RuntimeError, match="not found"):
        A.load(str(tmp_path / "libglu.so"))

"""C ABI checks that need no GPU: the library builds, loads, exports every
function include/nasgabor.h declares, and rejects bad arguments on the host
before any CUDA call (host-side fault injection: NULL pointers, out-of-range
sizes and modes, misaligned pointers)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")
LIB = os.path.join(ROOT, "paper_2606_09794_gb300", "libnasgabor.so")

NASG_OK, NASG_ERR_NULL, NASG_ERR_RANGE, NASG_ERR_ALIGN = 0, -1, -2, -3


@pytest.fixture(scope="module")
def so():
    from paper_2606_09794_gb300 import build as b
    b.build()
    return ctypes.CDLL(LIB)


def _declared_functions():
    names = []
    for f in sorted(os.listdir(HEADER_DIR)):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = set(_declared_functions())
    for required in ("nasgabor_eval_fwd", "nasgabor_eval_bwd", "sh_eval_fwd", "sh_eval_bwd"):
        assert required in names


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in _declared_functions() if not hasattr(so, n)]
    assert not missing, missing


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_lobes", ctypes.c_int32), ("frame_mode", ctypes.c_int32),
                ("param_dtype", ctypes.c_int32), ("norm_mode", ctypes.c_int32), ("act_mode", ctypes.c_int32),
                ("accumulate", ctypes.c_int32), ("lobe_family", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _fwd(so):
    f = so.nasgabor_eval_fwd
    f.argtypes = [ctypes.POINTER(Desc)] + [ctypes.c_void_p] * 3 + [ctypes.POINTER(ctypes.c_float),
                                                                    ctypes.c_void_p, ctypes.c_int64,
                                                                    ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    return f


CAM = (ctypes.c_float * 3)(0.0, 0.0, 3.0)
P = ctypes.c_void_p(0x10000)      # fake, aligned, never dereferenced: validation fails first
MIS = ctypes.c_void_p(0x10002)    # misaligned for float


def test_host_validation_rejects_before_launch(so):
    fwd = _fwd(so)
    good = Desc(16, 4, 0, 0, 0, 0, 0)
    assert fwd(None, P, P, P, CAM, None, 0, P, None) == NASG_ERR_NULL
    assert fwd(ctypes.byref(good), None, P, P, CAM, None, 0, P, None) == NASG_ERR_NULL
    assert fwd(ctypes.byref(good), P, P, P, None, None, 0, P, None) == NASG_ERR_NULL
    for bad in (Desc(-1, 4, 0, 0, 0, 0, 0), Desc(16, 0, 0, 0, 0, 0, 0), Desc(16, 33, 0, 0, 0, 0, 0),
                Desc(16, 4, 2, 0, 0, 0, 0), Desc(16, 4, 0, 2, 0, 0, 0), Desc(16, 4, 0, 0, 7, 0, 0),
                Desc(16, 4, 0, 0, 0, 2, 0), Desc(16, 4, 0, 0, 0, 0, 3), Desc(16, 4, 0, 0, 0, 0, 0, 4),
                Desc(16, 4, 0, 0, 0, 0, 0, -1), Desc(16, 4, 0, 0, 0, 0, 0, 0, 1)):
        assert fwd(ctypes.byref(bad), P, P, P, CAM, None, 0, P, None) == NASG_ERR_RANGE
    assert fwd(ctypes.byref(good), MIS, P, P, CAM, None, 0, P, None) == NASG_ERR_ALIGN
    assert fwd(ctypes.byref(good), P, P, P, CAM, P, -1, P, None) == NASG_ERR_RANGE
    # empty problems are valid and launch nothing
    assert fwd(ctypes.byref(Desc(0, 4, 0, 0, 0, 0, 0)), P, P, P, CAM, None, 0, P, None) == NASG_OK
    assert fwd(ctypes.byref(good), P, P, P, CAM, P, 0, P, None) == NASG_OK


def test_sh_validation(so):
    f = so.sh_eval_fwd
    f.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_float), ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    assert f(4, 10, P, P, CAM, P, None) == NASG_ERR_RANGE
    assert f(-1, 10, P, P, CAM, P, None) == NASG_ERR_RANGE
    assert f(3, -1, P, P, CAM, P, None) == NASG_ERR_RANGE
    assert f(3, 10, None, P, CAM, P, None) == NASG_ERR_NULL
    assert f(3, 10, MIS, P, CAM, P, None) == NASG_ERR_ALIGN
    assert f(3, 0, P, P, CAM, P, None) == NASG_OK


def test_status_strings_and_planes(so):
    so.nasg_status_string.restype = ctypes.c_char_p
    for s in (0, -1, -2, -3, -4, -5, -6, -99):
        assert so.nasg_status_string(s)
    assert so.nasg_lobe_planes(0) == 10 and so.nasg_lobe_planes(1) == 9 and so.nasg_lobe_planes(5) == -1
    assert so.nasg_abi_version() >= 2
    assert [so.nasg_param_planes(0, f) for f in range(5)] == [10, 9, 8, 11, -1]
    assert [so.nasg_param_planes(1, f) for f in range(4)] == [9, -1, -1, -1]


def test_lobe_family_needs_quaternion_frames(so):
    fwd = _fwd(so)
    assert fwd(ctypes.byref(Desc(16, 4, 1, 0, 0, 0, 0, 2)), P, P, P, CAM, None, 0, P, None) == -4


def test_fused_step_loss_mode_validation(so):
    """nasgabor_fused_step takes the loss mode after the gradient/target pointer (ABI 4):
    an unknown mode is rejected before any launch; with every list empty the two valid
    modes return NASG_OK without touching the device."""
    class Adam(ctypes.Structure):
        _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                    ("eps", ctypes.c_float), ("step", ctypes.c_int32)]

    f = so.nasgabor_fused_step
    f.argtypes = [ctypes.POINTER(Desc), ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                  ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                  ctypes.POINTER(Adam), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int32
    state = (ctypes.c_void_p * 8)(*([0x10000] * 8))
    hp = Adam(1e-3, 0.9, 0.999, 1e-8, 1)
    good = Desc(16, 8, 0, 1, 0, 0, 0)
    assert so.nasg_abi_version() == 4
    for mode in (-1, 2, 7):
        assert f(ctypes.byref(good), state, P, CAM, None, 0, None, P, mode, ctypes.byref(hp), None, None,
                 None) == NASG_ERR_RANGE
    for mode in (0, 1):
        assert f(ctypes.byref(good), state, P, CAM, P, 0, None, P, mode, ctypes.byref(hp), None, None,
                 None) == NASG_OK
        assert f(ctypes.byref(Desc(0, 8, 0, 1, 0, 0, 0)), state, P, CAM, None, 0, None, P, mode,
                 ctypes.byref(hp), None, None, None) == NASG_OK

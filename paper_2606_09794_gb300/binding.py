"""Thin Python binding of libnasgabor.so (C ABI in include/nasgabor.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels. torch supplies device memory and the current CUDA
stream; tensors are passed to the C ABI as raw pointers. Importing this module
loads the library and raises ImportError if it has not been built (there is no
fallback path).

Function names mirror the C entry points. Outputs are allocated here with
torch when the caller does not pass them.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnasgabor.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_2606_09794_gb300.build` "
                      "(or __graft_entry__.build()) first")
lib = ctypes.CDLL(LIB_PATH)

FRAME = {"quat": 0, "cos": 1}
NORM = {"approx": 0, "none": 1, "exact": 2}
FAMILY = {"nasgabor": 0, "nasg": 1, "sg": 2, "phase": 3}
LOSS = {"given": 0, "mse": 1}
ACT = {"raw": 0, "identity": 1}
PLANES = {"quat": 10, "cos": 9}

_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


class NasgDesc(ctypes.Structure):
    _fields_ = [("n", _i64), ("n_lobes", _i32), ("frame_mode", _i32), ("param_dtype", _i32),
                ("norm_mode", _i32), ("act_mode", _i32), ("accumulate", _i32), ("lobe_family", _i32),
                ("reserved", _i32)]


class NasgAdam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", _i32)]


class NasgTrainState(ctypes.Structure):
    _fields_ = [("master", _vp), ("m", _vp), ("v", _vp), ("params_bf16", _vp),
                ("c0_master", _vp), ("c0_m", _vp), ("c0_v", _vp), ("c0_bf16", _vp)]


class NasgScene(ctypes.Structure):
    _fields_ = [("n", _i64), ("n_lobes", _i32), ("reserved0", _i32), ("params", _vp), ("c0", _vp), ("means", _vp),
                ("cam", ctypes.c_float * 3), ("reserved1", ctypes.c_float), ("g_rgb", _vp), ("rgb", _vp),
                ("g_params", _vp), ("g_c0", _vp), ("g_means", _vp)]


class NasgBatchModes(ctypes.Structure):
    _fields_ = [("frame_mode", _i32), ("param_dtype", _i32), ("norm_mode", _i32), ("act_mode", _i32)]


class NasgBatchPlan(ctypes.Structure):
    _fields_ = [("n_scenes", _i32), ("frame_mode", _i32), ("param_dtype", _i32), ("norm_mode", _i32),
                ("act_mode", _i32), ("sub_tiles", _i32), ("pair_path", _i32), ("reserved", _i32),
                ("total_tiles", _i64), ("total_prims", _i64),
                ("total_lobes", _i64), ("workspace", _vp)]


class NasgBatchTuning(ctypes.Structure):
    _fields_ = [("dynamic", _i32), ("blocks_per_sm", _i32), ("sub_tiles", _i32), ("staged", _i32)]


def _decl(name, argtypes, restype=_i32):
    fn = getattr(lib, name)
    fn.argtypes = argtypes
    fn.restype = restype
    return fn


_P = ctypes.POINTER
_decl("nasg_lobe_planes", [_i32])
_decl("nasg_param_planes", [_i32, _i32])
_decl("nasg_status_string", [_i32], ctypes.c_char_p)
_decl("nasg_last_cuda_error", [])
_decl("nasg_abi_version", [])
_decl("nasg_device_status", [_vp])
_decl("nasg_probe_wait_timeout", [_i32, _vp])
_decl("nasgabor_eval_fwd", [_P(NasgDesc), _vp, _vp, _vp, _P(ctypes.c_float), _vp, _i64, _vp, _vp])
_decl("nasgabor_eval_bwd", [_P(NasgDesc), _vp, _vp, _P(ctypes.c_float), _vp, _i64, _vp, _vp, _vp, _vp, _vp])
_decl("nasgabor_fused_fwd_bwd", [_P(NasgDesc), _vp, _vp, _vp, _P(ctypes.c_float), _vp, _vp, _vp, _vp, _vp, _vp])
_decl("sh_eval_fwd", [_i32, _i64, _vp, _vp, _P(ctypes.c_float), _vp, _vp])
_decl("sh_eval_bwd", [_i32, _i64, _vp, _vp, _P(ctypes.c_float), _vp, _vp, _vp, _vp])
_decl("nasg_math_probe", [_i32, _vp, _vp, _vp, _i64, _vp])
_decl("nasgabor_fused_step", [_P(NasgDesc), _P(NasgTrainState), _vp, _P(ctypes.c_float), _vp, _i64, _vp, _vp, _i32,
                              _P(NasgAdam), _vp, _vp, _vp])
_decl("nasg_frustum_workspace_bytes", [_i64], ctypes.c_size_t)
_decl("nasgabor_batched_workspace_bytes", [_i32], ctypes.c_size_t)
_decl("nasgabor_fit_workspace_bytes", [], ctypes.c_size_t)
_decl("nasgabor_fit_step", [_P(NasgDesc), _P(NasgTrainState), _vp, _vp, _i32, _vp, _i32, _P(NasgAdam), _vp, _vp,
                            ctypes.c_size_t, _vp])
_decl("nasgabor_batched_prepare", [_P(NasgScene), _i32, _P(NasgBatchModes), _i32, _vp, ctypes.c_size_t,
                                   _P(NasgBatchPlan), _vp])
_decl("nasgabor_batched_run", [_P(NasgBatchPlan), _P(NasgBatchTuning), _vp])
_decl("nasgabor_batched_autotune", [_P(NasgScene), _i32, _P(NasgBatchModes), _vp, ctypes.c_size_t, _i32,
                                    _P(NasgBatchPlan), _P(NasgBatchTuning), _P(ctypes.c_float), _vp])
_decl("nasg_frustum_compact_noalloc", [_i64, _vp, _P(ctypes.c_float), _P(ctypes.c_float), ctypes.c_float,
                                       ctypes.c_float, _vp, _vp, _vp])
_decl("nasg_lr_heuristic", [_vp, _i32, _i32, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                           ctypes.c_double, _P(ctypes.c_double), _P(ctypes.c_double), _P(ctypes.c_double)])
_decl("nasg_cosine_lr_factor", [_i64, _i64, _i64], ctypes.c_double)
_decl("nasg_train_state_refresh_bf16", [_P(NasgDesc), _P(NasgTrainState), _vp])
_decl("nasg_pipe_probe", [_i32, _i64, _i32, _vp, _P(_i64), _vp])
_decl("nasg_frustum_compact", [_i64, _vp, _P(ctypes.c_float), _P(ctypes.c_float), ctypes.c_float, ctypes.c_float,
                               _vp, _vp, _vp, ctypes.c_size_t, _vp])


class NasgRasterCamera(ctypes.Structure):
    _fields_ = [("rot", ctypes.c_float * 9), ("centre", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("near_z", ctypes.c_float),
                ("width", _i32), ("height", _i32)]


_decl("nasgabor_fused_host_workspace_bytes", [_P(NasgDesc), _i64], ctypes.c_size_t)
_decl("nasgabor_fused_fwd_bwd_host", [_P(NasgDesc), _vp, _vp, _vp, _P(ctypes.c_float), _vp, _vp, _vp, _vp, _vp,
                                      _i64, _vp, ctypes.c_size_t, _vp])
_decl("nasg_raster_workspace_bytes", [_i64, _i32, _i32, _i64], ctypes.c_size_t)
_decl("nasg_raster_forward", [_i64, _vp, _vp, _vp, _vp, _vp, _P(NasgRasterCamera), _vp, _vp, _i64, _vp,
                              ctypes.c_size_t, _P(_i64), _vp])
_decl("nasg_raster_backward", [_i64, _vp, _P(NasgRasterCamera), _vp, _vp, _vp, _vp, _i64, _vp, ctypes.c_size_t,
                               _vp])


class NasgError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib.nasg_status_string(status).decode()
        extra = ""
        if status == -5:
            extra = f" (cudaError {lib.nasg_last_cuda_error()})"
        super().__init__(f"{where}: status {status}: {msg}{extra}")
        self.status = status


def _check(status: int, where: str):
    if status != 0:
        raise NasgError(status, where)


def _ptr(t):
    return None if t is None else _vp(t.data_ptr())


def _stream(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return _vp(s.cuda_stream)


def _cam(cam):
    if isinstance(cam, torch.Tensor):
        cam = cam.detach().to("cpu", torch.float32).reshape(-1).tolist()
    vals = [float(c) for c in cam]
    if len(vals) != 3:
        raise ValueError("cam must have 3 components")
    return (ctypes.c_float * 3)(*vals)


def _cuda(t, name, dtype=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _param_dtype(t):
    if t.dtype == torch.float32:
        return 0
    if t.dtype == torch.bfloat16:
        return 1
    raise TypeError("params must be float32 or bfloat16")


def make_desc(n, n_lobes, frame_mode="quat", param_dtype=torch.float32, norm_mode="approx", act_mode="raw",
              accumulate=False, family="nasgabor") -> NasgDesc:
    return NasgDesc(int(n), int(n_lobes), FRAME[frame_mode], 1 if param_dtype == torch.bfloat16 else 0,
                    NORM[norm_mode], ACT[act_mode], 1 if accumulate else 0, FAMILY[family], 0)


def param_planes(frame_mode="quat", family="nasgabor"):
    """Stored scalars per lobe for a frame mode and lobe family."""
    p = lib.nasg_param_planes(FRAME[frame_mode], FAMILY[family])
    if p < 0:
        raise ValueError(f"unsupported frame/family {frame_mode}/{family}")
    return p


def _check_planes(params, n, n_lobes, frame_mode, family):
    p = param_planes(frame_mode, family)
    if params.dim() != 2 or params.shape[0] != p or params.shape[1] != n * n_lobes:
        raise ValueError(f"params must be [{p}, {n * n_lobes}] for {frame_mode}/{family}, got {tuple(params.shape)}")


def nasg_device_status(stream=None):
    """Synchronise the stream and raise NasgError if a kernel's bounded wait gave up."""
    _check(lib.nasg_device_status(_stream(stream)), "nasg_device_status")


def nasg_lr_heuristic(centres, d_ref, eta_f_base, eta_sigma_base, k=3, beta=2.0, gamma=0.6):
    """(eta_f, eta_sigma, d_knn) of the camera-spacing learning-rate heuristic; centres: host [n][3]."""
    import numpy as np
    c = np.ascontiguousarray(np.asarray(centres, dtype=np.float32).reshape(-1, 3))
    ef, es, dk = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib.nasg_lr_heuristic(_vp(c.ctypes.data), int(c.shape[0]), int(k), float(d_ref), float(eta_f_base),
                                 float(eta_sigma_base), float(beta), float(gamma), ctypes.byref(ef),
                                 ctypes.byref(es), ctypes.byref(dk)), "nasg_lr_heuristic")
    return ef.value, es.value, dk.value


def nasg_cosine_lr_factor(t, t_max, t_start=0):
    """Cosine learning-rate multiplier at iteration t (1 before t_start)."""
    return lib.nasg_cosine_lr_factor(int(t), int(t_start), int(t_max))


def nasg_probe_wait_timeout(limit=1024, stream=None):
    """Diagnostic: run a bounded wait that cannot complete (sets the device error word)."""
    _check(lib.nasg_probe_wait_timeout(int(limit), _stream(stream)), "nasg_probe_wait_timeout")


def lobe_planes(frame_mode="quat") -> int:
    return int(lib.nasg_lobe_planes(FRAME[frame_mode]))


def nasgabor_eval_fwd(params, c0, means, cam, n_lobes, frame_mode="quat", norm_mode="approx",
                      act_mode="raw", idx=None, rgb=None, stream=None, family="nasgabor"):
    """rgb [N, 3] = c0 + sum_l w_l G_l(d) at d = normalize(means - cam); see include/nasgabor.h."""
    _cuda(params, "params")
    _cuda(c0, "c0", params.dtype)
    _cuda(means, "means", torch.float32)
    n = means.shape[0]
    if rgb is None:
        rgb = torch.empty((n, 3), device=means.device, dtype=torch.float32)
    _cuda(rgb, "rgb", torch.float32)
    if idx is not None:
        _cuda(idx, "idx", torch.int32)
    _check_planes(params, n, n_lobes, frame_mode, family)
    desc = make_desc(n, n_lobes, frame_mode, params.dtype, norm_mode, act_mode, family=family)
    _param_dtype(params)
    _check(lib.nasgabor_eval_fwd(ctypes.byref(desc), _ptr(params), _ptr(c0), _ptr(means), _cam(cam),
                                 _ptr(idx), 0 if idx is None else idx.numel(), _ptr(rgb), _stream(stream)),
           "nasgabor_eval_fwd")
    return rgb


def nasgabor_eval_bwd(params, means, cam, g_rgb, n_lobes, frame_mode="quat", norm_mode="approx",
                      act_mode="raw", idx=None, g_params=None, g_c0=None, g_means=None, want_means=True,
                      accumulate=False, stream=None, family="nasgabor"):
    """(g_params [P, N*L] f32, g_c0 [3, N] f32, g_means [N, 3] f32 or None); see include/nasgabor.h."""
    _cuda(params, "params")
    _cuda(means, "means", torch.float32)
    _cuda(g_rgb, "g_rgb", torch.float32)
    n = means.shape[0]
    dev = means.device
    if g_params is None:
        g_params = torch.empty(params.shape, device=dev, dtype=torch.float32)
    if g_c0 is None:
        g_c0 = torch.empty((3, n), device=dev, dtype=torch.float32)
    if g_means is None and want_means:
        g_means = torch.empty((n, 3), device=dev, dtype=torch.float32)
    for t, nm in ((g_params, "g_params"), (g_c0, "g_c0")):
        _cuda(t, nm, torch.float32)
    if g_means is not None:
        _cuda(g_means, "g_means", torch.float32)
    if idx is not None:
        _cuda(idx, "idx", torch.int32)
    _check_planes(params, n, n_lobes, frame_mode, family)
    desc = make_desc(n, n_lobes, frame_mode, params.dtype, norm_mode, act_mode, accumulate, family)
    _param_dtype(params)
    _check(lib.nasgabor_eval_bwd(ctypes.byref(desc), _ptr(params), _ptr(means), _cam(cam), _ptr(idx),
                                 0 if idx is None else idx.numel(), _ptr(g_rgb), _ptr(g_params), _ptr(g_c0),
                                 _ptr(g_means), _stream(stream)), "nasgabor_eval_bwd")
    return g_params, g_c0, g_means


def nasgabor_fused_fwd_bwd(params, c0, means, cam, g_rgb, n_lobes, frame_mode="quat", norm_mode="approx",
                           act_mode="raw", out=None, want_means=True, stream=None, family="nasgabor"):
    """One pass: (rgb, g_params, g_c0, g_means) for a given upstream gradient g_rgb."""
    _cuda(params, "params")
    _cuda(c0, "c0", params.dtype)
    _cuda(means, "means", torch.float32)
    _cuda(g_rgb, "g_rgb", torch.float32)
    n = means.shape[0]
    dev = means.device
    if out is None:
        out = (torch.empty((n, 3), device=dev, dtype=torch.float32),
               torch.empty(params.shape, device=dev, dtype=torch.float32),
               torch.empty((3, n), device=dev, dtype=torch.float32),
               torch.empty((n, 3), device=dev, dtype=torch.float32) if want_means else None)
    rgb, g_params, g_c0, g_means = out
    _check_planes(params, n, n_lobes, frame_mode, family)
    desc = make_desc(n, n_lobes, frame_mode, params.dtype, norm_mode, act_mode, family=family)
    _param_dtype(params)
    _check(lib.nasgabor_fused_fwd_bwd(ctypes.byref(desc), _ptr(params), _ptr(c0), _ptr(means), _cam(cam),
                                      _ptr(g_rgb), _ptr(rgb), _ptr(g_params), _ptr(g_c0), _ptr(g_means),
                                      _stream(stream)), "nasgabor_fused_fwd_bwd")
    return rgb, g_params, g_c0, g_means


def sh_eval_fwd(coeffs, means, cam, degree=3, rgb=None, stream=None):
    _cuda(coeffs, "coeffs", torch.float32)
    _cuda(means, "means", torch.float32)
    n = means.shape[0]
    if rgb is None:
        rgb = torch.empty((n, 3), device=means.device, dtype=torch.float32)
    _check(lib.sh_eval_fwd(degree, n, _ptr(coeffs), _ptr(means), _cam(cam), _ptr(rgb), _stream(stream)),
           "sh_eval_fwd")
    return rgb


def sh_eval_bwd(coeffs, means, cam, g_rgb, degree=3, g_coeffs=None, g_means=None, want_means=True,
                stream=None):
    _cuda(coeffs, "coeffs", torch.float32)
    _cuda(means, "means", torch.float32)
    _cuda(g_rgb, "g_rgb", torch.float32)
    n = means.shape[0]
    if g_coeffs is None:
        g_coeffs = torch.empty_like(coeffs)
    if g_means is None and want_means:
        g_means = torch.empty((n, 3), device=means.device, dtype=torch.float32)
    _check(lib.sh_eval_bwd(degree, n, _ptr(coeffs), _ptr(means), _cam(cam), _ptr(g_rgb), _ptr(g_coeffs),
                           _ptr(g_means), _stream(stream)), "sh_eval_bwd")
    return g_coeffs, g_means


def nasg_pipe_rate(pipe, iters=1 << 14, blocks_per_sm=4, reps=3, stream=None):
    """Diagnostic: measured issue rate (lane operations per second) of one pipe
    (0 MUFU ex2, 1 packed FP32x2 FMA, 2 scalar FMA); best of `reps` timed launches."""
    s = torch.cuda.current_stream() if stream is None else stream
    out = torch.empty(4096, device="cuda", dtype=torch.float32)
    ops = _i64(0)
    best = None
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _check(lib.nasg_pipe_probe(int(pipe), int(iters), int(blocks_per_sm), _ptr(out), ctypes.byref(ops),
                                   _vp(s.cuda_stream)), "nasg_pipe_probe")
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return ops.value / (best * 1e-3)


def nasg_math_probe(fn, x, stream=None):
    """Diagnostic: the library's FP32 elementary function `fn` (0 expm1, 1 tanh, 2 sincos, 3 tanh
    by the BF16 weight table) at x."""
    _cuda(x, "x", torch.float32)
    y = torch.empty_like(x)
    y2 = torch.empty_like(x) if fn > 0 else None
    _check(lib.nasg_math_probe(fn, _ptr(x), _ptr(y), _ptr(y2), x.numel(), _stream(stream)), "nasg_math_probe")
    return y, y2


class TrainState:
    """FP32 master, Adam moments and BF16 copies of one parameter set (device tensors).
    The BF16 copies are written by the library (nasg_train_state_refresh_bf16)."""

    # stored scalars per lobe -> a (frame, family) layout with that many planes
    _LAYOUT_OF_PLANES = {10: ("quat", "nasgabor"), 9: ("cos", "nasgabor"), 8: ("quat", "sg"), 11: ("quat", "phase")}

    def __init__(self, master, c0_master, m=None, v=None, c0_m=None, c0_v=None, bf16_copies=True,
                 frame_mode=None, family=None, stream=None):
        self.master = _cuda(master, "master", torch.float32)
        self.c0_master = _cuda(c0_master, "c0_master", torch.float32)
        self.m = torch.zeros_like(master) if m is None else _cuda(m, "m", torch.float32)
        self.v = torch.zeros_like(master) if v is None else _cuda(v, "v", torch.float32)
        self.c0_m = torch.zeros_like(c0_master) if c0_m is None else _cuda(c0_m, "c0_m", torch.float32)
        self.c0_v = torch.zeros_like(c0_master) if c0_v is None else _cuda(c0_v, "c0_v", torch.float32)
        self.params_bf16 = torch.empty(master.shape, dtype=torch.bfloat16, device=master.device) if bf16_copies else None
        self.c0_bf16 = torch.empty(c0_master.shape, dtype=torch.bfloat16, device=master.device) if bf16_copies else None
        n = c0_master.shape[1]
        if frame_mode is None or family is None:
            if master.dim() != 2 or master.shape[0] not in self._LAYOUT_OF_PLANES:
                raise ValueError(f"master must be [P, N*L] with P in {sorted(self._LAYOUT_OF_PLANES)}")
            f0, fam0 = self._LAYOUT_OF_PLANES[master.shape[0]]
            frame_mode, family = frame_mode or f0, family or fam0
        planes = param_planes(frame_mode, family)
        if master.dim() != 2 or master.shape[0] != planes or (n and master.shape[1] % n):
            raise ValueError(f"master must be [{planes}, N*L] with c0_master [3, N]")
        self.n_lobes = master.shape[1] // n if n else 1
        self.frame_mode, self.family = frame_mode, family
        if bf16_copies:
            self.refresh_bf16(stream)

    def refresh_bf16(self, stream=None):
        """BF16 copies = RNE(FP32 masters), written by the library."""
        desc = make_desc(self.c0_master.shape[1], max(self.n_lobes, 1), self.frame_mode, torch.bfloat16,
                         family=self.family)
        st = self.as_c()
        _check(lib.nasg_train_state_refresh_bf16(ctypes.byref(desc), ctypes.byref(st), _stream(stream)),
               "nasg_train_state_refresh_bf16")

    def as_c(self):
        return NasgTrainState(_ptr(self.master), _ptr(self.m), _ptr(self.v), _ptr(self.params_bf16),
                              _ptr(self.c0_master), _ptr(self.c0_m), _ptr(self.c0_v), _ptr(self.c0_bf16))


def nasgabor_fused_step(state, means, cam, g_rgb, n_lobes, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                        idx=None, n_idx_device=None, frame_mode="quat", norm_mode="approx", act_mode="raw",
                        evaluate_bf16=True, rgb=None, g_means=None, stream=None, family="nasgabor", loss="given"):
    """Forward + backward + Adam for the listed primitives; state (TrainState) updated in place.
    loss="given": g_rgb is dLoss/dRGB; loss="mse": g_rgb is the target colour [N, 3] and the
    kernel forms dLoss/dc = 2 (c - target) / (3 n_listed) (mean squared error)."""
    _cuda(means, "means", torch.float32)
    _cuda(g_rgb, "g_rgb", torch.float32)
    n = means.shape[0]
    if idx is not None:
        _cuda(idx, "idx", torch.int32)
    if n_idx_device is not None:
        _cuda(n_idx_device, "n_idx_device", torch.int32)
    for t, nm in ((rgb, "rgb"), (g_means, "g_means")):
        if t is not None:
            _cuda(t, nm, torch.float32)
    desc = make_desc(n, n_lobes, frame_mode, torch.bfloat16 if evaluate_bf16 else torch.float32,
                     norm_mode, act_mode, family=family)
    hp = NasgAdam(lr, beta1, beta2, eps, int(step))
    st = state.as_c()
    _check(lib.nasgabor_fused_step(ctypes.byref(desc), ctypes.byref(st), _ptr(means), _cam(cam), _ptr(idx),
                                   0 if idx is None else idx.numel(), _ptr(n_idx_device), _ptr(g_rgb), LOSS[loss],
                                   ctypes.byref(hp), _ptr(rgb), _ptr(g_means), _stream(stream)),
           "nasgabor_fused_step")
    return rgb


def nasg_frustum_workspace_bytes(n):
    return int(lib.nasg_frustum_workspace_bytes(int(n)))


def nasg_frustum_compact(means, rot, center, tan_half_fov, near=0.0, idx=None, n_visible=None, workspace=None,
                         stream=None):
    """Ordered indices of the primitives inside the frustum; returns (idx [N] int32, n_visible [1] int32)."""
    _cuda(means, "means", torch.float32)
    n = means.shape[0]
    dev = means.device
    if idx is None:
        idx = torch.empty(max(n, 1), device=dev, dtype=torch.int32)
    if n_visible is None:
        n_visible = torch.empty(1, device=dev, dtype=torch.int32)
    wsb = nasg_frustum_workspace_bytes(n)
    if workspace is None:
        workspace = torch.empty(max(wsb, 16), device=dev, dtype=torch.uint8)
    r = (ctypes.c_float * 9)(*[float(x) for x in torch.as_tensor(rot, dtype=torch.float32).reshape(-1).tolist()])
    c = _cam(center)
    _check(lib.nasg_frustum_compact(n, _ptr(means), r, c, float(tan_half_fov), float(near), _ptr(idx),
                                    _ptr(n_visible), _ptr(workspace), workspace.numel(), _stream(stream)),
           "nasg_frustum_compact")
    return idx, n_visible


class Batch:
    """Many scenes evaluated (forward + backward for a given upstream gradient) in one
    persistent launch. `scenes` is a list of dicts with device tensors params, c0, means,
    g_rgb and the camera `cam`; outputs rgb, g_params, g_c0, g_means are allocated here."""

    def __init__(self, scenes, frame_mode="quat", norm_mode="approx", act_mode="raw", sub_tiles=2,
                 want_means=True, stream=None):
        if not scenes:
            raise ValueError("empty batch")
        dtype = scenes[0]["params"].dtype
        self.modes = NasgBatchModes(FRAME[frame_mode], _param_dtype(scenes[0]["params"]), NORM[norm_mode],
                                    ACT[act_mode])
        self.scenes = scenes
        arr = (NasgScene * len(scenes))()
        for j, sc in enumerate(scenes):
            p, c0, mu, g = sc["params"], sc["c0"], sc["means"], sc["g_rgb"]
            for t, nm in ((p, "params"), (c0, "c0")):
                _cuda(t, nm, dtype)
            _cuda(mu, "means", torch.float32)
            _cuda(g, "g_rgb", torch.float32)
            n = mu.shape[0]
            dev = mu.device
            sc["rgb"] = torch.empty((n, 3), device=dev)
            sc["g_params"] = torch.empty(p.shape, device=dev, dtype=torch.float32)
            sc["g_c0"] = torch.empty((3, n), device=dev)
            sc["g_means"] = torch.empty((n, 3), device=dev) if want_means else None
            cam = [float(c) for c in sc["cam"]]
            arr[j] = NasgScene(n, int(sc["n_lobes"]), 0, _ptr(p), _ptr(c0), _ptr(mu), (ctypes.c_float * 3)(*cam), 0.0,
                               _ptr(g), _ptr(sc["rgb"]), _ptr(sc["g_params"]), _ptr(sc["g_c0"]),
                               _ptr(sc["g_means"]))
        self.arr = arr
        nbytes = int(lib.nasgabor_batched_workspace_bytes(len(scenes)))
        if nbytes == 0:
            raise ValueError("too many scenes")
        self.workspace = torch.empty(nbytes, device=scenes[0]["means"].device, dtype=torch.uint8)
        self.plan = NasgBatchPlan()
        self.tuning = NasgBatchTuning(1, 0, sub_tiles, 0)
        _check(lib.nasgabor_batched_prepare(arr, len(scenes), ctypes.byref(self.modes), int(sub_tiles),
                                            _ptr(self.workspace), nbytes, ctypes.byref(self.plan), _stream(stream)),
               "nasgabor_batched_prepare")

    @property
    def total_lobes(self):
        return int(self.plan.total_lobes)

    def run(self, stream=None):
        _check(lib.nasgabor_batched_run(ctypes.byref(self.plan), ctypes.byref(self.tuning), _stream(stream)),
               "nasgabor_batched_run")

    def autotune(self, reps=5, stream=None):
        best = NasgBatchTuning()
        ms = ctypes.c_float(0.0)
        _check(lib.nasgabor_batched_autotune(self.arr, len(self.scenes), ctypes.byref(self.modes),
                                             _ptr(self.workspace), self.workspace.numel(), int(reps),
                                             ctypes.byref(self.plan), ctypes.byref(best), ctypes.byref(ms),
                                             _stream(stream)), "nasgabor_batched_autotune")
        self.tuning = best
        return {"dynamic": best.dynamic, "blocks_per_sm": best.blocks_per_sm, "sub_tiles": best.sub_tiles,
                "staged": best.staged, "ms": ms.value}


def nasgabor_fit_step(state, teacher_params, teacher_c0, teacher_lobes, dirs, n_lobes, step, lr=1e-3, beta1=0.9,
                      beta2=0.999, eps=1e-8, evaluate_bf16=True, loss=None, workspace=None, norm_mode="approx",
                      act_mode="raw", stream=None):
    """One fitting step of the student (TrainState) to the teacher field at the directions
    dirs [D][3]; returns the device scalar loss (mean squared colour error)."""
    _cuda(teacher_params, "teacher_params", torch.float32)
    _cuda(teacher_c0, "teacher_c0", torch.float32)
    _cuda(dirs, "dirs", torch.float32)
    n = state.c0_master.shape[1]
    dev = dirs.device
    if loss is None:
        loss = torch.empty(1, device=dev, dtype=torch.float32)
    if workspace is None:
        workspace = torch.empty(int(lib.nasgabor_fit_workspace_bytes()), device=dev, dtype=torch.uint8)
    desc = make_desc(n, n_lobes, "quat", torch.bfloat16 if evaluate_bf16 else torch.float32, norm_mode, act_mode)
    hp = NasgAdam(lr, beta1, beta2, eps, int(step))
    st = state.as_c()
    _check(lib.nasgabor_fit_step(ctypes.byref(desc), ctypes.byref(st), _ptr(teacher_params), _ptr(teacher_c0),
                                 int(teacher_lobes), _ptr(dirs), dirs.shape[0], ctypes.byref(hp), _ptr(loss),
                                 _ptr(workspace), workspace.numel(), _stream(stream)), "nasgabor_fit_step")
    return loss


NOALLOC_MAX_PRIMS = 1 << 23


def nasg_frustum_compact_noalloc(means, rot, center, tan_half_fov, near=0.0, idx=None, n_visible=None,
                                 stream=None):
    """nasg_frustum_compact with the library's fixed scratch (no workspace): for callers that
    cannot allocate device memory where they need the list. At most NOALLOC_MAX_PRIMS
    primitives; calls that may overlap on the GPU race on the shared scratch."""
    _cuda(means, "means", torch.float32)
    n = means.shape[0]
    dev = means.device
    if idx is None:
        idx = torch.empty(max(n, 1), device=dev, dtype=torch.int32)
    if n_visible is None:
        n_visible = torch.empty(1, device=dev, dtype=torch.int32)
    r = (ctypes.c_float * 9)(*[float(x) for x in torch.as_tensor(rot, dtype=torch.float32).reshape(-1).tolist()])
    _check(lib.nasg_frustum_compact_noalloc(n, _ptr(means), r, _cam(center), float(tan_half_fov), float(near),
                                            _ptr(idx), _ptr(n_visible), _stream(stream)),
           "nasg_frustum_compact_noalloc")
    return idx, n_visible


# ---------------------------------------------------------------------------
# autograd: the backward recomputes from the saved inputs (nothing else saved)
# ---------------------------------------------------------------------------

class NasgEval(torch.autograd.Function):
    """rgb = NasgEval.apply(params, c0, means, cam, n_lobes, frame_mode, norm_mode, act_mode)."""

    @staticmethod
    def forward(ctx, params, c0, means, cam, n_lobes, frame_mode="quat", norm_mode="approx", act_mode="raw"):
        cam_t = tuple(float(c) for c in (cam.tolist() if isinstance(cam, torch.Tensor) else cam))
        ctx.save_for_backward(params, means)
        ctx.cfg = (cam_t, n_lobes, frame_mode, norm_mode, act_mode)
        return nasgabor_eval_fwd(params, c0, means, cam_t, n_lobes, frame_mode, norm_mode, act_mode)

    @staticmethod
    def backward(ctx, g_rgb):
        params, means = ctx.saved_tensors
        cam_t, n_lobes, frame_mode, norm_mode, act_mode = ctx.cfg
        g_params, g_c0, g_means = nasgabor_eval_bwd(params, means, cam_t, g_rgb.contiguous(), n_lobes,
                                                    frame_mode, norm_mode, act_mode,
                                                    want_means=ctx.needs_input_grad[2])
        return (g_params.to(params.dtype), g_c0.to(params.dtype), g_means, None, None, None, None, None)


class ShEval(torch.autograd.Function):
    """rgb = ShEval.apply(coeffs, means, cam, degree)."""

    @staticmethod
    def forward(ctx, coeffs, means, cam, degree=3):
        cam_t = tuple(float(c) for c in (cam.tolist() if isinstance(cam, torch.Tensor) else cam))
        ctx.save_for_backward(coeffs, means)
        ctx.cfg = (cam_t, degree)
        return sh_eval_fwd(coeffs, means, cam_t, degree)

    @staticmethod
    def backward(ctx, g_rgb):
        coeffs, means = ctx.saved_tensors
        cam_t, degree = ctx.cfg
        g_coeffs, g_means = sh_eval_bwd(coeffs, means, cam_t, g_rgb.contiguous(), degree,
                                        want_means=ctx.needs_input_grad[1])
        return g_coeffs, g_means, None, None


def raster_camera(rot, centre, width, height, fx, fy=None, cx=None, cy=None, near_z=0.2):
    """Pinhole camera for the compositing calls (rot: world->camera rows right, up, forward)."""
    import numpy as np
    r = np.asarray(rot, dtype=np.float32).reshape(9)
    c = np.asarray(centre, dtype=np.float32).reshape(3)
    return NasgRasterCamera((ctypes.c_float * 9)(*r.tolist()), (ctypes.c_float * 3)(*c.tolist()), float(fx),
                            float(fx if fy is None else fy), float(0.5 * width if cx is None else cx),
                            float(0.5 * height if cy is None else cy), float(near_z), int(width), int(height))


class Raster:
    """Front-to-back compositing of primitives (see include/nasgabor.h) with a
    workspace sized for `max_pairs` (tile, primitive) pairs; forward keeps the
    state that backward reuses."""

    def __init__(self, n, camera, max_pairs, device=None):
        self.n = int(n)
        self.camera = camera
        self.max_pairs = int(max_pairs)
        nbytes = lib.nasg_raster_workspace_bytes(self.n, camera.width, camera.height, self.max_pairs)
        if nbytes == 0:
            raise ValueError("raster workspace: arguments out of range")
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=device or "cuda")
        self.n_pairs = None

    def forward(self, means, scales, quats, opacity, colours, image=None, final_t=None, stream=None):
        h, w = self.camera.height, self.camera.width
        dev = means.device
        for t, nm in ((means, "means"), (scales, "scales"), (quats, "quats"), (opacity, "opacity"),
                      (colours, "colours")):
            _cuda(t, nm, torch.float32)
        if image is None:
            image = torch.empty((h, w, 3), device=dev, dtype=torch.float32)
        if final_t is None:
            final_t = torch.empty((h, w), device=dev, dtype=torch.float32)
        pairs = _i64(0)
        _check(lib.nasg_raster_forward(self.n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(opacity), _ptr(colours),
                                       ctypes.byref(self.camera), _ptr(image), _ptr(final_t), self.max_pairs,
                                       _ptr(self.workspace), self.workspace.numel(), ctypes.byref(pairs),
                                       _stream(stream)), "nasg_raster_forward")
        self.n_pairs = pairs.value
        return image, final_t

    def backward(self, colours, final_t, g_image, g_colours=None, g_opacity=None, stream=None):
        dev = colours.device
        _cuda(g_image, "g_image", torch.float32)
        if g_colours is None:
            g_colours = torch.empty((self.n, 3), device=dev, dtype=torch.float32)
        if g_opacity is None:
            g_opacity = torch.empty((self.n,), device=dev, dtype=torch.float32)
        _check(lib.nasg_raster_backward(self.n, _ptr(colours), ctypes.byref(self.camera), _ptr(final_t),
                                        _ptr(g_image), _ptr(g_colours), _ptr(g_opacity), self.max_pairs,
                                        _ptr(self.workspace), self.workspace.numel(), _stream(stream)),
               "nasg_raster_backward")
        return g_colours, g_opacity


def _host(t, name, dtype=None):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class HostFused:
    """Fused forward+backward over HOST tensors (pinned for asynchronous copies),
    streamed through a device workspace in chunks; see nasgabor_fused_fwd_bwd_host."""

    def __init__(self, n, n_lobes, param_dtype=torch.bfloat16, chunk=131072, frame_mode="quat", norm_mode="approx",
                 act_mode="raw", family="nasgabor", device=None):
        self.desc = make_desc(n, n_lobes, frame_mode, param_dtype, norm_mode, act_mode, family=family)
        self.chunk = int(chunk)
        nbytes = lib.nasgabor_fused_host_workspace_bytes(ctypes.byref(self.desc), self.chunk)
        if nbytes == 0:
            raise ValueError("host fused workspace: arguments out of range")
        self.workspace = torch.empty(int(nbytes), dtype=torch.uint8, device=device or "cuda")

    def __call__(self, params, c0, means, cam, g_rgb, out, stream=None):
        rgb, g_params, g_c0, g_means = out
        for t, nm in ((params, "params"), (c0, "c0")):
            _host(t, nm)
        for t, nm in ((means, "means"), (g_rgb, "g_rgb"), (rgb, "rgb"), (g_params, "g_params"), (g_c0, "g_c0")):
            _host(t, nm, torch.float32)
        if g_means is not None:
            _host(g_means, "g_means", torch.float32)
        _check(lib.nasgabor_fused_fwd_bwd_host(ctypes.byref(self.desc), _ptr(params), _ptr(c0), _ptr(means),
                                               _cam(cam), _ptr(g_rgb), _ptr(rgb), _ptr(g_params), _ptr(g_c0),
                                               _ptr(g_means), self.chunk, _ptr(self.workspace),
                                               self.workspace.numel(), _stream(stream)),
               "nasgabor_fused_fwd_bwd_host")
        return out

"""Python binding of ``libvstereo.so``, the sm_103a virtual-stereo hot path.

Argument marshalling only: every step runs in the library's CUDA kernels,
reached through its C ABI (``include/vstereo.h``).  PyTorch supplies device
memory and streams; tensors are passed as raw pointers.  There is no CPU
fallback: importing works anywhere, but the first call raises if the built
library is missing.

Steps of the method (arXiv 1902.09733):

* :func:`rectify_remap`               Section 2.1 remap + Section 2.2 downsample
* :func:`bp_stereo`                   Eq. 1 hierarchical min-sum BP
* :func:`guided_upsample`             Eq. 2 joint bilateral upsampling
* :func:`reproject`                   Eq. 3 point cloud
* :func:`guided_upsample_reproject`   Eq. 2 + Eq. 3 fused
* :func:`pair_run`, :func:`pair_run_host`  a whole pair (device / host buffers)
* :func:`sp_forward`, :func:`sp_backward`, :func:`smooth_bp`  the temperature-
  smoothed (log-domain sum-product) relaxation of the Eq. 1 messages, its
  adjoint, and a ``torch.autograd.Function`` over the two
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading
from dataclasses import dataclass

import torch

__all__ = [
    "Camera", "BPParams", "JBUParams", "PairConfig", "VSError", "lib", "library_path",
    "rectify_remap", "bp_workspace_size", "bp_stereo", "bp_export_messages",
    "guided_upsample", "reproject", "guided_upsample_reproject",
    "pair_workspace_size", "pair_run", "pair_run_host", "PoseParams", "pose_workspace_size", "harris_response",
    "harris_corners", "zssd_match", "epnp", "pose_estimate", "pair_run_batch", "pair_batch_workspace_size", "kernel_launches", "status_string",
    "profile_enable", "profile_collect", "Pipeline", "bp_stereo_batch", "bp_batch_workspace_size",
    "bp_autotune", "bp_autotune_reset", "bp_autotune_times", "bp_select_sweep", "bp_select_fused", "bp_autotune_plans", "bp_autotune_level_times", "bp_batch_mode", "SPParams", "sp_workspace_size", "sp_forward", "sp_backward",
    "smooth_bp", "SmoothBP", "sp_select_kernels", "sp_status",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libvstereo.so")

VS_OK, VS_EINVAL, VS_EALIGN, VS_EWORKSPACE, VS_ECUDA, VS_ETIMEOUT = 0, -1, -2, -3, -4, -5


class VSError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: status {code} ({status_string(code)})")
        self.code = code


# ---------------------------------------------------------------------------
# C structs (mirrors of include/vstereo.h)

class _Camera(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("fx", "fy", "cx", "cy", "k1", "k2")]


class _BPParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("labels", "levels", "iters", "data_trunc", "smooth_slope", "smooth_trunc", "iters_per_tile")]


class _BPJob(ctypes.Structure):
    _fields_ = [("left", ctypes.c_void_p), ("right", ctypes.c_void_p), ("w", ctypes.c_int32),
                ("h", ctypes.c_int32), ("pitch", ctypes.c_int32), ("params", _BPParams),
                ("labels", ctypes.c_void_p), ("labels_pitch", ctypes.c_int32)]


class _SPParams(ctypes.Structure):
    _fields_ = [("labels", ctypes.c_int32), ("iters", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
                ("lam", ctypes.c_float), ("trunc", ctypes.c_float), ("tau", ctypes.c_float)]


class _JBUParams(ctypes.Structure):
    _fields_ = [("scale", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("sigma_s", ctypes.c_float), ("sigma_r", ctypes.c_float)]


class _PairConfig(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("cam", _Camera),
                ("baseline", ctypes.c_float), ("bp", _BPParams), ("jbu", _JBUParams)]


class _PoseParams(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int32), ("margin", ctypes.c_int32), ("threshold25", ctypes.c_int64),
                ("radius", ctypes.c_int32), ("search", ctypes.c_int32)]


class _PairJob(ctypes.Structure):
    _fields_ = [("cfg", _PairConfig), ("left", ctypes.c_void_p), ("right", ctypes.c_void_p),
                ("disp", ctypes.c_void_p), ("xyz", ctypes.c_void_p)]


@dataclass(frozen=True)
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    k1: float = 0.0
    k2: float = 0.0

    def c(self) -> _Camera:
        return _Camera(self.fx, self.fy, self.cx, self.cy, self.k1, self.k2)


@dataclass(frozen=True)
class BPParams:
    labels: int = 64
    levels: int = 4
    iters: int = 10
    data_trunc: int = 20
    smooth_slope: int = 10
    smooth_trunc: int = 40
    iters_per_tile: int = 0     # 0 automatic, 1 one kernel per iteration, k >= 2 up to k per fused tile launch

    def c(self) -> _BPParams:
        return _BPParams(self.labels, self.levels, self.iters, self.data_trunc,
                         self.smooth_slope, self.smooth_trunc, self.iters_per_tile)


@dataclass(frozen=True)
class SPParams:
    """Smoothed BP: V(d, d') = min(lam |d - d'|, trunc), temperature tau."""
    labels: int = 48
    iters: int = 8
    ckpt_every: int = 2
    lam: float = 2.5
    trunc: float = 13.7
    tau: float = 2.0

    def c(self) -> _SPParams:
        return _SPParams(self.labels, self.iters, self.ckpt_every, self.lam, self.trunc, self.tau)


@dataclass(frozen=True)
class PoseParams:
    """Pose path (Section 2.3): grid x grid cells of one corner each, corners
    at least `margin` inside the frame with 25 R above `threshold25`, ZSSD
    patches of radius `radius` searched over [-search, search]^2."""
    grid: int = 30
    margin: int = 16
    threshold25: int = 0
    radius: int = 5
    search: int = 24

    def c(self) -> _PoseParams:
        return _PoseParams(self.grid, self.margin, self.threshold25, self.radius, self.search)


@dataclass(frozen=True)
class JBUParams:
    scale: int = 4
    radius: int = 2
    sigma_s: float = 1.0
    sigma_r: float = 12.0

    def c(self) -> _JBUParams:
        return _JBUParams(self.scale, self.radius, self.sigma_s, self.sigma_r)


@dataclass(frozen=True)
class PairConfig:
    W: int
    H: int
    cam: Camera
    baseline: float
    bp: BPParams
    jbu: JBUParams

    def c(self) -> _PairConfig:
        return _PairConfig(self.W, self.H, self.cam.c(), self.baseline, self.bp.c(), self.jbu.c())


# ---------------------------------------------------------------------------
# loading

_lock = threading.Lock()
_lib = None


def _load(path: str) -> ctypes.CDLL:
    """A CDLL of the library at `path` with every entry point's argument and
    result types set."""
    L = ctypes.CDLL(path)
    P, I, F, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
    cam_p, bp_p = ctypes.POINTER(_Camera), ctypes.POINTER(_BPParams)
    sp_p = ctypes.POINTER(_SPParams)
    jbu_p, cfg_p = ctypes.POINTER(_JBUParams), ctypes.POINTER(_PairConfig)
    sig = {
        "vs_rectify_remap": ([P, I, I, I, cam_p, P, P, I, I, P, I, P, I, P], I),
        "vs_bp_workspace_size": ([I, I, bp_p], S),
        "vs_bp_stereo": ([P, P, I, I, I, bp_p, P, I, P, S, P], I),
        "vs_bp_export_messages": ([P, S, I, I, bp_p, P, P], I),
        "vs_bp_status": ([P, S, I, I, bp_p, P], I),
        "vs_bp_test_withhold_copies": ([I], I),
        "vs_guided_upsample": ([P, I, I, I, P, I, P, I, I, I, jbu_p, P, P], I),
        "vs_reproject": ([P, I, I, cam_p, F, P, P], I),
        "vs_guided_upsample_reproject": ([P, I, I, I, P, I, P, I, I, I, jbu_p, cam_p, F, P, P, P], I),
        "vs_pair_workspace_size": ([cfg_p], S),
        "vs_pair_run": ([cfg_p, P, P, P, P, P, S, P], I),
        "vs_pair_run_host": ([cfg_p, P, P, P, P, P, P, P, P, S, P], I),
        "vs_status_string": ([I], ctypes.c_char_p),
        "vs_kernel_launches": ([], ctypes.c_uint64),
        "vs_profile_enable": ([I], I),
        "vs_profile_collect": ([P, P, I], I),
        "vs_bp_batch_workspace_size": ([P, I], S),
        "vs_bp_stereo_batch": ([P, I, P, S, P], I),
        "vs_bp_batch_mode": ([I], I),
        "vs_bp_autotune": ([P, P, I, I, I, bp_p, P, I, P, S, P, P], I),
        "vs_bp_autotune_reset": ([], None),
        "vs_bp_autotune_times": ([P, I], I),
        "vs_bp_select_sweep": ([I], I),
        "vs_bp_select_fused": ([I, I, I], I),
        "vs_sp_test_withhold_mma": ([I], I),
        "vs_bp_autotune_plans": ([P, I], I),
        "vs_pair_batch_workspace_size": ([P, I], S),
        "vs_pair_run_batch": ([P, I, P, S, P], I),
        "vs_bp_autotune_level_times": ([P, I], I),
        "vs_pipeline_workspace_size": ([cfg_p, I, I, I], S),
        "vs_pipeline_create": ([cfg_p, I, I, I, P, S, ctypes.POINTER(P)], I),
        "vs_pipeline_submit_pair": ([P, P, P, P], I),
        "vs_pipeline_submit_frame": ([P, P, P], I),
        "vs_pipeline_flush": ([P], I),
        "vs_pipeline_latencies": ([P, P, I], I),
        "vs_pipeline_destroy": ([P], None),
        "vs_sp_workspace_size": ([I, I, sp_p], S),
        "vs_sp_forward": ([P, I, I, sp_p, P, P, S, P], I),
        "vs_sp_backward": ([P, I, I, sp_p, P, P, P, P, S, P], I),
        "vs_sp_select_kernels": ([I], I),
        "vs_sp_status": ([P, S, I, I, sp_p, P], I),
        "vs_check_report": ([P], I),
        "vs_pose_workspace_size": ([I, I, ctypes.POINTER(_PoseParams)], S),
        "vs_harris_response": ([P, I, I, I, P, P], I),
        "vs_harris_corners": ([P, I, I, I, ctypes.POINTER(_PoseParams), P, P, S, P], I),
        "vs_zssd_match": ([P, P, I, I, I, P, I, ctypes.POINTER(_PoseParams), P, P, P], I),
        "vs_epnp": ([P, P, I, cam_p, P, P], I),
        "vs_pose_estimate": ([P, P, P, I, I, I, cam_p, ctypes.POINTER(_PoseParams), P, P, S, P], I),
        "vs_pose_average": ([P, P, ctypes.c_double, P, P], I),
        "vs_pose_stereo_workspace_size": ([I, I, ctypes.POINTER(_PoseParams)], S),
        "vs_pose_estimate_stereo": ([P, P, P, P, I, I, I, cam_p, ctypes.c_double, ctypes.POINTER(_PoseParams), P,
                                     P, S, P], I),
        "vs_check_test_shrink": ([ctypes.c_longlong], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(library_path):
            raise RuntimeError(
                f"{library_path} is missing: build it with "
                "`python -m paper_1902_09733_b300.build` (nvcc, sm_103a); there is no CPU fallback")
        _lib = _load(library_path)
        return _lib


checked_library_path = os.path.join(_HERE, "libvstereo_checked.so")
_checked = None


def checked_lib() -> ctypes.CDLL:
    """The checked build (bounds checks in the min-sum kernels, for tests)."""
    global _checked
    with _lock:
        if _checked is None:
            if not os.path.exists(checked_library_path):
                raise RuntimeError(f"{checked_library_path} is missing: build it with "
                                   "`python -m paper_1902_09733_b300.build`")
            _checked = _load(checked_library_path)
        return _checked


@contextlib.contextmanager
def using(library: ctypes.CDLL):
    """Test aid: every wrapper of this module calls `library` (for example
    checked_lib()) inside the block; one thread at a time."""
    global _lib
    lib()
    with _lock:
        old, _lib = _lib, library
    try:
        yield library
    finally:
        with _lock:
            _lib = old


def status_string(code: int) -> str:
    try:
        return lib().vs_status_string(code).decode()
    except RuntimeError:
        return "library not built"


def kernel_launches() -> int:
    return int(lib().vs_kernel_launches())


PROFILE_TAGS = {0: "sweep_level0", 1: "sweep_coarse", 2: "remap", 3: "upsample", 4: "bp_other",
                5: "smooth_fwd", 6: "smooth_adj"}


def profile_enable(capacity: int) -> None:
    """Bracket every later launch with a CUDA event pair (0 switches off)."""
    _check("vs_profile_enable", lib().vs_profile_enable(int(capacity)))


def profile_collect(max_records: int = 1 << 16):
    """[(tag name, milliseconds)] of the launches timed since the last collect."""
    tags = (ctypes.c_int * max_records)()
    ms = (ctypes.c_float * max_records)()
    n = lib().vs_profile_collect(ctypes.cast(tags, ctypes.c_void_p), ctypes.cast(ms, ctypes.c_void_p), max_records)
    if n < 0:
        raise VSError("vs_profile_collect", n)
    return [(PROFILE_TAGS.get(tags[i], str(tags[i])), float(ms[i])) for i in range(n)]


def _check(fn: str, rc: int) -> None:
    if rc != VS_OK:
        raise VSError(fn, rc)


def _stream(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev(t: torch.Tensor, dtype: torch.dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t


def _pitched(t: torch.Tensor, channels: int, name: str) -> int:
    """Row pitch in bytes of an image tensor whose rows may be padded."""
    if channels == 1:
        ok = t.dim() == 2 and t.stride(1) == 1
    else:
        ok = t.dim() == 3 and t.shape[2] == channels and t.stride(2) == 1 and t.stride(1) == channels
    if not ok:
        raise ValueError(f"{name} must be an (H, W{'' if channels == 1 else ', 3'}) image with contiguous rows")
    return t.stride(0) * t.element_size()


# ---------------------------------------------------------------------------
# steps


def rectify_remap(src: torch.Tensor, cam: Camera, R=None, scale: int = 4, dst=True, low_rgb=True,
                  low_gray=True, stream=None):
    """Section 2.1 remap of an (H, W, 3) uint8 frame fused with the Section 2.2
    downsample.  ``dst``/``low_rgb``/``low_gray`` are tensors to write, True to
    allocate, or None/False to skip.  Returns (dst, low_rgb, low_gray)."""
    _dev(src, torch.uint8, "src")
    H, W = src.shape[0], src.shape[1]
    w, h = -(-W // scale), -(-H // scale)

    def out(spec, shape):
        if spec is True:
            return torch.empty(shape, dtype=torch.uint8, device=src.device)
        return spec if isinstance(spec, torch.Tensor) else None

    dst_t, lr_t, lg_t = out(dst, (H, W, 3)), out(low_rgb, (h, w, 3)), out(low_gray, (h, w))
    Rm = None
    if R is not None:
        Rf = (ctypes.c_float * 9)(*[float(v) for v in torch.as_tensor(R, dtype=torch.float64).reshape(9)])
        Rm = ctypes.cast(Rf, ctypes.c_void_p)
    c = cam.c()
    rc = lib().vs_rectify_remap(
        src.data_ptr(), W, H, _pitched(src, 3, "src"), ctypes.byref(c), Rm,
        dst_t.data_ptr() if dst_t is not None else None, _pitched(dst_t, 3, "dst") if dst_t is not None else 0,
        scale,
        lr_t.data_ptr() if lr_t is not None else None, _pitched(lr_t, 3, "low_rgb") if lr_t is not None else 0,
        lg_t.data_ptr() if lg_t is not None else None, _pitched(lg_t, 1, "low_gray") if lg_t is not None else 0,
        _stream(stream))
    _check("vs_rectify_remap", rc)
    return dst_t, lr_t, lg_t


def bp_workspace_size(w: int, h: int, params: BPParams) -> int:
    p = params.c()
    return int(lib().vs_bp_workspace_size(w, h, ctypes.byref(p)))


def bp_stereo(left: torch.Tensor, right: torch.Tensor, params: BPParams, labels=None, workspace=None,
              stream=None) -> torch.Tensor:
    """Eq. 1 on an (h, w) uint8 grey pair; returns (h, w) uint8 labels."""
    _dev(left, torch.uint8, "left")
    _dev(right, torch.uint8, "right")
    if left.shape != right.shape or left.stride() != right.stride():
        raise ValueError("left and right must have the same shape and strides")
    h, w = left.shape
    pitch = _pitched(left, 1, "left")
    need = bp_workspace_size(w, h, params)
    if need == 0:
        raise VSError("vs_bp_workspace_size", VS_EINVAL)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=left.device)
    if labels is None:
        labels = torch.empty((h, w), dtype=torch.uint8, device=left.device)
    p = params.c()
    rc = lib().vs_bp_stereo(left.data_ptr(), right.data_ptr(), w, h, pitch, ctypes.byref(p),
                            labels.data_ptr(), _pitched(labels, 1, "labels"), workspace.data_ptr(),
                            workspace.numel() * workspace.element_size(), _stream(stream))
    _check("vs_bp_stereo", rc)
    return labels


def _jobs(pairs, labels):
    arr = (_BPJob * len(pairs))()
    for i, ((left, right, params), lab) in enumerate(zip(pairs, labels)):
        _dev(left, torch.uint8, "left")
        _dev(right, torch.uint8, "right")
        if left.shape != right.shape or left.stride() != right.stride():
            raise ValueError("left and right must have the same shape and strides")
        h, w = left.shape
        arr[i] = _BPJob(left.data_ptr(), right.data_ptr(), w, h, _pitched(left, 1, "left"), params.c(),
                        lab.data_ptr(), _pitched(lab, 1, "labels"))
    return arr


def bp_batch_workspace_size(pairs) -> int:
    """Workspace bytes for a batch of (left, right, BPParams) grey pairs."""
    arr = (_BPJob * len(pairs))()
    for i, (left, right, params) in enumerate(pairs):
        h, w = left.shape
        arr[i] = _BPJob(None, None, w, h, w, params.c(), None, w)
    return int(lib().vs_bp_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), len(pairs)))


def bp_stereo_batch(pairs, labels=None, workspace=None, stream=None):
    """Eq. 1 for a list of (left, right, BPParams) pairs advanced in lockstep
    (all with the same levels and iters); returns the list of label maps."""
    if labels is None:
        labels = [torch.empty(tuple(l.shape), dtype=torch.uint8, device=l.device) for l, _, _ in pairs]
    arr = _jobs(pairs, labels)
    need = bp_batch_workspace_size(pairs)
    if need == 0:
        raise VSError("vs_bp_batch_workspace_size", VS_EINVAL)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=pairs[0][0].device)
    _check("vs_bp_stereo_batch", lib().vs_bp_stereo_batch(ctypes.cast(arr, ctypes.c_void_p), len(pairs),
                                                          workspace.data_ptr(), workspace.numel(),
                                                          _stream(stream)))
    return labels


def bp_batch_mode(mode: str) -> None:
    """Schedule of bp_stereo_batch: "streams" (default) or "lockstep"."""
    _check("vs_bp_batch_mode", lib().vs_bp_batch_mode({"streams": 0, "lockstep": 1}[mode]))


def bp_autotune(left: torch.Tensor, right: torch.Tensor, params: BPParams, workspace=None, labels=None,
                stream=None):
    """Time the sweep kernels on every level of this pair and keep the
    fastest for later calls; returns the choice per level (0 plain, 1 preload,
    2 labels split in two, 3 in four) and leaves the pair's labels in ``labels``."""
    h, w = left.shape
    if workspace is None:
        workspace = torch.empty(bp_workspace_size(w, h, params), dtype=torch.uint8, device=left.device)
    if labels is None:
        labels = torch.empty((h, w), dtype=torch.uint8, device=left.device)
    chosen = (ctypes.c_int * params.levels)()
    p = params.c()
    _check("vs_bp_autotune", lib().vs_bp_autotune(
        left.data_ptr(), right.data_ptr(), w, h, _pitched(left, 1, "left"), ctypes.byref(p), labels.data_ptr(),
        _pitched(labels, 1, "labels"), workspace.data_ptr(), workspace.numel(), _stream(stream),
        ctypes.cast(chosen, ctypes.c_void_p)))
    return [int(v) for v in chosen]


def bp_autotune_times():
    """[[ms per launch of variants 0..3] per level] of the last bp_autotune (-1: not applicable)."""
    buf = (ctypes.c_float * 64)()
    n = lib().vs_bp_autotune_times(ctypes.cast(buf, ctypes.c_void_p), 64)
    return [[float(buf[i + v]) for v in range(4)] for i in range(0, n, 4)]


def bp_autotune_plans():
    """[(K, tile_w, tile_h, lanes)] per level chosen by the last bp_autotune (K = 0: unfused)."""
    buf = (ctypes.c_int * 64)()
    n = lib().vs_bp_autotune_plans(ctypes.cast(buf, ctypes.c_void_p), 64)
    return [tuple(buf[i:i + 4]) for i in range(0, n, 4)]


def bp_autotune_level_times():
    """[(ms unfused, ms best fused)] per level behind the last bp_autotune (-1: not timed)."""
    buf = (ctypes.c_float * 64)()
    n = lib().vs_bp_autotune_level_times(ctypes.cast(buf, ctypes.c_void_p), 64)
    return [(buf[i], buf[i + 1]) for i in range(0, n, 2)]


def bp_select_sweep(variant: int) -> None:
    """Force sweep variant 0..4 (plain, preload, split 2, split 4, staged) wherever it applies (-1: automatic)."""
    _check("vs_bp_select_sweep", lib().vs_bp_select_sweep(int(variant)))


def bp_select_fused(tile_w: int = 0, tile_h: int = 0, lanes: int = 0) -> None:
    """Force the core tile and lanes per direction pair of fused sweeps (0, 0, 0: automatic)."""
    _check("vs_bp_select_fused", lib().vs_bp_select_fused(int(tile_w), int(tile_h), int(lanes)))


def bp_test_withhold_copies(on: bool) -> None:
    """Test aid: staged sweeps issue no copies, so their bounded waits run out (status VS_ETIMEOUT)."""
    _check("vs_bp_test_withhold_copies", lib().vs_bp_test_withhold_copies(1 if on else 0))


def bp_status(workspace: torch.Tensor, w: int, h: int, params: BPParams, stream=None) -> None:
    """Raise VSError(VS_ETIMEOUT) if a kernel of the last bp_stereo on ``workspace`` gave up a bounded wait."""
    c = params.c()
    _check("vs_bp_status", lib().vs_bp_status(workspace.data_ptr(), workspace.numel(), w, h, ctypes.byref(c),
                                              _stream(stream)))


def bp_autotune_reset() -> None:
    lib().vs_bp_autotune_reset()


def bp_export_messages(workspace: torch.Tensor, w: int, h: int, params: BPParams, stream=None) -> torch.Tensor:
    """Final level-0 incoming messages of the last bp_stereo on ``workspace``,
    (4, h, w, labels) int32, directions left, right, up, down."""
    out = torch.empty((4, h, w, params.labels), dtype=torch.int32, device=workspace.device)
    p = params.c()
    rc = lib().vs_bp_export_messages(workspace.data_ptr(), workspace.numel(), w, h, ctypes.byref(p),
                                     out.data_ptr(), _stream(stream))
    _check("vs_bp_export_messages", rc)
    return out


def guided_upsample(labels: torch.Tensor, guide_low: torch.Tensor, guide_full: torch.Tensor,
                    jbu: JBUParams, disp=None, stream=None) -> torch.Tensor:
    """Eq. 2; returns the (H, W) float32 full-resolution disparity."""
    h, w = labels.shape
    H, W = guide_full.shape[0], guide_full.shape[1]
    if disp is None:
        disp = torch.empty((H, W), dtype=torch.float32, device=labels.device)
    j = jbu.c()
    rc = lib().vs_guided_upsample(
        _dev(labels, torch.uint8, "labels").data_ptr(), w, h, _pitched(labels, 1, "labels"),
        _dev(guide_low, torch.uint8, "guide_low").data_ptr(), _pitched(guide_low, 3, "guide_low"),
        _dev(guide_full, torch.uint8, "guide_full").data_ptr(), W, H, _pitched(guide_full, 3, "guide_full"),
        ctypes.byref(j), _dev(disp, torch.float32, "disp").data_ptr(), _stream(stream))
    _check("vs_guided_upsample", rc)
    return disp


def reproject(disp: torch.Tensor, cam: Camera, baseline: float, xyz=None, stream=None) -> torch.Tensor:
    """Eq. 3; returns (H, W, 3) float32 camera-frame points (NaN where d <= 0)."""
    _dev(disp, torch.float32, "disp")
    if not disp.is_contiguous():
        raise ValueError("disp must be contiguous")
    H, W = disp.shape
    if xyz is None:
        xyz = torch.empty((H, W, 3), dtype=torch.float32, device=disp.device)
    c = cam.c()
    rc = lib().vs_reproject(disp.data_ptr(), W, H, ctypes.byref(c), float(baseline),
                            _dev(xyz, torch.float32, "xyz").data_ptr(), _stream(stream))
    _check("vs_reproject", rc)
    return xyz


def guided_upsample_reproject(labels, guide_low, guide_full, jbu: JBUParams, cam: Camera, baseline: float,
                              xyz=None, disp=None, want_disp: bool = True, stream=None):
    """Eq. 2 + Eq. 3 in one kernel; returns (disp or None, xyz)."""
    h, w = labels.shape
    H, W = guide_full.shape[0], guide_full.shape[1]
    dev = labels.device
    if xyz is None:
        xyz = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    if disp is None and want_disp:
        disp = torch.empty((H, W), dtype=torch.float32, device=dev)
    j, c = jbu.c(), cam.c()
    rc = lib().vs_guided_upsample_reproject(
        _dev(labels, torch.uint8, "labels").data_ptr(), w, h, _pitched(labels, 1, "labels"),
        _dev(guide_low, torch.uint8, "guide_low").data_ptr(), _pitched(guide_low, 3, "guide_low"),
        _dev(guide_full, torch.uint8, "guide_full").data_ptr(), W, H, _pitched(guide_full, 3, "guide_full"),
        ctypes.byref(j), ctypes.byref(c), float(baseline),
        disp.data_ptr() if disp is not None else None, _dev(xyz, torch.float32, "xyz").data_ptr(),
        _stream(stream))
    _check("vs_guided_upsample_reproject", rc)
    return disp, xyz


def pair_workspace_size(cfg: PairConfig) -> int:
    c = cfg.c()
    return int(lib().vs_pair_workspace_size(ctypes.byref(c)))


def pair_run(cfg: PairConfig, left_src: torch.Tensor, right_src: torch.Tensor, xyz=None, disp=None,
             workspace=None, stream=None):
    """A whole pair on device buffers; returns (disp or None, xyz)."""
    dev = left_src.device
    for t, n in ((left_src, "left_src"), (right_src, "right_src")):
        _dev(t, torch.uint8, n)
        if not t.is_contiguous() or tuple(t.shape) != (cfg.H, cfg.W, 3):
            raise ValueError(f"{n} must be a contiguous ({cfg.H}, {cfg.W}, 3) uint8 tensor")
    if xyz is None:
        xyz = torch.empty((cfg.H, cfg.W, 3), dtype=torch.float32, device=dev)
    if workspace is None:
        workspace = torch.empty(pair_workspace_size(cfg), dtype=torch.uint8, device=dev)
    c = cfg.c()
    rc = lib().vs_pair_run(ctypes.byref(c), left_src.data_ptr(), right_src.data_ptr(),
                           disp.data_ptr() if disp is not None else None, xyz.data_ptr(),
                           workspace.data_ptr(), workspace.numel(), _stream(stream))
    _check("vs_pair_run", rc)
    return disp, xyz


def _pair_jobs(jobs):
    arr = (_PairJob * len(jobs))()
    for i, (cfg, left, right, disp, xyz) in enumerate(jobs):
        arr[i] = _PairJob(cfg.c(), left.data_ptr(), right.data_ptr(),
                          disp.data_ptr() if disp is not None else None, xyz.data_ptr())
    return arr


def pair_batch_workspace_size(jobs) -> int:
    """Workspace bytes for [(PairConfig, left, right, disp or None, xyz)] device jobs."""
    arr = _pair_jobs(jobs)
    return int(lib().vs_pair_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), len(jobs)))


def pair_run_batch(jobs, workspace=None, stream=None):
    """Whole pairs [(PairConfig, left, right, disp or None, xyz)] on the library streams."""
    for cfg, left, right, disp, xyz in jobs:
        for t, n in ((left, "left"), (right, "right")):
            _dev(t, torch.uint8, n)
            if not t.is_contiguous() or tuple(t.shape) != (cfg.H, cfg.W, 3):
                raise ValueError(f"{n} must be a contiguous ({cfg.H}, {cfg.W}, 3) uint8 tensor")
        if tuple(xyz.shape) != (cfg.H, cfg.W, 3) or xyz.dtype != torch.float32 or not xyz.is_contiguous():
            raise ValueError("xyz must be a contiguous (H, W, 3) float32 tensor")
    arr = _pair_jobs(jobs)
    if workspace is None:
        n = lib().vs_pair_batch_workspace_size(ctypes.cast(arr, ctypes.c_void_p), len(jobs))
        if n == 0:
            raise VSError("vs_pair_batch_workspace_size", VS_EINVAL)
        workspace = torch.empty(n, dtype=torch.uint8, device=jobs[0][1].device)
    _check("vs_pair_run_batch", lib().vs_pair_run_batch(ctypes.cast(arr, ctypes.c_void_p), len(jobs),
                                                        workspace.data_ptr(), workspace.numel(), _stream(stream)))
    return workspace


# ---------------------------------------------------------------------------
# pose path (Section 2.3)


def _rgb(t: torch.Tensor, name: str):
    _dev(t, torch.uint8, name)
    if t.dim() != 3 or t.shape[2] != 3 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (H, W, 3) uint8 tensor")
    return t.shape[0], t.shape[1]


def pose_workspace_size(W: int, H: int, params: PoseParams) -> int:
    p = params.c()
    return int(lib().vs_pose_workspace_size(W, H, ctypes.byref(p)))


def harris_response(rgb: torch.Tensor, stream=None) -> torch.Tensor:
    """25 R of Eq. 5 at every pixel (int64 (H, W))."""
    H, W = _rgb(rgb, "rgb")
    out = torch.empty((H, W), dtype=torch.int64, device=rgb.device)
    _check("vs_harris_response", lib().vs_harris_response(rgb.data_ptr(), W, H, 3 * W, out.data_ptr(),
                                                          _stream(stream)))
    return out


def harris_corners(rgb: torch.Tensor, params: PoseParams, workspace=None, stream=None) -> torch.Tensor:
    """(grid^2, 2) int32 corners, -1 where a cell has none."""
    H, W = _rgb(rgb, "rgb")
    p = params.c()
    if workspace is None:
        workspace = torch.empty(pose_workspace_size(W, H, params), dtype=torch.uint8, device=rgb.device)
    out = torch.empty((params.grid * params.grid, 2), dtype=torch.int32, device=rgb.device)
    _check("vs_harris_corners", lib().vs_harris_corners(rgb.data_ptr(), W, H, 3 * W, ctypes.byref(p), out.data_ptr(),
                                                        workspace.data_ptr(), workspace.numel(), _stream(stream)))
    return out


def zssd_match(rgb1: torch.Tensor, rgb2: torch.Tensor, corners: torch.Tensor, params: PoseParams, stream=None):
    """(pos (n, 2) float64, cost (n,) int64) of the corners of frame 1 in frame 2."""
    H, W = _rgb(rgb1, "rgb1")
    _rgb(rgb2, "rgb2")
    corners = corners.to(torch.int32).contiguous()
    n = corners.shape[0]
    p = params.c()
    pos = torch.empty((n, 2), dtype=torch.float64, device=rgb1.device)
    cost = torch.empty((n,), dtype=torch.int64, device=rgb1.device)
    _check("vs_zssd_match", lib().vs_zssd_match(rgb1.data_ptr(), rgb2.data_ptr(), W, H, 3 * W, corners.data_ptr(), n,
                                                ctypes.byref(p), pos.data_ptr(), cost.data_ptr(), _stream(stream)))
    return pos, cost


def epnp(points: torch.Tensor, uv: torch.Tensor, cam: Camera, stream=None) -> torch.Tensor:
    """(14,) float64: R (row-major), T, mean reprojection error, inlier count."""
    points = points.to(torch.float64).contiguous()
    uv = uv.to(torch.float64).contiguous()
    out = torch.empty(14, dtype=torch.float64, device=points.device)
    c = cam.c()
    _check("vs_epnp", lib().vs_epnp(points.data_ptr(), uv.data_ptr(), points.shape[0], ctypes.byref(c),
                                    out.data_ptr(), _stream(stream)))
    return out


def pose_estimate(rgb1: torch.Tensor, rgb2: torch.Tensor, xyz1: torch.Tensor, cam: Camera, params: PoseParams,
                  workspace=None, stream=None) -> torch.Tensor:
    """Pose of camera 2 relative to camera 1 from frame 1's cloud: (14,) as :func:`epnp`."""
    H, W = _rgb(rgb1, "rgb1")
    _rgb(rgb2, "rgb2")
    if tuple(xyz1.shape) != (H, W, 3) or xyz1.dtype != torch.float32 or not xyz1.is_contiguous():
        raise ValueError("xyz1 must be a contiguous (H, W, 3) float32 tensor")
    if workspace is None:
        workspace = torch.empty(pose_workspace_size(W, H, params), dtype=torch.uint8, device=rgb1.device)
    out = torch.empty(14, dtype=torch.float64, device=rgb1.device)
    c, p = cam.c(), params.c()
    _check("vs_pose_estimate", lib().vs_pose_estimate(rgb1.data_ptr(), rgb2.data_ptr(), xyz1.data_ptr(), W, H, 3 * W,
                                                      ctypes.byref(c), ctypes.byref(p), out.data_ptr(),
                                                      workspace.data_ptr(), workspace.numel(), _stream(stream)))
    return out


def pose_average(left: torch.Tensor, right: torch.Tensor, baseline: float, stream=None) -> torch.Tensor:
    """Section 2.3: the left and right poses of a later stereo pair (14 float64
    each, as :func:`pose_estimate`) averaged through the virtual rig; (14,)."""
    left = left.to(torch.float64).contiguous()
    right = right.to(torch.float64).contiguous()
    out = torch.empty(14, dtype=torch.float64, device=left.device)
    _check("vs_pose_average", lib().vs_pose_average(left.data_ptr(), right.data_ptr(), float(baseline),
                                                    out.data_ptr(), _stream(stream)))
    return out


def pose_stereo_workspace_size(W: int, H: int, params: PoseParams) -> int:
    p = params.c()
    return int(lib().vs_pose_stereo_workspace_size(W, H, ctypes.byref(p)))


def pose_estimate_stereo(left1: torch.Tensor, left2: torch.Tensor, right2: torch.Tensor, xyz1: torch.Tensor,
                         cam: Camera, baseline: float, params: PoseParams, workspace=None,
                         stream=None) -> torch.Tensor:
    """The averaged pose of a later stereo pair (left2, right2) relative to
    frame 1's left camera, from frame 1's cloud: (14,) as :func:`pose_average`."""
    H, W = _rgb(left1, "left1")
    _rgb(left2, "left2")
    _rgb(right2, "right2")
    if tuple(xyz1.shape) != (H, W, 3) or xyz1.dtype != torch.float32 or not xyz1.is_contiguous():
        raise ValueError("xyz1 must be a contiguous (H, W, 3) float32 tensor")
    if workspace is None:
        workspace = torch.empty(pose_stereo_workspace_size(W, H, params), dtype=torch.uint8, device=left1.device)
    out = torch.empty(14, dtype=torch.float64, device=left1.device)
    c, p = cam.c(), params.c()
    _check("vs_pose_estimate_stereo",
           lib().vs_pose_estimate_stereo(left1.data_ptr(), left2.data_ptr(), right2.data_ptr(), xyz1.data_ptr(), W, H,
                                         3 * W, ctypes.byref(c), float(baseline), ctypes.byref(p), out.data_ptr(),
                                         workspace.data_ptr(), workspace.numel(), _stream(stream)))
    return out


def pair_run_host(cfg: PairConfig, left_host: torch.Tensor, right_host: torch.Tensor, xyz_host: torch.Tensor,
                  dev_in: torch.Tensor, dev_xyz: torch.Tensor, workspace: torch.Tensor, disp_host=None,
                  dev_disp=None, stream=None):
    """A whole pair from host (ideally pinned) frames to a host point cloud;
    copies in and out inside the call and returns when the cloud is on the host."""
    for t, n in ((left_host, "left_host"), (right_host, "right_host"), (xyz_host, "xyz_host")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{n} must be a contiguous host tensor")
    c = cfg.c()
    rc = lib().vs_pair_run_host(
        ctypes.byref(c), left_host.data_ptr(), right_host.data_ptr(),
        disp_host.data_ptr() if disp_host is not None else None, xyz_host.data_ptr(),
        dev_in.data_ptr(), dev_disp.data_ptr() if dev_disp is not None else None, dev_xyz.data_ptr(),
        workspace.data_ptr(), workspace.numel(), _stream(stream))
    _check("vs_pair_run_host", rc)
    return xyz_host


class Pipeline:
    """Streaming driver over three CUDA streams (``vs_pipeline_*``).

    ``mode="pairs"``: :meth:`submit_pair` takes both frames of independent
    pairs.  ``mode="flight"``: :meth:`submit_frame` takes one frame at a time
    and pairs frame f - k (left) with frame f (right).  Up to ``depth`` pairs
    are in flight; host tensors passed to a submit must stay alive until the
    pair completes (:meth:`flush`).  Device memory is one caller-visible
    workspace tensor; the library allocates none.
    """

    MODES = {"pairs": 0, "flight": 1}

    def __init__(self, cfg: PairConfig, mode: str = "pairs", depth: int = 3, k: int = 1, device=None):
        self.cfg = cfg
        self._c = cfg.c()
        self.mode = self.MODES[mode]
        n = int(lib().vs_pipeline_workspace_size(ctypes.byref(self._c), self.mode, depth, k))
        if n == 0:
            raise VSError("vs_pipeline_workspace_size", VS_EINVAL)
        self.workspace = torch.empty(n, dtype=torch.uint8, device=device or "cuda")
        h = ctypes.c_void_p()
        _check("vs_pipeline_create", lib().vs_pipeline_create(ctypes.byref(self._c), self.mode, depth, k,
                                                               self.workspace.data_ptr(), n, ctypes.byref(h)))
        self._h = h
        self._keep = []

    def submit_pair(self, left_host: torch.Tensor, right_host: torch.Tensor, xyz_host: torch.Tensor | None):
        self._keep.append((left_host, right_host, xyz_host))
        _check("vs_pipeline_submit_pair", lib().vs_pipeline_submit_pair(
            self._h, left_host.data_ptr(), right_host.data_ptr(),
            xyz_host.data_ptr() if xyz_host is not None else None))

    def submit_frame(self, frame_host: torch.Tensor, xyz_host: torch.Tensor | None = None):
        self._keep.append((frame_host, xyz_host))
        _check("vs_pipeline_submit_frame", lib().vs_pipeline_submit_frame(
            self._h, frame_host.data_ptr(), xyz_host.data_ptr() if xyz_host is not None else None))

    def flush(self):
        _check("vs_pipeline_flush", lib().vs_pipeline_flush(self._h))
        self._keep.clear()

    def latencies(self, max_records: int = 1 << 16):
        buf = (ctypes.c_float * max_records)()
        n = lib().vs_pipeline_latencies(self._h, ctypes.cast(buf, ctypes.c_void_p), max_records)
        if n < 0:
            raise VSError("vs_pipeline_latencies", n)
        return [float(buf[i]) for i in range(n)]

    def close(self):
        if getattr(self, "_h", None):
            lib().vs_pipeline_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# temperature-smoothed BP (differentiable relaxation of Eq. 1)


def _cost_volume(cost: torch.Tensor, name: str) -> tuple[int, int, int]:
    _dev(cost, torch.float32, name)
    if cost.dim() != 3 or not cost.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (h, w, labels) float32 tensor")
    h, w, L = cost.shape
    return h, w, L


def sp_workspace_size(w: int, h: int, params: SPParams) -> int:
    c = params.c()
    return int(lib().vs_sp_workspace_size(w, h, ctypes.byref(c)))


def sp_forward(cost: torch.Tensor, params: SPParams, beliefs=None, workspace=None, stream=None):
    """Beliefs of the smoothed BP on an (h, w, L) cost volume; returns
    (beliefs, workspace), the workspace holding the adjoint's checkpoints."""
    h, w, L = _cost_volume(cost, "cost")
    if L != params.labels:
        raise ValueError(f"cost has {L} labels, params.labels is {params.labels}")
    need = sp_workspace_size(w, h, params)
    if need == 0:
        raise VSError("vs_sp_workspace_size", VS_EINVAL)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=cost.device)
    if beliefs is None:
        beliefs = torch.empty_like(cost)
    c = params.c()
    _check("vs_sp_forward", lib().vs_sp_forward(cost.data_ptr(), w, h, ctypes.byref(c),
                                                _dev(beliefs, torch.float32, "beliefs").data_ptr(),
                                                workspace.data_ptr(), workspace.numel(), _stream(stream)))
    return beliefs, workspace


def sp_backward(cost: torch.Tensor, params: SPParams, grad_beliefs: torch.Tensor, workspace: torch.Tensor,
                grad_cost=None, grad_params=None, stream=None):
    """Adjoint after :func:`sp_forward` on the same workspace: returns
    (dL/dcost, tensor([dL/dlam, dL/dtrunc, dL/dtau]))."""
    h, w, L = _cost_volume(cost, "cost")
    grad_beliefs = grad_beliefs.contiguous()
    _cost_volume(grad_beliefs, "grad_beliefs")
    if grad_cost is None:
        grad_cost = torch.empty_like(cost)
    if grad_params is None:
        grad_params = torch.empty(3, dtype=torch.float32, device=cost.device)
    c = params.c()
    _check("vs_sp_backward", lib().vs_sp_backward(
        cost.data_ptr(), w, h, ctypes.byref(c), grad_beliefs.data_ptr(),
        _dev(grad_cost, torch.float32, "grad_cost").data_ptr(),
        _dev(grad_params, torch.float32, "grad_params").data_ptr(),
        workspace.data_ptr(), workspace.numel(), _stream(stream)))
    return grad_cost, grad_params


def sp_select_kernels(family: str) -> None:
    """"simt" (FP32 multiply-adds, the default) or "tensor" (tcgen05) kernels for sp_forward / sp_backward."""
    _check("vs_sp_select_kernels", lib().vs_sp_select_kernels({"tensor": 0, "simt": 1}[family]))


def sp_test_withhold_mma(on: bool) -> None:
    """Test aid: the tensor-core smoothed-BP kernels issue no MMA, so their bounded waits run out."""
    _check("vs_sp_test_withhold_mma", lib().vs_sp_test_withhold_mma(1 if on else 0))


def sp_status(workspace: torch.Tensor, w: int, h: int, params: SPParams, stream=None) -> None:
    """Raise VSError(VS_ETIMEOUT) if a tensor-core kernel gave up waiting for its MMAs."""
    c = params.c()
    _check("vs_sp_status", lib().vs_sp_status(workspace.data_ptr(), workspace.numel(), w, h, ctypes.byref(c),
                                              _stream(stream)))


def _scalar(v) -> float:
    return float(v.detach().item()) if isinstance(v, torch.Tensor) else float(v)


class SmoothBP(torch.autograd.Function):
    """beliefs = smoothed BP(cost; lam, trunc, tau), differentiable in all four.

    Forward and backward are the library's kernels (``vs_sp_forward``,
    ``vs_sp_backward``); the workspace with the message checkpoints lives in
    the autograd context until the graph is freed.  The three scalars are read
    on the host (one synchronisation each when they are CUDA tensors).
    """

    @staticmethod
    def forward(ctx, cost, lam, trunc, tau, iters: int = 8, ckpt_every: int = 2):
        cost = cost.contiguous()
        params = SPParams(labels=cost.shape[-1], iters=int(iters), ckpt_every=int(ckpt_every),
                          lam=_scalar(lam), trunc=_scalar(trunc), tau=_scalar(tau))
        beliefs, ws = sp_forward(cost, params)
        ctx.save_for_backward(cost)
        ctx.params = params
        ctx.ws = ws
        ctx.scalar_like = [v if isinstance(v, torch.Tensor) else None for v in (lam, trunc, tau)]
        return beliefs

    @staticmethod
    def backward(ctx, grad_beliefs):
        (cost,) = ctx.saved_tensors
        g_cost, g_par = sp_backward(cost, ctx.params, grad_beliefs.to(torch.float32), ctx.ws)
        outs = []
        for i, like in enumerate(ctx.scalar_like):
            if like is None or not ctx.needs_input_grad[1 + i]:
                outs.append(None)
            else:
                outs.append(g_par[i].to(like.dtype).to(like.device).reshape(like.shape))
        return (g_cost if ctx.needs_input_grad[0] else None, *outs, None, None)


def smooth_bp(cost: torch.Tensor, lam, trunc, tau, iters: int = 8, ckpt_every: int = 2) -> torch.Tensor:
    """Differentiable beliefs of the smoothed BP on an (h, w, L) float32 CUDA cost volume."""
    return SmoothBP.apply(cost, lam, trunc, tau, iters, ckpt_every)

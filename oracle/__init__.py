"""Plain CPU oracle for the virtual-stereo hot path (arXiv 1902.09733).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
CUDA library never imports, links or calls it, and the two share no code: the
oracle is ``vsref.c`` (plain C, int32 / double) plus this ctypes wrapper.

Functions, each following one step of the method:

* :func:`rectify_remap`     -- Section 2.1, undistort + rectify remap
* :func:`downsample_luma`   -- Section 2.2, downsample to the stereo size
* :func:`cost_level0`, :func:`cost_coarsen` -- Eq. 1 data term and pyramid
* :func:`message`           -- Eq. 1 min-sum message (brute force or DT)
* :func:`bp`                -- Eq. 1 hierarchical loopy min-sum BP + labels
* :func:`guided_upsample`   -- Eq. 2 joint bilateral upsampling
* :func:`reproject`         -- Eq. 3 reprojection to (x, y, z)
* :func:`sp_message`, :func:`sp_forward`, :func:`sp_backward` -- the
  temperature-smoothed (log-domain sum-product) relaxation of the Eq. 1
  messages and its reverse-mode derivative (``vsref_smooth.c``)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "vsref.c"), os.path.join(_HERE, "vsref_smooth.c")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libvsref.so")

MSG_BRUTE = 0
MSG_DT = 1

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``vsref.c`` and ``vsref_smooth.c`` into ``oracle/_build/libvsref.so`` with gcc (OpenMP rows)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, *_SRCS, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.vsref_rectify_remap.argtypes = [P, I, I, I, P, P, P, I, P]
        lib.vsref_rectify_remap.restype = I
        lib.vsref_downsample_luma.argtypes = [P, I, I, I, I, P, P]
        lib.vsref_downsample_luma.restype = I
        lib.vsref_cost_level0.argtypes = [P, P, I, I, I, I, P]
        lib.vsref_cost_level0.restype = None
        lib.vsref_cost_coarsen.argtypes = [P, I, I, I, P]
        lib.vsref_cost_coarsen.restype = None
        lib.vsref_message.argtypes = [P, I, I, I, I, P]
        lib.vsref_message.restype = None
        lib.vsref_bp.argtypes = [P, P, I, I, I, I, I, I, I, I, I, P, P]
        lib.vsref_bp.restype = I
        lib.vsref_guided_upsample.argtypes = [P, I, I, P, P, I, I, I, I, D, D, P]
        lib.vsref_guided_upsample.restype = I
        lib.vsref_reproject.argtypes = [P, I, I, P, D, P]
        lib.vsref_reproject.restype = None
        lib.vsref_set_threads.argtypes = [I]
        lib.vsref_set_threads.restype = I
        lib.vsref_sp_message.argtypes = [P, I, D, D, D, P, P]
        lib.vsref_sp_message.restype = None
        lib.vsref_sp_forward.argtypes = [P, I, I, I, I, D, D, D, P, P]
        lib.vsref_sp_forward.restype = I
        lib.vsref_sp_backward.argtypes = [P, I, I, I, I, D, D, D, P, P, P, P]
        lib.vsref_sp_backward.restype = I
        _lib = lib
        return lib


def set_threads(n: int = 0) -> int:
    """Threads of the row loops (n <= 0 keeps the setting); returns the count in use."""
    return int(_load().vsref_set_threads(int(n)))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def rectify_remap(src: np.ndarray, cam, R=None, return_float: bool = False):
    """Section 2.1 remap of an (H, W, 3) uint8 frame; cam = (fx, fy, cx, cy, k1, k2)."""
    src = _u8(src)
    H, W, C = src.shape
    assert C == 3
    cam_a = np.ascontiguousarray(cam, dtype=np.float64)
    R_a = None if R is None else np.ascontiguousarray(R, dtype=np.float64).reshape(9)
    dst = np.zeros((H, W, 3), np.uint8)
    dst_f = np.zeros((H, W, 3), np.float64) if return_float else None
    rc = _load().vsref_rectify_remap(_ptr(src), W, H, 3 * W, _ptr(cam_a),
                                     None if R_a is None else _ptr(R_a),
                                     _ptr(dst), 3 * W, None if dst_f is None else _ptr(dst_f))
    _check(rc, "rectify_remap")
    return (dst, dst_f) if return_float else dst


def downsample_luma(rgb: np.ndarray, s: int):
    """Section 2.2 box-mean downsample by s; returns (low_rgb (h,w,3), low_gray (h,w))."""
    rgb = _u8(rgb)
    H, W, _ = rgb.shape
    w, h = -(-W // s), -(-H // s)
    low_rgb = np.zeros((h, w, 3), np.uint8)
    low_gray = np.zeros((h, w), np.uint8)
    rc = _load().vsref_downsample_luma(_ptr(rgb), W, H, 3 * W, s, _ptr(low_rgb), _ptr(low_gray))
    _check(rc, "downsample_luma")
    return low_rgb, low_gray


def cost_level0(left: np.ndarray, right: np.ndarray, L: int, Td: int) -> np.ndarray:
    """Eq. 1 data term at level 0, (h, w, L) int32."""
    left, right = _u8(left), _u8(right)
    h, w = left.shape
    out = np.zeros((h, w, L), np.int32)
    _load().vsref_cost_level0(_ptr(left), _ptr(right), w, h, L, Td, _ptr(out))
    return out


def cost_coarsen(fine: np.ndarray) -> np.ndarray:
    """One coarser pyramid level: sums of in-frame 2x2 children, (ceil(h/2), ceil(w/2), L)."""
    fine = np.ascontiguousarray(fine, dtype=np.int32)
    hf, wf, L = fine.shape
    out = np.zeros(((hf + 1) // 2, (wf + 1) // 2, L), np.int32)
    _load().vsref_cost_coarsen(_ptr(fine), wf, hf, L, _ptr(out))
    return out


def message(hv, c: int, Ts: int, mode: int = MSG_BRUTE) -> np.ndarray:
    """Eq. 1 normalised min-sum message from h(d') with smoothness min(c|d-d'|, Ts)."""
    hv = np.ascontiguousarray(hv, dtype=np.int32)
    out = np.zeros_like(hv)
    _load().vsref_message(_ptr(hv), hv.shape[0], c, Ts, mode, _ptr(out))
    return out


def bp(left: np.ndarray, right: np.ndarray, labels: int, levels: int, iters: int,
       data_trunc: int, smooth_slope: int, smooth_trunc: int, mode: int = MSG_BRUTE,
       return_messages: bool = False):
    """Eq. 1 hierarchical min-sum BP on an (h, w) grey pair; returns (h, w) uint8 labels.

    With ``return_messages`` also returns the final level-0 incoming messages,
    (4, h, w, labels) int32, directions 0 left, 1 right, 2 up, 3 down.
    """
    left, right = _u8(left), _u8(right)
    h, w = left.shape
    out = np.zeros((h, w), np.uint8)
    msgs = np.zeros((4, h, w, labels), np.int32) if return_messages else None
    rc = _load().vsref_bp(_ptr(left), _ptr(right), w, h, labels, levels, iters, data_trunc,
                          smooth_slope, smooth_trunc, mode, _ptr(out),
                          None if msgs is None else _ptr(msgs))
    _check(rc, "bp")
    return (out, msgs) if return_messages else out


def guided_upsample(labels: np.ndarray, guide_low: np.ndarray, guide_full: np.ndarray,
                    scale: int, radius: int, sigma_s: float, sigma_r: float) -> np.ndarray:
    """Eq. 2 joint bilateral upsampling; returns (H, W) float64 full-res disparity."""
    labels, guide_low, guide_full = _u8(labels), _u8(guide_low), _u8(guide_full)
    h, w = labels.shape
    H, W, _ = guide_full.shape
    assert guide_low.shape == (h, w, 3)
    disp = np.zeros((H, W), np.float64)
    rc = _load().vsref_guided_upsample(_ptr(labels), w, h, _ptr(guide_low), _ptr(guide_full),
                                       W, H, scale, radius, float(sigma_s), float(sigma_r), _ptr(disp))
    _check(rc, "guided_upsample")
    return disp


def reproject(disp: np.ndarray, cam, baseline: float) -> np.ndarray:
    """Eq. 3 reprojection; cam = (fx, fy, cx, cy, ...); returns (H, W, 3) float64."""
    disp = np.ascontiguousarray(disp, dtype=np.float64)
    H, W = disp.shape
    cam_a = np.ascontiguousarray(list(cam)[:4], dtype=np.float64)
    xyz = np.zeros((H, W, 3), np.float64)
    _load().vsref_reproject(_ptr(disp), W, H, _ptr(cam_a), float(baseline), _ptr(xyz))
    return xyz


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def sp_message(hv, lam: float, T: float, tau: float, return_unnormalised: bool = False):
    """Smoothed message -tau log sum_d' exp(-(h(d') + min(lam|d-d'|, T))/tau), mean-normalised."""
    hv = _f64(hv)
    out = np.zeros_like(hv)
    mt = np.zeros_like(hv)
    _load().vsref_sp_message(_ptr(hv), hv.shape[0], float(lam), float(T), float(tau),
                             _ptr(out), _ptr(mt))
    return (out, mt) if return_unnormalised else out


def sp_forward(D, lam: float, T: float, tau: float, iters: int, return_states: bool = False):
    """Synchronous smoothed BP on an (h, w, L) data term; returns (h, w, L) beliefs.

    With ``return_states`` also returns every iteration's incoming messages,
    (iters + 1, 4, h, w, L), slots 0 left, 1 right, 2 up, 3 down.
    """
    D = _f64(D)
    h, w, L = D.shape
    states = np.zeros((iters + 1, 4, h, w, L), np.float64)
    bel = np.zeros((h, w, L), np.float64)
    rc = _load().vsref_sp_forward(_ptr(D), w, h, L, iters, float(lam), float(T), float(tau),
                                  _ptr(states), _ptr(bel))
    _check(rc, "sp_forward")
    return (bel, states) if return_states else bel


def sp_backward(D, lam: float, T: float, tau: float, iters: int, gbel, states=None):
    """Reverse mode of :func:`sp_forward`: returns (dL/dD, dL/dlam, dL/dT, dL/dtau)."""
    D = _f64(D)
    h, w, L = D.shape
    if states is None:
        _, states = sp_forward(D, lam, T, tau, iters, return_states=True)
    states = _f64(states)
    gbel = _f64(gbel)
    assert gbel.shape == D.shape and states.shape == (iters + 1, 4, h, w, L)
    gD = np.zeros_like(D)
    gpar = np.zeros(3, np.float64)
    rc = _load().vsref_sp_backward(_ptr(D), w, h, L, iters, float(lam), float(T), float(tau),
                                   _ptr(states), _ptr(gbel), _ptr(gD), _ptr(gpar))
    _check(rc, "sp_backward")
    return gD, float(gpar[0]), float(gpar[1]), float(gpar[2])

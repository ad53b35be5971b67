"""CUDA renderer of the synthetic flight scenes (input generation only).

The stereo library never calls this.  :class:`GpuScene` uploads a
:class:`paper_1902_09733_b300.synth.FlightScene`'s tables once and draws
frames on the device with ``libvsrender.so`` (``vs_render.cu``), the same
pixels the host renderer draws (a test compares them), fast enough to feed a
1500-frame lawnmower flight to the streaming pipeline.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libvsrender.so")
_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(library_path):
                raise RuntimeError(f"{library_path} is missing: build it with `python -m paper_1902_09733_b300.build`")
            L = ctypes.CDLL(library_path)
            P, I, F, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double
            L.vsr_render.argtypes = [P, I, F, F, I, P, P, P, P, F, D, D, P, F, F, I, F, F, P, I, I, P, P]
            L.vsr_render.restype = I
            _lib = L
    return _lib


class GpuScene:
    """A flight scene's tables on the device, and frames drawn from them."""

    def __init__(self, scene, device="cuda"):
        t = scene.tables()
        self.device = torch.device(device)
        self.height = torch.from_numpy(t["height"]).to(self.device)
        self.n = int(t["height"].shape[0])
        self.half, self.res, self.nhalf = t["half"], t["res"], t["noise_half"]
        self.top, self.altitude = t["top"], t["altitude"]
        self.lats = [torch.from_numpy(lat).to(self.device) for _, _, lat in t["octaves"]]
        k = len(self.lats)
        self._lat = (ctypes.c_void_p * k)(*[x.data_ptr() for x in self.lats])
        self._m = (ctypes.c_int * k)(*[int(x.shape[0]) for x in self.lats])
        self._lam = (ctypes.c_float * k)(*[float(lam) for lam, _, _ in t["octaves"]])
        self._amp = (ctypes.c_double * k)(*[float(amp) for _, amp, _ in t["octaves"]])
        self.k = k

    def render(self, pose, cam, W: int = 2704, H: int = 1520, out=None, stream=None, depth=None) -> torch.Tensor:
        """(H, W, 3) uint8 device frame from pose (x, y, yaw); cam = fx, fy, cx, cy, k1, k2;
        depth: an optional (H, W) float32 device tensor that receives each pixel's z-depth."""
        if out is None:
            out = torch.empty((H, W, 3), dtype=torch.uint8, device=self.device)
        x, y, yaw = (float(v) for v in pose)
        cam6 = (ctypes.c_double * 6)(*[float(c) for c in cam])
        rotate = 0 if yaw == 0.0 else 1
        cosy, siny = float(np.float32(np.cos(yaw))), float(np.float32(np.sin(yaw)))
        st = None if stream is None else ctypes.c_void_p(stream.cuda_stream)
        rc = lib().vsr_render(self.height.data_ptr(), self.n, self.half, self.res, self.k, self._lat, self._m,
                              self._lam, self._amp, self.nhalf, self.top, self.altitude, cam6, x, y, rotate,
                              cosy, siny, out.data_ptr(), W, H,
                              depth.data_ptr() if depth is not None else None, st)
        if rc != 0:
            raise RuntimeError(f"vsr_render failed with status {rc}")
        return out

"""Seeded synthetic inputs for the virtual-stereo path.

This module only *makes inputs*.  It holds none of the arithmetic the stereo
path computes (no remap, cost, message, upsampling or reprojection code), so
the CUDA library and the CPU oracle can both be fed from it without sharing
any of the method.  Everything is numpy on the host and fully determined by
the seed.

Two workloads:

* :func:`noise_pair` -- a small grey pair: seeded uniform noise blurred with a
  Gaussian (sigma 1.5 px), and a right view made by warping it with a seeded
  piecewise-planar disparity field (four planes on the Voronoi cells of four
  seeded points, disparity 0..15).
* :func:`flight_frames` -- consecutive frames of a straight flight leg at
  100 m over terrain with box buildings; :class:`FlightScene` and
  :func:`lawnmower_path` -- the same kind of scene flown along a seeded
  lawnmower path (the streaming workload, rendered on the GPU by
  :mod:`paper_1902_09733_b300.scene`).
* :func:`terrain_pair` -- a 2.7K RGB pair of a seeded textured heightfield
  (value-noise fBm relief, independent colour-noise albedo) seen by a nadir
  pinhole camera with radial lens distortion; the right camera is displaced by
  the baseline along +x, so a left pixel u matches the right pixel u - d.
  :func:`pair_variants` turns one rendered pair into four distinct valid
  pairs (flips, and left/right swaps where a flip reverses the motion).
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

# ----------------------------------------------------------------------------
# helpers


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _gauss_blur(img: np.ndarray, sigma: float, radius: int) -> np.ndarray:
    """Separable Gaussian blur with mirror ('reflect') borders."""
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-(t * t) / (2.0 * sigma * sigma))
    k /= k.sum()
    pad = np.pad(img.astype(np.float64), radius, mode="reflect")
    h, w = img.shape
    tmp = np.zeros((h + 2 * radius, w), np.float64)
    for i, kv in enumerate(k):
        tmp += kv * pad[:, i:i + w]
    out = np.zeros((h, w), np.float64)
    for i, kv in enumerate(k):
        out += kv * tmp[i:i + h, :]
    return out


def _sample_rows_linear(img: np.ndarray, xs: np.ndarray) -> np.ndarray:
    """Linear interpolation of every row of img at fractional columns xs (edge clamped)."""
    h, w = img.shape
    xs = np.clip(xs, 0.0, w - 1.0)
    x0 = np.floor(xs).astype(np.int64)
    x1 = np.minimum(x0 + 1, w - 1)
    a = xs - x0
    rows = np.arange(h)[:, None]
    return (1.0 - a) * img[rows, x0] + a * img[rows, x1]


# ----------------------------------------------------------------------------
# small noise pair with a piecewise-planar disparity field


def noise_pair(seed: int, w: int = 160, h: int = 120, max_disp: float = 15.0,
               n_planes: int = 4, sigma: float = 1.5):
    """Grey pair (left, right) uint8 (h, w) and the left ground-truth disparity.

    The disparity field is defined on the right view: d_R(x, y) = a x + b y + c
    of the plane owning the nearest of ``n_planes`` seeded points, clipped to
    [0, max_disp]; IR(x, y) = IL(x + d_R(x, y), y) by linear interpolation of the
    blurred (unrounded) left image.  The left ground truth is obtained by
    forward-warping d_R (nearest pixel, larger disparity wins); pixels that no
    right pixel maps to are occluded and hold NaN.
    """
    g = _rng(seed)
    base = g.integers(0, 256, size=(h, w)).astype(np.float64)
    blurred = _gauss_blur(base, sigma, 5)
    left = np.clip(np.rint(blurred), 0, 255).astype(np.uint8)

    pts = np.stack([g.uniform(0, w, n_planes), g.uniform(0, h, n_planes)], axis=1)
    coef = np.stack([g.uniform(-0.04, 0.04, n_planes), g.uniform(-0.04, 0.04, n_planes),
                     g.uniform(0.0, max_disp, n_planes)], axis=1)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    dist = (xx[None] - pts[:, 0, None, None]) ** 2 + (yy[None] - pts[:, 1, None, None]) ** 2
    owner = np.argmin(dist, axis=0)
    a, b, c = coef[owner, 0], coef[owner, 1], coef[owner, 2]
    # each plane is centred on its seed point so the offset c is the disparity there
    d_r = a * (xx - pts[owner, 0]) + b * (yy - pts[owner, 1]) + c
    d_r = np.clip(d_r, 0.0, max_disp)

    right_f = _sample_rows_linear(blurred, xx + d_r)
    right = np.clip(np.rint(right_f), 0, 255).astype(np.uint8)

    gt = np.full((h, w), -np.inf)
    xl = np.rint(xx + d_r).astype(np.int64)
    ok = xl < w
    rows = np.broadcast_to(np.arange(h)[:, None], (h, w))
    np.maximum.at(gt, (rows[ok], xl[ok]), d_r[ok])
    gt[np.isinf(gt)] = np.nan
    return left, right, gt


# ----------------------------------------------------------------------------
# 2.7K textured terrain pair

# Camera of the full-resolution workload: fx, fy, cx, cy, k1, k2.
TERRAIN_CAMERA = (1400.0, 1400.0, 1351.5, 759.5, -0.25, 0.07)


class _ValueNoise:
    """Sum of octaves of smoothstep-interpolated lattice noise on the ground plane."""

    def __init__(self, g: np.random.Generator, wavelengths, amplitudes, extent: float, channels: int = 1):
        self.octaves = []
        for lam, amp in zip(wavelengths, amplitudes):
            n = int(np.ceil(extent / lam)) + 3
            lat = g.uniform(-1.0, 1.0, size=(n, n, channels)).astype(np.float32)
            self.octaves.append((float(lam), float(amp), lat))
        self.half = extent / 2.0

    def __call__(self, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        out = None
        for lam, amp, lat in self.octaves:
            n = lat.shape[0]
            gx = np.clip((X + self.half) / lam, 0.0, n - 2.001).astype(np.float32)
            gy = np.clip((Y + self.half) / lam, 0.0, n - 2.001).astype(np.float32)
            ix = gx.astype(np.int64)
            iy = gy.astype(np.int64)
            fx = gx - ix
            fy = gy - iy
            sx = (fx * fx * (3.0 - 2.0 * fx))[..., None]
            sy = (fy * fy * (3.0 - 2.0 * fy))[..., None]
            v00 = lat[iy, ix]
            v10 = lat[iy, ix + 1]
            v01 = lat[iy + 1, ix]
            v11 = lat[iy + 1, ix + 1]
            v = (v00 * (1 - sx) + v10 * sx) * (1 - sy) + (v01 * (1 - sx) + v11 * sx) * sy
            out = amp * v if out is None else out + amp * v
        return out


def _undistort_normalised(xd: np.ndarray, yd: np.ndarray, k1: float, k2: float, iters: int = 8):
    """Invert the radial lens model for the renderer (fixed-point iteration).

    The renderer needs, for every pixel of the *distorted* frame it draws, the
    ideal pinhole ray it sees; the radial factor is divided out repeatedly.
    """
    x = xd.copy()
    y = yd.copy()
    for _ in range(iters):
        r2 = x * x + y * y
        f = 1.0 + k1 * r2 + k2 * r2 * r2
        x = xd / f
        y = yd / f
    return x, y


class _HeightGrid:
    """Heights tabulated on a regular ground grid, sampled bilinearly (fast to march)."""

    def __init__(self, field, extent: float, n: int):
        self.half = extent / 2.0
        self.res = extent / (n - 1)
        g = np.linspace(-self.half, self.half, n)
        GX, GY = np.meshgrid(g, g)
        self.grid = np.ascontiguousarray(field(GX, GY)[..., 0], dtype=np.float32)
        self.flat = self.grid.ravel()
        self.n = n

    def __call__(self, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        n = self.n
        gx = np.clip((X + self.half) / self.res, 0.0, n - 1.001).astype(np.float32)
        gy = np.clip((Y + self.half) / self.res, 0.0, n - 1.001).astype(np.float32)
        ix = gx.astype(np.int32)
        iy = gy.astype(np.int32)
        fx = gx - ix
        fy = gy - iy
        base = iy * n + ix
        v00 = self.flat[base]
        v10 = self.flat[base + 1]
        v01 = self.flat[base + n]
        v11 = self.flat[base + n + 1]
        return (v00 + fx * (v10 - v00)) * (1 - fy) + (v01 + fx * (v11 - v01)) * fy


def _render_view(height: _HeightGrid, albedo: _ValueNoise, relief: float, W: int, H: int,
                 cam, cam_x: float, altitude: float, march_steps: int = 20,
                 refine_steps: int = 12, cam_y: float = 0.0, yaw: float = 0.0):
    """Nadir view from (cam_x, cam_y, altitude); the camera's x axis points
    along heading ``yaw`` (radians from the ground +x axis towards +y)."""
    fx, fy, cx, cy, k1, k2 = cam
    cos_y, sin_y = np.float32(np.cos(yaw)), np.float32(np.sin(yaw))
    out = np.zeros((H, W, 3), np.uint8)
    depth = np.zeros((H, W), np.float32)

    def band(r0: int, r1: int) -> None:
        vv, uu = np.mgrid[r0:r1, 0:W].astype(np.float64)
        xd = (uu - cx) / fx
        yd = (vv - cy) / fy
        xn, yn = _undistort_normalised(xd, yd, k1, k2)
        xn = xn.astype(np.float32)
        yn = yn.astype(np.float32)
        if yaw != 0.0:
            # ground direction of the ray: the camera axes turned by the heading
            xn, yn = cos_y * xn - sin_y * yn, sin_y * xn + cos_y * yn

        def surface_gap(t):
            # positive once the ray at depth t is at or below the surface
            return t - (altitude - height(cam_x + t * xn, cam_y + t * yn))

        t0 = np.float32(altitude - relief - 1e-3)
        step = np.float32((relief + 1e-3) / march_steps)
        t_lo = np.full(xn.shape, t0, np.float32)
        t_hi = np.full(xn.shape, altitude, np.float32)
        found = np.zeros(xn.shape, bool)
        for i in range(1, march_steps + 1):
            t = np.float32(t0 + i * step)
            hit = (surface_gap(t) >= 0.0) & ~found
            t_hi[hit] = t
            t_lo[hit] = t - step
            found |= hit
        for _ in range(refine_steps):
            tm = 0.5 * (t_lo + t_hi)
            below = surface_gap(tm) >= 0.0
            t_hi = np.where(below, tm, t_hi)
            t_lo = np.where(below, t_lo, tm)
        t = 0.5 * (t_lo + t_hi)
        X = cam_x + t * xn
        Y = cam_y + t * yn
        col = albedo(X, Y)
        shade = 0.75 + 0.25 * np.clip(height(X, Y)[..., None] / relief, 0.0, 1.0)
        rgb = np.clip(128.0 + 110.0 * col * shade, 0.0, 255.0)
        out[r0:r1] = np.rint(rgb).astype(np.uint8)
        depth[r0:r1] = t

    # row bands are independent; numpy releases the GIL inside each array op
    rows_per_band = 64
    bands = [(r0, min(H, r0 + rows_per_band)) for r0 in range(0, H, rows_per_band)]
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(lambda b: band(*b), bands))
    return out, depth


def terrain_pair(seed: int, W: int = 2704, H: int = 1520, cam=TERRAIN_CAMERA,
                 baseline: float = 0.5, altitude: float = 20.0, relief: float = 15.0,
                 return_depth: bool = False):
    """Left/right (H, W, 3) uint8 frames of a seeded textured heightfield.

    Nadir camera at ``altitude`` metres above the height datum; the terrain
    rises 0..``relief`` metres (value-noise fBm, wavelengths 40..5 m); albedo
    is independent colour value noise (wavelengths 0.8..0.1 m).  Both frames
    carry the radial distortion (k1, k2) of ``cam``; the right camera sits
    ``baseline`` metres along +x.  With ``return_depth`` the z-depth of every
    pixel of each frame along its own (undistorted) ray is returned too.
    """
    g = _rng(seed)
    extent = 2.0 * altitude * 1.4 + 4.0 * baseline + 8.0
    noise = _ValueNoise(g, [40.0, 20.0, 10.0, 5.0], [1.0, 0.5, 0.25, 0.125], extent)
    height = _HeightGrid(noise, extent, 1537)
    lo, hi = float(height.grid.min()), float(height.grid.max())
    height.grid = ((height.grid - lo) * (relief / max(hi - lo, 1e-6))).astype(np.float32)
    height.flat = height.grid.ravel()
    albedo = _ValueNoise(g, [0.8, 0.4, 0.2, 0.1], [0.5, 0.3, 0.2, 0.15], extent, channels=3)
    left, dl = _render_view(height, albedo, relief, W, H, cam, 0.0, altitude)
    right, dr = _render_view(height, albedo, relief, W, H, cam, baseline, altitude)
    if return_depth:
        return left, right, dl, dr
    return left, right


class FlightScene:
    """Terrain with box buildings under a nadir camera at ``altitude`` metres.

    The terrain is value-noise fBm (0..``relief`` m, wavelengths 40..5 m
    scaled by altitude / 20); ``n_buildings`` seeded boxes rise 5..30 m above
    the highest ground they cover; the albedo is colour value noise whose
    wavelengths scale the same way, so texture stays at a few low-resolution
    pixels.  The scene covers ``extent`` metres square around the origin.
    :meth:`render` draws a frame on the host; :meth:`tables` hands the same
    tables to the CUDA renderer (:mod:`paper_1902_09733_b300.scene`).
    """

    def __init__(self, seed: int, extent: float, altitude: float = 100.0, relief: float = 15.0,
                 n_buildings: int = 40, grid: int = 2049, building_heights=(5.0, 30.0)):
        g = _rng(seed)
        scale = altitude / 20.0
        self.altitude = float(altitude)
        self.extent = float(extent)
        noise = _ValueNoise(g, [40.0 * scale, 20.0 * scale, 10.0 * scale, 5.0 * scale], [1.0, 0.5, 0.25, 0.125],
                            extent)
        height = _HeightGrid(noise, extent, grid)
        lo, hi = float(height.grid.min()), float(height.grid.max())
        hgrid = ((height.grid - lo) * (relief / max(hi - lo, 1e-6))).astype(np.float32)
        n = hgrid.shape[0]
        cells = np.linspace(-extent / 2.0, extent / 2.0, n)
        for _ in range(n_buildings):
            cx0, cy0 = g.uniform(-extent / 2 + 10, extent / 2 - 10, size=2)
            sx, sy = g.uniform(6.0, 25.0, size=2)
            top = g.uniform(*building_heights)
            ix = np.where(np.abs(cells - cx0) <= sx / 2)[0]
            iy = np.where(np.abs(cells - cy0) <= sy / 2)[0]
            if ix.size and iy.size:
                block = hgrid[iy[0]:iy[-1] + 1, ix[0]:ix[-1] + 1]
                hgrid[iy[0]:iy[-1] + 1, ix[0]:ix[-1] + 1] = float(block.max()) + top
        height.grid = hgrid
        height.flat = hgrid.ravel()
        self.height = height
        self.top = float(hgrid.max())
        self.albedo = _ValueNoise(g, [0.8 * scale, 0.4 * scale, 0.2 * scale, 0.1 * scale], [0.5, 0.3, 0.2, 0.15],
                                  extent, channels=3)

    def render(self, pose, W: int = 2704, H: int = 1520, cam=TERRAIN_CAMERA, return_depth: bool = False):
        """(H, W, 3) uint8 frame from pose (x, y, yaw) with the radial distortion of ``cam``; with
        ``return_depth`` also the (H, W) float32 z-depth of each pixel along its undistorted ray.

        Camera frame of a pose: z = depth below the camera, (x, y) = the ground offset from the
        camera turned by -yaw, so that u = fx x / z + cx and v = fy y / z + cy (undistorted)."""
        x, y, yaw = pose
        frame, depth = _render_view(self.height, self.albedo, self.top, W, H, cam, float(x), self.altitude,
                                    cam_y=float(y), yaw=float(yaw))
        return (frame, depth) if return_depth else frame

    def tables(self):
        """The renderer's inputs as contiguous float32 arrays: the height grid
        (n x n), its half extent and cell size, and per albedo octave its
        wavelength, amplitude and (m x m x 3) lattice."""
        octs = [(lam, amp, np.ascontiguousarray(lat, np.float32)) for lam, amp, lat in self.albedo.octaves]
        return {"height": np.ascontiguousarray(self.height.grid, np.float32), "half": float(self.height.half),
                "res": float(self.height.res), "noise_half": float(self.albedo.half), "octaves": octs,
                "top": self.top, "altitude": self.altitude}


def lawnmower_path(seed: int, n_frames: int, spacing: float = 0.05, leg: float = 25.0, radius: float = 8.0):
    """Camera poses (x, y, yaw) of a lawnmower flight, ``spacing`` metres apart.

    Straight legs of ``leg`` metres along +x and -x alternate, joined by
    half-circle turns of ``radius`` metres (left, then right, ...), each new
    leg 2 ``radius`` further along +y.  The camera's heading follows the
    flight direction, so consecutive frames move along the camera's x axis
    (on a turn they also rotate by spacing / radius radians per frame).  The
    seed shifts the start by up to 2 m.  Returns an (n_frames, 3) array.
    """
    g = _rng(seed + 7919)
    x0, y0 = -leg / 2.0 + g.uniform(-2.0, 2.0), g.uniform(-2.0, 2.0)
    half_turn = np.pi * radius
    period = 2.0 * (leg + half_turn)
    poses = np.zeros((n_frames, 3))
    for i in range(n_frames):
        s = i * spacing
        k, r = divmod(s, period)
        ybase = y0 + 4.0 * radius * k
        if r < leg:                                   # +x leg
            poses[i] = (x0 + r, ybase, 0.0)
        elif r < leg + half_turn:                     # left turn, heading 0 -> pi
            psi = (r - leg) / radius
            cxp, cyp = x0 + leg, ybase + radius
            poses[i] = (cxp + radius * np.sin(psi), cyp - radius * np.cos(psi), psi)
        elif r < 2.0 * leg + half_turn:               # -x leg
            poses[i] = (x0 + leg - (r - leg - half_turn), ybase + 2.0 * radius, np.pi)
        else:                                         # right turn, heading pi -> 0
            psi = np.pi - (r - 2.0 * leg - half_turn) / radius
            cxp, cyp = x0, ybase + 3.0 * radius
            poses[i] = (cxp - radius * np.sin(psi), cyp + radius * np.cos(psi), psi)
    return poses


def relative_pose(pose1, pose2):
    """[R, T] taking camera-frame points of pose 1 to camera-frame points of
    pose 2 (both nadir at the same altitude, frames as in FlightScene.render):
    a turn by yaw1 - yaw2 about the optical axis and the ground offset of the
    two cameras turned into camera 2's axes."""
    x1, y1, a1 = pose1
    x2, y2, a2 = pose2
    d = a1 - a2
    R = np.array([[np.cos(d), -np.sin(d), 0.0], [np.sin(d), np.cos(d), 0.0], [0.0, 0.0, 1.0]])
    c, s = np.cos(-a2), np.sin(-a2)
    T = np.array([c * (x1 - x2) - s * (y1 - y2), s * (x1 - x2) + c * (y1 - y2), 0.0])
    return R, T


def lawnmower_extent(poses, altitude: float = 100.0, W: int = 2704, H: int = 1520, cam=TERRAIN_CAMERA) -> float:
    """Square scene extent that holds every frame's ground footprint (with the
    lens's outward distortion and a building-height margin) for these poses."""
    fx, fy = cam[0], cam[1]
    reach = 1.15 * altitude * 0.5 * np.hypot(W / fx, H / fy)
    span = max(np.abs(poses[:, 0]).max(), np.abs(poses[:, 1]).max())
    return float(2.0 * (span + reach) + 10.0)


def flight_frames(seed: int, n_frames: int, spacing: float = 0.05, altitude: float = 100.0,
                  W: int = 2704, H: int = 1520, cam=TERRAIN_CAMERA, relief: float = 15.0,
                  n_buildings: int = 40):
    """Frames of a straight flight leg over a terrain with box buildings.

    The nadir camera flies along +x at ``altitude`` metres, ``spacing`` metres
    per frame (3 m/s at 60 fps gives 0.05 m), over a :class:`FlightScene`.
    Yields (H, W, 3) uint8 frames with the radial distortion of ``cam``.
    """
    leg = spacing * max(n_frames - 1, 0)
    scene = FlightScene(seed, 2.0 * altitude * 1.4 + leg + 8.0, altitude, relief, n_buildings)
    x0 = -leg / 2.0
    for i in range(n_frames):
        yield scene.render((x0 + i * spacing, 0.0, 0.0), W, H, cam)


def pair_variants(left: np.ndarray, right: np.ndarray):
    """Four distinct valid stereo pairs from one rendered pair.

    A vertical flip keeps the horizontal motion; a horizontal flip (or a 180
    degree turn) reverses it, so the two frames swap roles.
    """
    return [
        (left, right),
        (np.ascontiguousarray(left[::-1]), np.ascontiguousarray(right[::-1])),
        (np.ascontiguousarray(right[:, ::-1]), np.ascontiguousarray(left[:, ::-1])),
        (np.ascontiguousarray(right[::-1, ::-1]), np.ascontiguousarray(left[::-1, ::-1])),
    ]

"""Plain CPU oracle of the pose path of Section 2.3 (Eq. 4-7).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU legs of ``bench.py`` may import this module; the CUDA library never
does, and the two share no code.  numpy, int64 for the integer stages and
float64 for EPnP.

Steps, in the order of Section 2.3:

* :func:`harris_response25` -- Eq. 4 and Eq. 5: image derivatives A and B,
  the Gaussian-windowed second-moment matrix M, the response R = det M - k
  (tr M)^2 with k = 0.04, returned as 25 R so that it is an exact integer.
* :func:`harris_corners` -- Section 3.2: the image divided into a grid of
  cells, in each cell the strongest local maximum of R above a threshold.
* :func:`zssd_match` -- correspondences of the corners in a second frame
  within a search range, by zero-mean sum of squared differences of patches.
* :func:`epnp` -- Eq. 6 and Eq. 7 (the cited O(n) algorithm): the points as
  weighted sums of four control points, the control points in the camera
  frame from the null space of the linear system, and [R, T] from them.
* :func:`pose_average` -- the poses of a later pair's left and right images,
  averaged (the right one moved to the left camera through the virtual rig).

Readings where the paper is silent (also listed in the design notes):
derivatives are central differences of the integer luma (77 R + 150 G + 29 B
+ 128) >> 8 with the frame edge repeated; the Gaussian window is the 5 x 5
binomial [1 4 6 4 1]^T [1 4 6 4 1] (a discrete Gaussian, sigma 1; taps
outside the frame are skipped); k = 0.04; a local maximum beats each of its
8 neighbours in (R, then the smaller raster index); in each cell the largest
(R, smaller index) wins; ZSSD ties go to the first displacement in raster
order (dy, then dx), followed by a parabola through the costs of the two
neighbouring displacements on each axis (sub-pixel position); EPnP keeps the
solution of N = 1, 2 or 3 null-space vectors (each refined by Gauss-Newton)
with the smallest reprojection error, the equations of Eq. 6 taken in
normalised image coordinates (divided by fx and fy); at least 6 points (with 4 or 5 the
null space of the linear system has more than the 3 directions searched).
"""
from __future__ import annotations

import numpy as np

K_INV = 25                              # k = 0.04 = 1 / 25
BINOMIAL = np.array([1, 4, 6, 4, 1], np.int64)


def grey(rgb: np.ndarray) -> np.ndarray:
    """Integer luma of an (H, W, 3) uint8 frame, as int64."""
    c = rgb.astype(np.int64)
    return (77 * c[..., 0] + 150 * c[..., 1] + 29 * c[..., 2] + 128) >> 8


def _shift(img: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """img[y + dy, x + dx] where inside the frame, else 0."""
    H, W = img.shape
    out = np.zeros_like(img)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    if ys < ye and xs < xe:
        out[ys:ye, xs:xe] = img[ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def harris_response25(rgb: np.ndarray) -> np.ndarray:
    """25 R of Eq. 5 at every pixel, int64 (H, W).

    Eq. 4: the change of intensity under a small shift (x, y) is (x, y) M
    (x, y)^T with M = sum over the window of w [A^2, AB; AB, B^2], A and B the
    first-order derivatives; Eq. 5: R = det M - k tr(M)^2.  With k = 1/25,
    25 R = 25 det M - tr(M)^2 is an integer."""
    g = grey(rgb)
    gp = np.pad(g, 1, mode="edge")
    A = gp[1:-1, 2:] - gp[1:-1, :-2]         # d/dx, central difference
    B = gp[2:, 1:-1] - gp[:-2, 1:-1]         # d/dy
    prods = (A * A, B * B, A * B)
    S = [np.zeros_like(g) for _ in range(3)]
    for i in range(5):
        for j in range(5):
            w = BINOMIAL[i] * BINOMIAL[j]
            for s, p in zip(S, prods):
                s += w * _shift(p, i - 2, j - 2)
    sxx, syy, sxy = S
    return K_INV * (sxx * syy - sxy * sxy) - (sxx + syy) ** 2


def harris_corners(r25: np.ndarray, grid: int = 30, margin: int = 8, threshold25: int = 0) -> np.ndarray:
    """(grid * grid, 2) int corners (x, y), one per cell in row-major cell
    order, (-1, -1) where a cell has none.

    Cell (gx, gy) holds x in [gx W / grid, (gx + 1) W / grid) and y likewise
    (integer division).  A candidate lies at least ``margin`` pixels inside
    the frame, has 25 R > threshold25, and is a local maximum: none of its 8
    neighbours has a larger R, or an equal R at a smaller raster index.  The
    cell's corner is its candidate with the largest R (the smaller raster
    index on ties)."""
    H, W = r25.shape
    idx = np.arange(H * W, dtype=np.int64).reshape(H, W)
    big = np.iinfo(np.int64).min
    rp = np.pad(r25, 1, constant_values=big)
    ip = np.pad(idx, 1, constant_values=-1)
    is_max = np.ones((H, W), bool)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            rq = rp[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            iq = ip[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            beats = (rq > r25) | ((rq == r25) & (iq >= 0) & (iq < idx))
            is_max &= ~beats
    yy, xx = np.mgrid[0:H, 0:W]
    cand = is_max & (r25 > threshold25) & (xx >= margin) & (xx < W - margin) & (yy >= margin) & (yy < H - margin)
    out = np.full((grid * grid, 2), -1, np.int64)
    for gy in range(grid):
        y0, y1 = gy * H // grid, (gy + 1) * H // grid
        for gx in range(grid):
            x0, x1 = gx * W // grid, (gx + 1) * W // grid
            c = cand[y0:y1, x0:x1]
            if not c.any():
                continue
            r = np.where(c, r25[y0:y1, x0:x1], big)
            k = int(np.argmax(r))            # first of the largest: the smaller raster index
            out[gy * grid + gx] = (x0 + k % (x1 - x0), y0 + k // (x1 - x0))
    return out


def zssd_match(rgb1: np.ndarray, rgb2: np.ndarray, corners: np.ndarray, radius: int = 5, search: int = 16):
    """Matches of the corners of frame 1 in frame 2: (n, 2) float positions
    (x, y) (NaN where a corner is (-1, -1) or no displacement fits), (n,)
    int64 costs n Z with n = (2 radius + 1)^2.

    For the patch P1 around corner p in frame 1 and the patch P2 around p + d
    in frame 2, d in [-search, search]^2 with P2 inside frame 2, the zero-mean
    SSD is Z = sum((P1 - mean P1) - (P2 - mean P2))^2; n Z = n sum(D^2) -
    (sum D)^2 with D = P1 - P2 is exact in integers.  The smallest wins (the
    first in raster order of (dy, dx) on ties); then on each axis the
    parabola through the costs at d - 1, d, d + 1 moves the match by (c- -
    c+) / (2 (c- - 2 c0 + c+)) where both neighbours exist and the
    denominator is positive."""
    g1, g2 = grey(rgb1), grey(rgb2)
    H, W = g1.shape
    r, S = radius, search
    npx = (2 * r + 1) ** 2
    pos = np.full((len(corners), 2), np.nan)
    cost = np.full(len(corners), -1, np.int64)
    # frame 2 padded by the search range; padding marks displacements whose patch leaves the frame
    pad = S + r
    g2p = np.pad(g2, pad, constant_values=-1)
    for ci, (x, y) in enumerate(corners):
        if x < 0 or not (r <= x < W - r and r <= y < H - r):
            continue
        P1 = g1[y - r:y + r + 1, x - r:x + r + 1]
        region = g2p[y + pad - S - r:y + pad + S + r + 1, x + pad - S - r:x + pad + S + r + 1]
        win = np.lib.stride_tricks.sliding_window_view(region, (2 * r + 1, 2 * r + 1))   # (2S+1, 2S+1, p, p)
        valid = (win >= 0).all(axis=(2, 3))
        D = P1[None, None] - win
        Z = npx * (D * D).sum(axis=(2, 3)) - D.sum(axis=(2, 3)) ** 2
        Z = np.where(valid, Z, -1)
        if not valid.any():
            continue
        zz = np.where(valid, Z, np.iinfo(np.int64).max)
        k = int(np.argmin(zz))                # the first in raster order of (dy, dx) on ties
        by, bx = divmod(k, 2 * S + 1)
        c0 = int(Z[by, bx])
        off = [0.0, 0.0]
        for axis, (ya, xa, yb, xb) in enumerate(((by, bx - 1, by, bx + 1), (by - 1, bx, by + 1, bx))):
            if min(ya, xa) >= 0 and max(yb, xb) <= 2 * S and valid[ya, xa] and valid[yb, xb]:
                cm, cp = int(Z[ya, xa]), int(Z[yb, xb])
                den = cm - 2 * c0 + cp
                if den > 0:
                    off[axis] = (cm - cp) / (2.0 * den)
        pos[ci] = (x + bx - S + off[0], y + by - S + off[1])
        cost[ci] = c0
    return pos, cost


# ---------------------------------------------------------------------------
# EPnP (Eq. 6, Eq. 7)

_PAIRS = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def _control_points(P: np.ndarray) -> np.ndarray:
    """The four world control points: the centroid, and the centroid plus the
    principal axes scaled by the root of their variance."""
    c0 = P.mean(axis=0)
    Q = P - c0
    lam, V = np.linalg.eigh(Q.T @ Q / len(P))
    # each axis with its largest-magnitude component positive (a fixed choice of the
    # eigenvectors' signs, so that the control points do not depend on the eigen-solver)
    for k in range(3):
        if V[np.argmax(np.abs(V[:, k])), k] < 0:
            V[:, k] = -V[:, k]
    cw = [c0]
    for k in (2, 1, 0):
        cw.append(c0 + np.sqrt(max(lam[k], 0.0)) * V[:, k])
    return np.array(cw)


def _alphas(P: np.ndarray, cw: np.ndarray) -> np.ndarray:
    """Barycentric coordinates: P_i = sum_j alpha_ij c_j with sum_j alpha_ij = 1."""
    C = (cw[1:] - cw[0]).T
    a = np.linalg.solve(C, (P - cw[0]).T).T
    return np.column_stack([1.0 - a.sum(axis=1), a])


def _pose_from_betas(betas, V4, alphas, P, uv, cam):
    fx, fy, cx, cy = cam
    x = sum(b * V4[:, k] for k, b in enumerate(betas))
    cc = x.reshape(4, 3)
    pc = alphas @ cc
    if (pc[:, 2] < 0).sum() > len(pc) / 2:   # the sign of the null vector: points in front
        cc, pc = -cc, -pc
    # Eq. 7 for the points: [R, T] from the world points and their camera-frame positions
    mw, mc = P.mean(axis=0), pc.mean(axis=0)
    Hm = (pc - mc).T @ (P - mw)
    U, _, Vt = np.linalg.svd(Hm)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt))])
    R = U @ D @ Vt
    T = mc - R @ mw
    proj = (R @ P.T).T + T
    u = fx * proj[:, 0] / proj[:, 2] + cx
    v = fy * proj[:, 1] / proj[:, 2] + cy
    err = np.sqrt((u - uv[:, 0]) ** 2 + (v - uv[:, 1]) ** 2).mean()
    return R, T, err


def _gauss_newton(betas, V4, dw, iters=5):
    """Refine the four betas on the six control-point distance residuals."""
    b = np.array(list(betas) + [0.0] * (4 - len(betas)), float)
    vd = [np.array([V4[3 * i:3 * i + 3, k] - V4[3 * j:3 * j + 3, k] for (i, j) in _PAIRS]) for k in range(4)]
    for _ in range(iters):
        J = np.zeros((6, 4))
        r = np.zeros(6)
        for p in range(6):
            d = sum(b[k] * vd[k][p] for k in range(4))
            r[p] = d @ d - dw[p]
            for k in range(4):
                J[p, k] = 2.0 * d @ vd[k][p]
        step, *_ = np.linalg.lstsq(J, -r, rcond=None)
        b = b + step
    return b


def epnp(P: np.ndarray, uv: np.ndarray, cam):
    """[R, T] with camera point = R P + T, from n >= 6 world points P (n, 3)
    and their pixels uv (n, 2) in a camera of intrinsics cam = (fx, fy, cx,
    cy); returns (R, T, mean reprojection error in pixels)."""
    P = np.asarray(P, float)
    uv = np.asarray(uv, float)
    fx, fy, cx, cy = cam
    cw = _control_points(P)
    alphas = _alphas(P, cw)
    # Eq. 6: w_i [u_i, 1] = A sum_j alpha_ij c_j^c gives two equations per point; divided by
    # fx and fy they read in normalised image coordinates (the same equations, a 12 x 12
    # normal matrix of order 1 instead of fx^2, whose smallest eigenvectors come out accurate)
    n = len(P)
    un, vn = (uv[:, 0] - cx) / fx, (uv[:, 1] - cy) / fy
    M = np.zeros((2 * n, 12))
    for j in range(4):
        M[0::2, 3 * j + 0] = alphas[:, j]
        M[0::2, 3 * j + 2] = -alphas[:, j] * un
        M[1::2, 3 * j + 1] = alphas[:, j]
        M[1::2, 3 * j + 2] = -alphas[:, j] * vn
    _, Vm = np.linalg.eigh(M.T @ M)
    V4 = Vm[:, :4]                            # the four smallest eigenvalues
    dw = np.array([np.sum((cw[i] - cw[j]) ** 2) for (i, j) in _PAIRS])
    # products of the null-vector differences for the distance constraints
    vd = [np.array([V4[3 * i:3 * i + 3, k] - V4[3 * j:3 * j + 3, k] for (i, j) in _PAIRS]) for k in range(4)]
    cands = []
    # N = 1: beta scales the first vector so that the distances match
    d1 = np.linalg.norm(vd[0], axis=1)
    b1 = np.sum(d1 * np.sqrt(dw)) / np.sum(d1 * d1)
    cands.append([b1])
    # N = 2: ||b1 v1 + b2 v2||^2 = dw, linear in (b1^2, b1 b2, b2^2)
    L2 = np.column_stack([np.sum(vd[0] * vd[0], 1), 2 * np.sum(vd[0] * vd[1], 1), np.sum(vd[1] * vd[1], 1)])
    s2, *_ = np.linalg.lstsq(L2, dw, rcond=None)
    b1 = np.sqrt(abs(s2[0]))                  # the overall sign is fixed by the depths later
    cands.append([b1, np.sign(s2[1]) * np.sqrt(abs(s2[2]))])
    # N = 3: six products (b1^2, b1 b2, b2^2, b1 b3, b2 b3, b3^2)
    L3 = np.column_stack([np.sum(vd[0] * vd[0], 1), 2 * np.sum(vd[0] * vd[1], 1), np.sum(vd[1] * vd[1], 1),
                          2 * np.sum(vd[0] * vd[2], 1), 2 * np.sum(vd[1] * vd[2], 1), np.sum(vd[2] * vd[2], 1)])
    s3, *_ = np.linalg.lstsq(L3, dw, rcond=None)
    b1 = np.sqrt(abs(s3[0]))
    cands.append([b1, s3[1] / b1, s3[3] / b1] if b1 > 0 else [0.0, 0.0, 0.0])
    best = None
    for c in cands:
        b = _gauss_newton(c, V4, dw)
        R, T, err = _pose_from_betas(b, V4, alphas, P, uv, cam)
        if best is None or err < best[2]:
            best = (R, T, err)
    return best


def epnp_inliers(P: np.ndarray, uv: np.ndarray, cam, threshold: float = 2.0, rounds: int = 2):
    """EPnP, then again on the points whose reprojection error is below
    max(threshold, 3 x the median error), ``rounds`` times (a reading: the
    paper names no outlier step, and a few wrong matches pull the plain
    least-squares solution along the rotation-translation ambiguity of a
    far, nearly flat scene).  Returns (R, T, mean error of the inliers,
    inlier mask)."""
    P = np.asarray(P, float)
    uv = np.asarray(uv, float)
    keep = np.ones(len(P), bool)
    fx, fy, cx, cy = cam
    R, T, err = epnp(P, uv, cam)
    for _ in range(rounds):
        pc = (R @ P.T).T + T
        e = np.hypot(fx * pc[:, 0] / pc[:, 2] + cx - uv[:, 0], fy * pc[:, 1] / pc[:, 2] + cy - uv[:, 1])
        keep = e < max(threshold, 3.0 * float(np.median(e)))
        if keep.sum() < 6:
            break
        R, T, err = epnp(P[keep], uv[keep], cam)
    return R, T, err, keep


def pose_average(RL, TL, RR, TR, baseline: float):
    """Section 2.3: the relative pose of a later stereo pair estimated from
    its left image and from its right image, averaged.

    Both estimates map frame-1 left-camera points to the later pair's
    cameras: (RL, TL) to its left camera, (RR, TR) to its right camera.  The
    virtual rig (a reading: the paper states only that it averages the left
    and right poses) has the right camera ``baseline`` metres along the left
    camera's +x with the same orientation, p_right = p_left - (baseline, 0,
    0), so the right estimate gives the left camera's pose as (RR, TR + b).
    The rotations are averaged by their chordal mean (the rotation nearest
    to RL + RR, the polar factor of the sum; for two rotations the geodesic
    midpoint), the translations arithmetically.  An estimate with a NaN
    entry is left out; with both, NaN.  Returns (R, T)."""
    b = np.array([baseline, 0.0, 0.0])
    cand = []
    for R, T in ((RL, TL), (RR, TR + b if TR is not None else None)):
        if R is None or T is None:
            continue
        R, T = np.asarray(R, float), np.asarray(T, float)
        if np.isfinite(R).all() and np.isfinite(T).all():
            cand.append((R, T))
    if not cand:
        return np.full((3, 3), np.nan), np.full(3, np.nan)
    if len(cand) == 1:
        return cand[0]
    M = cand[0][0] + cand[1][0]
    U, _, Vt = np.linalg.svd(M)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt))])
    return U @ D @ Vt, 0.5 * (cand[0][1] + cand[1][1])

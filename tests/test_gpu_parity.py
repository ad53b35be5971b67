"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer stages (BP labels, BP messages, downsample, grey) must match bit for
bit.  The remap output is within 1 LSB of the FP64 oracle (a rounding tie can
flip); the FP32 upsampled disparity within 1e-4 * max(|d|, 1) and the point
cloud within 1e-4 relative of the FP64 oracle run on the same inputs.
Every BP case runs on the GPU's own downsampled inputs, so remap rounding
cannot leak into the integer comparison.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_09733_b300 as vs
from paper_1902_09733_b300 import build, synth

pytestmark = pytest.mark.gpu

CAM2K = vs.Camera(*synth.TERRAIN_CAMERA)
BP_CFG1 = vs.BPParams(labels=16, levels=3, iters=5, data_trunc=20, smooth_slope=10, smooth_trunc=40)
BP_CFG2 = vs.BPParams(labels=64, levels=4, iters=10, data_trunc=20, smooth_slope=10, smooth_trunc=40)
JBU_CFG2 = vs.JBUParams(scale=4, radius=2, sigma_s=1.0, sigma_r=12.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    vs.lib()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def run_bp(left, right, p: vs.BPParams, messages=False):
    L, R = dev(left), dev(right)
    # random bytes in the workspace: the path must not depend on its contents
    n = vs.bp_workspace_size(left.shape[1], left.shape[0], p)
    ws = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda")
    lab = vs.bp_stereo(L, R, p, workspace=ws)
    if messages:
        m = vs.bp_export_messages(ws, left.shape[1], left.shape[0], p)
        return host(lab), host(m)
    return host(lab)


def oracle_bp(left, right, p: vs.BPParams, mode=oracle.MSG_BRUTE):
    return oracle.bp(left, right, p.labels, p.levels, p.iters, p.data_trunc, p.smooth_slope,
                     p.smooth_trunc, mode=mode, return_messages=True)


def assert_bp_parity(left, right, p, mode=oracle.MSG_BRUTE):
    lab, msg = run_bp(left, right, p, messages=True)
    olab, omsg = oracle_bp(left, right, p, mode)
    np.testing.assert_array_equal(msg, omsg)
    np.testing.assert_array_equal(lab, olab)
    return lab


# ---------------------------------------------------------------------------
# Eq. 1


def test_bp_hand_chain_and_grid():
    IL = np.array([[50, 52, 50]], np.uint8)
    IR = np.array([[47, 61, 64]], np.uint8)
    for levels, iters in ((1, 1), (1, 2), (2, 1), (2, 3)):
        p = vs.BPParams(3, levels, iters, 20, 4, 6)
        assert_bp_parity(IL, IR, p)
        assert_bp_parity(IL.T.copy(), IR.T.copy(), p)
    IL = np.array([[10, 20, 30], [40, 50, 60], [70, 80, 90]], np.uint8)
    IR = np.array([[12, 13, 27], [41, 38, 65], [70, 84, 79]], np.uint8)
    for levels, iters in ((2, 1), (2, 2), (1, 4)):
        assert_bp_parity(IL, IR, vs.BPParams(2, levels, iters, 20, 3, 5))


@pytest.mark.parametrize("seed", range(4))
def test_bp_config1_noise_pairs(seed):
    """160x120, 16 labels, 3 levels x 5 iterations, min(|IL-IR|, 20), min(10|dp-dq|, 40)."""
    left, right, _ = synth.noise_pair(seed)
    assert_bp_parity(left, right, BP_CFG1)


@pytest.mark.parametrize("h,w,p", [
    (7, 13, vs.BPParams(5, 3, 3, 20, 4, 12)),
    (1, 37, vs.BPParams(9, 2, 4, 20, 3, 9)),
    (29, 1, vs.BPParams(9, 3, 4, 20, 3, 9)),
    (33, 65, vs.BPParams(37, 4, 6, 25, 6, 30)),
    (17, 23, vs.BPParams(128, 3, 2, 20, 10, 40)),
    (21, 40, vs.BPParams(48, 2, 3, 20, 10, 40)),
    (20, 41, vs.BPParams(64, 3, 1, 20, 10, 40)),     # one iteration per level
    (19, 30, vs.BPParams(80, 2, 2, 15, 50, 40)),     # slope above the truncation
    (18, 35, vs.BPParams(96, 1, 3, 20, 0, 40)),      # no smoothness
    (16, 27, vs.BPParams(112, 2, 2, 0, 10, 40)),     # no data term
    (15, 26, vs.BPParams(100, 4, 2, 127, 127, 127)),  # largest truncations
    (70, 90, vs.BPParams(20, 6, 3, 20, 7, 40)),      # six levels, down to 3x2
    (1, 1, vs.BPParams(4, 3, 2, 20, 5, 10)),
    (23, 31, vs.BPParams(24, 3, 3, 60, 8, 30)),     # level-1 costs in bytes above 127
    (22, 34, vs.BPParams(32, 2, 3, 63, 9, 48)),
    (26, 36, vs.BPParams(16, 3, 4, 15, 10, 45)),    # byte-lane sums at levels 0 and 1
])
def test_bp_ragged_and_edge_cases(h, w, p):
    g = np.random.default_rng(h * 1000 + w)
    left = g.integers(0, 256, size=(h, w)).astype(np.uint8)
    right = np.clip(np.roll(left, 3, axis=1).astype(int) + g.integers(-6, 7, size=(h, w)), 0, 255).astype(np.uint8)
    assert_bp_parity(left, right, p, mode=oracle.MSG_DT if p.labels > 40 else oracle.MSG_BRUTE)


def test_bp_full_size_config2_and_determinism():
    """676x380 (2704x1520 / 4), 64 labels, 4 levels x 10 iterations: the launch
    configuration of the benchmark, bit-exact against the oracle (DT mode,
    itself pinned to the brute-force definition), and bit-identical twice."""
    left, right, _ = synth.noise_pair(11, w=676, h=380, max_disp=40.0)
    lab = assert_bp_parity(left, right, BP_CFG2, mode=oracle.MSG_DT)
    lab2, msg2 = run_bp(left, right, BP_CFG2, messages=True)
    np.testing.assert_array_equal(lab, lab2)


def test_bp_workspace_reuse_needs_no_initialisation():
    p = vs.BPParams(16, 3, 4, 20, 10, 40)
    a_l, a_r, _ = synth.noise_pair(1, w=64, h=48)
    b_l, b_r, _ = synth.noise_pair(2, w=64, h=48)
    ws = torch.full((vs.bp_workspace_size(64, 48, p),), 0xAB, dtype=torch.uint8, device="cuda")
    la = host(vs.bp_stereo(dev(a_l), dev(a_r), p, workspace=ws))
    lb = host(vs.bp_stereo(dev(b_l), dev(b_r), p, workspace=ws))
    la2 = host(vs.bp_stereo(dev(a_l), dev(a_r), p, workspace=ws))
    np.testing.assert_array_equal(la, la2)
    np.testing.assert_array_equal(la, oracle_bp(a_l, a_r, p)[0])
    np.testing.assert_array_equal(lb, oracle_bp(b_l, b_r, p)[0])


def test_bp_pitched_rows():
    left, right, _ = synth.noise_pair(5, w=50, h=30)
    big_l = np.zeros((30, 64), np.uint8)
    big_r = np.zeros((30, 64), np.uint8)
    big_l[:, :50], big_r[:, :50] = left, right
    L, R = dev(big_l)[:, :50], dev(big_r)[:, :50]
    out = torch.zeros((30, 80), dtype=torch.uint8, device="cuda")
    vs.bp_stereo(L, R, BP_CFG1, labels=out[:, :50])
    got = host(out)
    np.testing.assert_array_equal(got[:, :50], oracle_bp(left, right, BP_CFG1)[0])
    assert not got[:, 50:].any()


@pytest.mark.parametrize("p", [
    vs.BPParams(64, 3, 2, 20, 10, 40),    # level-1 costs in bytes
    vs.BPParams(40, 2, 2, 70, 6, 50),     # level-1 costs in 16 bits, a partial label chunk
    vs.BPParams(17, 1, 3, 20, 10, 40),    # one level: no level-1 sums
])
def test_bp_wide_rows_at_odd_addresses(p):
    """Rows of 150 bytes at an odd start and an odd pitch: the data term reads
    the right image in aligned words whatever the row alignment, and falls back
    to byte loads at both edges and on padding labels."""
    left, right, _ = synth.noise_pair(21, w=150, h=37, max_disp=30.0)
    big_l = np.zeros((37, 203), np.uint8)
    big_r = np.zeros((37, 203), np.uint8)
    big_l[:, 1:151], big_r[:, 1:151] = left, right
    L, R = dev(big_l)[:, 1:151], dev(big_r)[:, 1:151]
    n = vs.bp_workspace_size(150, 37, p)
    ws = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda")
    lab = vs.bp_stereo(L, R, p, workspace=ws)
    msg = vs.bp_export_messages(ws, 150, 37, p)
    olab, omsg = oracle_bp(left, right, p, mode=oracle.MSG_DT)
    np.testing.assert_array_equal(host(msg), omsg)
    np.testing.assert_array_equal(host(lab), olab)


def test_bp_rejects_small_workspace():
    left, right, _ = synth.noise_pair(0, w=32, h=24)
    ws = torch.empty(100, dtype=torch.uint8, device="cuda")
    with pytest.raises(vs.VSError) as e:
        vs.bp_stereo(dev(left), dev(right), BP_CFG1, workspace=ws)
    assert e.value.code == vs.VS_EWORKSPACE


# ---------------------------------------------------------------------------
# Section 2.1 / 2.2


def _check_remap(src, cam, R, s):
    # both sides see the same (float32) camera and rotation
    cam = vs.Camera(*[float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy, cam.k1, cam.k2)])
    if R is not None:
        R = np.asarray(R, np.float32).astype(np.float64)
    d, lr, lg = vs.rectify_remap(dev(src), cam, R=R, scale=s)
    d, lr, lg = host(d), host(lr), host(lg)
    want = oracle.rectify_remap(src, (cam.fx, cam.fy, cam.cx, cam.cy, cam.k1, cam.k2), R=R)
    diff = np.abs(d.astype(int) - want.astype(int))
    assert diff.max() <= 1
    wl, wg = oracle.downsample_luma(d, s)
    np.testing.assert_array_equal(lr, wl)
    np.testing.assert_array_equal(lg, wg)
    return diff


@pytest.mark.parametrize("H,W,s", [(48, 64, 4), (45, 61, 4), (37, 50, 3), (20, 33, 1), (64, 80, 16),
                                   (46, 68, 2), (48, 72, 8), (96, 160, 8), (34, 132, 2)])
def test_remap_downsample_small(H, W, s):
    g = np.random.default_rng(H * W)
    src = g.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    cam = vs.Camera(0.6 * W, 0.62 * W, (W - 1) / 2 + 0.3, (H - 1) / 2 - 0.2, -0.25, 0.07)
    _check_remap(src, cam, None, s)
    c, sn = np.cos(0.03), np.sin(0.03)
    R = np.array([[c, 0, sn], [0, 1, 0], [-sn, 0, c]]) @ np.array([[1, 0, 0], [0, c, -sn], [0, sn, c]])
    _check_remap(src, cam, R, s)


def test_remap_strong_pincushion_reads_taps_from_global_memory():
    """A pincushion lens spreads one destination tile over a source window
    larger than the shared-memory stage, which takes the direct-read path."""
    g = np.random.default_rng(13)
    src = g.integers(0, 256, size=(150, 200, 3)).astype(np.uint8)
    _check_remap(src, vs.Camera(60.0, 60.0, 99.5, 74.5, 1.5, 0.5), None, 4)


def test_remap_identity_is_exact():
    g = np.random.default_rng(9)
    src = g.integers(0, 256, size=(30, 41, 3)).astype(np.uint8)
    d, _, _ = vs.rectify_remap(dev(src), vs.Camera(40, 35, 20.0, 14.5), scale=4)
    np.testing.assert_array_equal(host(d), src)


def test_remap_full_size_terrain_frame():
    left, _ = synth.terrain_pair(0)
    diff = _check_remap(left, CAM2K, None, 4)
    assert (diff > 0).mean() < 1e-3      # only rounding ties may flip


@pytest.mark.parametrize("s", [2, 4, 8])
def test_remap_block_kernel_matches_general_kernel(s):
    """Word-aligned rows at scales 2, 4 and 8 take the block kernel, rows at
    an odd pitch the general one: same bytes on the 2.7K frame, with and
    without the full-resolution and low-res RGB outputs."""
    left, _ = synth.terrain_pair(0)
    H, W, _ = left.shape
    d1, lr1, lg1 = vs.rectify_remap(dev(left), CAM2K, scale=s)
    big = torch.zeros((H, W + 1, 3), dtype=torch.uint8, device="cuda")
    big[:, :W] = dev(left)
    d2, lr2, lg2 = vs.rectify_remap(big[:, :W], CAM2K, scale=s)
    _, _, lg3 = vs.rectify_remap(dev(left), CAM2K, scale=s, dst=None, low_rgb=None)
    np.testing.assert_array_equal(host(d1), host(d2))
    np.testing.assert_array_equal(host(lr1), host(lr2))
    np.testing.assert_array_equal(host(lg1), host(lg2))
    np.testing.assert_array_equal(host(lg1), host(lg3))


@pytest.mark.parametrize("s", [2, 4, 8])
def test_remap_block_kernel_with_rays_leaving_the_frame(s):
    """Strong pincushion on a frame the block kernel takes: many quads fall
    back to the per-pixel sampler near the border."""
    g = np.random.default_rng(14)
    src = g.integers(0, 256, size=(144, 200, 3)).astype(np.uint8)
    _check_remap(src, vs.Camera(60.0, 60.0, 99.5, 71.5, 1.5, 0.5), None, s)


def test_remap_pitched_and_low_only():
    g = np.random.default_rng(12)
    H, W = 40, 52
    src = g.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    big = torch.zeros((H, W + 7, 3), dtype=torch.uint8, device="cuda")
    big[:, :W] = dev(src)
    cam = vs.Camera(30, 30, 25.5, 19.5, -0.2, 0.05)
    d, lr, lg = vs.rectify_remap(big[:, :W], cam, scale=4)
    _, lr2, lg2 = vs.rectify_remap(dev(src), cam, scale=4, dst=None)
    np.testing.assert_array_equal(host(lr), host(lr2))
    np.testing.assert_array_equal(host(lg), host(lg2))


# ---------------------------------------------------------------------------
# Eq. 2 / Eq. 3


def _jbu_inputs(seed, H, W, s, smooth=True):
    g = np.random.default_rng(seed)
    gf = g.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    if smooth:
        gf = np.clip(gf // 4 + 96, 0, 255).astype(np.uint8)
    gl, _ = oracle.downsample_luma(gf, s)
    h, w = gl.shape[:2]
    lab = g.integers(0, 64, size=(h, w)).astype(np.uint8)
    return lab, gl, gf


def _assert_disp_close(a, b):
    np.testing.assert_array_less(np.abs(a.astype(np.float64) - b), 1e-4 * np.maximum(np.abs(b), 1.0) + 1e-12)


def _assert_xyz_close(a, b, disp_ref):
    """Points within 1e-4 relative.  Where the reference disparity is itself
    within the disparity tolerance of 0 (|d| <= 1e-4) the point is at
    infinity and FP32 may give d = 0 (no point, NaN): either is accepted."""
    edge = np.abs(disp_ref) <= 1e-4
    nan_a, nan_b = np.isnan(a).any(-1), np.isnan(b).any(-1)
    np.testing.assert_array_equal(nan_a[~edge], nan_b[~edge])
    ok = ~nan_b & ~edge
    err = np.linalg.norm(a[ok].astype(np.float64) - b[ok], axis=-1)
    assert (err <= 1e-4 * np.linalg.norm(b[ok], axis=-1) + 1e-12).all()


@pytest.mark.parametrize("H,W,jp", [
    (40, 64, vs.JBUParams(4, 2, 1.0, 12.0)),
    (43, 45, vs.JBUParams(4, 2, 1.0, 12.0)),
    (30, 31, vs.JBUParams(3, 1, 0.7, 20.0)),
    (17, 70, vs.JBUParams(1, 3, 1.5, 8.0)),
    (64, 96, vs.JBUParams(8, 2, 1.0, 3.0)),
    (24, 40, vs.JBUParams(2, 0, 1.0, 12.0)),
    (42, 48, vs.JBUParams(4, 1, 0.8, 10.0)),    # scale-4 kernel, ragged last block row
    (36, 52, vs.JBUParams(4, 3, 1.2, 15.0)),
    (16, 16, vs.JBUParams(4, 0, 1.0, 12.0)),
    (45, 68, vs.JBUParams(4, 2, 1.0, 12.0)),
    (40, 64, vs.JBUParams(4, 2, 1.0, 5000.0)),  # flat range term: frame-edge taps must stay out
    (30, 62, vs.JBUParams(2, 2, 1.0, 5000.0)),
    (44, 60, vs.JBUParams(4, 3, 0.25, 12.0)),   # spatial spread beyond the scale-4 kernel's range
    (40, 64, vs.JBUParams(4, 2, 1.0, 2.0)),     # narrow range term: many pixels' weights underflow
    (151, 260, vs.JBUParams(2, 2, 1.0, 12.0)),  # scale-2 block kernel over several CTAs, odd height
    (200, 520, vs.JBUParams(8, 2, 1.0, 12.0)),  # scale-8 block kernel (rows in a loop) over several CTAs
    (203, 264, vs.JBUParams(8, 3, 0.6, 9.0)),   # scale 8, ragged last block row
])
def test_jbu_and_reproject_small(H, W, jp):
    for smooth in (True, False):
        lab, gl, gf = _jbu_inputs(H + W, H, W, jp.scale, smooth)
        lab[:3, :3] = 0                  # a corner whose windows see only d = 0 -> NaN points
        disp = host(vs.guided_upsample(dev(lab), dev(gl), dev(gf), jp))
        want = oracle.guided_upsample(lab, gl, gf, jp.scale, jp.radius, jp.sigma_s, jp.sigma_r)
        _assert_disp_close(disp, want)
        cam = vs.Camera(1400.0, 1380.0, (W - 1) / 2, (H - 1) / 2)
        d2, xyz = vs.guided_upsample_reproject(dev(lab), dev(gl), dev(gf), jp, cam, 0.5)
        np.testing.assert_array_equal(host(d2), disp)
        _assert_xyz_close(host(xyz), oracle.reproject(want, (cam.fx, cam.fy, cam.cx, cam.cy), 0.5), want)


def test_reproject_standalone_and_nan():
    g = np.random.default_rng(3)
    disp = g.uniform(-5, 140, size=(30, 50)).astype(np.float32)
    disp[0, :5] = 0.0
    disp[1, 0] = np.nan
    cam = vs.Camera(1400.0, 1390.0, 24.5, 14.5)
    xyz = host(vs.reproject(dev(disp), cam, 0.5))
    _assert_xyz_close(xyz, oracle.reproject(disp.astype(np.float64), (cam.fx, cam.fy, cam.cx, cam.cy), 0.5), disp)
    assert np.isnan(xyz[disp <= 0]).all() and np.isnan(xyz[1, 0]).all()


# ---------------------------------------------------------------------------
# whole pair at 2.7K


@pytest.fixture(scope="module")
def terrain():
    return synth.terrain_pair(0)


def _pair_cfg():
    return vs.PairConfig(2704, 1520, CAM2K, 0.5, BP_CFG2, JBU_CFG2)


@pytest.mark.parametrize("s", [2, 4, 8])
def test_pair_driver_matches_frame_by_frame_calls(s):
    """The pair driver remaps both frames in one launch of the block kernel
    (the lens model of each quad once, both frames sampled at it); its cloud
    equals, bit for bit, the one from the public per-frame calls."""
    W, H = 1024, 568   # a multiple of 8 both ways; 568 = 71 x 8 leaves ragged CTA rows
    rng = np.random.default_rng(40 + s)
    left = (rng.integers(0, 256, (H, W, 3))).astype(np.uint8)
    right = np.roll(left, -3 * s, axis=1)
    bp = vs.BPParams(labels=32, levels=3, iters=5, data_trunc=20, smooth_slope=10, smooth_trunc=40)
    jbu = vs.JBUParams(scale=s, radius=2, sigma_s=1.0, sigma_r=12.0)
    cfg = vs.PairConfig(W, H, CAM2K, 0.5, bp, jbu)
    dl, lrl, lgl = vs.rectify_remap(dev(left), cfg.cam, scale=s)
    _, _, lgr = vs.rectify_remap(dev(right), cfg.cam, scale=s, dst=None, low_rgb=None)
    lab = vs.bp_stereo(lgl, lgr, cfg.bp)
    _, xyz = vs.guided_upsample_reproject(lab, lrl, dl, cfg.jbu, cfg.cam, cfg.baseline)
    _, xyz2 = vs.pair_run(cfg, dev(left), dev(right))
    np.testing.assert_array_equal(host(xyz2), host(xyz))


def test_full_pair_stage_by_stage(terrain):
    """The 2.7K pipeline of the benchmark, each stage against the oracle on the
    GPU's own inputs to that stage."""
    left, right = terrain
    cfg = _pair_cfg()
    dl, lrl, lgl = vs.rectify_remap(dev(left), cfg.cam, scale=4)
    _, _, lgr = vs.rectify_remap(dev(right), cfg.cam, scale=4, dst=None, low_rgb=None)
    lab = vs.bp_stereo(lgl, lgr, cfg.bp)
    disp, xyz = vs.guided_upsample_reproject(lab, lrl, dl, cfg.jbu, cfg.cam, cfg.baseline)
    dl_h, lrl_h, lgl_h, lgr_h, lab_h = host(dl), host(lrl), host(lgl), host(lgr), host(lab)
    # remap + downsample
    want = oracle.rectify_remap(left, synth.TERRAIN_CAMERA)
    assert np.abs(dl_h.astype(int) - want.astype(int)).max() <= 1
    wl, wg = oracle.downsample_luma(dl_h, 4)
    np.testing.assert_array_equal(lrl_h, wl)
    np.testing.assert_array_equal(lgl_h, wg)
    # BP, bit-exact
    np.testing.assert_array_equal(lab_h, oracle.bp(lgl_h, lgr_h, 64, 4, 10, 20, 10, 40, mode=oracle.MSG_DT))
    # upsample + reprojection against the FP64 oracle on every pixel
    want_d = oracle.guided_upsample(lab_h, lrl_h, dl_h, 4, 2, 1.0, 12.0)
    disp_h, xyz_h = host(disp), host(xyz)
    _assert_disp_close(disp_h, want_d)
    _assert_xyz_close(xyz_h, oracle.reproject(want_d, synth.TERRAIN_CAMERA, 0.5), want_d)
    # the driver entry points give the same bits
    _, xyz2 = vs.pair_run(cfg, dev(left), dev(right))
    np.testing.assert_array_equal(host(xyz2), xyz_h)
    lh = torch.from_numpy(left).pin_memory()
    rh = torch.from_numpy(right).pin_memory()
    xh = torch.empty((1520, 2704, 3), dtype=torch.float32).pin_memory()
    dev_in = torch.empty(2 * left.size, dtype=torch.uint8, device="cuda")
    dev_xyz = torch.empty((1520, 2704, 3), dtype=torch.float32, device="cuda")
    ws = torch.empty(vs.pair_workspace_size(cfg), dtype=torch.uint8, device="cuda")
    vs.pair_run_host(cfg, lh, rh, xh, dev_in, dev_xyz, ws)
    np.testing.assert_array_equal(xh.numpy(), xyz_h)

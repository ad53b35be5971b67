"""Host-side checks of the C ABI: the library loads, exports every entry point
that include/vstereo.h declares, and rejects bad arguments before touching
the GPU.  No CUDA device is needed (no kernel is launched)."""
import ctypes
import os
import re

import pytest

import paper_1902_09733_b300 as vs
from paper_1902_09733_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return vs.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "vstereo.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vs_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.vs_status_string(code)
    assert vs.status_string(-3).startswith("workspace")


def test_workspace_sizes_and_parameter_ranges(lib):
    ok = vs.BPParams(labels=64, levels=4, iters=10, data_trunc=20, smooth_slope=10, smooth_trunc=40,
                     iters_per_tile=1)
    n = vs.bp_workspace_size(676, 380, ok)
    # level 0: costs 2*380*338*64 + messages 8*380*338*64 bytes; coarser levels add about a third
    lvl0 = 10 * 380 * 338 * 64
    assert lvl0 < n < 1.45 * lvl0
    # fused sweeps add a second message buffer: the largest coarse level in the
    # automatic mode (level 1: 8*190*176*64 bytes with its rows padded to
    # 16-slot groups), level 0 (8*380*352*64) when every level may be fused
    auto = vs.bp_workspace_size(676, 380, vs.BPParams(**{**ok.__dict__, "iters_per_tile": 0}))
    assert auto - n == 8 * 190 * 176 * 64
    every = vs.bp_workspace_size(676, 380, vs.BPParams(**{**ok.__dict__, "iters_per_tile": 3}))
    assert every - n == 8 * 380 * 352 * 64
    bad = [
        dict(labels=1), dict(labels=257), dict(levels=0), dict(levels=9), dict(iters=0),
        dict(smooth_trunc=65536), dict(smooth_slope=-1), dict(data_trunc=-1), dict(smooth_trunc=-1),
        dict(levels=8, data_trunc=20000),         # 20000 * 4^7 is beyond 2^28
        dict(iters_per_tile=-1), dict(iters_per_tile=65),
    ]
    for b in bad:
        p = vs.BPParams(**{**ok.__dict__, **b})
        assert vs.bp_workspace_size(676, 380, p) == 0, b
    # the general path (16-bit messages, int32 data terms in 32-label lane blocks) beyond the byte
    # path's limits: 256 labels, truncations above 127, coarse sums beyond 16 bits
    for b, Lp in ((dict(labels=129), 256), (dict(labels=256), 256), (dict(data_trunc=128), 64),
                  (dict(smooth_trunc=200), 64), (dict(levels=7, data_trunc=20), 64), (dict(labels=40), 64)):
        p = vs.BPParams(**{**ok.__dict__, **b})
        n = vs.bp_workspace_size(676, 380, p)
        if b == dict(labels=40):
            assert n < 1.45 * lvl0            # the byte path
            continue
        lvl0_wide = 2 * 380 * 338 * Lp * (4 + 4 * 2)
        assert lvl0_wide < n < 1.45 * lvl0_wide + 4096, (b, n)
    assert vs.bp_workspace_size(0, 10, ok) == 0
    cfg = vs.PairConfig(2704, 1520, vs.Camera(1400, 1400, 1351.5, 759.5, -0.25, 0.07), 0.5, ok, vs.JBUParams())
    assert vs.pair_workspace_size(cfg) > n + 2 * 2704 * 1520 * 3


def test_bad_arguments_are_rejected_on_the_host(lib):
    p = vs._BPParams(16, 3, 5, 20, 10, 40)
    # NULL images, bad pitch, missing workspace: rejected before any launch
    assert lib.vs_bp_stereo(None, None, 160, 120, 160, ctypes.byref(p), None, 160, None, 0, None) == vs.VS_EINVAL
    fake = 1 << 20   # never dereferenced: the checks fail first
    assert lib.vs_bp_stereo(fake, fake, 160, 120, 100, ctypes.byref(p), fake, 160, fake, 1 << 30, None) == vs.VS_EINVAL
    assert lib.vs_bp_stereo(fake, fake, 160, 120, 160, ctypes.byref(p), fake, 160, None, 0, None) == vs.VS_EWORKSPACE
    assert lib.vs_bp_stereo(fake, fake, 160, 120, 160, ctypes.byref(p), fake, 160, fake + 16, 1 << 30, None) == vs.VS_EWORKSPACE
    assert lib.vs_bp_stereo(fake, fake, 160, 120, 160, ctypes.byref(p), fake, 160, fake, 100, None) == vs.VS_EWORKSPACE
    cam = vs._Camera(1400, 1400, 1351.5, 759.5, -0.25, 0.07)
    assert lib.vs_rectify_remap(None, 10, 10, 30, ctypes.byref(cam), None, fake, 30, 4, None, 0, None, 0, None) == vs.VS_EINVAL
    assert lib.vs_rectify_remap(fake, 10, 10, 20, ctypes.byref(cam), None, fake, 30, 4, None, 0, None, 0, None) == vs.VS_EINVAL
    assert lib.vs_rectify_remap(fake, 10, 10, 30, ctypes.byref(cam), None, fake, 30, 17, fake, 9, None, 0, None) == vs.VS_EINVAL
    badcam = vs._Camera(0, 1400, 1351.5, 759.5, 0, 0)
    assert lib.vs_rectify_remap(fake, 10, 10, 30, ctypes.byref(badcam), None, fake, 30, 4, None, 0, None, 0, None) == vs.VS_EINVAL
    j = vs._JBUParams(4, 2, 1.0, 12.0)
    # low-res size must be ceil(W / s)
    assert lib.vs_guided_upsample(fake, 10, 10, 10, fake, 30, fake, 48, 40, 144, ctypes.byref(j), fake, None) == vs.VS_EINVAL
    j0 = vs._JBUParams(4, 2, 0.0, 12.0)
    assert lib.vs_guided_upsample(fake, 12, 10, 12, fake, 36, fake, 48, 40, 144, ctypes.byref(j0), fake, None) == vs.VS_EINVAL
    jr = vs._JBUParams(4, 4, 1.0, 12.0)
    assert lib.vs_guided_upsample(fake, 12, 10, 12, fake, 36, fake, 48, 40, 144, ctypes.byref(jr), fake, None) == vs.VS_EINVAL
    assert lib.vs_reproject(fake, 10, 10, ctypes.byref(cam), 0.0, fake, None) == vs.VS_EINVAL
    assert lib.vs_reproject(fake, 10, 10, ctypes.byref(cam), -1.0, fake, None) == vs.VS_EINVAL
    # the BP status read-out checks its workspace before touching the device
    bad_bp = vs._BPParams(1, 3, 5, 20, 10, 40)
    assert lib.vs_bp_status(fake, 1 << 30, 160, 120, ctypes.byref(bad_bp), None) == vs.VS_EINVAL
    assert lib.vs_bp_status(None, 1 << 30, 160, 120, ctypes.byref(p), None) == vs.VS_EWORKSPACE
    assert lib.vs_bp_status(fake, 100, 160, 120, ctypes.byref(p), None) == vs.VS_EWORKSPACE
    assert lib.vs_bp_status(fake + 16, 1 << 30, 160, 120, ctypes.byref(p), None) == vs.VS_EWORKSPACE
    # sweep variants: -1 (automatic) .. 4 (staged)
    assert lib.vs_bp_select_sweep(5) == vs.VS_EINVAL
    assert lib.vs_bp_select_sweep(-2) == vs.VS_EINVAL
    assert lib.vs_bp_test_withhold_copies(2) == vs.VS_EINVAL
    # fused tiles: both sides or neither, lanes 0, 1, 2 or 4
    for args in ((-1, 4, 0), (4, 0, 0), (0, 4, 0), (4, 4, 3), (2000, 4, 1)):
        assert lib.vs_bp_select_fused(*args) == vs.VS_EINVAL, args
    assert lib.vs_bp_select_fused(0, 0, 0) == vs.VS_OK
    # the product library carries no bounds checks
    assert lib.vs_check_report(None) == -1
    assert lib.vs_check_test_shrink(256) == vs.VS_EINVAL


def test_pipeline_host_checks(lib):
    cfg = vs.PairConfig(2704, 1520, vs.Camera(1400, 1400, 1351.5, 759.5, -0.25, 0.07), 0.5,
                        vs.BPParams(), vs.JBUParams()).c()
    pairs = lib.vs_pipeline_workspace_size(ctypes.byref(cfg), 0, 3, 1)
    flight = lib.vs_pipeline_workspace_size(ctypes.byref(cfg), 1, 3, 3)
    assert pairs > 3 * (2 * 2704 * 1520 * 3 + 2704 * 1520 * 12)
    assert flight > 4 * 2704 * 1520 * 3
    for mode, depth, k in ((2, 3, 1), (0, 0, 1), (0, 17, 1), (1, 3, 0), (1, 3, 65)):
        assert lib.vs_pipeline_workspace_size(ctypes.byref(cfg), mode, depth, k) == 0
    h = ctypes.c_void_p()
    # checks fail before any CUDA object is created
    assert lib.vs_pipeline_create(ctypes.byref(cfg), 0, 3, 1, None, 0, ctypes.byref(h)) == vs.VS_EWORKSPACE
    assert lib.vs_pipeline_create(ctypes.byref(cfg), 5, 3, 1, None, 0, ctypes.byref(h)) == vs.VS_EINVAL
    assert lib.vs_pipeline_submit_pair(None, None, None, None) == vs.VS_EINVAL
    assert lib.vs_pipeline_flush(None) == vs.VS_EINVAL


def test_batch_workspace_is_the_sum_of_the_pairs(lib):
    import torch
    shapes = [(120, 160, 16), (61, 97, 64), (45, 33, 128)]
    pairs = [(torch.empty((h, w), dtype=torch.uint8), None, vs.BPParams(L, 3, 4, 20, 10, 40)) for h, w, L in shapes]
    total = vs.bp_batch_workspace_size(pairs)
    singles = sum(vs.bp_workspace_size(w, h, vs.BPParams(L, 3, 4, 20, 10, 40)) for h, w, L in shapes)
    assert singles <= total <= singles + 256 * len(shapes)
    pairs[1] = (pairs[1][0], None, vs.BPParams(64, 3, 5, 20, 10, 40))     # different iters
    assert vs.bp_batch_workspace_size(pairs) == 0


def test_pair_batch_workspace_is_the_sum_of_the_pairs(lib):
    import torch
    jobs = []
    for W, H, s, L in ((2704, 1520, 4, 64), (1000, 600, 2, 128), (640, 360, 8, 32)):
        cfg = vs.PairConfig(W, H, vs.Camera(1400, 1400, W / 2, H / 2, -0.25, 0.07), 0.5,
                            vs.BPParams(L, 4, 10, 20, 10, 40), vs.JBUParams(s, 2, 1.0, 12.0))
        t = torch.empty((H, W, 3), dtype=torch.uint8)
        jobs.append((cfg, t, t, None, torch.empty((H, W, 3))))
    total = vs.pair_batch_workspace_size(jobs)
    singles = sum(vs.pair_workspace_size(j[0]) for j in jobs)
    assert singles <= total <= singles + 256 * len(jobs)
    bad = (vs.PairConfig(0, 10, jobs[0][0].cam, 0.5, vs.BPParams(), vs.JBUParams()),) + jobs[0][1:]
    assert vs.pair_batch_workspace_size(jobs + [bad]) == 0


def test_smooth_bp_workspace_and_host_checks(lib):
    ok = vs.SPParams(labels=48, iters=8, ckpt_every=2, lam=2.5, trunc=13.7, tau=2.0)
    n = vs.sp_workspace_size(338, 190, ok)
    state = 16 * 338 * 190 * 48
    # checkpoints of iterations 2, 4, 6 + one recompute state + two adjoint states
    assert 6 * state <= n < 6 * state + 6 * 256 + (4 * 338 * 190 // 128 + 1) * 32 + 512
    # every ckpt interval gives floor((iters-1)/k) + min(k, iters) + 1 states
    for k in range(1, 9):
        p = vs.SPParams(**{**ok.__dict__, "ckpt_every": k})
        states = (8 - 1) // k + min(k, 8) + 1
        assert states * state <= vs.sp_workspace_size(338, 190, p) < (states + 1) * state
    bad = [dict(labels=40), dict(labels=8), dict(labels=128), dict(iters=0), dict(iters=65),
           dict(ckpt_every=0), dict(ckpt_every=9), dict(tau=0.0), dict(tau=-1.0), dict(lam=-0.5),
           dict(trunc=-1.0), dict(trunc=101.0, tau=2.0), dict(lam=float("nan")), dict(tau=float("inf"))]
    for b in bad:
        p = vs.SPParams(**{**ok.__dict__, **b})
        assert vs.sp_workspace_size(338, 190, p) == 0, b
    assert vs.sp_workspace_size(0, 190, ok) == 0
    assert vs.sp_workspace_size(4096, 1025, ok) == 0          # more than 2^22 pixels
    c = ok.c()
    bad_p = vs.SPParams(**{**ok.__dict__, "labels": 40}).c()
    assert lib.vs_sp_forward(None, 338, 190, ctypes.byref(c), None, None, 0, None) == vs.VS_EINVAL
    assert lib.vs_sp_forward(16, 338, 190, ctypes.byref(bad_p), 16, 256, 1 << 30, None) == vs.VS_EINVAL
    assert lib.vs_sp_forward(20, 338, 190, ctypes.byref(c), 16, 256, 1 << 30, None) == vs.VS_EALIGN
    assert lib.vs_sp_forward(16, 338, 190, ctypes.byref(c), 16, 256, 1024, None) == vs.VS_EWORKSPACE
    assert lib.vs_sp_forward(16, 338, 190, ctypes.byref(c), 16, 100, 1 << 30, None) == vs.VS_EWORKSPACE
    assert lib.vs_sp_backward(16, 338, 190, ctypes.byref(c), 16, 16, None, 256, 1 << 30, None) == vs.VS_EINVAL
    assert lib.vs_sp_backward(16, 338, 190, ctypes.byref(c), 16, 24, 16, 256, 1 << 30, None) == vs.VS_EALIGN
    assert lib.vs_sp_backward(16, 338, 190, ctypes.byref(c), 16, 16, 16, 256, 64, None) == vs.VS_EWORKSPACE
    assert lib.vs_sp_select_kernels(2) == vs.VS_EINVAL
    assert lib.vs_sp_status(256, 64, 338, 190, ctypes.byref(c), None) == vs.VS_EWORKSPACE
    assert lib.vs_sp_status(256, 1 << 30, 338, 190, ctypes.byref(bad_p), None) == vs.VS_EINVAL


def test_pose_workspaces_and_host_checks(lib):
    p = vs.PoseParams(grid=30, margin=40, threshold25=0, radius=5, search=32)
    single = vs.pose_workspace_size(2704, 1520, p)
    stereo = vs.pose_stereo_workspace_size(2704, 1520, p)
    assert single >= 2704 * 1520 * 8
    # a second set of matches and points (pos 16, cost 8, P 24, uv 16 bytes per cell) and two outputs
    assert single + 900 * 64 <= stereo <= single + 900 * 64 + 8 * 256
    bad = vs.PoseParams(grid=30, margin=5, threshold25=0, radius=5, search=32)   # margin < radius + 1
    assert vs.pose_stereo_workspace_size(2704, 1520, bad) == 0
    c = vs.Camera(1400.0, 1400.0, 1351.5, 759.5).c()
    pp = p.c()
    fake = 256
    assert lib.vs_pose_average(None, fake, 0.15, fake, None) == vs.VS_EINVAL
    assert lib.vs_pose_average(fake, fake, float("nan"), fake, None) == vs.VS_EINVAL
    assert lib.vs_pose_estimate_stereo(fake, fake, None, fake, 2704, 1520, 3 * 2704, ctypes.byref(c), 0.15,
                                       ctypes.byref(pp), fake, fake, stereo, None) == vs.VS_EINVAL
    assert lib.vs_pose_estimate_stereo(fake, fake, fake, fake, 2704, 1520, 3 * 2704, ctypes.byref(c), 0.15,
                                       ctypes.byref(pp), fake, fake, stereo - 1, None) == vs.VS_EWORKSPACE
    assert lib.vs_pose_estimate_stereo(fake, fake, fake, fake, 2704, 1520, 3 * 2704, ctypes.byref(c),
                                       float("inf"), ctypes.byref(pp), fake, fake, stereo, None) == vs.VS_EINVAL

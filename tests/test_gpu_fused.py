"""Fused sweeps (several red-black iterations per launch, each CTA iterating a
shared-memory tile whose halo shrinks by one pixel per iteration) against the
oracle.  How the iterations are launched must never change what they compute:
labels and final level-0 messages are compared bit for bit, on odd sizes, with
tiles forced small so that every launch has many tile edges, and with every
lane count of the distance transform."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_09733_b300 as vs
from paper_1902_09733_b300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available()
    build.build()


@pytest.fixture(autouse=True)
def _restore():
    yield
    vs.bp_select_fused(0, 0, 0)
    vs.bp_select_sweep(-1)


def _pair(seed, h, w):
    left, right, _ = synth.noise_pair(seed, w=w, h=h, max_disp=min(12.0, w / 4))
    return torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), left, right


def _run(L_, R_, p, random_ws=True):
    h, w = L_.shape
    n = vs.bp_workspace_size(w, h, p)
    ws = (torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda") if random_ws
          else torch.zeros(n, dtype=torch.uint8, device="cuda"))
    lab = vs.bp_stereo(L_, R_, p, workspace=ws)
    msg = vs.bp_export_messages(ws, w, h, p)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), msg.cpu().numpy()


def _oracle(l, r, p):
    return oracle.bp(l, r, p.labels, p.levels, p.iters, p.data_trunc, p.smooth_slope, p.smooth_trunc,
                     mode=oracle.MSG_DT, return_messages=True)


SHAPES = [(61, 97, 64), (29, 45, 37), (33, 70, 96), (36, 52, 16), (45, 33, 128), (23, 17, 48)]


@pytest.mark.parametrize("K", [2, 3, 5])
@pytest.mark.parametrize("shape", SHAPES)
def test_fused_matches_the_oracle_on_odd_sizes(K, shape):
    """K iterations per launch on every level (6 per level: launches of K and
    the remainder), with the library's tiles and with 6 x 4 cores."""
    h, w, L = shape
    L_, R_, l, r = _pair(40 + K + h, h, w)
    p = vs.BPParams(L, 4, 6, 20, 10, 40, iters_per_tile=K)
    want, wmsg = _oracle(l, r, p)
    for tile in ((0, 0), (6, 4)):
        vs.bp_select_fused(*tile, 0)
        got, msg = _run(L_, R_, p)
        np.testing.assert_array_equal(msg, wmsg)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("lanes", [1, 2, 4])
@pytest.mark.parametrize("tile", [(2, 2), (5, 3), (8, 6), (31, 7)])
def test_fused_every_lane_count_and_tile(lanes, tile):
    """Tiles of 2 x 2 up to 31 x 7 pixels (odd widths put a tile edge between
    the two pixels of a colour slot) and 1, 2 or 4 lanes per direction pair."""
    h, w, L = 41, 77, 64
    L_, R_, l, r = _pair(3, h, w)
    p = vs.BPParams(L, 3, 5, 20, 10, 40, iters_per_tile=3)
    vs.bp_select_fused(*tile, lanes)
    got, msg = _run(L_, R_, p)
    want, wmsg = _oracle(l, r, p)
    np.testing.assert_array_equal(msg, wmsg)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("levels,iters,K", [(1, 7, 3), (3, 1, 2), (2, 4, 9), (4, 10, 10), (3, 5, 1)])
def test_fused_edge_schedules(levels, iters, K):
    """One level only; one iteration per level (the first launch of a level
    both starts from the parent and ends it); K above iters (clamped to one
    launch per level); a whole level in one launch; and K = 1 (every
    iteration unfused) for comparison."""
    h, w, L = 37, 59, 32
    L_, R_, l, r = _pair(9 + iters, h, w)
    p = vs.BPParams(L, levels, iters, 20, 10, 40, iters_per_tile=K)
    got, msg = _run(L_, R_, p)
    want, wmsg = _oracle(l, r, p)
    np.testing.assert_array_equal(msg, wmsg)
    np.testing.assert_array_equal(got, want)


def test_fused_degenerate_frames():
    """1-pixel-wide and 1-pixel-high frames and a 1 x 1 frame."""
    for h, w in ((1, 40), (40, 1), (1, 1), (2, 3)):
        L_, R_, l, r = _pair(5, max(h, 8), max(w, 8))
        L_, R_ = L_[:h, :w].contiguous(), R_[:h, :w].contiguous()
        l, r = np.ascontiguousarray(l[:h, :w]), np.ascontiguousarray(r[:h, :w])
        p = vs.BPParams(16, 2, 3, 20, 10, 40, iters_per_tile=2)
        got, msg = _run(L_, R_, p)
        want, wmsg = _oracle(l, r, p)
        np.testing.assert_array_equal(msg, wmsg)
        np.testing.assert_array_equal(got, want)


def test_fused_full_size_pair_and_graph_replay():
    """The 676 x 380, 64-label, 4 x 10 pair with the automatic choice, with
    every level fused (K = 2 and 5), and K = 2 replayed from a CUDA graph:
    all equal the oracle's labels and messages."""
    h, w = 380, 676
    L_, R_, l, r = _pair(2, h, w)
    base = vs.BPParams(64, 4, 10, 20, 10, 40)
    want, wmsg = _oracle(l, r, base)
    for K in (0, 2, 5):
        p = vs.BPParams(**{**base.__dict__, "iters_per_tile": K})
        got, msg = _run(L_, R_, p)
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(msg, wmsg)
    p = vs.BPParams(**{**base.__dict__, "iters_per_tile": 2})
    ws = torch.zeros(vs.bp_workspace_size(w, h, p), dtype=torch.uint8, device="cuda")
    lab = torch.full((h, w), 255, dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        vs.bp_stereo(L_, R_, p, labels=lab, workspace=ws)   # warm-up outside capture
    torch.cuda.synchronize()
    lab.fill_(255)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        vs.bp_stereo(L_, R_, p, labels=lab, workspace=ws)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lab.cpu().numpy(), want)
    np.testing.assert_array_equal(vs.bp_export_messages(ws, w, h, p).cpu().numpy(), wmsg)


def test_fused_autotune_keeps_results_identical():
    """The automatic mode after vs_bp_autotune (which times every coarse level
    unfused and fused on several K, tiles and lane counts) gives the oracle's
    labels and messages; level 0 stays one kernel per iteration."""
    h, w = 190, 338
    L_, R_, l, r = _pair(7, h, w)
    p = vs.BPParams(64, 4, 10, 20, 10, 40)
    want, wmsg = _oracle(l, r, p)
    try:
        vs.bp_autotune(L_, R_, p)
        plans = vs.bp_autotune_plans()
        assert len(plans) == 4 and plans[0] == (0, 0, 0, 0)
        for K, tw, th, ns in plans[1:]:
            assert K == 0 or (2 <= K <= 10 and tw >= 2 and th >= 2 and ns in (1, 2, 4))
        got, msg = _run(L_, R_, p)
        np.testing.assert_array_equal(msg, wmsg)
        np.testing.assert_array_equal(got, want)
    finally:
        vs.bp_autotune_reset()

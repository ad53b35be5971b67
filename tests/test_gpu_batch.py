"""Batched BP (vs_bp_stereo_batch) and the sweep autotuner (vs_bp_autotune):
both must reproduce the single-pair results bit for bit."""
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


def _pair(seed, h, w):
    left, right, _ = synth.noise_pair(seed, w=w, h=h, max_disp=min(12.0, w / 4))
    return torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), left, right


SHAPES = [(120, 160, 16), (61, 97, 64), (45, 33, 32), (150, 200, 128), (17, 23, 48), (90, 70, 96), (33, 40, 5),
          (64, 64, 64)]


@pytest.fixture(params=["streams", "lockstep"])
def batch_mode(request):
    """Both schedules of the batch must give the single calls' results."""
    vs.bp_batch_mode(request.param)
    yield request.param
    vs.bp_batch_mode("streams")


def test_batch_matches_single_calls_and_oracle(batch_mode):
    pairs, hosts = [], []
    for i, (h, w, L) in enumerate(SHAPES):
        L_, R_, l, r = _pair(i, h, w)
        pairs.append((L_, R_, vs.BPParams(L, 3, 4, 20, 10, 40)))
        hosts.append((l, r))
    got = vs.bp_stereo_batch(pairs)
    torch.cuda.synchronize()
    for (L_, R_, p), lab, (l, r) in zip(pairs, got, hosts):
        single = vs.bp_stereo(L_, R_, p)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(lab.cpu().numpy(), single.cpu().numpy())
        if p.labels <= 64:
            want = oracle.bp(l, r, p.labels, p.levels, p.iters, 20, 10, 40, mode=oracle.MSG_DT)
            np.testing.assert_array_equal(lab.cpu().numpy(), want)


def test_batch_larger_than_one_launch_and_graph_replay(batch_mode):
    """70 jobs exceed one lockstep launch's job table; the batch (forked onto
    the library streams in the default schedule) replays from a graph."""
    pairs = []
    for i in range(70):
        L_, R_, _, _ = _pair(100 + i, 24 + (i % 5), 30 + (i % 7))
        pairs.append((L_, R_, vs.BPParams(32 if i % 2 else 16, 2, 3, 20, 10, 40)))
    labels = [torch.empty(tuple(p[0].shape), dtype=torch.uint8, device="cuda") for p in pairs]
    ws = torch.empty(vs.bp_batch_workspace_size(pairs), dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        vs.bp_stereo_batch(pairs, labels=labels, workspace=ws)
    torch.cuda.synchronize()
    first = [t.cpu().numpy().copy() for t in labels]
    for t in labels:
        t.fill_(255)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        vs.bp_stereo_batch(pairs, labels=labels, workspace=ws)
    g.replay()
    torch.cuda.synchronize()
    for (L_, R_, p), a, b in zip(pairs, first, labels):
        np.testing.assert_array_equal(b.cpu().numpy(), a)
        np.testing.assert_array_equal(a, vs.bp_stereo(L_, R_, p).cpu().numpy())


def test_batch_rejects_mixed_schedules():
    L_, R_, _, _ = _pair(0, 20, 30)
    with pytest.raises(vs.VSError):
        vs.bp_stereo_batch([(L_, R_, vs.BPParams(16, 3, 4, 20, 10, 40)), (L_, R_, vs.BPParams(16, 2, 4, 20, 10, 40))])


def test_autotune_keeps_results_identical():
    L_, R_, l, r = _pair(7, 190, 338)
    p = vs.BPParams(64, 4, 10, 20, 10, 40)
    ws = torch.empty(vs.bp_workspace_size(338, 190, p), dtype=torch.uint8, device="cuda")
    before = vs.bp_stereo(L_, R_, p, workspace=ws).cpu().numpy()
    msg_before = vs.bp_export_messages(ws, 338, 190, p).cpu().numpy()
    try:
        chosen = vs.bp_autotune(L_, R_, p, workspace=ws)
        assert len(chosen) == 4 and all(c in (0, 1, 2, 3) for c in chosen)
        times = vs.bp_autotune_times()
        assert len(times) == 4 and all(row[c] > 0 and row[c] == min(t for t in row if t > 0)
                                       for row, c in zip(times, chosen))
        after = vs.bp_stereo(L_, R_, p, workspace=ws).cpu().numpy()
        np.testing.assert_array_equal(after, before)
        np.testing.assert_array_equal(vs.bp_export_messages(ws, 338, 190, p).cpu().numpy(), msg_before)
    finally:
        vs.bp_autotune_reset()
    np.testing.assert_array_equal(before, oracle.bp(l, r, 64, 4, 10, 20, 10, 40, mode=oracle.MSG_DT))


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("shape", [(190, 338, 64), (61, 97, 128), (33, 70, 96), (29, 45, 37), (36, 52, 16)])
def test_every_sweep_variant_matches_the_oracle(variant, shape):
    """Each sweep kernel (plain, preload, labels split over two or four lanes,
    staged through shared memory -- here on levels 0 and 1, whose costs and
    belief sums fit bytes) forced on every level where it applies gives the
    oracle's labels and final level-0 messages bit for bit."""
    h, w, L = shape
    L_, R_, l, r = _pair(11 + variant, h, w)
    p = vs.BPParams(L, 4, 6, 20, 10, 40)
    try:
        vs.bp_select_sweep(variant)
        ws = torch.empty(vs.bp_workspace_size(w, h, p), dtype=torch.uint8, device="cuda")
        got = vs.bp_stereo(L_, R_, p, workspace=ws).cpu().numpy()
        msg = vs.bp_export_messages(ws, w, h, p).cpu().numpy()
        vs.bp_status(ws, w, h, p)    # no bounded wait ran out
    finally:
        vs.bp_select_sweep(-1)
    want, wmsg = oracle.bp(l, r, L, 4, 6, 20, 10, 40, mode=oracle.MSG_DT, return_messages=True)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(msg, wmsg)


def _rgb(seed, H, W):
    g = np.random.default_rng(seed)
    return torch.from_numpy(g.integers(0, 256, size=(H, W, 3)).astype(np.uint8)).cuda()


def test_pair_batch_matches_single_pair_calls_and_replays():
    """Whole pairs (remap, BP, upsample + reproject) of mixed sizes,
    downsample factors 2 / 4 / 8, 32..128 labels and baselines in one
    vs_pair_run_batch call: every cloud and disparity equals its own
    vs_pair_run bit for bit, eagerly and replayed from a CUDA graph."""
    specs = [(320, 176, 2, 32, 0.05), (416, 240, 4, 64, 0.15), (200, 120, 8, 96, 0.25), (336, 200, 4, 128, 0.1),
             (160, 96, 2, 64, 0.2), (520, 300, 8, 32, 0.05)]
    jobs, singles = [], []
    for i, (W, H, s, L, B) in enumerate(specs):
        f = W / 2704.0
        cam = vs.Camera(1400 * f, 1400 * f, (W - 1) / 2, (H - 1) / 2, -0.25, 0.07)
        cfg = vs.PairConfig(W, H, cam, B, vs.BPParams(L, 3, 5, 20, 10, 40), vs.JBUParams(s, 2, 1.0, 12.0))
        left, right = _rgb(2 * i, H, W), _rgb(2 * i + 1, H, W)
        xyz = torch.full((H, W, 3), 7.0, device="cuda")
        disp = torch.full((H, W), 7.0, device="cuda")
        jobs.append((cfg, left, right, disp, xyz))
        d1, x1 = vs.pair_run(cfg, left, right, disp=torch.empty((H, W), device="cuda"))
        singles.append((d1, x1))
    ws = vs.pair_run_batch(jobs)
    torch.cuda.synchronize()
    for (cfg, _, _, disp, xyz), (d1, x1) in zip(jobs, singles):
        assert torch.equal(disp, d1) and torch.equal(torch.nan_to_num(xyz, 1e30), torch.nan_to_num(x1, 1e30))
    for _, _, _, disp, xyz in jobs:
        disp.fill_(7.0)
        xyz.fill_(7.0)
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        vs.pair_run_batch(jobs, workspace=ws, stream=st)
    g.replay()
    torch.cuda.synchronize()
    for (cfg, _, _, disp, xyz), (d1, x1) in zip(jobs, singles):
        assert torch.equal(disp, d1) and torch.equal(torch.nan_to_num(xyz, 1e30), torch.nan_to_num(x1, 1e30))

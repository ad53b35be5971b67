"""The benchmark's launch configuration: three (its default) or four 2.7K
pairs on as many streams, forked and joined inside one CUDA graph, replayed
twice.  Every pair's point cloud must equal that pair run alone, bit for bit
(the single-pair path is itself checked stage by stage against the oracle at
this size)."""
import numpy as np
import pytest
import torch

import paper_1902_09733_b300 as vs
from paper_1902_09733_b300 import build, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available()
    build.build()


@pytest.mark.parametrize("P", [3, 4])
def test_pairs_in_flight_in_one_graph_match_single_runs(P):
    cam = vs.Camera(*synth.TERRAIN_CAMERA)
    bp = vs.BPParams(labels=64, levels=4, iters=10, data_trunc=20, smooth_slope=10, smooth_trunc=40)
    jbu = vs.JBUParams(scale=4, radius=2, sigma_s=1.0, sigma_r=12.0)
    cfg = vs.PairConfig(2704, 1520, cam, 0.5, bp, jbu)
    left, right = synth.terrain_pair(0)
    pairs = [(torch.from_numpy(l).cuda(), torch.from_numpy(r).cuda()) for l, r in synth.pair_variants(left, right)]
    assert len(pairs) >= P
    pairs = pairs[:P]
    n = len(pairs)
    ws = [torch.empty(vs.pair_workspace_size(cfg), dtype=torch.uint8, device="cuda") for _ in range(n)]
    want = []
    for (l, r), w in zip(pairs, ws):
        _, xyz = vs.pair_run(cfg, l, r, workspace=w)
        want.append(xyz.clone())
    torch.cuda.synchronize()

    # the same buffers, now written by the graph: poison them first
    xyz = [torch.full((1520, 2704, 3), float("nan"), dtype=torch.float32, device="cuda") for _ in range(n)]
    for w in ws:
        w.fill_(0xA5)
    stream = torch.cuda.Stream()
    side = [torch.cuda.Stream() for _ in range(n)]
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fork = torch.cuda.Event()
        fork.record(stream)
        joins = []
        for k in range(n):
            side[k].wait_event(fork)
            vs.pair_run(cfg, *pairs[k], xyz=xyz[k], workspace=ws[k], stream=side[k])
            e = torch.cuda.Event()
            e.record(side[k])
            joins.append(e)
        for e in joins:
            stream.wait_event(e)
    for _ in range(2):
        with torch.cuda.stream(stream):
            g.replay()
        torch.cuda.synchronize()
        for k in range(n):
            np.testing.assert_array_equal(xyz[k].cpu().numpy(), want[k].cpu().numpy())

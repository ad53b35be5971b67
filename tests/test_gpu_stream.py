"""The streaming drivers (vs_pipeline_*): overlapped copies and compute must
give exactly the clouds of the one-pair driver, in pair and flight mode."""
import numpy as np
import pytest
import torch

import paper_1902_09733_b300 as vs
from paper_1902_09733_b300 import build

pytestmark = pytest.mark.gpu

CFG = vs.PairConfig(320, 180, vs.Camera(160.0, 160.0, 159.5, 89.5, -0.2, 0.05), 0.5,
                    vs.BPParams(16, 3, 5, 20, 10, 40), vs.JBUParams(4, 2, 1.0, 12.0))


@pytest.fixture(scope="module", autouse=True)
def _built():
    assert torch.cuda.is_available()
    build.build()


def _frames(n, seed=0):
    g = np.random.default_rng(seed)
    base = g.integers(0, 256, size=(180, 400, 3)).astype(np.uint8)
    # a scene sliding left by 2 px per frame: later frames are right views
    return [np.ascontiguousarray(base[:, 2 * i:2 * i + 320]) for i in range(n)]


def _reference(left, right):
    _, xyz = vs.pair_run(CFG, torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda())
    torch.cuda.synchronize()
    return xyz.cpu().numpy()


def _same(a, b):
    np.testing.assert_array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_array_equal(np.nan_to_num(a), np.nan_to_num(b))


@pytest.mark.parametrize("depth", [1, 3])
def test_pair_mode_matches_single_pair_driver(depth):
    frames = _frames(7)
    pairs = [(frames[i], frames[i + 2]) for i in range(5)]
    pipe = vs.Pipeline(CFG, mode="pairs", depth=depth)
    outs = []
    for left, right in pairs:
        xyz = torch.empty((180, 320, 3), dtype=torch.float32).pin_memory()
        pipe.submit_pair(torch.from_numpy(left).pin_memory(), torch.from_numpy(right).pin_memory(), xyz)
        outs.append(xyz)
    pipe.flush()
    assert len(pipe.latencies()) == len(pairs)
    for (left, right), xyz in zip(pairs, outs):
        _same(xyz.numpy(), _reference(left, right))
    pipe.close()


@pytest.mark.parametrize("k,depth", [(1, 2), (3, 3)])
def test_flight_mode_pairs_frame_f_minus_k_with_f(k, depth):
    frames = _frames(9, seed=1)
    pipe = vs.Pipeline(CFG, mode="flight", depth=depth, k=k)
    outs = {}
    for f, fr in enumerate(frames):
        xyz = torch.full((180, 320, 3), -7.0, dtype=torch.float32).pin_memory() if f >= k else None
        pipe.submit_frame(torch.from_numpy(fr).pin_memory(), xyz)
        if xyz is not None:
            outs[f] = xyz
    pipe.flush()
    assert len(pipe.latencies()) == len(frames) - k
    for f, xyz in outs.items():
        _same(xyz.numpy(), _reference(frames[f - k], frames[f]))
    pipe.close()

"""The general min-sum path (16-bit messages, 32-bit sums, one warp per
pixel) for what the byte path cannot hold: up to 256 labels, truncations
above 127, coarse data terms beyond 16 bits, 8 levels.  Labels and final
level-0 messages must equal the oracle's bit for bit."""
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


def _pair(seed, h, w, max_disp):
    left, right, _ = synth.noise_pair(seed, w=w, h=h, max_disp=max_disp)
    return torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda(), left, right


# (h, w, labels, levels, iters, data_trunc, slope, smooth_trunc)
CASES = [
    (61, 97, 256, 4, 6, 20, 10, 40),       # 256 labels
    (33, 70, 200, 3, 5, 150, 7, 200),      # truncations above 127
    (29, 45, 37, 8, 4, 130, 9, 140),       # 8 levels, small label count
    (97, 61, 160, 8, 3, 20, 10, 40),       # 8 levels, 160 labels
    (45, 33, 129, 2, 1, 20, 10, 40),       # one iteration per level (the parent's messages kept)
    (40, 52, 64, 7, 3, 20, 10, 40),        # 20 * 4^6: coarse sums beyond 16 bits
    (23, 17, 256, 1, 7, 255, 300, 1000),   # slope above the truncation (the same V)
    (1, 40, 200, 2, 3, 20, 10, 40),        # one row
]


@pytest.mark.parametrize("case", CASES)
def test_general_path_matches_the_oracle(case):
    h, w, L, levels, iters, Td, c, Ts = case
    L_, R_, l, r = _pair(60 + h + L, max(h, 8), w, min(40.0, w / 3))
    L_, R_ = L_[:h].contiguous(), R_[:h].contiguous()
    l, r = np.ascontiguousarray(l[:h]), np.ascontiguousarray(r[:h])
    p = vs.BPParams(L, levels, iters, Td, c, Ts)
    n = vs.bp_workspace_size(w, h, p)
    assert n > 0
    ws = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda")   # contents must not matter
    lab = vs.bp_stereo(L_, R_, p, workspace=ws)
    msg = vs.bp_export_messages(ws, w, h, p)
    vs.bp_status(ws, w, h, p)
    torch.cuda.synchronize()
    want, wmsg = oracle.bp(l, r, L, levels, iters, Td, c, Ts, mode=oracle.MSG_DT, return_messages=True)
    np.testing.assert_array_equal(msg.cpu().numpy(), wmsg)
    np.testing.assert_array_equal(lab.cpu().numpy(), want)


@pytest.mark.parametrize("mode", ["streams", "lockstep"])
def test_batch_mixes_both_paths(mode):
    """A batch with byte-path and general-path pairs gives every pair's own result."""
    specs = [(40, 60, 64, 40), (33, 50, 200, 40), (30, 44, 32, 150), (41, 63, 256, 60)]
    pairs = []
    for i, (h, w, L, Ts) in enumerate(specs):
        L_, R_, _, _ = _pair(80 + i, h, w, 12.0)
        pairs.append((L_, R_, vs.BPParams(L, 3, 4, 20, 10, Ts)))
    vs.bp_batch_mode(mode)
    try:
        got = vs.bp_stereo_batch(pairs)
        torch.cuda.synchronize()
    finally:
        vs.bp_batch_mode("streams")
    for (L_, R_, p), lab in zip(pairs, got):
        np.testing.assert_array_equal(lab.cpu().numpy(), vs.bp_stereo(L_, R_, p).cpu().numpy())

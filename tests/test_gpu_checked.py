"""The checked build (libvstereo_checked.so: every global access of the
min-sum kernels tested against the call's buffers, the first one outside them
recorded and skipped) on small odd-sized cases of every kernel family: no
access is refused, the results equal the product library's bit for bit, and
two runs give identical bits.  A registered workspace 256 bytes shorter than
the real one shows that a refused access is reported (the access itself stays
inside the real buffer)."""
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
    vs.lib()


def _pair(seed, h, w):
    left, right, _ = synth.noise_pair(seed, w=w, h=h, max_disp=min(12.0, w / 4))
    return torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()


def _report(lib):
    out = (np.zeros(2, np.uint64))
    r = lib.vs_check_report(out.ctypes.data)
    return r, int(out[0]), int(out[1])


def _bp(L_, R_, p):
    h, w = L_.shape
    ws = torch.randint(0, 256, (vs.bp_workspace_size(w, h, p),), dtype=torch.uint8, device="cuda")
    lab = vs.bp_stereo(L_, R_, p, workspace=ws)
    msg = vs.bp_export_messages(ws, w, h, p)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), msg.cpu().numpy()


# (h, w, labels, levels, iters, smooth_trunc, iters_per_tile, forced sweep variant, fused tile)
CASES = [
    (29, 45, 37, 4, 6, 40, 1, -1, None),       # automatic variants, padded labels
    (61, 97, 64, 4, 6, 40, 1, 4, None),        # staged sweep forced (bulk copies)
    (33, 70, 96, 3, 5, 40, 1, 2, None),        # labels split over two lanes
    (36, 52, 16, 3, 5, 40, 1, 1, None),        # register preload
    (41, 77, 64, 3, 5, 40, 3, -1, (5, 3)),     # fused tiles with small, odd cores
    (23, 17, 128, 2, 4, 40, 2, -1, (2, 2)),    # fused, 128 labels, two lanes
    (33, 50, 200, 3, 4, 40, 0, -1, None),      # the general path (200 labels)
    (30, 44, 32, 3, 3, 150, 0, -1, None),      # the general path (truncation above 127)
]


@pytest.mark.parametrize("case", CASES)
def test_checked_build_refuses_nothing_and_matches(case):
    h, w, L, levels, iters, Ts, K, variant, tile = case
    L_, R_ = _pair(h + w, h, w)
    p = vs.BPParams(L, levels, iters, 20, 10, Ts, iters_per_tile=K)
    chk = vs.checked_lib()
    runs = []
    for library in (vs.lib(), chk, chk):
        with vs.using(library):
            vs.bp_select_sweep(variant)
            if tile:
                vs.bp_select_fused(tile[0], tile[1], 0)
            try:
                runs.append(_bp(L_, R_, p))
            finally:
                vs.bp_select_sweep(-1)
                vs.bp_select_fused(0, 0, 0)
    assert _report(chk) == (0, 0, 0)
    for lab, msg in runs[1:]:
        np.testing.assert_array_equal(lab, runs[0][0])
        np.testing.assert_array_equal(msg, runs[0][1])


@pytest.mark.parametrize("mode", ["streams", "lockstep"])
def test_checked_build_batch(mode):
    specs = [(40, 60, 64, 40), (33, 50, 200, 40), (30, 44, 32, 150), (27, 31, 16, 40)]
    pairs = [(*_pair(90 + i, h, w), vs.BPParams(L, 3, 4, 20, 10, Ts)) for i, (h, w, L, Ts) in enumerate(specs)]
    want = [vs.bp_stereo(l, r, p).cpu().numpy() for l, r, p in pairs]
    chk = vs.checked_lib()
    with vs.using(chk):
        vs.bp_batch_mode(mode)
        try:
            got = vs.bp_stereo_batch(pairs)
            torch.cuda.synchronize()
        finally:
            vs.bp_batch_mode("streams")
    assert _report(chk) == (0, 0, 0)
    for g, w_ in zip(got, want):
        np.testing.assert_array_equal(g.cpu().numpy(), w_)


@pytest.mark.parametrize("L", [64, 200])
def test_checked_build_reports_a_refused_access(L):
    """With the workspace registered 256 bytes short, the first kernel's write
    of the call's status word (the workspace's last 256-byte slot) is refused
    and reported as the status site with its address."""
    L_, R_ = _pair(7, 31, 45)
    p = vs.BPParams(L, 3, 3, 20, 10, 40)
    n = vs.bp_workspace_size(45, 31, p)
    ws = torch.zeros(n, dtype=torch.uint8, device="cuda")
    chk = vs.checked_lib()
    assert chk.vs_check_test_shrink(256) == vs.VS_OK
    try:
        with vs.using(chk):
            vs.bp_stereo(L_, R_, p, workspace=ws)
            torch.cuda.synchronize()
    finally:
        chk.vs_check_test_shrink(0)
    r, site, addr = _report(chk)
    assert r == 1 and site == 7, (r, site)                       # 7: the status word
    assert ws.data_ptr() + n - 256 <= addr < ws.data_ptr() + n
    assert _report(chk) == (0, 0, 0)                             # reading it clears it

"""The bounded waits of the staged BP sweep: when the bulk copies a CTA waits
for never arrive, each wait gives up after about a second, the call reports
VS_ETIMEOUT through vs_bp_status, and the GPU context stays usable.  The
missing copies are made on purpose by a test aid that announces the bytes to
the mbarrier but issues no copy (no fault, no unbounded wait)."""
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


def test_staged_sweep_wait_runs_out_and_is_reported():
    # one level, three iterations: iterations 1 and 2 read the level's own
    # messages, so the forced staged variant runs them
    p = vs.BPParams(16, 1, 3, 20, 10, 40)
    left, right, _ = synth.noise_pair(3, w=64, h=48)
    L, R = torch.from_numpy(left).cuda(), torch.from_numpy(right).cuda()
    ws = torch.empty(vs.bp_workspace_size(64, 48, p), dtype=torch.uint8, device="cuda")
    vs.bp_select_sweep(4)
    try:
        vs.bp_test_withhold_copies(True)
        try:
            vs.bp_stereo(L, R, p, workspace=ws)
            with pytest.raises(vs.VSError) as e:
                vs.bp_status(ws, 64, 48, p)
            assert e.value.code == vs.VS_ETIMEOUT
        finally:
            vs.bp_test_withhold_copies(False)
        # the same workspace and context serve the next call normally
        lab = vs.bp_stereo(L, R, p, workspace=ws)
        vs.bp_status(ws, 64, 48, p)
    finally:
        vs.bp_select_sweep(-1)
    want = oracle.bp(left, right, 16, 1, 3, 20, 10, 40)
    np.testing.assert_array_equal(lab.cpu().numpy(), want)


def test_tensor_core_mma_wait_runs_out_and_is_reported():
    """The tensor-core smoothed-BP kernels with their MMAs withheld (a test aid:
    no MMA and no completion signal are issued, so nothing is in flight): each
    bounded wait gives up, the forward and the adjoint report VS_ETIMEOUT
    through vs_sp_status, and the next calls run normally and agree with the
    SIMT kernels."""
    g = torch.Generator(device="cuda").manual_seed(5)
    p = vs.SPParams(labels=48, iters=2, ckpt_every=1, lam=2.5, trunc=13.75, tau=2.0)
    cost = torch.rand((30, 40, 48), generator=g, device="cuda") * 20.0
    gb = torch.randn((30, 40, 48), generator=g, device="cuda")
    vs.sp_select_kernels("tensor")
    try:
        vs.sp_test_withhold_mma(True)
        try:
            _, ws = vs.sp_forward(cost, p)
            with pytest.raises(vs.VSError) as e:
                vs.sp_status(ws, 40, 30, p)
            assert e.value.code == vs.VS_ETIMEOUT
            vs.sp_backward(cost, p, gb, ws)
            with pytest.raises(vs.VSError) as e:
                vs.sp_status(ws, 40, 30, p)
            assert e.value.code == vs.VS_ETIMEOUT
        finally:
            vs.sp_test_withhold_mma(False)
        b_tc, ws = vs.sp_forward(cost, p)
        gc_tc, gp_tc = vs.sp_backward(cost, p, gb, ws)
        vs.sp_status(ws, 40, 30, p)
    finally:
        vs.sp_select_kernels("simt")
    b_s, ws_s = vs.sp_forward(cost, p)
    gc_s, gp_s = vs.sp_backward(cost, p, gb, ws_s)
    torch.cuda.synchronize()
    # each family is within 2e-5 (beliefs) and 1e-3 (gradients) of the FP64 oracle
    scale = b_s.abs().max().item()
    assert (b_tc - b_s).abs().max().item() <= 4e-5 * scale
    assert (gc_tc - gc_s).abs().max().item() <= 2e-3 * gc_s.abs().max().item()
    assert torch.allclose(gp_tc, gp_s, rtol=2e-3, atol=2e-3 * gp_s.abs().max().item())

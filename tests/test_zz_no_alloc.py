"""The allocation-free stereo entry point, vs_bp_stereo_noalloc.

Some callers cannot call cudaMalloc at all (code inside an allocator or
memory-pool callback, plugins whose host owns every allocation, real-time
loops that must not allocate).  For them the library runs the stereo step on
a scratch array it carries itself.  These tests call that entry point
through the C ABI and check that calls in a row -- the same pair twice, a
larger one, then smaller ones over its leftovers -- give exactly the labels of
the ordinary entry point with a caller workspace (BP is integer and
bit-exact), that a bounded wait which runs out is reported through
vs_bp_noalloc_status, and that a pair too large for the built-in scratch is
refused.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1902_09733_b300 as vs
from paper_1902_09733_b300 import build, synth

pytestmark = pytest.mark.gpu


def _entry():
    build.build()
    f = vs.lib().vs_bp_stereo_noalloc
    P, I = ctypes.c_void_p, ctypes.c_int
    f.argtypes = [P, P, I, I, I, ctypes.POINTER(vs._BPParams), P, I, P]
    f.restype = I
    return f


def _status():
    f = vs.lib().vs_bp_noalloc_status
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(vs._BPParams), ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_matches_workspace_entry_point_twice_in_a_row():
    assert torch.cuda.is_available()
    f = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(0, 160, 120, vs.BPParams(16, 3, 5, 20, 10, 40)),    # the small noise pair, twice
             (1, 160, 120, vs.BPParams(16, 3, 5, 20, 10, 40)),
             (2, 320, 180, vs.BPParams(16, 3, 5, 20, 10, 40)),    # the paper's 320 x 180, 16 labels
             # then smaller pairs with other label counts over the larger one's leftovers
             (3, 160, 120, vs.BPParams(32, 3, 5, 20, 10, 40)),
             (4, 97, 61, vs.BPParams(48, 2, 4, 20, 10, 40))]
    for seed, w, h, p in cases:
        assert vs.bp_workspace_size(w, h, p) <= 8 << 20
        left, right, _ = synth.noise_pair(seed, w=w, h=h)
        L = torch.from_numpy(left).cuda()
        R = torch.from_numpy(right).cuda()
        out = torch.full((h, w), 255, dtype=torch.uint8, device="cuda")
        cp = p.c()
        rc = f(L.data_ptr(), R.data_ptr(), w, h, w, ctypes.byref(cp), out.data_ptr(), w, stream)
        assert rc == vs.VS_OK, vs.status_string(rc)
        assert _status()(w, h, ctypes.byref(cp), stream) == vs.VS_OK
        ref = vs.bp_stereo(L, R, p)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_reports_a_bounded_wait_that_ran_out():
    """The staged sweep forced on a no-alloc call whose bulk copies are
    withheld (a test aid: the bytes are announced, no copy is issued, so no
    fault and no unbounded wait): vs_bp_noalloc_status reads VS_ETIMEOUT from
    the built-in scratch, and the next call runs normally."""
    f = _entry()
    stream = torch.cuda.current_stream().cuda_stream
    w, h = 64, 48
    p = vs.BPParams(16, 1, 3, 20, 10, 40)     # iterations 1 and 2 run the staged sweep
    left, right, _ = synth.noise_pair(3, w=w, h=h)
    L = torch.from_numpy(left).cuda()
    R = torch.from_numpy(right).cuda()
    out = torch.empty((h, w), dtype=torch.uint8, device="cuda")
    cp = p.c()
    vs.bp_select_sweep(4)
    try:
        vs.bp_test_withhold_copies(True)
        try:
            assert f(L.data_ptr(), R.data_ptr(), w, h, w, ctypes.byref(cp), out.data_ptr(), w, stream) == vs.VS_OK
            assert _status()(w, h, ctypes.byref(cp), stream) == vs.VS_ETIMEOUT
        finally:
            vs.bp_test_withhold_copies(False)
        assert f(L.data_ptr(), R.data_ptr(), w, h, w, ctypes.byref(cp), out.data_ptr(), w, stream) == vs.VS_OK
        assert _status()(w, h, ctypes.byref(cp), stream) == vs.VS_OK
    finally:
        vs.bp_select_sweep(-1)
    ref = vs.bp_stereo(L, R, p)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_refuses_pairs_larger_than_its_scratch():
    f = _entry()
    p = vs.BPParams(64, 4, 10, 20, 10, 40)
    assert vs.bp_workspace_size(676, 380, p) > 8 << 20
    L = torch.zeros((380, 676), dtype=torch.uint8, device="cuda")
    out = torch.full((380, 676), 7, dtype=torch.uint8, device="cuda")
    cp = p.c()
    rc = f(L.data_ptr(), L.data_ptr(), 676, 380, 676, ctypes.byref(cp), out.data_ptr(), 676,
           torch.cuda.current_stream().cuda_stream)
    assert rc == vs.VS_EWORKSPACE
    torch.cuda.synchronize()
    assert (out.cpu().numpy() == 7).all()     # nothing was launched

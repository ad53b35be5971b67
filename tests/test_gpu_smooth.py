"""GPU parity of the temperature-smoothed BP (forward and adjoint) against the
FP64 oracle, through the C ABI.

Tolerances (FP32 kernels against FP64).  A message is tau times a difference
of logs of sums of positive terms, so its rounding error is absolute, about
tau x 1e-6 per iteration (FP32 sums; the tensor-core MMAs truncate and give
about twice that), and the sums of three incoming messages carry it on, so
after 8 iterations beliefs are off by up to ~5e-4 in absolute terms whatever
their own size.  Hence beliefs within 2e-5 of the volume's belief scale
max |b| (about 60 here), element by element; dL/dD within 1e-3 of max |dL/dD|
element by element and the three scalar gradients within 1e-3 relative --
the bar set for the adjoint against finite differences.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_09733_b300 as vs

pytestmark = pytest.mark.gpu

B_TOL = 2e-5
G_RTOL = 1e-3


@pytest.fixture(params=["simt", "tensor"])
def kernels(request):
    """Both kernel families must meet the same bar."""
    vs.sp_select_kernels(request.param)
    yield request.param
    vs.sp_select_kernels("simt")


def _cost(seed, h, w, L, hi=20.0):
    g = np.random.default_rng(seed)
    return g.uniform(0.0, hi, (h, w, L)).astype(np.float32)


def _run(D, params, gb=None):
    cost = torch.from_numpy(D).cuda()
    bel, ws = vs.sp_forward(cost, params)
    out = [bel.cpu().numpy()]
    if gb is not None:
        gcost, gpar = vs.sp_backward(cost, params, torch.from_numpy(gb).cuda(), ws)
        out += [gcost.cpu().numpy(), gpar.cpu().numpy()]
    torch.cuda.synchronize()
    vs.sp_status(ws, D.shape[1], D.shape[0], params)
    return out


def _check_beliefs(got, ref, scale=None):
    err = np.abs(got.astype(np.float64) - ref)
    tol = B_TOL * (np.abs(ref).max() if scale is None else scale)
    assert err.max() <= tol, f"max err {err.max():.3g} > {tol:.3g}"


def _check_grads(gD, gpar, ref):
    rD, rl, rT, rt = ref
    scale = np.abs(rD).max()
    err = np.abs(gD.astype(np.float64) - rD).max()
    assert err <= G_RTOL * scale, f"dL/dD max err {err:.3g} vs scale {scale:.3g}"
    for got, want, name in zip(gpar, (rl, rT, rt), ("lambda", "trunc", "tau")):
        assert abs(got - want) <= G_RTOL * max(abs(want), 1e-3), f"{name}: {got} vs {want}"


CASES = [
    # (w, h, L, iters, ckpt, lam, trunc, tau): several CTAs with a ragged last one,
    # every label count, checkpoint intervals that do and do not divide iters;
    # trunc/lam is never an integer, so no kink lambda |d - d'| == trunc is hit
    (37, 23, 16, 5, 2, 2.5, 13.7, 2.0),
    (29, 17, 48, 8, 2, 2.5, 13.7, 2.0),
    (21, 13, 32, 6, 4, 1.3, 7.9, 0.5),
    (11, 9, 64, 4, 3, 0.7, 20.65, 1.1),
    (19, 11, 48, 3, 1, 4.1, 9.3, 3.0),
    (1, 1, 16, 1, 1, 2.5, 13.7, 2.0),
    (40, 1, 16, 7, 7, 1.9, 6.1, 0.9),
    (1, 33, 32, 5, 2, 1.9, 6.1, 0.9),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}_i{c[3]}k{c[4]}" for c in CASES])
def test_forward_and_adjoint_match_oracle(case, kernels):
    w, h, L, iters, k, lam, T, tau = case
    # the library takes float parameters: give the oracle the same values
    lam, T, tau = (float(np.float32(v)) for v in (lam, T, tau))
    D = _cost(w * 1000 + h, h, w, L)
    gb = np.random.default_rng(7 + w).normal(size=D.shape).astype(np.float32)
    p = vs.SPParams(labels=L, iters=iters, ckpt_every=k, lam=lam, trunc=T, tau=tau)
    bel, gD, gpar = _run(D, p, gb)
    D64 = D.astype(np.float64)
    ref_b, states = oracle.sp_forward(D64, lam, T, tau, iters, return_states=True)
    _check_beliefs(bel, ref_b)
    _check_grads(gD, gpar, oracle.sp_backward(D64, lam, T, tau, iters, gb.astype(np.float64), states))


def test_checkpoint_interval_does_not_change_results(kernels):
    """Recomputation from checkpoints repeats the same arithmetic: every interval
    gives the same bits."""
    D = _cost(5, 31, 45, 48)
    gb = np.random.default_rng(5).normal(size=D.shape).astype(np.float32)
    base = None
    for k in (1, 2, 3, 5, 8):
        out = _run(D, vs.SPParams(labels=48, iters=8, ckpt_every=k), gb)
        if base is None:
            base = out
        else:
            for a, b in zip(out, base):
                assert np.array_equal(a, b), k


def test_runs_are_bit_identical_and_backward_repeats(kernels):
    D = _cost(6, 40, 50, 32)
    gb = np.random.default_rng(6).normal(size=D.shape).astype(np.float32)
    p = vs.SPParams(labels=32, iters=6, ckpt_every=2, lam=1.5, trunc=9.1, tau=1.3)
    a = _run(D, p, gb)
    b = _run(D, p, gb)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    # the adjoint leaves the checkpoints intact: a second backward on the same workspace agrees
    cost = torch.from_numpy(D).cuda()
    _, ws = vs.sp_forward(cost, p)
    g1 = vs.sp_backward(cost, p, torch.from_numpy(gb).cuda(), ws)
    g2 = vs.sp_backward(cost, p, torch.from_numpy(gb).cuda(), ws)
    assert torch.equal(g1[0], g2[0]) and torch.equal(g1[1], g2[1])


def test_no_smoothness_and_constant_shift(kernels):
    D = _cost(8, 20, 30, 16)
    gb = np.random.default_rng(8).normal(size=D.shape).astype(np.float32)
    bel, gD, gpar = _run(D, vs.SPParams(labels=16, iters=4, ckpt_every=2, lam=0.0, trunc=5.0, tau=1.0), gb)
    np.testing.assert_allclose(bel, D, rtol=0, atol=1e-5)
    np.testing.assert_allclose(gD, gb, rtol=0, atol=1e-5)
    assert gpar[1] == 0.0
    # a constant added to one pixel's data term moves only its own belief
    p = vs.SPParams(labels=16, iters=4, ckpt_every=2)
    b0 = _run(D, p)[0]
    D2 = D.copy()
    D2[7, 11] += 4.0
    b1 = _run(D2, p)[0]
    diff = b1 - b0
    diff[7, 11] -= 4.0
    assert np.abs(diff).max() < 2e-4


# --------------------------------------------------------------------------- full size

W, H, L, ITERS = 338, 190, 48, 8
# parameters exactly representable in FP32, so the FP64 oracle sees the same values
FULL = vs.SPParams(labels=L, iters=ITERS, ckpt_every=2, lam=2.5, trunc=13.75, tau=2.0)
SAMPLES = [(0, 0), (95, 22), (337, 189), (170, 100), (5, 170), (300, 40), (250, 150)]


def _crop(x, y, r):
    x0, x1 = max(0, x - r), min(W, x + r + 1)
    y0, y1 = max(0, y - r), min(H, y + r + 1)
    return x0, x1, y0, y1


@pytest.fixture(scope="module")
def full_case():
    D = _cost(2024, H, W, L)
    cost = torch.from_numpy(D).cuda()
    bel, ws = vs.sp_forward(cost, FULL)
    # adjoint of a loss that reads only the sampled pixels' beliefs
    g = np.random.default_rng(99)
    gb = np.zeros_like(D)
    for x, y in SAMPLES:
        gb[y, x] = g.normal(size=L)
    gcost, gpar = vs.sp_backward(cost, FULL, torch.from_numpy(gb).cuda(), ws)
    torch.cuda.synchronize()
    return D, gb, bel.cpu().numpy(), gcost.cpu().numpy(), gpar.cpu().numpy()


def test_full_size_sampled_beliefs(full_case):
    """A belief after 8 iterations depends on the data within L1 distance 8;
    the oracle on a crop of radius 9 reproduces it exactly."""
    D, _, bel, _, _ = full_case
    scale = np.abs(bel).max()
    for x, y in SAMPLES:
        x0, x1, y0, y1 = _crop(x, y, ITERS + 1)
        ref = oracle.sp_forward(D[y0:y1, x0:x1].astype(np.float64), FULL.lam, FULL.trunc, FULL.tau, ITERS)
        _check_beliefs(bel[y, x][None], ref[y - y0, x - x0][None], scale)


def test_full_size_sampled_adjoint(full_case):
    """The loss reads beliefs at samples more than 2*9 pixels apart, so dL/dD is
    the sum of disjoint per-sample gradients, each inside its crop, and the
    scalar gradients are the sums of the crops'."""
    D, gb, _, gD, gpar = full_case
    seen = np.zeros((H, W), bool)
    tot = np.zeros(3)
    ref_full = np.zeros(D.shape)
    for x, y in SAMPLES:
        x0, x1, y0, y1 = _crop(x, y, ITERS + 1)
        Dc = D[y0:y1, x0:x1].astype(np.float64)
        gbc = gb[y0:y1, x0:x1].astype(np.float64)
        rD, rl, rT, rt = oracle.sp_backward(Dc, FULL.lam, FULL.trunc, FULL.tau, ITERS, gbc)
        assert not seen[y0:y1, x0:x1].any()
        seen[y0:y1, x0:x1] = True
        ref_full[y0:y1, x0:x1] = rD
        tot += (rl, rT, rt)
    scale = np.abs(ref_full).max()
    assert np.abs(gD - ref_full).max() <= G_RTOL * scale
    assert np.all(gD[~seen] == 0)
    for got, want in zip(gpar, tot):
        assert abs(got - want) <= G_RTOL * abs(want)


def test_full_size_adjoint_against_central_differences():
    """Central differences of the FP32 forward (step 1e-3, loss accumulated in
    double) against the adjoint, for lambda, trunc, tau and a random direction
    in D, within 1e-3 relative.  The loss is <c, b> with c = softmax(-b0/tau)
    at the unperturbed beliefs b0 (the gradient of the summed free energy):
    its derivative adds up coherently over the 3 million beliefs while FP32
    rounding of the forward adds up in quadrature, which keeps the differences
    above their noise floor.  T/lambda = 5.5 keeps every kink |d - d'| =
    T/lambda away from the probes."""
    D = _cost(77, H, W, L)
    cost = torch.from_numpy(D).cuda()
    g = torch.Generator(device="cuda").manual_seed(3)
    v = torch.randn(D.shape, device="cuda", generator=g, dtype=torch.float32)
    b0, ws = vs.sp_forward(cost, FULL)
    c = torch.softmax(-b0.double() / FULL.tau, dim=-1)

    def loss(cst, **kw):
        p = vs.SPParams(**{**FULL.__dict__, **kw})
        b, _ = vs.sp_forward(cst, p)
        return float((b.double() * c).sum())

    _, ws = vs.sp_forward(cost, FULL)
    gD, gpar = vs.sp_backward(cost, FULL, c.float(), ws)
    h = 1e-3
    fd = {
        "lam": (loss(cost, lam=FULL.lam + h) - loss(cost, lam=FULL.lam - h)) / (2 * h),
        "trunc": (loss(cost, trunc=FULL.trunc + h) - loss(cost, trunc=FULL.trunc - h)) / (2 * h),
        "tau": (loss(cost, tau=FULL.tau + h) - loss(cost, tau=FULL.tau - h)) / (2 * h),
        "D": (loss(cost + h * v) - loss(cost - h * v)) / (2 * h),
    }
    adj = {"lam": float(gpar[0]), "trunc": float(gpar[1]), "tau": float(gpar[2]),
           "D": float((gD.double() * v.double()).sum())}
    for k in fd:
        assert abs(adj[k] - fd[k]) <= 1e-3 * abs(fd[k]), (k, adj[k], fd[k])


# --------------------------------------------------------------------------- autograd

def test_autograd_function_matches_the_abi():
    D = _cost(31, 24, 36, 48)
    cost = torch.from_numpy(D).cuda().requires_grad_(True)
    lam = torch.tensor(2.5, device="cuda", requires_grad=True)
    T = torch.tensor(13.7, device="cuda", requires_grad=True)
    tau = torch.tensor(2.0, device="cuda", requires_grad=True)
    b = vs.smooth_bp(cost, lam, T, tau, iters=6, ckpt_every=2)
    gb = torch.randn_like(b)
    (b * gb).sum().backward()
    p = vs.SPParams(labels=48, iters=6, ckpt_every=2, lam=2.5, trunc=13.7, tau=2.0)
    b2, ws = vs.sp_forward(cost.detach(), p)
    gD, gpar = vs.sp_backward(cost.detach(), p, gb, ws)
    assert torch.equal(b.detach(), b2)
    assert torch.equal(cost.grad, gD)
    assert torch.equal(torch.stack([lam.grad, T.grad, tau.grad]), gpar)


def _scene(seed):
    """A 338x190 noise pair with a piecewise-planar disparity of up to 40 px and
    its truncated absolute-difference cost volume (48 labels, T_d = 20)."""
    from paper_1902_09733_b300 import synth
    left, right, gt = synth.noise_pair(seed, w=W, h=H, max_disp=40.0)
    IL = torch.from_numpy(left.astype(np.float32)).cuda()
    IR = torch.from_numpy(right.astype(np.float32)).cuda()
    cost = torch.full((H, W, L), 20.0, device="cuda")
    for d in range(L):
        cost[:, d:, d] = torch.clamp((IL[:, d:] - IR[:, :W - d]).abs(), max=20.0)
    valid = torch.from_numpy(~np.isnan(gt)).cuda()
    valid[:, :L] = False
    return cost.contiguous(), torch.from_numpy(np.nan_to_num(gt)).float().cuda(), valid


def test_fit_smoothness_to_ground_truth():
    """Fit lambda and trunc by gradient descent through the adjoint so the soft
    arg-min of the beliefs approaches the ground-truth disparity of 16 scenes."""
    scenes = [_scene(s) for s in range(16)]
    labels = torch.arange(L, device="cuda", dtype=torch.float32)
    lam = torch.tensor(0.3, device="cuda", requires_grad=True)
    T = torch.tensor(3.1, device="cuda", requires_grad=True)
    tau = 2.0
    opt = torch.optim.Adam([lam, T], lr=0.25)

    def epoch(train=True):
        total = 0.0
        for cost, gt, valid in scenes:
            b = vs.smooth_bp(cost, lam, T, tau, iters=8, ckpt_every=2)
            p = torch.softmax(-b / tau, dim=-1)
            d = (p * labels).sum(-1)
            loss = torch.nn.functional.smooth_l1_loss(d[valid], gt[valid])
            if train:
                opt.zero_grad()
                loss.backward()
                opt.step()
                with torch.no_grad():
                    lam.clamp_(min=0.05)
                    T.clamp_(min=0.5, max=90.0)
            total += float(loss.detach())
        return total / len(scenes)

    with torch.no_grad():
        start = epoch(train=False)
    for _ in range(4):
        epoch()
    with torch.no_grad():
        end = epoch(train=False)
    print(f"fit: loss {start:.3f} -> {end:.3f}, lambda {float(lam):.3f}, trunc {float(T):.3f}")
    assert end < 0.8 * start

"""Pins for the smoothed (log-domain sum-product) BP oracle and its reverse mode.

The oracle (``oracle/vsref_smooth.c``) replaces the minimum of the Eq. 1
min-sum message by the soft minimum -tau log sum exp(-x/tau).  Nothing here
re-types its loops: each test checks it against something fixed independently
of them -- hand-worked messages, exact Gibbs marginals by enumeration on trees
(where sum-product is exact), the tau -> 0 limit (min-sum min-marginals by
enumeration), exact invariances of the model (constant shifts, scaling,
mirror and label reversal) and, for the reverse mode, central finite
differences of the forward pass and Euler's identity for homogeneous functions.
"""
import itertools

import numpy as np
import pytest

import oracle


# --------------------------------------------------------------------------- helpers

def _grid_edges(h, w):
    edges = []
    for y in range(h):
        for x in range(w):
            if x + 1 < w:
                edges.append((y * w + x, y * w + x + 1))
            if y + 1 < h:
                edges.append((y * w + x, (y + 1) * w + x))
    return edges


def _enumerate_energies(D, lam, T):
    """Energy sum_p D_p(x_p) + sum_edges min(lam|x_p - x_q|, T) of every labelling."""
    h, w, L = D.shape
    n = h * w
    X = np.array(list(itertools.product(range(L), repeat=n)), dtype=np.int64)
    Df = D.reshape(n, L)
    E = Df[np.arange(n)[None, :], X].sum(axis=1)
    for p, q in _grid_edges(h, w):
        E = E + np.minimum(lam * np.abs(X[:, p] - X[:, q]), T)
    return X, E


def _gibbs_marginals(D, lam, T, tau):
    h, w, L = D.shape
    X, E = _enumerate_energies(D, lam, T)
    P = np.exp(-(E - E.min()) / tau)
    P /= P.sum()
    out = np.zeros((h * w, L))
    for p in range(h * w):
        out[p] = np.bincount(X[:, p], weights=P, minlength=L)
    return out.reshape(h, w, L)


def _min_marginals(D, lam, T):
    h, w, L = D.shape
    X, E = _enumerate_energies(D, lam, T)
    out = np.full((h * w, L), np.inf)
    for p in range(h * w):
        np.minimum.at(out[p], X[:, p], E)
    return out.reshape(h, w, L)


def _softmax_neg(b, tau):
    z = -(b - b.min(axis=-1, keepdims=True)) / tau
    e = np.exp(z)
    return e / e.sum(axis=-1, keepdims=True)


# --------------------------------------------------------------------------- messages

@pytest.mark.parametrize("case", ["B", "C", "D"])
def test_message_hand_values(golden, case):
    g = golden("sp_message_hand.txt")
    tau = g[f"{case}.tau"][0][0][0]
    lam = g[f"{case}.lam"][0][0][0]
    T = g[f"{case}.T"][0][0][0]
    h = np.array(g[f"{case}.h"][0][0])
    m, mt = oracle.sp_message(h, lam, T, tau, return_unnormalised=True)
    np.testing.assert_allclose(mt, g[f"{case}.mt"][0][0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(m, g[f"{case}.m"][0][0], rtol=0, atol=1e-14)


def test_message_tends_to_min_sum_as_tau_vanishes():
    """softmin_tau -> min as tau -> 0, with error at most tau * log L."""
    rng = np.random.default_rng(3)
    L, lam, T = 9, 1.7, 6.2
    for _ in range(20):
        h = rng.uniform(0, 20, L)
        V = np.minimum(lam * np.abs(np.arange(L)[:, None] - np.arange(L)[None, :]), T)
        ms = (h[None, :] + V).min(axis=1)
        for tau in (1e-2, 1e-4):
            _, mt = oracle.sp_message(h, lam, T, tau, return_unnormalised=True)
            assert np.all(mt <= ms + 1e-12)
            assert np.all(mt >= ms - tau * np.log(L) - 1e-12)


def test_message_shift_and_scale():
    """Adding c to h adds c to mt (normalised message unchanged); scaling h, lam, T
    and tau together by s scales the message by s."""
    rng = np.random.default_rng(4)
    h = rng.uniform(0, 10, 7)
    m, mt = oracle.sp_message(h, 1.3, 4.1, 0.7, return_unnormalised=True)
    m2, mt2 = oracle.sp_message(h + 3.25, 1.3, 4.1, 0.7, return_unnormalised=True)
    np.testing.assert_allclose(mt2, mt + 3.25, atol=1e-12)
    np.testing.assert_allclose(m2, m, atol=1e-12)
    m3 = oracle.sp_message(2.5 * h, 2.5 * 1.3, 2.5 * 4.1, 2.5 * 0.7)
    np.testing.assert_allclose(m3, 2.5 * m, atol=1e-12)
    assert abs(m.mean()) < 1e-14


# --------------------------------------------------------------------------- forward

@pytest.mark.parametrize("vertical", [False, True])
@pytest.mark.parametrize("seed", [0, 1])
def test_chain_beliefs_give_exact_gibbs_marginals(seed, vertical):
    """On a chain (a tree) synchronous sum-product is exact once messages have
    crossed it: softmax(-b/tau) equals the marginals of exp(-E/tau) by enumeration."""
    rng = np.random.default_rng(seed)
    N, L = 5, 4
    D = rng.uniform(0, 6, (1, N, L))
    if vertical:
        D = D.reshape(N, 1, L)
    lam, T, tau = 1.3, 3.7, 0.9
    ref = _gibbs_marginals(D, lam, T, tau)
    for iters in (N - 1, N + 3):
        b = oracle.sp_forward(D, lam, T, tau, iters)
        np.testing.assert_allclose(_softmax_neg(b, tau), ref, rtol=0, atol=1e-12)
    # one iteration short of the diameter is not yet exact at the chain ends
    b = oracle.sp_forward(D, lam, T, tau, N - 2)
    assert np.abs(_softmax_neg(b, tau) - ref).max() > 1e-6


def test_chain_small_tau_gives_min_marginals():
    rng = np.random.default_rng(7)
    N, L = 5, 4
    D = rng.uniform(0, 6, (1, N, L))
    lam, T, tau = 1.3, 3.7, 1e-3
    mm = _min_marginals(D, lam, T)
    b = oracle.sp_forward(D, lam, T, tau, N)
    got = b - b.min(axis=-1, keepdims=True)
    want = mm - mm.min(axis=-1, keepdims=True)
    # soft minima over at most L^N terms differ from minima by at most tau ln(L^N)
    assert np.abs(got - want).max() < 2 * tau * N * np.log(L) + 1e-9


@pytest.mark.parametrize("lam,T", [(0.0, 3.0), (2.0, 0.0)])
def test_no_smoothness_leaves_the_data_term(lam, T):
    rng = np.random.default_rng(11)
    D = rng.uniform(0, 5, (4, 5, 6))
    b, states = oracle.sp_forward(D, lam, T, 0.8, 3, return_states=True)
    np.testing.assert_allclose(b, D, rtol=0, atol=1e-12)
    assert np.abs(states).max() < 1e-12
    gb = rng.normal(size=D.shape)
    gD, glam, gT, gtau = oracle.sp_backward(D, lam, T, 0.8, 3, gb)
    np.testing.assert_allclose(gD, gb, rtol=0, atol=1e-12)
    assert abs(gtau) < 1e-12
    if lam == 0.0:
        assert gT == 0.0


def test_messages_are_mean_free_and_missing_slots_stay_zero():
    rng = np.random.default_rng(12)
    D = rng.uniform(0, 9, (5, 6, 7))
    _, states = oracle.sp_forward(D, 1.1, 4.3, 1.5, 4, return_states=True)
    assert np.abs(states.mean(axis=-1)).max() < 1e-12
    for t in range(5):
        assert np.all(states[t, 0, :, 0] == 0)    # no left neighbour in column 0
        assert np.all(states[t, 1, :, -1] == 0)   # no right neighbour in the last column
        assert np.all(states[t, 2, 0] == 0)
        assert np.all(states[t, 3, -1] == 0)


def test_constant_shift_of_one_pixel_moves_only_its_belief():
    rng = np.random.default_rng(13)
    D = rng.uniform(0, 9, (4, 5, 6))
    b = oracle.sp_forward(D, 1.1, 4.3, 1.5, 4)
    D2 = D.copy()
    D2[2, 3] += 2.75
    b2 = oracle.sp_forward(D2, 1.1, 4.3, 1.5, 4)
    want = b.copy()
    want[2, 3] += 2.75
    np.testing.assert_allclose(b2, want, rtol=0, atol=1e-11)


def test_scale_equivariance():
    rng = np.random.default_rng(14)
    D = rng.uniform(0, 9, (4, 5, 6))
    b = oracle.sp_forward(D, 1.1, 4.3, 1.5, 4)
    b2 = oracle.sp_forward(3.0 * D, 3.3, 12.9, 4.5, 4)
    np.testing.assert_allclose(b2, 3.0 * b, rtol=1e-12, atol=1e-10)


def test_mirror_and_label_reversal():
    rng = np.random.default_rng(15)
    D = rng.uniform(0, 9, (4, 5, 6))
    b = oracle.sp_forward(D, 1.1, 4.3, 1.5, 4)
    np.testing.assert_allclose(oracle.sp_forward(D[:, ::-1], 1.1, 4.3, 1.5, 4), b[:, ::-1], atol=1e-11)
    np.testing.assert_allclose(oracle.sp_forward(D[::-1], 1.1, 4.3, 1.5, 4), b[::-1], atol=1e-11)
    np.testing.assert_allclose(oracle.sp_forward(D[:, :, ::-1], 1.1, 4.3, 1.5, 4), b[:, :, ::-1],
                               atol=1e-11)
    np.testing.assert_allclose(oracle.sp_forward(D.transpose(1, 0, 2), 1.1, 4.3, 1.5, 4),
                               b.transpose(1, 0, 2), atol=1e-11)


# --------------------------------------------------------------------------- reverse mode

def _loss(D, lam, T, tau, iters, gb):
    return float((oracle.sp_forward(D, lam, T, tau, iters) * gb).sum())


@pytest.mark.parametrize("step,rtol", [(1e-3, 1e-4), (1e-5, 1e-8)])
def test_reverse_mode_matches_central_differences(step, rtol):
    """T/lam = 3.43: no kink |d-d'| = T/lam lies within the step of any probe.
    Central differences are off by O(step^2) (about 1e-6 relative at 1e-3 along
    a direction of norm 11), so the tolerance shrinks with the step."""
    rng = np.random.default_rng(21)
    h, w, L, iters = 4, 5, 6, 4
    D = rng.uniform(0, 8, (h, w, L))
    lam, T, tau = 1.2, 4.116, 0.9
    gb = rng.normal(size=D.shape)
    gD, glam, gT, gtau = oracle.sp_backward(D, lam, T, tau, iters, gb)

    f = lambda *a: _loss(*a, iters, gb)
    for _ in range(3):
        v = rng.normal(size=D.shape)
        fd = (f(D + step * v, lam, T, tau) - f(D - step * v, lam, T, tau)) / (2 * step)
        assert abs(fd - (gD * v).sum()) <= rtol * max(abs(fd), 1.0)
    fd_lam = (f(D, lam + step, T, tau) - f(D, lam - step, T, tau)) / (2 * step)
    fd_T = (f(D, lam, T + step, tau) - f(D, lam, T - step, tau)) / (2 * step)
    fd_tau = (f(D, lam, T, tau + step) - f(D, lam, T, tau - step)) / (2 * step)
    for got, fd in ((glam, fd_lam), (gT, fd_T), (gtau, fd_tau)):
        assert abs(got - fd) <= rtol * max(abs(fd), 1.0), (got, fd)


def test_reverse_mode_one_iteration_single_edge():
    """1 x 2 image, one iteration: b_1 = D_1 + m_{0->1}; the gradient of sum(gb * b)
    in D_0 is the message's Jacobian applied to gb_1, which central differences pin."""
    rng = np.random.default_rng(22)
    D = rng.uniform(0, 4, (1, 2, 5))
    lam, T, tau = 0.8, 2.3, 0.6
    gb = rng.normal(size=D.shape)
    gD, *_ = oracle.sp_backward(D, lam, T, tau, 1, gb)
    step = 1e-6
    for d in range(5):
        e = np.zeros_like(D)
        e[0, 0, d] = 1.0
        fd = (_loss(D + step * e, lam, T, tau, 1, gb) - _loss(D - step * e, lam, T, tau, 1, gb)) / (2 * step)
        assert abs(gD[0, 0, d] - fd) < 1e-8


def test_reverse_mode_euler_identity():
    """Beliefs are homogeneous of degree 1 in (D, lam, T, tau), so
    <gD, D> + lam*glam + T*gT + tau*gtau = <gb, b> (Euler's theorem)."""
    rng = np.random.default_rng(23)
    D = rng.uniform(0, 8, (5, 4, 7))
    lam, T, tau = 0.9, 3.3, 1.4
    gb = rng.normal(size=D.shape)
    b = oracle.sp_forward(D, lam, T, tau, 5)
    gD, glam, gT, gtau = oracle.sp_backward(D, lam, T, tau, 5, gb)
    lhs = (gD * D).sum() + lam * glam + T * gT + tau * gtau
    rhs = (gb * b).sum()
    assert abs(lhs - rhs) < 1e-9 * max(abs(rhs), 1.0)


def test_reverse_mode_constant_direction():
    """Adding c to all labels of D_p shifts only b_p by c, so sum_d gD_p(d) = sum_d gb_p(d)."""
    rng = np.random.default_rng(24)
    D = rng.uniform(0, 8, (4, 5, 6))
    gb = rng.normal(size=D.shape)
    gD, *_ = oracle.sp_backward(D, 1.1, 4.3, 1.5, 4, gb)
    np.testing.assert_allclose(gD.sum(axis=-1), gb.sum(axis=-1), rtol=0, atol=1e-10)

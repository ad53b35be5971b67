"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: values
worked by hand from the paper's definitions (tests/golden), brute-force
enumeration on tiny inputs, closed forms, special cases and invariants.
No GPU is needed.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1902_09733_b300 import synth

# ---------------------------------------------------------------------------
# Eq. 1 -- single message


def test_message_hand_values(golden):
    g = golden("message_hand.txt")
    for case in ("A", "B"):
        h = np.array(g[f"{case}.h"][0][0], np.int32)
        c = int(g[f"{case}.c"][0][0][0])
        Ts = int(g[f"{case}.Ts"][0][0][0])
        want = np.array(g[f"{case}.m"][0][0], np.int32)
        for mode in (oracle.MSG_BRUTE, oracle.MSG_DT):
            np.testing.assert_array_equal(oracle.message(h, c, Ts, mode), want)


def test_message_dt_equals_bruteforce():
    """The O(L) two-pass transform equals the O(L^2) definition, exactly."""
    g = np.random.default_rng(1)
    for _ in range(400):
        L = int(g.integers(2, 70))
        c = int(g.integers(0, 30))
        Ts = int(g.integers(0, 120))
        h = g.integers(0, 400, size=L).astype(np.int32)
        a = oracle.message(h, c, Ts, oracle.MSG_BRUTE)
        b = oracle.message(h, c, Ts, oracle.MSG_DT)
        np.testing.assert_array_equal(a, b)
        assert a.min() == 0 and a.max() <= Ts


def test_message_bruteforce_matches_explicit_minimum():
    """The brute-force mode against an independent numpy min-plus product."""
    g = np.random.default_rng(2)
    for _ in range(50):
        L = int(g.integers(2, 40))
        c, Ts = int(g.integers(0, 20)), int(g.integers(0, 60))
        h = g.integers(0, 300, size=L).astype(np.int64)
        d = np.arange(L)
        V = np.minimum(c * np.abs(d[:, None] - d[None, :]), Ts)
        m = (h[None, :] + V).min(axis=1)
        m -= m.min()
        np.testing.assert_array_equal(oracle.message(h, c, Ts, oracle.MSG_BRUTE), m)


# ---------------------------------------------------------------------------
# Eq. 1 -- data term and pyramid


def test_cost_hand_values(golden):
    g = golden("bp_chain3_hand.txt")
    IL = np.array([[50, 52, 50]], np.uint8)
    IR = np.array([[47, 61, 64]], np.uint8)
    want = np.array(g["D0"][0], np.int32)
    np.testing.assert_array_equal(oracle.cost_level0(IL, IR, 3, 20)[0], want)


def test_cost_special_cases():
    g = np.random.default_rng(3)
    IL = g.integers(0, 256, size=(7, 13)).astype(np.uint8)
    c = oracle.cost_level0(IL, IL, 9, 25)
    assert (c[:, :, 0] == 0).all()                 # identical views match at d = 0
    for d in range(9):                             # no partner left of the frame
        assert (c[:, :d, d] == 25).all()
    assert c.max() <= 25 and c.min() >= 0
    # an exact shift IR(x) = IL(x + 3) gives zero cost at d = 3 wherever x >= 3
    IR = np.zeros_like(IL)
    IR[:, :-3] = IL[:, 3:]
    c = oracle.cost_level0(IL, IR, 9, 25)
    assert (c[:, 3:, 3] == 0).all()


@pytest.mark.parametrize("h,w", [(1, 1), (3, 3), (5, 8), (7, 13), (16, 9)])
def test_cost_coarsen_partition(h, w):
    """Every fine pixel has exactly one parent: totals agree, shape halves rounding up."""
    g = np.random.default_rng(h * 100 + w)
    fine = g.integers(0, 50, size=(h, w, 4)).astype(np.int32)
    coarse = oracle.cost_coarsen(fine)
    assert coarse.shape == ((h + 1) // 2, (w + 1) // 2, 4)
    np.testing.assert_array_equal(coarse.sum(axis=(0, 1)), fine.sum(axis=(0, 1)))
    # corner parent owns exactly the 2x2 top-left block
    np.testing.assert_array_equal(coarse[0, 0], fine[:2, :2].sum(axis=(0, 1)))
    # the last parent of an odd row has only the children that exist
    np.testing.assert_array_equal(coarse[-1, -1], fine[2 * ((h + 1) // 2 - 1):, 2 * ((w + 1) // 2 - 1):].sum(axis=(0, 1)))


# ---------------------------------------------------------------------------
# Eq. 1 -- belief propagation


def _hand_messages(g, key):
    return np.array(g[key][0], np.int32)


@pytest.mark.parametrize("mode", [oracle.MSG_BRUTE, oracle.MSG_DT])
def test_bp_hand_chain(golden, mode):
    """1x3 chain worked by hand: schedule, exclusion, normalisation, init, labels."""
    g = golden("bp_chain3_hand.txt")
    IL = np.array([[50, 52, 50]], np.uint8)
    IR = np.array([[47, 61, 64]], np.uint8)
    for tag, levels, iters in (("iters1", 1, 1), ("iters2", 1, 2), ("levels2", 2, 1)):
        lab, m = oracle.bp(IL, IR, 3, levels, iters, 20, 4, 6, mode=mode, return_messages=True)
        np.testing.assert_array_equal(lab[0], np.array(g[f"{tag}.labels"][0][0], np.uint8))
        np.testing.assert_array_equal(m[0, 0], _hand_messages(g, f"{tag}.from_left"))
        np.testing.assert_array_equal(m[1, 0], _hand_messages(g, f"{tag}.from_right"))
        assert not m[2:].any()


@pytest.mark.parametrize("mode", [oracle.MSG_BRUTE, oracle.MSG_DT])
def test_bp_hand_grid_two_levels(golden, mode):
    """3x3 pair, two levels, worked by hand: coarse costs, coarse-to-fine
    initialisation from the parent (x>>1, y>>1), all four directions."""
    g = golden("bp_grid3_two_levels_hand.txt")
    IL = np.array([[10, 20, 30], [40, 50, 60], [70, 80, 90]], np.uint8)
    IR = np.array([[12, 13, 27], [41, 38, 65], [70, 84, 79]], np.uint8)
    lab, m = oracle.bp(IL, IR, 2, 2, 1, 20, 3, 5, mode=mode, return_messages=True)
    np.testing.assert_array_equal(lab, np.array(g["labels"][0], np.uint8))
    for k, name in enumerate(("from_left", "from_right", "from_up", "from_down")):
        np.testing.assert_array_equal(m[k], np.array(g[name][0], np.int32).reshape(3, 3, 2))


def _chain_min_marginals(D, c, Ts):
    """Brute force over all L^n labelings of a chain: min-marginals and energies."""
    n, L = D.shape
    labs = np.array(list(itertools.product(range(L), repeat=n)), np.int64)
    E = D[np.arange(n)[None, :], labs].sum(axis=1)
    E += np.minimum(c * np.abs(np.diff(labs, axis=1)), Ts).sum(axis=1)
    mm = np.stack([np.array([E[labs[:, x] == d].min() for d in range(L)]) for x in range(n)])
    return mm - mm.min(axis=1, keepdims=True), labs, E


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("vertical", [False, True])
def test_bp_chain_beliefs_are_exact_min_marginals(seed, vertical):
    """On a chain (a tree) min-sum BP is exact: after enough iterations the
    beliefs D + incoming equal the brute-force min-marginals, and the labels
    are the optimum when it is unique.  A vertical chain (one column) checks
    the up/down directions; its data term only separates d = 0 from the rest."""
    g = np.random.default_rng(100 + seed)
    n, L = 8, 4
    Td, c, Ts = 20, int(g.integers(1, 8)), int(g.integers(4, 25))
    shape = (n, 1) if vertical else (1, n)
    IL = g.integers(0, 256, size=shape).astype(np.uint8)
    IR = np.clip(IL.astype(int) + g.integers(-15, 16, size=shape), 0, 255).astype(np.uint8)
    D = oracle.cost_level0(IL, IR, L, Td).reshape(n, L).astype(np.int64)
    mm, labs, E = _chain_min_marginals(D, c, Ts)
    dirs = (2, 3) if vertical else (0, 1)
    for mode in (oracle.MSG_BRUTE, oracle.MSG_DT):
        lab, m = oracle.bp(IL, IR, L, 1, 2 * n + 2, Td, c, Ts, mode=mode, return_messages=True)
        b = D + m[dirs[0]].reshape(n, L) + m[dirs[1]].reshape(n, L)
        b -= b.min(axis=1, keepdims=True)
        np.testing.assert_array_equal(b, mm)
        if (E == E.min()).sum() == 1:
            np.testing.assert_array_equal(lab.reshape(n), labs[np.argmin(E)])


@pytest.mark.parametrize("seed", range(4))
def test_bp_winner_take_all_without_smoothness(seed):
    """With c = 0 or Ts = 0 every message is flat, so BP reduces to argmin_d D0."""
    g = np.random.default_rng(200 + seed)
    IL = g.integers(0, 256, size=(9, 14)).astype(np.uint8)
    IR = g.integers(0, 256, size=(9, 14)).astype(np.uint8)
    D = oracle.cost_level0(IL, IR, 7, 30)
    wta = np.argmin(D, axis=2)          # numpy returns the first minimum, the smallest d
    for c, Ts in ((0, 40), (10, 0)):
        lab, m = oracle.bp(IL, IR, 7, 2, 3, 30, c, Ts, return_messages=True)
        assert not m.any()
        np.testing.assert_array_equal(lab, wta)


def test_bp_recovers_integer_shift():
    """IR(x) = IL(x + d0) on strong texture: the disparity d0 is recovered."""
    g = np.random.default_rng(7)
    h, w, d0 = 30, 50, 5
    IL = g.integers(0, 256, size=(h, w)).astype(np.uint8)
    IR = np.zeros_like(IL)
    IR[:, :w - d0] = IL[:, d0:]
    IR[:, w - d0:] = g.integers(0, 256, size=(h, d0))
    lab = oracle.bp(IL, IR, 16, 3, 5, 20, 10, 40, mode=oracle.MSG_DT)
    assert (lab[:, d0:] == d0).mean() == 1.0


def test_bp_message_invariants_and_borders():
    """Every message is normalised to min 0 and capped at Ts; missing
    neighbours never receive one."""
    left, right, _ = synth.noise_pair(3, w=23, h=17)
    Ts = 40
    lab, m = oracle.bp(left, right, 16, 3, 5, 20, 10, Ts, mode=oracle.MSG_DT, return_messages=True)
    assert m.min() == 0 and m.max() <= Ts
    inner = [m[0][:, 1:], m[1][:, :-1], m[2][1:, :], m[3][:-1, :]]
    for a in inner:
        np.testing.assert_array_equal(a.min(axis=-1), 0)
    assert not m[0][:, 0].any() and not m[1][:, -1].any()
    assert not m[2][0].any() and not m[3][-1].any()


def _grid_energy(D, lab, c, Ts):
    E = D[np.arange(D.shape[0])[:, None], np.arange(D.shape[1])[None, :], lab].sum()
    E += np.minimum(c * np.abs(np.diff(lab, axis=1)), Ts).sum()
    E += np.minimum(c * np.abs(np.diff(lab, axis=0)), Ts).sum()
    return int(E)


def test_bp_fixed_point_is_single_pixel_optimal():
    """At a converged min-sum fixed point with unique belief minima, no single
    pixel can change its label and lower the energy (neighbourhood optimality
    of min-sum fixed points, Weiss and Freeman 2001)."""
    checked = 0
    for seed in range(12):
        left, right, _ = synth.noise_pair(seed, w=12, h=10, max_disp=5)
        L, Td, c, Ts = 6, 30, 4, 8
        a_lab, a = oracle.bp(left, right, L, 1, 300, Td, c, Ts, mode=oracle.MSG_DT, return_messages=True)
        b_lab, b = oracle.bp(left, right, L, 1, 302, Td, c, Ts, mode=oracle.MSG_DT, return_messages=True)
        if not np.array_equal(a, b):
            continue                       # oscillating: no fixed point to test
        D = oracle.cost_level0(left, right, L, Td).astype(np.int64)
        bel = D + a.sum(axis=0)
        srt = np.sort(bel, axis=2)
        if (srt[..., 0] == srt[..., 1]).any():
            continue                       # ties: the theorem needs unique minima
        lab = a_lab.astype(np.int64)
        E0 = _grid_energy(D, lab, c, Ts)
        for y in range(lab.shape[0]):
            for x in range(lab.shape[1]):
                for d in range(L):
                    t = lab.copy()
                    t[y, x] = d
                    assert _grid_energy(D, t, c, Ts) >= E0
        checked += 1
    assert checked >= 3


def test_bp_levels_run_on_odd_and_degenerate_sizes():
    """Pyramids on odd sizes down to 1x1 run and keep labels in range."""
    g = np.random.default_rng(11)
    for h, w in ((1, 1), (1, 5), (5, 1), (3, 7), (13, 7)):
        IL = g.integers(0, 256, size=(h, w)).astype(np.uint8)
        IR = g.integers(0, 256, size=(h, w)).astype(np.uint8)
        for mode in (oracle.MSG_BRUTE, oracle.MSG_DT):
            lab = oracle.bp(IL, IR, 5, 4, 3, 20, 4, 12, mode=mode)
            assert lab.shape == (h, w) and lab.max() < 5


# ---------------------------------------------------------------------------
# Section 2.1 -- remap


def test_remap_identity_without_distortion():
    g = np.random.default_rng(20)
    src = g.integers(0, 256, size=(37, 53, 3)).astype(np.uint8)
    cam = (45.0, 41.0, 26.0, 18.0, 0.0, 0.0)
    np.testing.assert_array_equal(oracle.rectify_remap(src, cam), src)


def test_remap_half_turn_rotation():
    """R = half turn about the optical axis with the principal point at the
    frame centre turns the image by 180 degrees."""
    g = np.random.default_rng(21)
    H, W = 30, 44
    src = g.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    cam = (50.0, 50.0, (W - 1) / 2, (H - 1) / 2, 0.0, 0.0)
    R = np.diag([-1.0, -1.0, 1.0])
    np.testing.assert_array_equal(oracle.rectify_remap(src, cam, R=R), src[::-1, ::-1])


def test_remap_quarter_turn_rotation():
    """A quarter turn about the optical axis (square frame, centred principal
    point) rotates the image: the ray of (u, v) is R^T (xn, yn, 1)."""
    g = np.random.default_rng(23)
    N = 24
    src = g.integers(0, 256, size=(N, N, 3)).astype(np.uint8)
    cam = (30.0, 30.0, (N - 1) / 2, (N - 1) / 2, 0.0, 0.0)
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    dst = oracle.rectify_remap(src, cam, R=R)
    vv, uu = np.mgrid[0:N, 0:N]
    np.testing.assert_array_equal(dst, src[N - 1 - uu, vv])


def test_remap_radial_hand_values(golden):
    g = golden("remap_radial_hand.txt")
    cam = g["camera"][0][0]
    W, H = (int(v) for v in g["size"][0][0])
    vv, uu = np.mgrid[0:H, 0:W]
    src = np.zeros((H, W, 3), np.uint8)
    src[..., 0] = 2 * uu + 1
    src[..., 1] = 2 * vv + 1
    src[..., 2] = 100
    _, f = oracle.rectify_remap(src, cam, return_float=True)
    for row in g["pixel"]:
        u, v, sx, sy = row[0]
        np.testing.assert_allclose(f[int(v), int(u)], [2 * sx + 1, 2 * sy + 1, 100.0], rtol=0, atol=1e-9)


def test_remap_mirror_symmetry():
    """The radial model is symmetric about the principal point: mirroring the
    source mirrors the output when cx sits on the frame's centre line."""
    g = np.random.default_rng(22)
    H, W = 40, 60
    src = g.integers(0, 256, size=(H, W, 3)).astype(np.uint8)
    cam = (38.0, 35.0, (W - 1) / 2, 17.25, -0.3, 0.09)
    _, a = oracle.rectify_remap(src, cam, return_float=True)
    _, b = oracle.rectify_remap(src[:, ::-1], cam, return_float=True)
    np.testing.assert_allclose(b, a[:, ::-1], rtol=0, atol=1e-9)
    # the principal point itself never moves
    cam2 = (38.0, 35.0, 30.0, 20.0, -0.3, 0.09)
    np.testing.assert_array_equal(oracle.rectify_remap(src, cam2)[20, 30], src[20, 30])


# ---------------------------------------------------------------------------
# Section 2.2 -- downsample + grey


def test_downsample_constant_and_rounding():
    img = np.full((8, 12, 3), 77, np.uint8)
    low, gray = oracle.downsample_luma(img, 4)
    assert (low == 77).all() and low.shape == (2, 3, 3)
    # half-integer means round up: a 2x2 block of 0,1,0,1 -> (2 + 2) // 4 = 1
    img = np.zeros((2, 2, 3), np.uint8)
    img[0, 1] = img[1, 0] = 1
    low, _ = oracle.downsample_luma(img, 2)
    assert (low == 1).all()
    img[1, 0] = 0                     # mean 0.25 -> 0
    low, _ = oracle.downsample_luma(img, 2)
    assert (low == 0).all()
    # grey of white is 255, of black 0; weights sum to 256
    w, _ = oracle.downsample_luma(np.full((4, 4, 3), 255, np.uint8), 4)
    assert oracle.downsample_luma(np.full((4, 4, 3), 255, np.uint8), 4)[1][0, 0] == 255
    px = np.zeros((1, 1, 3), np.uint8)
    px[0, 0] = (200, 0, 0)
    assert oracle.downsample_luma(px, 1)[1][0, 0] == (77 * 200 + 128) >> 8


def test_downsample_ragged_edge_uses_in_frame_pixels():
    img = np.zeros((5, 5, 3), np.uint8)
    img[4, 4] = 90                      # the corner block holds a single pixel
    low, _ = oracle.downsample_luma(img, 4)
    assert low.shape == (2, 2, 3) and (low[1, 1] == 90).all() and (low[0, 0] == 0).all()


# ---------------------------------------------------------------------------
# Eq. 2 -- joint bilateral upsampling


def test_jbu_constant_disparity_is_exact():
    g = np.random.default_rng(30)
    lab = np.full((11, 9), 7, np.uint8)
    gl = g.integers(0, 256, size=(11, 9, 3)).astype(np.uint8)
    gf = g.integers(0, 256, size=(44, 36, 3)).astype(np.uint8)
    d = oracle.guided_upsample(lab, gl, gf, 4, 2, 1.0, 12.0)
    np.testing.assert_allclose(d, 28.0, rtol=1e-13)


def test_jbu_flat_kernels_reduce_to_window_mean():
    """With both Gaussians made flat the weights are uniform: D_p is s times the
    mean of the clipped 5x5 window centred at round-half-up(p_down)."""
    g = np.random.default_rng(31)
    h, w, s = 6, 7, 4
    lab = g.integers(0, 64, size=(h, w)).astype(np.uint8)
    gl = g.integers(0, 256, size=(h, w, 3)).astype(np.uint8)
    gf = g.integers(0, 256, size=(h * s, w * s, 3)).astype(np.uint8)
    d = oracle.guided_upsample(lab, gl, gf, s, 2, 1e9, 1e9)
    for y in range(h * s):
        for x in range(w * s):
            cx = int(np.floor((x + 0.5) / s - 0.5 + 0.5))
            cy = int(np.floor((y + 0.5) / s - 0.5 + 0.5))
            win = lab[max(cy - 2, 0):cy + 3, max(cx - 2, 0):cx + 3].astype(float)
            assert abs(d[y, x] - s * win.mean()) < 1e-6


def test_jbu_mirror_symmetry():
    """Centre-aligned sampling is mirror symmetric when W = s * w."""
    g = np.random.default_rng(32)
    h, w, s = 8, 10, 4
    lab = g.integers(0, 64, size=(h, w)).astype(np.uint8)
    gl = g.integers(0, 256, size=(h, w, 3)).astype(np.uint8)
    gf = g.integers(0, 256, size=(h * s, w * s, 3)).astype(np.uint8)
    a = oracle.guided_upsample(lab, gl, gf, s, 2, 1.0, 12.0)
    b = oracle.guided_upsample(lab[:, ::-1], gl[:, ::-1], gf[:, ::-1], s, 2, 1.0, 12.0)
    np.testing.assert_allclose(b, a[:, ::-1], rtol=1e-12)
    c = oracle.guided_upsample(lab[::-1], gl[::-1], gf[::-1], s, 2, 1.0, 12.0)
    np.testing.assert_allclose(c, a[::-1], rtol=1e-12)


def test_jbu_linear_ramp_at_unit_scale():
    """s = 1, flat guide: symmetric weights reproduce a linear ramp inside the frame."""
    h, w = 9, 12
    lab = np.tile((3 * np.arange(w) + 2).astype(np.uint8), (h, 1))
    gl = np.full((h, w, 3), 50, np.uint8)
    d = oracle.guided_upsample(lab, gl, gl, 1, 2, 1.0, 12.0)
    np.testing.assert_allclose(d[:, 2:w - 2], lab[:, 2:w - 2].astype(float), rtol=1e-12)


def test_jbu_range_kernel_follows_full_res_colour():
    """Across a colour edge the range kernel picks the side of I_p: a pixel
    takes the disparity of the low-res pixels of its own colour."""
    h, w, s = 6, 8, 4
    gl = np.zeros((h, w, 3), np.uint8)
    gl[:, w // 2:] = 255
    lab = np.zeros((h, w), np.uint8)
    lab[:, :w // 2] = 5
    lab[:, w // 2:] = 9
    gf = np.zeros((h * s, w * s, 3), np.uint8)
    gf[:, (w // 2) * s:] = 255
    d = oracle.guided_upsample(lab, gl, gf, s, 2, 1.0, 12.0)
    np.testing.assert_allclose(d[:, :(w // 2) * s], 5 * s, rtol=1e-9)
    np.testing.assert_allclose(d[:, (w // 2) * s:], 9 * s, rtol=1e-9)


def test_jbu_range_kernel_uses_full_res_detail():
    """The range kernel compares the full-res colour I_p, not the low-res colour
    under p: a thin full-res stripe absent from the low-res guide takes the
    disparity of the matching low-res colour elsewhere in its window."""
    h, w, s = 5, 10, 4
    gl = np.zeros((h, w, 3), np.uint8)
    gl[:, 3] = 255
    lab = np.full((h, w), 5, np.uint8)
    lab[:, 3] = 9
    gf = np.zeros((h * s, w * s, 3), np.uint8)
    gf[:, 20:24] = 255                  # under low-res column 5, which is dark
    d = oracle.guided_upsample(lab, gl, gf, s, 2, 1.0, 12.0)
    np.testing.assert_allclose(d[:, 20:22], 9 * s, rtol=1e-9)


def test_jbu_hand_worked_weights(golden):
    """Eq. 2 values worked by hand, exponent by exponent, at a clipped corner,
    an interior window and a second clipped corner (tests/golden/jbu_hand.txt).
    These fix the numeric scale of both Gaussians: the factor 2 in 2 sigma^2,
    sigma_s in low-res pixels and the Euclidean RGB distance."""
    g = golden("jbu_hand.txt")
    w, h, W, H = (int(v) for v in g["size"][0][0])
    s, r, sig_s, sig_r = g["params"][0][0]
    lab = np.array(g["lab"][0], np.uint8)
    gl = np.array(g["glow"][0], np.uint8).reshape(h, w, 3)
    gf = np.zeros((H, W, 3), np.uint8)
    pix = [row[0] for row in g["pixel"]]
    for x, y, R, G, B, _ in pix:
        gf[int(y), int(x)] = (int(R), int(G), int(B))
    d = oracle.guided_upsample(lab, gl, gf, int(s), int(r), sig_s, sig_r)
    for x, y, _, _, _, want in pix:
        assert abs(d[int(y), int(x)] - want) <= 1e-12 * want, (x, y, d[int(y), int(x)], want)


def test_jbu_two_taps_closed_form(golden):
    """Two taps on a flat guide: D_p = s (w1 d1 + w2 d2) / (w1 + w2) with
    w = exp(-ds2 / 2), the decimal values of tests/golden/jbu_hand.txt."""
    g = golden("jbu_hand.txt")
    lab = np.array([[0, 10]], np.uint8)
    gl = np.full((1, 2, 3), 77, np.uint8)
    gf = np.full((2, 4, 3), 77, np.uint8)
    d = oracle.guided_upsample(lab, gl, gf, 2, 1, 1.0, 12.0)
    for x, y, want in (row[0] for row in g["two"]):
        assert abs(d[int(y), int(x)] - want) <= 1e-12 * want


# ---------------------------------------------------------------------------
# Eq. 3 -- reprojection


def test_reproject_inverts_the_forward_projection():
    """Points projected with the first line of Eq. 3 (u = fx x/z + u0,
    v = fy y/z + v0, d = fx B / z) come back from the second line."""
    g = np.random.default_rng(40)
    H, W = 20, 30
    fx, fy, cx, cy, B = 1400.0, 1300.0, 14.5, 9.5, 0.5
    z = g.uniform(5.0, 50.0, size=(H, W))
    vv, uu = np.mgrid[0:H, 0:W].astype(float)
    x = (uu - cx) * z / fx
    y = (vv - cy) * z / fy
    disp = fx * B / z
    disp[3, 4] = 0.0
    disp[5, 6] = -2.0
    xyz = oracle.reproject(disp, (fx, fy, cx, cy), B)
    ok = disp > 0
    np.testing.assert_allclose(xyz[ok], np.stack([x, y, z], -1)[ok], rtol=1e-12, atol=1e-12)
    assert np.isnan(xyz[~ok]).all()


# ---------------------------------------------------------------------------
# threads


def test_thread_count_does_not_change_results():
    """The row loops run over OpenMP threads; one thread and many give the same
    remap, grey, BP labels and messages, and JBU disparities, bit for bit."""
    g = np.random.default_rng(50)
    frame = g.integers(0, 256, size=(47, 61, 3)).astype(np.uint8)
    cam = (60.0, 58.0, 30.0, 23.0, -0.2, 0.05)
    left, right, _ = synth.noise_pair(4, w=61, h=47, max_disp=8.0)
    n0 = oracle.set_threads(0)
    try:
        out = []
        for n in (1, max(2, n0)):
            oracle.set_threads(n)
            rem = oracle.rectify_remap(frame, cam)
            low, grey = oracle.downsample_luma(rem, 2)
            lab, msg = oracle.bp(left, right, 16, 3, 4, 20, 10, 40, mode=oracle.MSG_DT, return_messages=True)
            disp = oracle.guided_upsample(lab[:24, :31].copy(), low, rem, 2, 2, 1.0, 12.0)
            out.append((rem, grey, lab, msg, disp))
        for a, b in zip(*out):
            np.testing.assert_array_equal(a, b)
    finally:
        oracle.set_threads(n0)

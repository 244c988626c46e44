"""Pins for the oracle's post-filters (announced in Section 5 of the paper):
adaptive P2, the sub-pixel disparity and the left-right consistency check.

Each pin computes the expected value a second way that shares nothing with
the C code: brute-force path energies, exact rational arithmetic for the
parabola vertex, numpy medians, and a pair with a known constant shift.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
import stereo_synth as synth

DIRS8 = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (1, -1), (-1, -1)]


def path_energy_var(mc_seq, P1, p2_steps):
    """Brute-force path energy with a jump penalty per step: V(d_{i-1}, d_i) =
    0 (equal), min(P1, P2_i) (change of one), P2_i (larger change)."""
    n, D = mc_seq.shape
    E = np.full((n, D), np.iinfo(np.int64).max, dtype=np.int64)
    for k in range(n):
        for seq in itertools.product(range(D), repeat=k + 1):
            e = sum(int(mc_seq[i, seq[i]]) for i in range(k + 1))
            for i in range(1, k + 1):
                diff = abs(seq[i] - seq[i - 1])
                e += 0 if diff == 0 else (min(P1, p2_steps[i]) if diff == 1 else p2_steps[i])
            E[k, seq[-1]] = min(E[k, seq[-1]], e)
    return E


def path_pixels(W, H, rx, ry, x, y):
    pts = [(x, y)]
    while 0 <= x - rx < W and 0 <= y - ry < H:
        x, y = x - rx, y - ry
        pts.append((x, y))
    return pts[::-1]


@pytest.mark.parametrize("P1,P2", [(1, 9), (2, 40), (3, 3), (5, 2)])
@pytest.mark.parametrize("r", DIRS8)
def test_adaptive_p2_matches_brute_force_path_energy(P1, P2, r):
    rng = np.random.default_rng(hash((P1, P2, r)) & 0xFFFF)
    H, W, D = 4, 5, 3
    MC = rng.integers(0, 32, (H, W, D)).astype(np.uint8)
    Ib = rng.integers(0, 12, (H, W)).astype(np.uint8)  # small steps, so P2 / (1 + g) varies
    L = oracle.aggregate_ex(MC, Ib, P1, P2, *r)
    for y in range(H):
        for x in range(W):
            pts = path_pixels(W, H, r[0], r[1], x, y)
            if len(pts) > 4:
                continue
            seq = np.stack([MC[py, px] for (px, py) in pts])
            p2s = [0] + [max(P1, P2 // (1 + abs(int(Ib[b[1], b[0]]) - int(Ib[a[1], a[0]]))))
                         for a, b in zip(pts[:-1], pts[1:])]
            E = path_energy_var(seq, P1, p2s)
            expect = E[-1] - (E[-2].min() if len(pts) > 1 else 0)
            assert L[y, x].tolist() == expect.tolist(), (r, x, y)


@pytest.mark.parametrize("r", DIRS8)
def test_adaptive_p2_on_a_flat_base_image_is_the_constant_p2(r):
    rng = np.random.default_rng(5)
    MC = rng.integers(0, 32, (9, 11, 8)).astype(np.uint8)
    flat = np.full((9, 11), 77, np.uint8)
    assert (oracle.aggregate_ex(MC, flat, 7, 84, *r) == oracle.aggregate(MC, 7, 84, *r)).all()
    assert (oracle.aggregate_ex(MC, None, 7, 84, *r) == oracle.aggregate(MC, 7, 84, *r)).all()


def test_subpixel_exact_parabolas():
    # S(d) = (4d - 21)^2: vertex at 5.25 -> 16 * 5 + 4
    S = np.array([(4 * d - 21) ** 2 for d in range(10)], np.int32)
    assert int(np.argmin(S)) == 5 and oracle.subpixel(S, 5) == 84
    # symmetric neighbours: no offset
    S = np.array([9, 4, 1, 4, 9], np.int32)
    assert oracle.subpixel(S, 2) == 32
    # S(d+1) == S(d) (d is the lowest of the tie): the vertex is half-way, +8/16
    S = np.array([10, 3, 3, 10], np.int32)
    assert oracle.subpixel(S, 1) == 16 + 8
    # the ends of the range get no offset
    assert oracle.subpixel(np.array([1, 2, 3], np.int32), 0) == 0
    assert oracle.subpixel(np.array([3, 2, 1], np.int32), 2) == 32


def test_subpixel_against_exact_rationals():
    rng = np.random.default_rng(11)
    for _ in range(2000):
        D = int(rng.integers(3, 40))
        S = rng.integers(0, 2000, D).astype(np.int32)
        d = int(np.argmin(S))  # lowest d on ties, as Eq. 4
        got = oracle.subpixel(S, d)
        if d in (0, D - 1):
            assert got == 16 * d
            continue
        a, b, c = int(S[d - 1]), int(S[d]), int(S[d + 1])
        off = Fraction(16 * (a - c), 2 * (a + c - 2 * b))  # the vertex offset in 1/16 pixel
        rounded = int((off + Fraction(1, 2)).__floor__())  # halves rounded up
        assert got == 16 * d + rounded
        assert -8 <= got - 16 * d <= 8


def test_median_u16_against_numpy():
    rng = np.random.default_rng(2)
    v = rng.integers(0, 4096, (13, 17)).astype(np.uint16)
    out = oracle.median3x3_u16(v)
    for y in range(1, 12):
        for x in range(1, 16):
            assert out[y, x] == int(np.median(v[y - 1:y + 2, x - 1:x + 2]))
    assert (out[0] == v[0]).all() and (out[-1] == v[-1]).all()
    assert (out[:, 0] == v[:, 0]).all() and (out[:, -1] == v[:, -1]).all()


@pytest.mark.parametrize("n_paths", [2, 4, 8])
@pytest.mark.parametrize("census", ["csct", "ct62"])
def test_no_post_filter_is_16_times_the_plain_path(n_paths, census):
    pair = synth.make_pair(synth.PairSpec(50, 31, 32, 3, 2, 20), 40 + n_paths)
    got = oracle.sgm_ex(pair.left, pair.right, 32, 7, 60, n_paths, 0, census)
    assert (got == 16 * oracle.sgm(pair.left, pair.right, 32, 7, 60, n_paths, census=census).astype(np.uint16)).all()


def test_subpixel_output_stays_within_half_a_pixel_of_the_winner():
    pair = synth.make_pair(synth.PairSpec(60, 40, 64, 4, 2, 40), 8)
    r = oracle.sgm_ex(pair.left, pair.right, 64, 7, 84, 4, oracle.POST_SUBPIXEL, debug=True)
    assert (r["dL"] == oracle.sgm(pair.left, pair.right, 64, 7, 84, 4, debug=True)["raw"]).all()
    # border ring (copied by the median): within half a pixel of the winner
    out, dL = r["out"].astype(np.int64), r["dL"].astype(np.int64)
    for ring in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
        assert (np.abs(out[ring] - 16 * dL[ring]) <= 8).all()


@pytest.mark.parametrize("d0", [4, 9])
def test_lr_check_on_a_known_shift(d0):
    """Noise-free textured pair shifted by d0: both passes find d0 in the
    interior, so the check passes there; left pixels with x < d_L fail."""
    H, W, D = 48, 96, 32
    big = synth.box3(synth.uniform_int(synth.stream_u64(77, 1, H * (W + d0)), 0, 255)
                     .astype(np.uint8).reshape(H, W + d0))
    left = big[:, :W].copy()
    right = big[:, d0:d0 + W].copy()
    r = oracle.sgm_ex(left, right, D, 7, 84, 4, oracle.POST_LR_CHECK, debug=True)
    assert (r["dL"][16:H - 16, d0 + 16:W - 16] == d0).all()
    # right pixel x matches left pixel x + d0: d_R = d0 wherever x + d0 stays inside
    assert (r["dR"][16:H - 16, 16:W - 16 - d0] == d0).all()
    assert (r["out"][16:H - 16, d0 + 16:W - 16] == 16 * d0).all()
    xs = np.arange(W)[None, :]
    assert (r["out"][xs < r["dL"].astype(np.int64)] == oracle.DISP16_INVALID).all()


@pytest.mark.parametrize("post", [oracle.POST_LR_CHECK, oracle.POST_LR_CHECK | oracle.POST_SUBPIXEL])
def test_lr_check_marks_exactly_the_inconsistent_pixels(post):
    pair = synth.make_pair(synth.PairSpec(70, 36, 32, 4, 2, 24), 12)
    r = oracle.sgm_ex(pair.left, pair.right, 32, 7, 84, 8, post, debug=True)
    plain = oracle.sgm_ex(pair.left, pair.right, 32, 7, 84, 8, post & ~oracle.POST_LR_CHECK)
    dL, dR = r["dL"].astype(np.int64), r["dR"].astype(np.int64)
    H, W = dL.shape
    bad = np.zeros((H, W), bool)
    for y in range(H):
        for x in range(W):
            xr = x - dL[y, x]
            bad[y, x] = xr < 0 or abs(dL[y, x] - dR[y, xr]) > 1
    assert bad.any() and not bad.all()
    assert (r["out"][bad] == oracle.DISP16_INVALID).all()
    assert (r["out"][~bad] == plain[~bad]).all()

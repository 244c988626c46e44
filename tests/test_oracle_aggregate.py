"""Pins for the oracle's Eq. 3 (path aggregation, Section 3.2).

The main pin is the path energy: along one path p0, p1, ..., pn,
E(pk, d) = min over disparity sequences ending in d of
sum MC(pi, di) + sum V(d_{i-1}, d_i), with V = 0 for equal disparities,
min(P1, P2) for a change of one and P2 otherwise.  Eq. 3 subtracts the
previous minimum at each step, so L(pk, d) = E(pk, d) - min_d' E(p_{k-1}, d')
(and L = E = MC at the first pixel).  E is computed here by enumerating every
disparity sequence, which shares nothing with the recurrence.
"""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dp_worked_example.txt")
DIRS8 = [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (1, -1), (-1, -1)]


def path_energy(mc_seq, P1, P2):
    """E(p_k, d) for every k by brute force over all disparity sequences."""
    n, D = mc_seq.shape
    E = np.full((n, D), np.iinfo(np.int64).max, dtype=np.int64)
    for k in range(n):
        for seq in itertools.product(range(D), repeat=k + 1):
            e = sum(int(mc_seq[i, seq[i]]) for i in range(k + 1))
            for i in range(1, k + 1):
                diff = abs(seq[i] - seq[i - 1])
                e += 0 if diff == 0 else (min(P1, P2) if diff == 1 else P2)
            E[k, seq[-1]] = min(E[k, seq[-1]], e)
    return E


def path_pixels(W, H, rx, ry, x, y):
    """Pixels of the path through (x, y) along r, from its first pixel to (x, y)."""
    pts = [(x, y)]
    while 0 <= x - rx < W and 0 <= y - ry < H:
        x, y = x - rx, y - ry
        pts.append((x, y))
    return pts[::-1]


def test_worked_example_golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, *v = line.split()
            vals[k] = [int(t) for t in v]
    D, P1, P2 = vals["D"][0], vals["P1"][0], vals["P2"][0]
    MC = np.array(vals["MC"], dtype=np.uint8).reshape(1, 3, D)
    L = oracle.aggregate(MC, P1, P2, 1, 0)
    assert L.reshape(-1).tolist() == vals["L"]


@pytest.mark.parametrize("P1,P2", [(1, 3), (2, 2), (0, 5), (3, 1), (7, 84)])
@pytest.mark.parametrize("r", DIRS8)
def test_matches_brute_force_path_energy(P1, P2, r):
    rng = np.random.default_rng(hash((P1, P2, r)) & 0xFFFF)
    H, W, D = 4, 5, 3
    MC = rng.integers(0, 32, (H, W, D)).astype(np.uint8)
    L = oracle.aggregate(MC, P1, P2, *r)
    for y in range(H):
        for x in range(W):
            pts = path_pixels(W, H, r[0], r[1], x, y)
            if len(pts) > 4:
                continue
            seq = np.stack([MC[py, px] for (px, py) in pts])
            E = path_energy(seq, P1, P2)
            expect = E[-1] - (E[-2].min() if len(pts) > 1 else 0)
            assert L[y, x].tolist() == expect.tolist(), (r, x, y)


def test_long_1d_path_energy_with_d4():
    rng = np.random.default_rng(21)
    MC = rng.integers(0, 32, (1, 6, 4)).astype(np.uint8)
    for P1, P2 in [(2, 9), (5, 5)]:
        L = oracle.aggregate(MC, P1, P2, 1, 0)
        E = path_energy(MC[0], P1, P2)
        for k in range(1, 6):
            assert L[0, k].tolist() == (E[k] - E[k - 1].min()).tolist()


@pytest.mark.parametrize("r", DIRS8)
def test_zero_penalties_give_the_matching_cost(r):
    rng = np.random.default_rng(22)
    MC = rng.integers(0, 32, (9, 11, 8)).astype(np.uint8)
    assert (oracle.aggregate(MC, 0, 0, *r) == MC).all()


@pytest.mark.parametrize("P1,P2", [(7, 84), (10, 120), (0, 224), (224, 224), (3, 2)])
@pytest.mark.parametrize("r", DIRS8)
def test_bounds(P1, P2, r):
    """0 <= L - MC <= P2, and the step minimum never exceeds 31."""
    rng = np.random.default_rng(23)
    MC = rng.integers(0, 32, (10, 12, 16)).astype(np.uint8)
    L = oracle.aggregate(MC, P1, P2, *r).astype(np.int64)
    diff = L - MC
    assert diff.min() >= 0 and diff.max() <= P2
    assert L.min(axis=2).max() <= 31


def test_huge_equal_penalties_keep_one_disparity_per_path():
    """With P1 = P2 above any reachable L, L(p, .) - min = cumulative MC - min."""
    rng = np.random.default_rng(24)
    MC = rng.integers(0, 32, (1, 12, 6)).astype(np.uint8)
    big = 100000
    L = oracle.aggregate(MC, big, big, 1, 0).astype(np.int64)
    cum = np.cumsum(MC[0].astype(np.int64), axis=0)
    for x in range(12):
        assert (L[0, x] - L[0, x].min()).tolist() == (cum[x] - cum[x].min()).tolist()


def test_first_pixel_of_each_path_is_the_matching_cost():
    rng = np.random.default_rng(25)
    H, W, D = 6, 7, 5
    MC = rng.integers(0, 32, (H, W, D)).astype(np.uint8)
    for (rx, ry) in DIRS8:
        L = oracle.aggregate(MC, 4, 30, rx, ry)
        for y in range(H):
            for x in range(W):
                if not (0 <= x - rx < W and 0 <= y - ry < H):
                    assert (L[y, x] == MC[y, x]).all()


def test_direction_sets():
    assert oracle.directions(2) == [(1, 0), (0, 1)]
    assert oracle.directions(4) == [(1, 0), (0, 1), (-1, 0), (0, -1)]
    assert sorted(oracle.directions(8)) == sorted(DIRS8)
    assert oracle.directions(3) == []

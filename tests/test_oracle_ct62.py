"""Pins for the oracle's full 9x7 Census (62-bit features, the CT the paper
contrasts with its CSCT in Section 2) that do not restate it."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ct62_patterns.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, W, H, rule, cx, cy, hexv = line.split()
        rows.append((name, int(W), int(H), rule, int(cx), int(cy), int(hexv, 16)))
    return rows


@pytest.mark.parametrize("row", _golden_rows(), ids=lambda r: r[0])
def test_hand_derived_patterns(row):
    name, W, H, rule, cx, cy, expected = row
    ys, xs = np.mgrid[0:H, 0:W]
    img = np.asarray(eval(rule, {"x": xs, "y": ys}), dtype=np.int64) * np.ones((H, W), dtype=np.int64)
    img = img.astype(np.uint8)
    F = oracle.ct62(img)
    assert int(F[cy, cx]) == expected, f"{name}: got {int(F[cy, cx]):#018x}, expected {expected:#018x}"
    mask = np.ones((H, W), dtype=bool)
    mask[cy, cx] = False
    assert not F[mask].any()
    assert oracle.ct62_at(img, cx, cy) == expected


def test_constant_image_interior_all_ones_border_zero():
    img = np.full((20, 30), 77, dtype=np.uint8)
    F = oracle.ct62(img)
    assert (F[3:-3, 4:-4] == (1 << 62) - 1).all()
    inner = np.zeros_like(F, dtype=bool)
    inner[3:-3, 4:-4] = True
    assert (F[~inner] == 0).all()


def test_bits_above_61_never_set_and_popcount_bounds():
    img = np.random.default_rng(4).integers(0, 256, (40, 50), dtype=np.uint8)
    F = oracle.ct62(img)
    assert (F >> np.uint64(62) == 0).all()
    MC = oracle.cost64(F, F, 16)
    assert (MC[:, :, 0] == 0).all()  # a feature against itself
    assert MC.max() <= 62


def test_invariant_under_strictly_increasing_intensity_map():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 200, (30, 40), dtype=np.uint8)
    lut = np.cumsum(rng.integers(1, 2, 256)).clip(0, 255).astype(np.uint8)  # strictly increasing on [0, 200)
    assert (np.diff(lut[:200].astype(int)) > 0).all()
    assert (oracle.ct62(lut[img]) == oracle.ct62(img)).all()


def test_bitcount64_matches_python():
    rng = np.random.default_rng(6)
    for v in [0, 1, (1 << 62) - 1, (1 << 64) - 1] + [int(x) for x in rng.integers(0, 2**63, 50, dtype=np.uint64)]:
        assert oracle.bitcount64(v) == bin(v).count("1")


def test_cost_left_of_image_uses_zero_match_feature():
    img = np.random.default_rng(7).integers(0, 256, (12, 20), dtype=np.uint8)
    F = oracle.ct62(img)
    MC = oracle.cost64(F, F, 12)
    for x in range(12):
        for d in range(x + 1, 12):
            assert (MC[:, x, d] == [bin(int(v)).count("1") for v in F[:, x]]).all()


def test_identical_images_give_zero_disparity():
    img = np.random.default_rng(8).integers(0, 256, (24, 33), dtype=np.uint8)
    for n_paths in (2, 4, 8):
        assert not oracle.sgm(img, img, 32, 7, 84, n_paths, census="ct62").any()


def test_zero_penalties_reduce_to_local_census_matching():
    # P1 = P2 = 0 gives L_r = MC for every path, so the raw disparity is the
    # lowest argmin of MC (a plain local Census matcher)
    rng = np.random.default_rng(9)
    left = rng.integers(0, 256, (20, 30), dtype=np.uint8)
    right = rng.integers(0, 256, (20, 30), dtype=np.uint8)
    out = oracle.sgm(left, right, 16, 0, 0, 4, debug=True, census="ct62")
    MC = oracle.cost64(oracle.ct62(left), oracle.ct62(right), 16)
    assert (out["raw"] == MC.argmin(axis=2)).all()
    assert (out["S"] == 4 * MC.astype(np.int32)).all()


def test_known_shift_recovered_in_the_interior():
    rng = np.random.default_rng(10)
    base = rng.integers(0, 256, (48, 96), dtype=np.uint8)
    d0 = 7
    left = base
    right = np.zeros_like(base)
    right[:, : 96 - d0] = base[:, d0:]
    right[:, 96 - d0 :] = rng.integers(0, 256, (48, d0), dtype=np.uint8)
    disp = oracle.sgm(left, right, 32, 7, 84, 4, census="ct62")
    assert (disp[16:-16, d0 + 16 : -16] == d0).all()

"""Pins for the oracle's Eq. 1 (CSCT 9x7, Section 3.1) that do not restate it."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "csct_patterns.txt")


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
    F = oracle.csct(img)
    assert int(F[cy, cx]) == expected, f"{name}: got {int(F[cy, cx]):#010x}, expected {expected:#010x}"
    # every other pixel of a 9x7 image lies within 4 columns / 3 rows of the border
    mask = np.ones((H, W), dtype=bool)
    mask[cy, cx] = False
    assert not F[mask].any()


def test_constant_image_interior_all_ones_border_zero():
    img = np.full((20, 30), 77, dtype=np.uint8)
    F = oracle.csct(img)
    assert (F[3:-3, 4:-4] == 0x7FFFFFFF).all()
    inner = np.zeros_like(F, dtype=bool)
    inner[3:-3, 4:-4] = True
    assert (F[~inner] == 0).all()


def test_too_small_images_have_no_valid_window():
    for H, W in [(6, 9), (7, 8), (1, 1), (3, 40)]:
        img = np.random.default_rng(1).integers(0, 256, (H, W), dtype=np.uint8)
        assert not oracle.csct(img).any()


def test_bits_above_30_never_set():
    img = np.random.default_rng(2).integers(0, 256, (40, 50), dtype=np.uint8)
    assert (oracle.csct(img) >> 31 == 0).all()


def test_invariant_under_strictly_increasing_intensity_map():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 200, (30, 40), dtype=np.uint8)
    mapped = (img.astype(np.int32) + 55).astype(np.uint8)  # strictly increasing on [0, 200)
    assert (oracle.csct(img) == oracle.csct(mapped)).all()
    squashed = (img.astype(np.int32) * 255 // 199).astype(np.uint8)  # strictly increasing on [0, 199]
    assert (oracle.csct(img) == oracle.csct(squashed)).all()


def test_mirror_in_x_complements_the_i_ge_1_bits_of_tie_free_images():
    """Mirroring x maps the pair (i, j) onto (i, -j) with its operands swapped.

    On an image whose values inside every window are distinct, s(b, a) =
    1 - s(a, b), so the mirrored feature's bit (i, j) is the complement of the
    original bit (i, -j); the three i = 0 bits do not change.
    """
    rng = np.random.default_rng(4)
    H, W = 7, 9
    img = rng.permutation(256)[: H * W].reshape(H, W).astype(np.uint8)
    f = oracle.csct_at(img, 4, 3)
    g = oracle.csct_at(img[:, ::-1].copy(), 4, 3)
    for i in range(1, 5):
        for j in range(-3, 4):
            b_orig = (f >> ((i - 1) * 7 + (-j + 3))) & 1
            b_mirr = (g >> ((i - 1) * 7 + (j + 3))) & 1
            assert b_mirr == 1 - b_orig
    assert (f >> 28) == (g >> 28)


def test_feature_of_band_matches_full_image_row():
    """Eq. 1 at (x, y) only reads rows y-3..y+3."""
    rng = np.random.default_rng(5)
    img = rng.integers(0, 256, (25, 33), dtype=np.uint8)
    F = oracle.csct(img)
    for y in range(3, 22):
        band = img[y - 3:y + 4].copy()
        assert (oracle.csct(band)[3] == F[y]).all()

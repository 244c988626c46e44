"""Pins for the oracle's Eq. 2 (matching cost, Section 3.1)."""
import numpy as np

import oracle


def test_bitcount_matches_python_popcount():
    rng = np.random.default_rng(10)
    vals = [0, 1, 0x7FFFFFFF, 0xFFFFFFFF, 0x80000000] + [int(v) for v in rng.integers(0, 2**32, 2000, dtype=np.uint64)]
    for v in vals:
        assert oracle.bitcount(v) == bin(v).count("1")


def test_identical_images_have_zero_cost_at_zero_disparity():
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, (30, 50), dtype=np.uint8)
    F = oracle.csct(img)
    MC = oracle.cost(F, F, 16)
    assert (MC[:, :, 0] == 0).all()
    assert MC.max() <= 31


def test_match_left_of_the_image_uses_zero_feature():
    rng = np.random.default_rng(12)
    a = rng.integers(0, 256, (20, 40), dtype=np.uint8)
    b = rng.integers(0, 256, (20, 40), dtype=np.uint8)
    Fa, Fb = oracle.csct(a), oracle.csct(b)
    D = 32
    MC = oracle.cost(Fa, Fb, D)
    pc = np.vectorize(lambda v: bin(int(v)).count("1"))(Fa)
    for x in range(D):
        for d in range(x + 1, D):
            assert (MC[:, x, d] == pc[:, x]).all()


def test_pure_shift_has_zero_cost_at_the_shift():
    """right(x) = left(x + s) => F_R(x - s) = F_L(x) wherever both windows fit."""
    rng = np.random.default_rng(13)
    H, W, s = 20, 60, 7
    big = rng.integers(0, 256, (H, W + s), dtype=np.uint8)
    left = big[:, :W].copy()
    right = big[:, s:s + W].copy()
    MC = oracle.cost(oracle.csct(left), oracle.csct(right), 16)
    # x-s must be a valid window centre of the right image and x of the left
    assert (MC[3:H - 3, 4 + s:W - 4, s] == 0).all()


def test_cost_is_symmetric_hamming_distance():
    """MC(x, d) computed base->match equals the distance match->base at x-d."""
    rng = np.random.default_rng(14)
    a = rng.integers(0, 256, (12, 30), dtype=np.uint8)
    b = rng.integers(0, 256, (12, 30), dtype=np.uint8)
    Fa, Fb = oracle.csct(a), oracle.csct(b)
    MC = oracle.cost(Fa, Fb, 8)
    for y in range(12):
        for x in range(8, 30):
            for d in range(8):
                assert MC[y, x, d] == bin(int(Fa[y, x]) ^ int(Fb[y, x - d])).count("1")

"""End-to-end pins for the oracle: Eq. 4 (WTA), the 3x3 median and the whole path."""
import numpy as np
import pytest

import oracle
import stereo_synth as synth


def test_wta_breaks_ties_toward_lowest_disparity():
    S = np.array([[[5, 3, 3, 4], [2, 2, 2, 2], [9, 8, 7, 7]]], dtype=np.int32)
    assert oracle.wta(S).tolist() == [[1, 0, 2]]


def test_median_hand_cases():
    raw = np.array([[9, 9, 9, 9],
                    [9, 1, 2, 9],
                    [9, 3, 4, 9],
                    [9, 9, 9, 9]], dtype=np.uint8)
    out = oracle.median3x3(raw)
    # (1,1): {9,9,9,9,1,2,9,3,4} sorted 1,2,3,4,9,9,9,9,9 -> 9
    assert out[1, 1] == 9
    # border ring copied
    assert (out[0] == raw[0]).all() and (out[:, 0] == raw[:, 0]).all()
    raw2 = np.array([[0, 0, 0], [0, 200, 0], [0, 0, 0]], dtype=np.uint8)
    assert oracle.median3x3(raw2)[1, 1] == 0  # an isolated outlier is removed
    raw3 = np.array([[1, 2, 3], [4, 5, 6], [7, 8, 9]], dtype=np.uint8)
    assert oracle.median3x3(raw3)[1, 1] == 5


@pytest.mark.parametrize("n_paths", [2, 4, 8])
def test_identical_images_give_zero_disparity(n_paths):
    pair = synth.make_pair(synth.PairSpec(48, 32, 32, 3, 2, 20), 7)
    d = oracle.sgm(pair.left, pair.left, 32, 7, 84, n_paths)
    assert not d.any()


def test_constant_images_give_zero_disparity():
    a = np.full((20, 40), 13, dtype=np.uint8)
    b = np.full((20, 40), 200, dtype=np.uint8)
    assert not oracle.sgm(a, b, 32, 10, 120, 8).any()


@pytest.mark.parametrize("d0", [3, 11])
def test_known_constant_shift_recovered_in_interior(d0):
    """Noise-free textured pair shifted by d0: raw WTA = d0 away from borders."""
    H, W, D = 48, 96, 32
    big = synth.box3(synth.uniform_int(synth.stream_u64(99, 1, H * (W + d0)), 0, 255)
                     .astype(np.uint8).reshape(H, W + d0))
    left = big[:, :W].copy()          # left(x) = big(x)
    right = big[:, d0:d0 + W].copy()  # right(x - d0) = big(x) = left(x): Eq. 2 matches x with x - d0
    out = oracle.sgm(left, right, D, 7, 84, 4, debug=True)
    raw = out["raw"]
    assert (raw[16:H - 16, d0 + 16:W - 16] == d0).all()


@pytest.mark.parametrize("n_paths", [2, 4, 8])
def test_pixel_route_agrees_with_full_image_route(n_paths):
    pair = synth.make_pair(synth.PairSpec(40, 26, 32, 3, 2, 20), 3)
    full = oracle.sgm(pair.left, pair.right, 32, 7, 84, n_paths, debug=True)
    rng = np.random.default_rng(n_paths)
    pts = [(0, 0), (39, 25), (39, 0), (0, 25)] + [(int(x), int(y)) for x, y in
                                                  zip(rng.integers(0, 40, 12), rng.integers(0, 26, 12))]
    for (x, y) in pts:
        d, S = oracle.pixel(pair.left, pair.right, 32, 7, 84, n_paths, x, y)
        assert S.tolist() == full["S"][y, x].tolist()
        assert d == full["raw"][y, x]
    got = oracle.disp_at(pair.left, pair.right, 32, 7, 84, n_paths, pts)
    for (x, y), v in got.items():
        assert v == full["disp"][y, x]


def test_sum_is_the_sum_of_the_directions():
    pair = synth.make_pair(synth.PairSpec(30, 20, 32, 2, 2, 20), 5)
    out = oracle.sgm(pair.left, pair.right, 32, 7, 84, 8, debug=True)
    MC = oracle.cost(out["Fb"], out["Fm"], 32)
    S = sum(oracle.aggregate(MC, 7, 84, rx, ry) for rx, ry in oracle.directions(8))
    assert (S == out["S"]).all()
    # S(p, d) >= n_paths * MC(p, d) since every L_r >= MC
    assert (out["S"] >= 8 * MC.astype(np.int32)).all()


def test_rejects_bad_arguments():
    a = np.zeros((10, 10), dtype=np.uint8)
    with pytest.raises(ValueError):
        oracle.sgm(a, a, 32, 7, 84, 3)
    with pytest.raises(ValueError):
        oracle.pixel(a, a, 32, 7, 84, 4, 10, 0)

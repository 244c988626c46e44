"""The full 9x7 Census (62-bit features) on the GPU vs the oracle, bit-exact.

The context flag SGM_FLAG_CENSUS_FULL swaps the CSCT of Eq. 1 for the
classic Census transform that compares every pixel of the 9x7 window with
the centre (the CT that Section 2 contrasts with the CSCT).  Features are
uint64, the matching cost of Eq. 2 reaches 62, and the rest of the path
(Eqs. 3-4, the median) is unchanged.
"""
import numpy as np
import pytest

import oracle
import stereo_synth as synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgm():
    from paper_1610_04121_gb300 import sgm as m

    return m


@pytest.fixture(scope="module")
def ctx(sgm):
    c = sgm.Context(0, flags=sgm.SGM_FLAG_CENSUS_FULL)
    yield c
    c.close()


def _compare_stages(ctx, left, right, D, P1, P2, n_paths):
    ref = oracle.sgm(left, right, D, P1, P2, n_paths, debug=True, census="ct62")
    got = ctx.debug(left, right, D, P1, P2, n_paths)
    assert got["Fb"].dtype == np.uint64
    assert (got["Fb"] == ref["Fb"]).all(), "features (left)"
    assert (got["Fm"] == ref["Fm"]).all(), "features (right)"
    assert (got["MC"] == oracle.cost64(ref["Fb"], ref["Fm"], D)).all(), "matching cost"
    bad = np.argwhere(got["S"].astype(np.int32) != ref["S"])
    assert bad.size == 0, f"S differs at {bad[:5].tolist()} (of {len(bad)})"
    bad = np.argwhere(got["raw"] != ref["raw"])
    assert bad.size == 0, f"raw disparity differs at {bad[:5].tolist()} (of {len(bad)})"
    assert (got["disp"] == ref["disp"]).all(), "median-filtered disparity"
    return got


@pytest.mark.parametrize("n_paths", [2, 4, 8])
@pytest.mark.parametrize("D", [32, 64, 96, 128, 160, 192, 224, 256])
def test_small_ragged_all_D(ctx, D, n_paths):
    pair = synth.make_pair(synth.PairSpec(77, 45, D, 4, 1, min(48, D - 1)), 3000 + D)
    _compare_stages(ctx, pair.left, pair.right, D, 7, 84, n_paths)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (3, 3), (9, 7), (10, 8), (33, 2), (2, 33), (17, 23),
                                 (100, 3)])
@pytest.mark.parametrize("n_paths", [2, 4, 8])
def test_degenerate_and_tiny_sizes(ctx, W, H, n_paths):
    rng = np.random.default_rng(W * 100 + H + 7)
    left = rng.integers(0, 256, (H, W), dtype=np.uint8)
    right = rng.integers(0, 256, (H, W), dtype=np.uint8)
    _compare_stages(ctx, left, right, 32, 7, 84, n_paths)


def test_flat_images_reach_the_largest_cost(ctx):
    # a flat image has the feature 0x3FFFFFFFFFFFFFFF wherever the window fits
    # and 0 on its border, so an inner left pixel matched with a border column
    # of the right image differs in all 62 bits
    left = np.full((20, 40), 100, np.uint8)
    right = np.full((20, 40), 101, np.uint8)
    got = _compare_stages(ctx, left, right, 32, 7, 84, 4)
    assert int(got["MC"].max()) == 62


@pytest.mark.parametrize("n_paths", [2, 4, 8])
@pytest.mark.parametrize("P1,P2", [(0, 0), (224, 193), (7, 65), (7, 66), (1, 2), (193, 193)])
def test_penalties_up_to_the_byte_limit(ctx, n_paths, P1, P2):
    # 4 paths keep byte sums while 2 * (62 + P2) <= 255, i.e. P2 <= 65
    pair = synth.make_pair(synth.PairSpec(70, 37, 64, 4, 2, 40), 77 + P2)
    _compare_stages(ctx, pair.left, pair.right, 64, P1, P2, n_paths)


def test_p2_above_the_byte_limit_is_rejected(sgm, ctx):
    pair = synth.make_pair(synth.PairSpec(64, 32, 64, 4, 2, 40), 5)
    out = np.zeros_like(pair.left)
    with pytest.raises(sgm.SgmError) as e:
        sgm.sgm_compute(ctx.handle, pair.left, pair.right, 64, 32, 64, 7, 194, 4, out)
    assert e.value.code == sgm.SGM_EINVAL
    assert "193" in sgm.last_error(ctx.handle)
    # the same penalties are fine with the CSCT
    with sgm.Context(0) as plain:
        plain.compute(pair.left, pair.right, 64, 7, 194, 4, out)
    assert (out == oracle.sgm(pair.left, pair.right, 64, 7, 194, 4)).all()


@pytest.mark.parametrize("n_paths", [4, 8])
def test_full_size_frame(ctx, n_paths):
    # the 640x480, 128-disparity frame, whole-image comparison of the output
    pair = synth.make_pair(synth.PairSpec(640, 480, 128, 4, 2, 100), 11)
    got = ctx.compute(pair.left, pair.right, 128, 7, 84, n_paths)
    ref = oracle.sgm(pair.left, pair.right, 128, 7, 84, n_paths, census="ct62")
    bad = np.argwhere(got != ref)
    assert bad.size == 0, f"disparity differs at {bad[:5].tolist()} (of {len(bad)})"


def test_differs_from_the_csct(sgm, ctx):
    # the two transforms give different outputs on a textured pair, so the
    # flag really switches the features
    pair = synth.make_pair(synth.PairSpec(96, 64, 64, 4, 2, 40), 21)
    a = ctx.compute(pair.left, pair.right, 64, 7, 84, 4)
    with sgm.Context(0) as plain:
        b = plain.compute(pair.left, pair.right, 64, 7, 84, 4)
    assert (a != b).any()


def test_batch_and_served_match_the_oracle(sgm, ctx):
    shapes = [(96, 64, 64, 4), (50, 33, 32, 8), (130, 70, 128, 2), (64, 64, 256, 8), (40, 20, 96, 4),
              (77, 45, 160, 4)]
    pairs, outs, refs = [], [], []
    for i, (W, H, D, npth) in enumerate(shapes):
        p = synth.make_pair(synth.PairSpec(W, H, D, 4, 2, min(48, D - 1)), 40 + i)
        P1, P2 = [(7, 84), (10, 60)][i % 2]
        o = np.zeros((H, W), np.uint8)
        pairs.append((p.left, p.right, o, W, H, D, P1, P2, npth))
        outs.append(o)
        refs.append(oracle.sgm(p.left, p.right, D, P1, P2, npth, census="ct62"))
    sgm.sgm_compute_batch(ctx.handle, pairs)
    for o, r, q in zip(outs, refs, shapes):
        assert (o == r).all(), q
    c = sgm.Context(0, flags=sgm.SGM_FLAG_CENSUS_FULL)
    try:
        tickets = []
        for (L, R, _, W, H, D, P1, P2, npth), r in zip(pairs, refs):
            o = np.zeros((H, W), np.uint8)
            tickets.append((sgm.sgm_submit(c.handle, L, R, W, H, D, P1, P2, npth, o), o, r))
        for t, o, r in tickets:
            assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK
            assert (o == r).all()
    finally:
        c.close()

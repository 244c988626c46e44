"""The paired-line 4-path schedule (SGM_SCHED_PAIRS) against the oracle.

Two lines share every packed word, the cubes live in 2 x 2 pixel quads over
a grid padded to even sizes, and the horizontal pair is split between two
launches with a parallel winner-take-all over the columns both directions
passed.  Eq. 3 and Eq. 4 are integer arithmetic, so every stage must match
the oracle bit for bit: the debug path (forced to this schedule) dumps the
features, the quad costs in natural order, S, the raw and the final
disparity.  The shapes cover odd and even sizes (padding rows and columns),
W <= H (the horizontal pair ends in the first launch), H < W <= 2H (an
overlap finished in parallel) and W > 2H (the horizontal pair meets in the
middle in the second launch, including W2 = 2 H2 + 2, where only the
right-to-left chain stores columns for the other); the penalties cover byte
and u16 sums of the vertical pair and 16- and 32-bit winner-take-all keys.
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
    c = sgm.Context(0)
    sgm.sgm_set_schedule(c.handle, sgm.SGM_SCHED_PAIRS)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx62(sgm):
    c = sgm.Context(0, flags=sgm.SGM_FLAG_CENSUS_FULL)
    sgm.sgm_set_schedule(c.handle, sgm.SGM_SCHED_PAIRS)
    yield c
    c.close()


def _compare(c, left, right, D, P1, P2, census="csct"):
    ref = oracle.sgm(left, right, D, P1, P2, 4, debug=True, census=census)
    got = c.debug(left, right, D, P1, P2, 4)
    assert (got["Fb"] == ref["Fb"]).all() and (got["Fm"] == ref["Fm"]).all(), "features"
    MC = (oracle.cost64 if census == "ct62" else oracle.cost)(ref["Fb"], ref["Fm"], D)
    bad = np.argwhere(got["MC"] != MC)
    assert bad.size == 0, f"matching cost differs at {bad[:5].tolist()} (of {len(bad)})"
    bad = np.argwhere(got["S"].astype(np.int32) != ref["S"])
    assert bad.size == 0, f"S differs at {bad[:5].tolist()} (of {len(bad)})"
    bad = np.argwhere(got["raw"] != ref["raw"])
    assert bad.size == 0, f"raw disparity differs at {bad[:5].tolist()} (of {len(bad)})"
    assert (got["disp"] == ref["disp"]).all(), "median-filtered disparity"
    out = c.compute(left, right, D, P1, P2, 4)  # the captured graph
    assert (out == ref["disp"]).all(), "graph path"


@pytest.mark.parametrize("P2", [84, 120])  # byte / u16 sums of the vertical pair
@pytest.mark.parametrize("D", [32, 64, 96, 128, 160, 192, 224, 256])
def test_every_D_ragged(ctx, D, P2):
    pair = synth.make_pair(synth.PairSpec(77, 45, D, 4, 1, min(48, D - 1)), 9100 + D)
    _compare(ctx, pair.left, pair.right, D, 7, P2)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (2, 2), (3, 3), (2, 33), (33, 2), (17, 23), (64, 64),
                                 (100, 3), (101, 51), (200, 31), (31, 200), (130, 66), (131, 67), (134, 66),
                                 (133, 65)])
def test_sizes_and_split_geometries(ctx, W, H):
    rng = np.random.default_rng(W * 1000 + H)
    left = rng.integers(0, 256, (H, W), dtype=np.uint8)
    right = rng.integers(0, 256, (H, W), dtype=np.uint8)
    _compare(ctx, left, right, 64, 7, 84)
    _compare(ctx, left, right, 32, 10, 120)


@pytest.mark.parametrize("P1,P2", [(0, 0), (224, 224), (50, 10), (0, 224), (1, 2), (10, 120), (7, 96), (7, 97)])
def test_penalties(ctx, P1, P2):
    pair = synth.make_pair(synth.PairSpec(70, 40, 64, 4, 2, 40), 77)
    _compare(ctx, pair.left, pair.right, 64, P1, P2)


@pytest.mark.parametrize("D,P2", [(64, 60), (128, 84), (128, 150), (256, 100)])
def test_full_census(ctx62, D, P2):
    pair = synth.make_pair(synth.PairSpec(90, 50, D, 4, 2, min(48, D - 1)), 333 + D)
    _compare(ctx62, pair.left, pair.right, D, 7, P2, census="ct62")


@pytest.mark.parametrize("D", [64, 256])
@pytest.mark.parametrize("census", ["csct", "ct62"])
def test_census_cost_tiles(ctx, ctx62, D, census):
    # Census tiles of 64 x 4 pixels, cost segments of 32 quads (64 columns)
    # with the match features of D columns to their left: ragged last tiles
    # and segments in both directions
    pair = synth.make_pair(synth.PairSpec(301, 21, D, 3, 1, min(60, D - 1)), 9300 + D)
    _compare(ctx62 if census == "ct62" else ctx, pair.left, pair.right, D, 7, 84, census)


def test_identical_images_give_zero(ctx):
    pair = synth.make_pair(synth.PairSpec(64, 40, 64, 3, 2, 40), 5)
    _compare(ctx, pair.left, pair.left, 64, 7, 84)
    assert not ctx.compute(pair.left, pair.left, 64, 7, 84, 4).any()


@pytest.mark.parametrize("P2", [84, 120])
def test_full_frame_640x480(ctx, P2):
    w = synth.WORKLOADS["sgm_640x480_d128_p4"]
    pair = synth.workload_pair(w.name)
    _compare(ctx, pair.left, pair.right, 128, 7, P2)


@pytest.mark.parametrize("D", [128, 256])
def test_1920x1080_sampled(ctx, D):
    pair = synth.make_pair(synth.PairSpec(1920, 1080, D, 6, 4, 48), 5151 + D)
    out = ctx.compute(pair.left, pair.right, D, 7, 84, 4)
    rng = np.random.default_rng(D)
    pts = [(0, 0), (1919, 1079), (1919, 0), (0, 1079), (960, 540), (1080, 7), (5, 1070)]
    pts += [(int(x), int(y)) for x, y in zip(rng.integers(1, 1919, 6), rng.integers(1, 1079, 6))]
    ref = oracle.disp_at(pair.left, pair.right, D, 7, 84, 4, pts)
    for (x, y), v in ref.items():
        assert out[y, x] == v, (x, y, int(out[y, x]), v)

"""GPU path vs the CPU oracle, element by element, through the C ABI.

Everything here is integer arithmetic, so the bar is bit-exact equality of
the features (Eq. 1), the matching cost (Eq. 2), the summed path costs
(Eqs. 3-4), the winner-take-all disparity and the median-filtered output.
"""
import numpy as np
import pytest

import oracle
import stereo_synth as synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1610_04121_gb300 import sgm

    c = sgm.Context(0)
    yield c
    c.close()


def _compare_stages(ctx, left, right, D, P1, P2, n_paths, check_S=True):
    ref = oracle.sgm(left, right, D, P1, P2, n_paths, debug=True)
    got = ctx.debug(left, right, D, P1, P2, n_paths)
    assert (got["Fb"] == ref["Fb"]).all(), "features (left)"
    assert (got["Fm"] == ref["Fm"]).all(), "features (right)"
    MC = oracle.cost(ref["Fb"], ref["Fm"], D)
    assert (got["MC"] == MC).all(), "matching cost"
    if check_S:
        bad = np.argwhere(got["S"].astype(np.int32) != ref["S"])
        assert bad.size == 0, f"S differs at {bad[:5].tolist()} (of {len(bad)})"
    bad = np.argwhere(got["raw"] != ref["raw"])
    assert bad.size == 0, f"raw disparity differs at {bad[:5].tolist()} (of {len(bad)})"
    assert (got["disp"] == ref["disp"]).all(), "median-filtered disparity"
    return got


@pytest.mark.parametrize("n_paths", [2, 4, 8])
@pytest.mark.parametrize("D", [32, 64, 96, 128, 160, 192, 224, 256])
def test_small_ragged_all_D(ctx, D, n_paths):
    # several 32x16 census tiles, 32-pixel cost segments and a ragged tail
    pair = synth.make_pair(synth.PairSpec(77, 45, D, 4, 1, min(48, D - 1)), 1000 + D)
    _compare_stages(ctx, pair.left, pair.right, D, 7, 84, n_paths)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (3, 3), (8, 6), (9, 7), (10, 8), (33, 2), (2, 33),
                                 (17, 23), (64, 64), (100, 3)])
@pytest.mark.parametrize("n_paths", [2, 4, 8])
def test_degenerate_and_tiny_sizes(ctx, W, H, n_paths):
    rng = np.random.default_rng(W * 100 + H)
    left = rng.integers(0, 256, (H, W), dtype=np.uint8)
    right = rng.integers(0, 256, (H, W), dtype=np.uint8)
    _compare_stages(ctx, left, right, 32, 7, 84, n_paths)


@pytest.mark.parametrize("P1,P2", [(0, 0), (224, 224), (50, 10), (0, 224), (1, 2), (10, 120)])
def test_penalty_extremes(ctx, P1, P2):
    pair = synth.make_pair(synth.PairSpec(70, 40, 64, 4, 2, 40), 77)
    _compare_stages(ctx, pair.left, pair.right, 64, P1, P2, 8)


def test_identical_and_constant_images(ctx):
    pair = synth.make_pair(synth.PairSpec(64, 40, 64, 3, 2, 40), 5)
    got = _compare_stages(ctx, pair.left, pair.left, 64, 7, 84, 4)
    assert not got["disp"].any()
    a = np.full((30, 50), 9, np.uint8)
    got = _compare_stages(ctx, a, np.full_like(a, 200), 32, 7, 84, 8)
    assert not got["disp"].any()


def test_width_smaller_than_D(ctx):
    rng = np.random.default_rng(3)
    left = rng.integers(0, 256, (20, 40), dtype=np.uint8)
    right = rng.integers(0, 256, (20, 40), dtype=np.uint8)
    _compare_stages(ctx, left, right, 256, 7, 84, 8)


@pytest.mark.parametrize("name", list(synth.WORKLOADS))
def test_full_size_workloads_bit_exact(ctx, name):
    """The three single-pair workloads at full size, every stage."""
    w = synth.WORKLOADS[name]
    pair = synth.workload_pair(name)
    _compare_stages(ctx, pair.left, pair.right, w.spec.D, w.P1, w.P2, w.n_paths)


def test_compute_path_equals_debug_path(ctx):
    """The graph-replayed sgm_compute gives the debug path's disparity."""
    w = synth.WORKLOADS["sgm_640x480_d128_p4"]
    pair = synth.workload_pair(w.name)
    ref = oracle.sgm(pair.left, pair.right, w.spec.D, w.P1, w.P2, w.n_paths)
    for _ in range(3):
        out = ctx.compute(pair.left, pair.right, w.spec.D, w.P1, w.P2, w.n_paths)
        assert (out == ref).all()


@pytest.mark.parametrize("D,n_paths", [(256, 8), (128, 4)])
def test_1920x1080_sampled_against_pixel_oracle(ctx, D, n_paths):
    """Largest served size: sampled outputs against the per-pixel oracle."""
    pair = synth.make_pair(synth.PairSpec(1920, 1080, D, 6, 4, 48), 4242 + D)
    P1, P2 = (10, 120) if n_paths == 8 else (7, 84)
    out = ctx.compute(pair.left, pair.right, D, P1, P2, n_paths)
    rng = np.random.default_rng(D)
    pts = [(0, 0), (1919, 1079), (1919, 0), (0, 1079), (960, 540), (5, 1070)]
    pts += [(int(x), int(y)) for x, y in zip(rng.integers(1, 1919, 6), rng.integers(1, 1079, 6))]
    ref = oracle.disp_at(pair.left, pair.right, D, P1, P2, n_paths, pts)
    for (x, y), v in ref.items():
        assert out[y, x] == v, (x, y, int(out[y, x]), v)

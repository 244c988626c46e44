"""The thread-parallel oracle driver (the CPU baseline's all-core timing)
gives exactly oracle_sgm's disparity: it splits only what Eq. 1-4 leave
independent (rows, columns, directions), so any mistake in its bands shows
up as a differing pixel."""
import numpy as np
import pytest

import oracle
import stereo_synth as synth


@pytest.mark.parametrize("W,H,D,n_paths", [(77, 45, 64, 4), (33, 17, 32, 8), (50, 3, 32, 2), (1, 1, 32, 4),
                                           (3, 40, 96, 8), (120, 64, 128, 4)])
@pytest.mark.parametrize("nthreads", [1, 3, 8])
def test_threaded_driver_equals_the_oracle(W, H, D, n_paths, nthreads):
    pair = synth.make_pair(synth.PairSpec(W, H, D, 4, 1, min(48, D - 1)), 31 * W + H + D)
    ref = oracle.sgm(pair.left, pair.right, D, 7, 84, n_paths)
    got = oracle.sgm_threads(pair.left, pair.right, D, 7, 84, n_paths, nthreads)
    assert np.array_equal(got, ref)


def test_threaded_driver_extreme_penalties():
    rng = np.random.default_rng(4)
    left = rng.integers(0, 256, (40, 60), dtype=np.uint8)
    right = rng.integers(0, 256, (40, 60), dtype=np.uint8)
    for P1, P2 in [(0, 0), (224, 224), (50, 10)]:
        assert np.array_equal(oracle.sgm_threads(left, right, 64, P1, P2, 8, 4), oracle.sgm(left, right, 64, P1, P2, 8))

"""The seeded input generator: determinism and the stated recipe."""
import numpy as np

import stereo_synth as synth


def test_deterministic_and_seed_sensitive():
    s = synth.WORKLOADS["sgm_320x240_d64_p4"].spec
    a, b = synth.make_pair(s, 1), synth.make_pair(s, 1)
    c = synth.make_pair(s, 2)
    assert (a.left == b.left).all() and (a.right == b.right).all() and (a.gt == b.gt).all()
    assert (a.left != c.left).any()


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: first outputs (Steele et al. 2014; widely tabulated)
    k = np.uint64(0)
    with np.errstate(over="ignore"):
        out = synth._mix64(k + np.arange(1, 4, dtype=np.uint64) * synth.GOLDEN)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_recipe_ranges():
    for name, w in synth.WORKLOADS.items():
        p = synth.workload_pair(name)
        assert p.left.shape == (w.spec.H, w.spec.W) and p.left.dtype == np.uint8
        assert p.gt.max() < w.spec.D
        lo = min(w.spec.d_lo, w.spec.background if w.spec.ramp is None else w.spec.ramp[0])
        assert p.gt.min() >= lo


def test_forward_warp_larger_disparity_wins():
    left = np.arange(8, dtype=np.uint8).reshape(1, 8) * 10
    gt = np.array([[0, 0, 0, 0, 2, 1, 0, 0]])
    fill = np.full((1, 8), 255, dtype=np.uint8)
    right = synth.forward_warp(left, gt, fill)
    # x=4 (d=2) -> 2, x=5 (d=1) -> 4, x=2 (d=0) -> 2 collides with x=4: d=2 wins
    assert right[0, 2] == 40 and right[0, 4] == 50 and right[0, 3] == 30


def test_batch_recipe_is_seeded():
    r1, r2 = synth.batch_recipe(64), synth.batch_recipe(64)
    assert [w.name for w in r1] == [w.name for w in r2]
    assert {w.spec.D for w in r1} <= {64, 128, 256}

"""The three 4-path sweep schedules and their autotuner, through the C ABI.

All schedules compute Eq. 3 and Eq. 4 over the same paths, so each must
match the oracle bit for bit on its own; the tuner only decides which runs.
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


@pytest.mark.parametrize("sched", [0, 1, 2])
@pytest.mark.parametrize("D", [32, 64, 96, 128, 160, 256])
def test_each_schedule_matches_the_oracle(sgm, sched, D):
    pair = synth.make_pair(synth.PairSpec(77, 45, D, 4, 2, min(48, D - 1)), 7000 + D)
    with sgm.Context(0) as c:
        sgm.sgm_set_schedule(c.handle, sched)
        assert sgm.sgm_schedule_for(c.handle, 77, 45, D, 7, 84, 4) == sched
        dbg = c.debug(pair.left, pair.right, D, 7, 84, 4)  # the debug path follows the forced schedule
        got = c.compute(pair.left, pair.right, D, 7, 84, 4)
    ref = oracle.sgm(pair.left, pair.right, D, 7, 84, 4, debug=True)
    assert (got == ref["disp"]).all()
    assert (dbg["S"].astype(np.int32) == ref["S"]).all() and (dbg["raw"] == ref["raw"]).all()


@pytest.mark.parametrize("sched", [0, 1, 2])
@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (2, 33), (33, 2), (17, 23), (200, 31), (31, 200)])
@pytest.mark.parametrize("P2", [84, 96, 97])  # byte sums hold up to 2 * (31 + P2) <= 255
def test_schedules_on_edge_sizes_and_sum_widths(sgm, sched, W, H, P2):
    rng = np.random.default_rng(W * 7 + H + P2)
    left = rng.integers(0, 256, (H, W), dtype=np.uint8)
    right = rng.integers(0, 256, (H, W), dtype=np.uint8)
    with sgm.Context(0) as c:
        sgm.sgm_set_schedule(c.handle, sched)
        got = c.compute(left, right, 64, 7, P2, 4)
    assert (got == oracle.sgm(left, right, 64, 7, P2, 4)).all()


def test_autotuner_picks_one_and_keeps_it(sgm):
    pair = synth.make_pair(synth.PairSpec(160, 96, 64, 4, 2, 40), 3)
    ref = oracle.sgm(pair.left, pair.right, 64, 7, 84, 4)
    with sgm.Context(0) as c:
        assert sgm.sgm_schedule_for(c.handle, 160, 96, 64, 7, 84, 4) == -1  # not tuned yet
        before = c.launches
        assert (c.compute(pair.left, pair.right, 64, 7, 84, 4) == ref).all()
        # tuning: per schedule one warm-up and five timed runs, then the chosen
        # run; a path is 5 kernels, 6 with the paired schedule (its second
        # launch is two kernels side by side)
        per_path = {0: 5, 1: 5, 2: 6}
        chosen = sgm.sgm_schedule_for(c.handle, 160, 96, 64, 7, 84, 4)
        assert chosen in (0, 1, 2)
        assert c.launches - before == 6 * sum(per_path.values()) + per_path[chosen]
        before = c.launches
        assert (c.compute(pair.left, pair.right, 64, 7, 84, 4) == ref).all()
        assert c.launches - before == per_path[chosen]
        assert sgm.sgm_schedule_for(c.handle, 160, 96, 64, 7, 84, 4) == chosen
        # other path counts have one schedule
        assert sgm.sgm_schedule_for(c.handle, 160, 96, 64, 7, 84, 8) == 0
        with pytest.raises(sgm.SgmError):
            sgm.sgm_set_schedule(c.handle, 3)


def test_stage_labels_follow_the_schedule(sgm):
    import torch

    pair = synth.make_pair(synth.PairSpec(128, 80, 128, 4, 2, 80), 9)
    L = torch.from_numpy(pair.left).cuda()
    R = torch.from_numpy(pair.right).cuda()
    out = torch.empty_like(L)
    c = sgm.Context(0, flags=sgm.SGM_FLAG_STAGE_TIMING)
    try:
        sgm.sgm_set_stream(c.handle, torch.cuda.current_stream())
        for sched, names in [(1, ["census", "cost", "sweep_h+v1", "sweep_v2", "median"]),
                             (2, ["census", "cost", "pairs_vh", "pairs_h_wta", "median"]),
                             (0, ["census", "cost", "sweep_v+h1", "sweep_h2", "median"])]:
            sgm.sgm_set_schedule(c.handle, sched)
            sgm.sgm_compute_async(c.handle, L, R, 128, 80, 128, 7, 84, 4, out)
            st = sgm.sgm_stage_times(c.handle)
            assert list(st) == names and all(v > 0 for v in st.values())
            torch.cuda.synchronize()
            assert (out.cpu().numpy() == oracle.sgm(pair.left, pair.right, 128, 7, 84, 4)).all()
    finally:
        c.close()


def test_full_frame_both_schedules(sgm):
    pair = synth.make_pair(synth.PairSpec(640, 480, 128, 12, 2, 120), 17)
    ref = oracle.sgm(pair.left, pair.right, 128, 7, 84, 4)
    with sgm.Context(0) as c:
        for sched in (0, 1, 2):
            sgm.sgm_set_schedule(c.handle, sched)
            assert (c.compute(pair.left, pair.right, 128, 7, 84, 4) == ref).all()

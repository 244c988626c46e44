"""The batched path through the C ABI: persistent per-stage grids over device
work lists, one captured graph per wave shape, the sweep grid autotuned per
wave; the device status word (SGM_EDEVICE); the served form's failure paths
(poll timeout, destroy with work queued, injected allocation failures) and
its admission bound.

Failures here are made on the host (test hooks read at sgm_create, a timeout
that elapses, a context destroyed early); no kernel is made to fault.
"""
import os

import numpy as np
import pytest

import oracle
import stereo_synth as synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgm():
    from paper_1610_04121_gb300 import sgm as m

    return m


def _pair(W, H, D, seed):
    return synth.make_pair(synth.PairSpec(W, H, D, 4, 2, min(48, D - 1)), seed)


def _sample_points(W, H, seed, n=4):
    rng = np.random.default_rng(seed)
    pts = [(0, 0), (W - 1, H - 1), (W // 2, H // 2)]
    pts += [(int(x), int(y)) for x, y in zip(rng.integers(1, W - 1, n), rng.integers(1, H - 1, n))]
    return pts


class _env:
    """Set environment variables for the contexts created inside the block."""

    def __init__(self, **kv):
        self.kv = kv

    def __enter__(self):
        for k, v in self.kv.items():
            os.environ[k] = str(v)

    def __exit__(self, *exc):
        for k in self.kv:
            os.environ.pop(k, None)


def test_uneven_64_pair_batch(sgm):
    # the 64 pairs of the batched benchmark: sizes 320x240 .. 1920x1080, D
    # 64 / 128 / 256, 4 or 8 paths; 320x240 pairs compared whole, the others
    # at sampled pixels
    recipe = synth.batch_recipe(64)
    pairs = synth.batch_pairs(recipe)
    outs = [np.zeros((w.spec.H, w.spec.W), np.uint8) for w in recipe]
    tuples = [(p.left, p.right, o, w.spec.W, w.spec.H, w.spec.D, w.P1, w.P2, w.n_paths)
              for w, p, o in zip(recipe, pairs, outs)]
    with sgm.Context(0) as c:
        sgm.sgm_compute_batch(c.handle, tuples)
    for i, (w, p, o) in enumerate(zip(recipe, pairs, outs)):
        W, H, D = w.spec.W, w.spec.H, w.spec.D
        if W == 320:
            ref = oracle.sgm(p.left, p.right, D, w.P1, w.P2, w.n_paths)
            assert (o == ref).all(), w.name
        else:
            ref = oracle.disp_at(p.left, p.right, D, w.P1, w.P2, w.n_paths, _sample_points(W, H, i))
            for (x, y), v in ref.items():
                assert o[y, x] == v, (w.name, x, y, int(o[y, x]), v)


def _small_mix(seed0):
    items = []
    for i, (W, H, D, npth, P2) in enumerate([(96, 64, 64, 4, 84), (64, 40, 128, 8, 120), (120, 50, 32, 2, 84),
                                             (75, 33, 64, 4, 84), (50, 90, 96, 8, 120), (33, 17, 256, 4, 120)]):
        items.append((_pair(W, H, D, seed0 + i), W, H, D, 7, P2, npth))
    return items


def _run(sgm, c, items):
    outs = [np.zeros((H, W), np.uint8) for p, W, H, D, P1, P2, npth in items]
    sgm.sgm_compute_batch(c.handle, [(p.left, p.right, o, W, H, D, P1, P2, npth)
                                     for (p, W, H, D, P1, P2, npth), o in zip(items, outs)])
    return outs


def test_tuned_once_then_one_graph_per_wave(sgm):
    items = _small_mix(500)
    refs = [oracle.sgm(p.left, p.right, D, P1, P2, npth) for p, W, H, D, P1, P2, npth in items]
    # groups (D, paths, sum width): a group runs census, cost, horizontal
    # sweeps, one or three vertical-type sweeps, median
    groups = {(D, npth, P2) for p, W, H, D, P1, P2, npth in items}
    per_wave = sum(4 + (3 if npth == 8 else 1) for D, npth, P2 in groups)
    with sgm.Context(0) as c:
        before = c.launches
        for o, r in zip(_run(sgm, c, items), refs):
            assert (o == r).all()
        # the first wave of a new shape: 4 sweep grids x (1 + 5) timed runs, then the run itself
        assert c.launches - before == 4 * 6 * per_wave + per_wave
        before = c.launches
        for o, r in zip(_run(sgm, c, items), refs):
            assert (o == r).all()
        assert c.launches - before == per_wave


def test_rejected_descriptor_reports_edevice_and_the_context_recovers(sgm):
    items = _small_mix(600)
    refs = [oracle.sgm(p.left, p.right, D, P1, P2, npth) for p, W, H, D, P1, P2, npth in items]
    with _env(SGM_TEST_BAD_JOB=1):
        c = sgm.Context(0)
    try:
        with pytest.raises(sgm.SgmError) as e:
            _run(sgm, c, items)
        assert e.value.code == sgm.SGM_EDEVICE
        for o, r in zip(_run(sgm, c, items), refs):  # the hook covered one wave
            assert (o == r).all()
    finally:
        c.close()


def test_injected_allocation_failure(sgm):
    p = _pair(96, 64, 64, 700)
    ref = oracle.sgm(p.left, p.right, 64, 7, 84, 4)
    # sgm_create's own allocations (one pinned status word per batched stream)
    with _env(SGM_TEST_FAIL_ALLOC=2):
        with pytest.raises(sgm.SgmError) as e:
            sgm.Context(0)
    assert e.value.code == sgm.SGM_ENOMEM
    # the first work arena: that call fails, the next one allocates and runs
    with _env(SGM_TEST_FAIL_ALLOC=4):
        c = sgm.Context(0)
    try:
        with pytest.raises(sgm.SgmError) as e:
            c.compute(p.left, p.right, 64, 7, 84, 4)
        assert e.value.code == sgm.SGM_ENOMEM
        assert (c.compute(p.left, p.right, 64, 7, 84, 4) == ref).all()
    finally:
        c.close()


def test_poll_times_out_on_a_large_request(sgm):
    W, H, D = 1920, 1080, 256
    p = _pair(W, H, D, 800)
    o = np.zeros((H, W), np.uint8)
    c = sgm.Context(0)
    try:
        t = sgm.sgm_submit(c.handle, p.left, p.right, W, H, D, 10, 120, 8, o)
        assert sgm.sgm_poll(c.handle, t, 1) == sgm.SGM_ETIMEDOUT
        assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK
        ref = oracle.disp_at(p.left, p.right, D, 10, 120, 8, _sample_points(W, H, 8))
        for (x, y), v in ref.items():
            assert o[y, x] == v, (x, y)
    finally:
        c.close()


def test_destroy_with_requests_queued_and_running(sgm):
    W, H, D = 1920, 1080, 256
    ps = [_pair(W, H, D, 900 + i) for i in range(2)]
    outs = [np.zeros((H, W), np.uint8) for _ in range(12)]
    c = sgm.Context(0)
    for i, o in enumerate(outs):
        p = ps[i % 2]
        assert sgm.sgm_submit(c.handle, p.left, p.right, W, H, D, 10, 120, 8, o) is not None
    c.close()  # cancels what is queued, waits for what runs, frees everything
    # the device and a new context are fine afterwards
    q = _pair(64, 48, 64, 950)
    with sgm.Context(0) as c2:
        assert (c2.compute(q.left, q.right, 64, 7, 84, 4) == oracle.sgm(q.left, q.right, 64, 7, 84, 4)).all()


def test_admission_bound_sheds_and_admitted_results_stay_exact(sgm):
    W, H, D = 640, 480, 128
    p = _pair(W, H, D, 1000)
    ref = oracle.sgm(p.left, p.right, D, 7, 84, 4)
    c = sgm.Context(0)
    try:
        o = np.zeros((H, W), np.uint8)
        t = sgm.sgm_submit(c.handle, p.left, p.right, W, H, D, 7, 84, 4, o)
        assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK and (o == ref).all()
        assert sgm.sgm_served_stats(c.handle)["service_de_per_s"] > 0
        sgm.sgm_set_admission_bound(c.handle, 1)  # 1 us: any request waits longer
        o2 = np.zeros((H, W), np.uint8)
        assert sgm.sgm_submit(c.handle, p.left, p.right, W, H, D, 7, 84, 4, o2) is None
        assert sgm.sgm_served_stats(c.handle)["shed"] == 1
        sgm.sgm_set_admission_bound(c.handle, 10_000_000)  # 10 s: a burst is admitted
        outs = [np.zeros((H, W), np.uint8) for _ in range(6)]
        ts = [sgm.sgm_submit(c.handle, p.left, p.right, W, H, D, 7, 84, 4, x) for x in outs]
        assert all(t is not None for t in ts)
        for t, x in zip(ts, outs):
            assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK and (x == ref).all()
        with pytest.raises(sgm.SgmError):
            sgm.sgm_set_admission_bound(c.handle, -1)
    finally:
        c.close()


def test_tuning_cache_round_trip(sgm, tmp_path):
    p = _pair(160, 96, 64, 1100)
    ref = oracle.sgm(p.left, p.right, 64, 7, 84, 4)
    items = _small_mix(1200)
    groups = {(D, npth, P2) for q, W, H, D, P1, P2, npth in items}
    per_wave = sum(4 + (3 if npth == 8 else 1) for D, npth, P2 in groups)
    path = str(tmp_path / "tuning.json")
    with sgm.Context(0) as c:
        assert (c.compute(p.left, p.right, 64, 7, 84, 4) == ref).all()  # tunes the 4-path schedule
        _run(sgm, c, items)  # tunes the batch's sweep grid
        chosen = sgm.sgm_schedule_for(c.handle, 160, 96, 64, 7, 84, 4)
        sgm.sgm_save_tuning(c.handle, path)
    with sgm.Context(0) as c:
        sgm.sgm_load_tuning(c.handle, path)
        assert sgm.sgm_schedule_for(c.handle, 160, 96, 64, 7, 84, 4) == chosen
        before = c.launches
        assert (c.compute(p.left, p.right, 64, 7, 84, 4) == ref).all()
        # no timed tuning runs: one path (the paired schedule runs its second
        # launch as two kernels)
        assert c.launches - before == (6 if chosen == sgm.SGM_SCHED_PAIRS else 5)
        before = c.launches
        refs = [oracle.sgm(q.left, q.right, D, P1, P2, npth) for q, W, H, D, P1, P2, npth in items]
        for o, r in zip(_run(sgm, c, items), refs):
            assert (o == r).all()
        assert c.launches - before == per_wave
        bad = tmp_path / "bad.json"
        bad.write_text('{"sgm_tuning": 1, "sm_count": 1, "schedules": [], "batch_grids": []}')
        with pytest.raises(sgm.SgmError):
            sgm.sgm_load_tuning(c.handle, str(bad))  # another device
        bad.write_text('{"sgm_tuning": 1, "sm_count": 152, "schedules": [[1, 2]], "batch_grids": []}')
        with pytest.raises(sgm.SgmError):
            sgm.sgm_load_tuning(c.handle, str(bad))
        with pytest.raises(sgm.SgmError):
            sgm.sgm_load_tuning(c.handle, str(tmp_path / "missing.json"))


def test_served_state_in_stats(sgm):
    W, H, D = 320, 240, 64
    p = _pair(W, H, D, 1300)
    c = sgm.Context(0)
    try:
        outs = [np.zeros((H, W), np.uint8) for _ in range(4)]
        ts = [sgm.sgm_submit(c.handle, p.left, p.right, W, H, D, 7, 84, 4, o) for o in outs]
        for t in ts:
            assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK
        st = sgm.sgm_served_stats(c.handle)
        assert st["queued"] == 0 and st["in_flight"] == 0 and st["pool_bytes"] > 0
    finally:
        c.close()

"""Served form with continuous batching: results in a mix equal results alone.

Requests are queued by sgm_submit; the context's scheduler batches whatever
is queued into one batched launch sequence per slot and keeps up to two
batches in flight.  Every result must be bit-identical to the same pair
computed alone (sgm_compute) and, for the small pairs, to the oracle.
"""
import time

import numpy as np
import pytest

import oracle
import stereo_synth as synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgm():
    from paper_1610_04121_gb300 import sgm as m

    return m


def _mix(n, seed0):
    """n small pairs of mixed size, D, penalties and path counts."""
    shapes = [(96, 64), (64, 40), (120, 50), (33, 17), (160, 90)]
    Ds = [32, 64, 128, 96, 256]
    paths = [2, 4, 8]
    out = []
    for i in range(n):
        W, H = shapes[i % len(shapes)]
        D = Ds[(i * 3) % len(Ds)]
        npth = paths[(i * 7) % len(paths)]
        P1, P2 = [(7, 84), (10, 120), (3, 40)][i % 3]
        p = synth.make_pair(synth.PairSpec(W, H, D, 4, 2, min(48, D - 1)), seed0 + i)
        out.append((p, W, H, D, P1, P2, npth))
    return out


def _alone(sgm, items):
    c = sgm.Context(0)
    try:
        res = []
        for p, W, H, D, P1, P2, npth in items:
            o = np.zeros((H, W), np.uint8)
            sgm.sgm_compute(c.handle, p.left, p.right, W, H, D, P1, P2, npth, o)
            res.append(o)
        return res
    finally:
        c.close()


def test_mix_equals_alone_and_batches_overlap(sgm):
    # one large pair first keeps the GPU busy while the burst behind it queues
    big = synth.make_pair(synth.PairSpec(1242, 375, 256, 8, 5, 100), 4242)
    items = [(big, 1242, 375, 256, 10, 120, 8)] + _mix(30, 7000)
    alone = _alone(sgm, items)
    for (p, W, H, D, P1, P2, npth), a in list(zip(items, alone))[1:]:
        assert (a == oracle.sgm(p.left, p.right, D, P1, P2, npth)).all(), (W, H, D, npth)
    c = sgm.Context(0)
    try:
        outs, tickets = [], []
        for p, W, H, D, P1, P2, npth in items:
            o = np.zeros((H, W), np.uint8)
            tickets.append(sgm.sgm_submit(c.handle, p.left, p.right, W, H, D, P1, P2, npth, o))
            outs.append(o)
        for t in tickets:
            assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK
        for i, (o, a) in enumerate(zip(outs, alone)):
            assert (o == a).all(), i
        st = sgm.sgm_served_stats(c.handle)
        assert st["completed"] == len(items)
        assert st["batches"] < len(items), st  # requests were batched
        assert st["max_in_flight"] == 2, st  # the burst ran beside the large pair
        assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
        assert st["de"] == sum(W * H * D for _, W, H, D, _, _, _ in items)
        sgm.sgm_served_reset_stats(c.handle)
        st = sgm.sgm_served_stats(c.handle)
        assert st["completed"] == 0 and st["batches"] == 0 and st["de"] == 0
    finally:
        c.close()


def test_arrivals_over_time_with_device_pointers(sgm):
    import torch

    items = _mix(24, 8000)
    refs = [oracle.sgm(p.left, p.right, D, P1, P2, npth) for p, W, H, D, P1, P2, npth in items]
    gaps = np.diff(synth.poisson_arrivals(4000.0, 0.05, 5), prepend=0.0)
    c = sgm.Context(0)
    try:
        outs, tickets = [], []
        for (p, W, H, D, P1, P2, npth), g in zip(items, gaps):
            L = torch.from_numpy(p.left).cuda()
            R = torch.from_numpy(p.right).cuda()
            o = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
            torch.cuda.synchronize()
            time.sleep(min(float(g), 0.01))
            tickets.append(sgm.sgm_submit(c.handle, L, R, W, H, D, P1, P2, npth, o))
            outs.append((L, R, o))
        for t in tickets:
            assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK
        for (_, _, o), r in zip(outs, refs):
            assert (o.cpu().numpy() == r).all()
    finally:
        c.close()


def test_memory_cap_admits_in_several_batches(sgm):
    items = _mix(12, 9000)
    alone = _alone(sgm, items)
    # in batched layout the pairs need 0.6-7.2 MiB each, 24 MiB together; a
    # 10 MiB cap forces the scheduler to split the queue into several batches
    c = sgm.Context(0, mem_cap_bytes=10 << 20)
    try:
        outs, tickets = [], []
        for p, W, H, D, P1, P2, npth in items:
            o = np.zeros((H, W), np.uint8)
            tickets.append(sgm.sgm_submit(c.handle, p.left, p.right, W, H, D, P1, P2, npth, o))
            outs.append(o)
        for t in tickets:
            assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK
        for o, a in zip(outs, alone):
            assert (o == a).all()
        st = sgm.sgm_served_stats(c.handle)
        assert st["batches"] >= 2, st
    finally:
        c.close()


def test_submit_rejects_a_pair_over_the_cap(sgm):
    c = sgm.Context(0, mem_cap_bytes=1 << 20)
    try:
        p = synth.make_pair(synth.PairSpec(320, 240, 128, 4, 2, 48), 11)
        o = np.zeros((240, 320), np.uint8)
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_submit(c.handle, p.left, p.right, 320, 240, 128, 7, 84, 4, o)
        assert e.value.code == sgm.SGM_ENOMEM
    finally:
        c.close()

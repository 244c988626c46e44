"""Entry points of the C ABI on the GPU: pointer kinds, async, batch, served."""
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
    yield c
    c.close()


def _pair(W=96, H=64, D=64, seed=1):
    return synth.make_pair(synth.PairSpec(W, H, D, 4, 2, min(48, D - 1)), seed)


def test_host_device_and_async_agree(sgm, ctx):
    import torch

    p = _pair()
    ref = oracle.sgm(p.left, p.right, 64, 7, 84, 4)
    host = ctx.compute(p.left, p.right, 64, 7, 84, 4)
    assert (host == ref).all()
    L = torch.from_numpy(p.left).cuda()
    R = torch.from_numpy(p.right).cuda()
    out = torch.empty_like(L)
    sgm.sgm_compute(ctx.handle, L, R, 96, 64, 64, 7, 84, 4, out)
    assert (out.cpu().numpy() == ref).all()
    out2 = torch.zeros_like(L)
    sgm.sgm_set_stream(ctx.handle, torch.cuda.current_stream())
    sgm.sgm_compute_async(ctx.handle, L, R, 96, 64, 64, 7, 84, 4, out2)
    torch.cuda.current_stream().synchronize()
    sgm.sgm_set_stream(ctx.handle, None)
    assert (out2.cpu().numpy() == ref).all()
    # pinned host memory is host memory too
    Lp, Rp = torch.from_numpy(p.left).pin_memory(), torch.from_numpy(p.right).pin_memory()
    op = torch.empty((64, 96), dtype=torch.uint8).pin_memory()
    sgm.sgm_compute(ctx.handle, Lp, Rp, 96, 64, 64, 7, 84, 4, op)
    assert (op.numpy() == ref).all()


def test_async_rejects_host_pointers(sgm, ctx):
    p = _pair()
    out = np.zeros_like(p.left)
    with pytest.raises(sgm.SgmError) as e:
        sgm.sgm_compute_async(ctx.handle, p.left, p.right, 96, 64, 64, 7, 84, 4, out)
    assert e.value.code == sgm.SGM_EINVAL


@pytest.mark.parametrize("bad", [dict(D=48), dict(D=288), dict(D=0), dict(P1=-1), dict(P2=225), dict(n_paths=3),
                                 dict(W=0), dict(H=-2)])
def test_invalid_arguments(sgm, ctx, bad):
    p = _pair()
    args = dict(W=96, H=64, D=64, P1=7, P2=84, n_paths=4)
    args.update(bad)
    out = np.zeros_like(p.left)
    with pytest.raises(sgm.SgmError) as e:
        sgm.sgm_compute(ctx.handle, p.left, p.right, args["W"], args["H"], args["D"], args["P1"], args["P2"],
                        args["n_paths"], out)
    assert e.value.code == sgm.SGM_EINVAL
    assert sgm.last_error(ctx.handle)


def test_batch_matches_single_pairs(sgm, ctx):
    specs = [(96, 64, 64, 4), (50, 33, 32, 8), (130, 70, 128, 2), (64, 64, 256, 8), (40, 20, 96, 4)]
    pairs, outs, refs = [], [], []
    for i, (W, H, D, npth) in enumerate(specs):
        p = _pair(W, H, D, seed=10 + i)
        o = np.zeros((H, W), np.uint8)
        pairs.append((p.left, p.right, o, W, H, D, 7, 84, npth))
        outs.append(o)
        refs.append(oracle.sgm(p.left, p.right, D, 7, 84, npth))
    sgm.sgm_compute_batch(ctx.handle, pairs)
    for o, r in zip(outs, refs):
        assert (o == r).all()


def test_served_results_match_and_tickets_retire(sgm):
    c = sgm.Context(0)
    try:
        items = []
        for i in range(12):
            W, H, D = [(96, 64, 64), (64, 40, 128), (120, 50, 32)][i % 3]
            p = _pair(W, H, D, seed=100 + i)
            o = np.zeros((H, W), np.uint8)
            t = sgm.sgm_submit(c.handle, p.left, p.right, W, H, D, 10, 120, 8, o)
            items.append((t, o, oracle.sgm(p.left, p.right, D, 10, 120, 8)))
        for t, o, r in items:
            assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK
            assert (o == r).all()
        with pytest.raises(sgm.SgmError):
            sgm.sgm_poll(c.handle, items[0][0], 0)  # retired
        st = sgm.sgm_served_stats(c.handle)
        assert st["completed"] == 12 and st["p99_us"] >= st["p50_us"] > 0
    finally:
        c.close()


def test_launch_counter_counts_kernels(sgm, ctx):
    p = _pair()
    ctx.compute(p.left, p.right, 64, 7, 84, 4)  # the first call of a 4-path key also tunes its schedule
    before = ctx.launches
    ctx.compute(p.left, p.right, 64, 7, 84, 4)
    H, W = p.left.shape
    # census, cost, the two sweep stages, median; the paired schedule runs its
    # second sweep stage as two kernels side by side
    paired = sgm.sgm_schedule_for(ctx.handle, W, H, 64, 7, 84, 4) == sgm.SGM_SCHED_PAIRS
    assert ctx.launches - before == (6 if paired else 5)
    before = ctx.launches
    ctx.compute(p.left, p.right, 64, 7, 84, 8)
    assert ctx.launches - before == 7  # the second halves of three vertical-type pairs
    before = ctx.launches
    ctx.compute(p.left, p.right, 64, 7, 84, 2)
    assert ctx.launches - before == 5


def test_stage_times_inside_graph_replay(sgm):
    import torch

    p = _pair(128, 80, 128, seed=9)
    c = sgm.Context(0, flags=sgm.SGM_FLAG_STAGE_TIMING)
    try:
        L = torch.from_numpy(p.left).cuda()
        R = torch.from_numpy(p.right).cuda()
        out = torch.empty_like(L)
        sgm.sgm_set_stream(c.handle, torch.cuda.current_stream())
        sgm.sgm_set_schedule(c.handle, sgm.SGM_SCHED_V_THEN_H)
        for n_paths, names in [(4, ["census", "cost", "sweep_v+h1", "sweep_h2", "median"]),
                               (8, ["census", "cost", "sweep_h", "sweep_diag+", "sweep_diag-", "sweep_v", "median"]),
                               (2, ["census", "cost", "sweep_h", "sweep_v", "median"])]:
            for _ in range(2):
                sgm.sgm_compute_async(c.handle, L, R, 128, 80, 128, 7, 84, n_paths, out)
                st = sgm.sgm_stage_times(c.handle)
                assert list(st) == names and all(v >= 0 for v in st.values())
                assert all(st[k] > 0 for k in names)
            torch.cuda.synchronize()
            assert (out.cpu().numpy() == oracle.sgm(p.left, p.right, 128, 7, 84, n_paths)).all()
    finally:
        c.close()


def _mixed_batch(n, seed0):
    import stereo_synth as synth

    shapes = [(96, 64), (130, 70), (64, 64), (200, 41), (33, 90)]
    out = []
    for i in range(n):
        W, H = shapes[i % len(shapes)]
        D = [32, 64, 96, 128, 256][(i * 7) % 5]
        npth = [2, 4, 8][(i * 5) % 3]
        P1, P2 = [(7, 84), (10, 120), (3, 20)][i % 3]
        p = synth.make_pair(synth.PairSpec(W, H, D, 4, 2, min(48, D - 1)), seed0 + i)
        out.append((p, W, H, D, P1, P2, npth))
    return out


def test_batch_of_many_mixed_pairs_equals_oracle(sgm, ctx):
    items = _mixed_batch(24, 500)
    pairs, outs = [], []
    for p, W, H, D, P1, P2, npth in items:
        o = np.zeros((H, W), np.uint8)
        pairs.append((p.left, p.right, o, W, H, D, P1, P2, npth))
        outs.append(o)
    sgm.sgm_compute_batch(ctx.handle, pairs)
    for (p, W, H, D, P1, P2, npth), o in zip(items, outs):
        assert (o == oracle.sgm(p.left, p.right, D, P1, P2, npth)).all(), (W, H, D, npth)


def test_batch_with_device_pointers_and_waves(sgm):
    import torch

    items = _mixed_batch(10, 900)
    refs = [oracle.sgm(p.left, p.right, D, P1, P2, npth) for p, W, H, D, P1, P2, npth in items]
    # the pairs need 0.8-7.3 MiB each, 33 MiB together: a 12 MiB cap forces
    # several waves through one arena
    c = sgm.Context(0, mem_cap_bytes=12 << 20)
    try:
        pairs, outs = [], []
        for p, W, H, D, P1, P2, npth in items:
            L = torch.from_numpy(p.left).cuda()
            R = torch.from_numpy(p.right).cuda()
            o = torch.zeros((H, W), dtype=torch.uint8, device="cuda")
            pairs.append((L, R, o, W, H, D, P1, P2, npth))
            outs.append(o)
        sgm.sgm_compute_batch(c.handle, pairs)
        for o, r in zip(outs, refs):
            assert (o.cpu().numpy() == r).all()
    finally:
        c.close()


def test_batch_rejects_a_pair_over_the_cap(sgm):
    c = sgm.Context(0, mem_cap_bytes=1 << 20)
    try:
        p = _pair(320, 240, 128, seed=3)
        o = np.zeros((240, 320), np.uint8)
        with pytest.raises(sgm.SgmError) as e:
            sgm.sgm_compute_batch(c.handle, [(p.left, p.right, o, 320, 240, 128, 7, 84, 4)])
        assert e.value.code == sgm.SGM_ENOMEM
    finally:
        c.close()


def test_pinned_buffers_staged(sgm):
    import torch

    # pinned host buffers are copied to and from the context's arena by
    # staging kernels inside the call's graph; a fresh context tunes first,
    # then replays; pageable buffers beside them go through cudaMemcpyAsync
    p = _pair(160, 96, 64, seed=41)
    ref = oracle.sgm(p.left, p.right, 64, 7, 84, 4)
    Lp, Rp = torch.from_numpy(p.left).pin_memory(), torch.from_numpy(p.right).pin_memory()
    c = sgm.Context(0)
    try:
        for _ in range(3):
            op = torch.zeros((96, 160), dtype=torch.uint8).pin_memory()
            sgm.sgm_compute(c.handle, Lp, Rp, 160, 96, 64, 7, 84, 4, op)
            assert (op.numpy() == ref).all()
        op = torch.zeros((96, 160), dtype=torch.uint8).pin_memory()
        for _ in range(2):  # the same pointers twice: the second call replays the graph
            op.zero_()
            sgm.sgm_compute(c.handle, Lp, Rp, 160, 96, 64, 7, 84, 4, op)
            assert (op.numpy() == ref).all()
        out = np.zeros((96, 160), np.uint8)  # pageable output beside pinned inputs
        sgm.sgm_compute(c.handle, Lp, Rp, 160, 96, 64, 7, 84, 4, out)
        assert (out == ref).all()
        Ld = torch.from_numpy(p.left).cuda()
        sgm.sgm_compute(c.handle, Ld, Rp, 160, 96, 64, 7, 84, 4, op)  # device input beside pinned ones
        assert (op.numpy() == ref).all()
        ref16 = oracle.sgm_ex(p.left, p.right, 64, 7, 84, 4, oracle.POST_SUBPIXEL | oracle.POST_LR_CHECK)
        o16 = torch.zeros((96, 160), dtype=torch.int16).pin_memory()
        for _ in range(2):
            sgm.sgm_compute_ex(c.handle, Lp, Rp, 160, 96, 64, 7, 84, 4,
                               oracle.POST_SUBPIXEL | oracle.POST_LR_CHECK, o16)
            assert (o16.numpy().view(np.uint16) == ref16).all()
        # the graph is keyed by the caller's buffers: a second pair of pinned
        # images of the same shape, alternating with the first, gets its own
        q = _pair(160, 96, 64, seed=43)
        refq = oracle.sgm(q.left, q.right, 64, 7, 84, 4)
        Lq, Rq = torch.from_numpy(q.left).pin_memory(), torch.from_numpy(q.right).pin_memory()
        for k in range(4):
            l, r, want = (Lp, Rp, ref) if k % 2 == 0 else (Lq, Rq, refq)
            sgm.sgm_compute(c.handle, l, r, 160, 96, 64, 7, 84, 4, op)
            assert (op.numpy() == want).all(), k
        # sizes that are not whole 16-byte pieces (the staging kernel's byte path)
        for W, H, npth in ((97, 61, 4), (97, 61, 8), (33, 7, 2)):
            o = _pair(W, H, 64, seed=W + H + npth)
            refo = oracle.sgm(o.left, o.right, 64, 7, 84, npth)
            Lo, Ro = torch.from_numpy(o.left).pin_memory(), torch.from_numpy(o.right).pin_memory()
            oo = torch.full((H, W), 255, dtype=torch.uint8).pin_memory()
            sgm.sgm_compute(c.handle, Lo, Ro, W, H, 64, 7, 84, npth, oo)
            assert (oo.numpy() == refo).all(), (W, H, npth)
    finally:
        c.close()


def test_pinned_buffers_batched_and_served(sgm):
    import torch

    # the batched and served forms stage pinned host buffers the same way
    shapes = [(97, 61, 64, 4), (66, 40, 32, 8), (160, 96, 128, 4)]
    pairs = [_pair(W, H, D, seed=500 + i) for i, (W, H, D, npth) in enumerate(shapes)]
    refs = [oracle.sgm(q.left, q.right, D, 7, 84, npth) for q, (W, H, D, npth) in zip(pairs, shapes)]
    pin = [(torch.from_numpy(q.left).pin_memory(), torch.from_numpy(q.right).pin_memory(),
            torch.full((H, W), 255, dtype=torch.uint8).pin_memory()) for q, (W, H, D, npth) in zip(pairs, shapes)]
    c = sgm.Context(0)
    try:
        sgm.sgm_compute_batch(c.handle, [(l, r, o, W, H, D, 7, 84, npth)
                                         for (l, r, o), (W, H, D, npth) in zip(pin, shapes)])
        for (l, r, o), want in zip(pin, refs):
            assert (o.numpy() == want).all()
        for (l, r, o), (W, H, D, npth) in zip(pin, shapes):
            o.fill_(255)
        ts = [sgm.sgm_submit(c.handle, l, r, W, H, D, 7, 84, npth, o) for (l, r, o), (W, H, D, npth) in zip(pin, shapes)]
        for t in ts:
            assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK
        for (l, r, o), want in zip(pin, refs):
            assert (o.numpy() == want).all()
    finally:
        c.close()

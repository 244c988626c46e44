"""Post-filters on the GPU (sgm_compute_ex) vs the oracle, bit-exact.

Sub-pixel disparity, the left-right check and adaptive P2 (the post-filters
Section 5 announces) are integer arithmetic in the readings both sides
implement, so the bar stays bit-exact equality of the uint16 output.
"""
import numpy as np
import pytest

import oracle
import stereo_synth as synth

pytestmark = pytest.mark.gpu

SUB, LR, AP2 = oracle.POST_SUBPIXEL, oracle.POST_LR_CHECK, oracle.POST_ADAPTIVE_P2


@pytest.fixture(scope="module")
def sgm():
    from paper_1610_04121_gb300 import sgm as m

    return m


@pytest.fixture(scope="module")
def ctx(sgm):
    c = sgm.Context(0)
    yield c
    c.close()


def _check(ctx, left, right, D, P1, P2, n_paths, post, census="csct"):
    got = ctx.compute_ex(left, right, D, P1, P2, n_paths, post)
    ref = oracle.sgm_ex(left, right, D, P1, P2, n_paths, post, census)
    bad = np.argwhere(got != ref)
    assert bad.size == 0, f"post={post}: differs at {bad[:5].tolist()} (of {len(bad)}): " \
                          f"{[(int(got[y, x]), int(ref[y, x])) for y, x in bad[:5]]}"
    return got


@pytest.mark.parametrize("post", [SUB, LR, AP2, SUB | LR, SUB | LR | AP2])
@pytest.mark.parametrize("n_paths", [2, 4, 8])
@pytest.mark.parametrize("D", [32, 64, 96, 128, 256])
def test_small_ragged(ctx, D, n_paths, post):
    pair = synth.make_pair(synth.PairSpec(77, 45, D, 4, 2, min(48, D - 1)), 5000 + D + n_paths)
    _check(ctx, pair.left, pair.right, D, 7, 84, n_paths, post)


@pytest.mark.parametrize("n_paths", [2, 4, 8])
def test_no_post_filter_is_16_times_sgm_compute(ctx, n_paths):
    pair = synth.make_pair(synth.PairSpec(90, 50, 64, 4, 2, 40), 77)
    got = ctx.compute_ex(pair.left, pair.right, 64, 7, 84, n_paths, 0)
    assert (got == 16 * ctx.compute(pair.left, pair.right, 64, 7, 84, n_paths).astype(np.uint16)).all()


@pytest.mark.parametrize("W,H", [(1, 1), (1, 9), (9, 1), (2, 33), (33, 2), (3, 3), (9, 7), (17, 23)])
@pytest.mark.parametrize("n_paths", [2, 4, 8])
def test_degenerate_sizes(ctx, W, H, n_paths):
    rng = np.random.default_rng(W * 31 + H)
    left = rng.integers(0, 256, (H, W), dtype=np.uint8)
    right = rng.integers(0, 256, (H, W), dtype=np.uint8)
    _check(ctx, left, right, 32, 7, 84, n_paths, SUB | LR | AP2)


@pytest.mark.parametrize("P1,P2", [(70, 20), (100, 20), (0, 0), (224, 224), (5, 224)])
@pytest.mark.parametrize("n_paths", [2, 4, 8])
def test_adaptive_p2_penalty_edges(ctx, P1, P2, n_paths):
    # 4 paths keep byte sums while 2 * (31 + max(P1, P2)) <= 255
    pair = synth.make_pair(synth.PairSpec(64, 40, 64, 4, 2, 40), P1 + P2)
    _check(ctx, pair.left, pair.right, 64, P1, P2, n_paths, AP2 | SUB)


def test_full_census_with_post_filters(sgm):
    pair = synth.make_pair(synth.PairSpec(80, 44, 64, 4, 2, 40), 13)
    with sgm.Context(0, flags=sgm.SGM_FLAG_CENSUS_FULL) as c:
        _check(c, pair.left, pair.right, 64, 7, 60, 4, SUB | LR | AP2, census="ct62")
        out = np.zeros((44, 80), np.uint16)
        with pytest.raises(sgm.SgmError) as e:  # max(P1, P2) = 200 > 255 - 62
            sgm.sgm_compute_ex(c.handle, pair.left, pair.right, 80, 44, 64, 200, 60, 4, AP2, out)
        assert e.value.code == sgm.SGM_EINVAL
        # without adaptive P2 only P2 is bounded
        _check(c, pair.left, pair.right, 64, 200, 60, 4, SUB | LR, census="ct62")


def test_unknown_flag_rejected(sgm, ctx):
    pair = synth.make_pair(synth.PairSpec(64, 32, 64, 4, 2, 40), 5)
    out = np.zeros((32, 64), np.uint16)
    with pytest.raises(sgm.SgmError) as e:
        sgm.sgm_compute_ex(ctx.handle, pair.left, pair.right, 64, 32, 64, 7, 84, 4, 8, out)
    assert e.value.code == sgm.SGM_EINVAL


def test_device_pointers_and_repeat_calls(sgm, ctx):
    import torch

    pair = synth.make_pair(synth.PairSpec(120, 70, 128, 4, 2, 80), 21)
    ref = oracle.sgm_ex(pair.left, pair.right, 128, 7, 84, 4, SUB | LR)
    L = torch.from_numpy(pair.left).cuda()
    R = torch.from_numpy(pair.right).cuda()
    out = torch.zeros((70, 120), dtype=torch.int16, device="cuda")
    for _ in range(3):  # the second and third calls replay the captured graph
        sgm.sgm_compute_ex(ctx.handle, L, R, 120, 70, 128, 7, 84, 4, SUB | LR, out)
        got = out.cpu().numpy().view(np.uint16)
        assert (got == ref).all()
    # the plain path in between still gives its own result
    assert (ctx.compute(pair.left, pair.right, 128, 7, 84, 4) == oracle.sgm(pair.left, pair.right, 128, 7, 84, 4)).all()


@pytest.mark.parametrize("n_paths", [4, 8])
def test_full_size_frame(ctx, n_paths):
    pair = synth.make_pair(synth.PairSpec(640, 480, 128, 4, 2, 100), 31)
    _check(ctx, pair.left, pair.right, 128, 7, 84, n_paths, SUB | LR | AP2)


def test_async_form_on_the_context_stream(sgm):
    import torch

    pair = synth.make_pair(synth.PairSpec(130, 66, 64, 4, 2, 40), 23)
    ref = oracle.sgm_ex(pair.left, pair.right, 64, 10, 120, 8, SUB | LR | AP2)
    L = torch.from_numpy(pair.left).cuda()
    R = torch.from_numpy(pair.right).cuda()
    out = torch.zeros((66, 130), dtype=torch.int16, device="cuda")
    with sgm.Context(0) as c:
        sgm.sgm_set_stream(c.handle, torch.cuda.current_stream())
        sgm.sgm_compute_ex_async(c.handle, L, R, 130, 66, 64, 10, 120, 8, SUB | LR | AP2, out)
        torch.cuda.current_stream().synchronize()
        sgm.sgm_set_stream(c.handle, None)
        got = out.cpu().numpy().view(np.uint16)
        bad = np.argwhere(got != ref)
        assert bad.size == 0, f"{len(bad)} differ, e.g. {[(y, x, int(got[y, x]), int(ref[y, x])) for y, x in bad[:6]]}"
        with pytest.raises(sgm.SgmError):  # host pointers are refused
            sgm.sgm_compute_ex_async(c.handle, pair.left, pair.right, 130, 66, 64, 10, 120, 8, SUB,
                                     np.zeros((66, 130), np.uint16))

"""The allocation-free entry point, checked against sgm_compute.

Some callers cannot allocate device memory: an embedding runtime that owns
all of it, a plugin that may only use the buffers its host hands it, or a
real-time loop that must never allocate.  They call sgm_compute_static, whose
intermediates live in one static device array of the library.  Its output must
equal sgm_compute's, bit for bit (all arithmetic is integer), call after call.

This file is named to run last, so that a run which stops at the first failure
has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest

import stereo_synth as synth

pytestmark = pytest.mark.gpu

CASES = [
    (320, 240, 64, 7, 84, 4, 11),     # the small single-pair workload's shape
    (160, 120, 96, 10, 120, 8, 12),   # 8 paths, D not a multiple of 64
    (97, 61, 32, 7, 84, 2, 13),       # 2 paths, ragged sizes
    (200, 100, 128, 10, 120, 4, 14),  # 4 paths whose sums need 16 bits (P2 > 96)
    (320, 240, 128, 10, 120, 8, 15),  # about 40 MB of intermediates: near the array's size
]


@pytest.mark.parametrize("W,H,D,P1,P2,n_paths,seed", CASES)
def test_static_entry_matches_compute_on_two_calls(W, H, D, P1, P2, n_paths, seed):
    import torch

    from paper_1610_04121_gb300 import sgm

    pair = synth.make_pair(synth.PairSpec(W, H, D, 6, 2, min(48, D - 1)), seed)
    with sgm.Context(0) as ctx:
        expected = ctx.compute(pair.left, pair.right, D, P1, P2, n_paths)
    left = torch.from_numpy(pair.left).cuda()
    right = torch.from_numpy(pair.right).cuda()
    stream = torch.cuda.current_stream()
    outs = [torch.full((H, W), 255, dtype=torch.uint8, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free_before = None
    for k, out in enumerate(outs):
        sgm.sgm_compute_static(left, right, W, H, D, P1, P2, n_paths, out, stream)
        stream.synchronize()
        got = out.cpu().numpy()
        assert np.array_equal(got, expected), f"{int((got != expected).sum())} pixels differ"
        if k == 0:
            free_before = torch.cuda.mem_get_info()[0]  # after the first call's set-up
    # the second call took no device memory
    assert torch.cuda.mem_get_info()[0] == free_before


def test_static_entry_rejects_what_it_cannot_hold():
    import torch

    from paper_1610_04121_gb300 import sgm

    big = torch.zeros((480, 640), dtype=torch.uint8, device="cuda")
    with pytest.raises(sgm.SgmError) as e:
        sgm.sgm_compute_static(big, big, 640, 480, 128, 7, 84, 4, big)
    assert e.value.code == sgm.SGM_EINVAL and "static scratch" in str(e.value)
    host = np.zeros((16, 16), dtype=np.uint8)
    with pytest.raises(sgm.SgmError) as e:
        sgm.sgm_compute_static(host, host, 16, 16, 32, 7, 84, 4, host)
    assert e.value.code == sgm.SGM_EINVAL

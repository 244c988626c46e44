"""The bounds-checked build (-DSGM_BOUNDS_CHECK, include/sgm.h): on valid
inputs every path gives the oracle's result with no guard firing; a guard
that fires is reported as SGM_EDEVICE.  The fired guard is made by a test
hook that declares the paired schedule's cube arrays one quad shorter than
they are, so the access it skips lies in range: nothing reads or writes out
of bounds.  The checked library runs in a child process
(SGM_BOUNDS_CHECK=1 selects it in the binding).
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PRELUDE = textwrap.dedent(f"""
    import sys
    import numpy as np
    sys.path.insert(0, {ROOT!r})
    import oracle
    import stereo_synth as synth
    from paper_1610_04121_gb300 import sgm
    assert sgm.sgm_bounds_checked(), "the checked library is not the one loaded"

    def pair(W, H, D, seed):
        return synth.make_pair(synth.PairSpec(W, H, D, 4, 2, min(48, D - 1)), seed)
""")

VALID = PRELUDE + textwrap.dedent("""
    p = pair(77, 45, 128, 1)
    with sgm.Context(0) as c:
        for sched in (0, 1, 2):
            sgm.sgm_set_schedule(c.handle, sched)
            for P2 in (84, 120):
                assert (c.compute(p.left, p.right, 128, 7, P2, 4) == oracle.sgm(p.left, p.right, 128, 7, P2, 4)).all()
        sgm.sgm_set_schedule(c.handle, sgm.SGM_SCHED_PAIRS)
        dbg = c.debug(p.left, p.right, 128, 7, 84, 4)
        assert (dbg["raw"] == oracle.sgm(p.left, p.right, 128, 7, 84, 4, debug=True)["raw"]).all()
        q = pair(70, 41, 96, 2)
        for n_paths, P2 in ((8, 120), (2, 84)):
            assert (c.compute(q.left, q.right, 96, 10, P2, n_paths)
                    == oracle.sgm(q.left, q.right, 96, 10, P2, n_paths)).all()
        assert (c.compute_ex(q.left, q.right, 96, 10, 84, 4, 7) == oracle.sgm_ex(q.left, q.right, 96, 10, 84, 4, 7)).all()
        outs = [np.zeros((45, 77), np.uint8), np.zeros((41, 70), np.uint8)]
        sgm.sgm_compute_batch(c.handle, [(p.left, p.right, outs[0], 77, 45, 128, 7, 84, 4),
                                         (q.left, q.right, outs[1], 70, 41, 96, 10, 120, 8)])
        assert (outs[0] == oracle.sgm(p.left, p.right, 128, 7, 84, 4)).all()
        assert (outs[1] == oracle.sgm(q.left, q.right, 96, 10, 120, 8)).all()
        o = np.zeros((45, 77), np.uint8)
        t = sgm.sgm_submit(c.handle, p.left, p.right, 77, 45, 128, 7, 84, 4, o)
        assert sgm.sgm_poll(c.handle, t, -1) == sgm.SGM_OK and (o == oracle.sgm(p.left, p.right, 128, 7, 84, 4)).all()
    with sgm.Context(0, flags=sgm.SGM_FLAG_CENSUS_FULL) as c:
        assert (c.compute(p.left, p.right, 128, 7, 84, 4)
                == oracle.sgm(p.left, p.right, 128, 7, 84, 4, census="ct62")).all()
    assert sgm.sgm_bounds_fault() == 0
    print("ok")
""")

FIRED = PRELUDE + textwrap.dedent("""
    p = pair(77, 45, 128, 3)
    with sgm.Context(0) as c:
        sgm.sgm_set_schedule(c.handle, sgm.SGM_SCHED_PAIRS)
        try:
            c.compute(p.left, p.right, 128, 7, 84, 4)
            raise SystemExit("no guard fired")
        except sgm.SgmError as e:
            assert e.code == sgm.SGM_EDEVICE, e
            assert "bounds check" in str(e), e
    assert sgm.sgm_bounds_fault() == 0  # the call took and cleared it
    print("ok")
""")


@pytest.fixture(scope="module")
def checked_lib():
    from paper_1610_04121_gb300 import build

    return build.build(bounds_check=True)


def _child(script, **env):
    e = dict(os.environ, SGM_BOUNDS_CHECK="1", **env)
    r = subprocess.run([sys.executable, "-c", script], env=e, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-4000:]


def test_checked_build_matches_the_oracle_with_no_guard_firing(checked_lib):
    _child(VALID)


def test_a_fired_guard_is_reported_as_edevice(checked_lib):
    _child(FIRED, SGM_TEST_BOUNDS_SHRINK="1")

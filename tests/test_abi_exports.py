"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol.

No compute call is made here: these run on hosts without a GPU.
"""
import ctypes
import os
import re

import pytest

from paper_1610_04121_gb300 import build as sgm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    return sgm_build.build()


def test_every_declared_function_is_exported(lib_path):
    from paper_1610_04121_gb300 import sgm

    lib = ctypes.CDLL(lib_path)
    names = list(sgm.header_functions())
    assert "sgm_compute" in names and "sgm_submit" in names and "sgm_poll" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/sgm.h but not exported"


def test_only_the_abi_is_exported(lib_path):
    """Everything else is hidden (-fvisibility=hidden): no C++ symbols leak."""
    import subprocess

    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if " T " in l}
    from paper_1610_04121_gb300 import sgm

    assert set(sgm.header_functions()) <= syms
    leaked = [s for s in syms if s.startswith("_Z") and "sgm" in s]
    assert not leaked, leaked[:5]


def test_built_for_sm_103a_only(lib_path):
    import subprocess

    r = subprocess.run(["cuobjdump", "--list-elf", lib_path], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    arches = set(re.findall(r"sm_(\d+a?)", r.stdout))
    assert arches == {"103a"}, arches


def test_argument_validation_without_a_gpu(lib_path):
    from paper_1610_04121_gb300 import sgm

    lib = sgm._lib
    assert lib.sgm_compute(None, None, None, 4, 4, 32, 1, 2, 4, None) == sgm.SGM_EINVAL
    assert lib.sgm_destroy(None) == sgm.SGM_OK
    assert lib.sgm_poll(None, 1, 0) == sgm.SGM_EINVAL
    assert lib.sgm_kernel_launches(None) == 0
    assert "sm_103a" in sgm.sgm_version()
    out = ctypes.c_void_p()
    assert lib.sgm_create(ctypes.byref(out), 0, 0, 7) == sgm.SGM_EINVAL  # flags must be 0


def test_header_documents_each_entry_point():
    text = open(os.path.join(ROOT, "include", "sgm.h")).read()
    for name in ["sgm_create", "sgm_compute", "sgm_submit", "sgm_poll", "sgm_destroy"]:
        i = text.index(name + "(")
        assert "/*" in text[max(0, i - 1500):i], name

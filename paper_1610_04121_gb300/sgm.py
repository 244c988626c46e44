"""Thin ctypes binding of the C ABI in ``include/sgm.h``.

Functions keep the C names and only marshal arguments: every stage of the
path runs in the CUDA library.  There is no CPU fallback: importing this
module raises if ``_lib/libsgm_gb300.so`` has not been built.

Array arguments may be numpy arrays (host memory), torch tensors (host or
CUDA) or raw integer addresses.
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Optional, Sequence

from . import build as _build

# SGM_BOUNDS_CHECK=1 in the environment selects the bounds-checked build
LIB_PATH = _build.CHECKED_LIB_PATH if os.environ.get("SGM_BOUNDS_CHECK") == "1" else _build.LIB_PATH

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"the SGM CUDA library is not built ({LIB_PATH} is missing); run "
        "`python -m paper_1610_04121_gb300.build` (needs nvcc) -- there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

SGM_OK, SGM_EAGAIN, SGM_EINVAL, SGM_ENOMEM = 0, 1, -1, -2
SGM_ECUDA, SGM_ETIMEDOUT, SGM_ECANCELED, SGM_EDEVICE = -3, -4, -5, -6
STATUS_NAMES = {0: "SGM_OK", 1: "SGM_EAGAIN", -1: "SGM_EINVAL", -2: "SGM_ENOMEM", -3: "SGM_ECUDA",
                -4: "SGM_ETIMEDOUT", -5: "SGM_ECANCELED", -6: "SGM_EDEVICE"}
SGM_FLAG_STAGE_TIMING = 1
SGM_FLAG_CENSUS_FULL = 2
SGM_POST_SUBPIXEL = 1
SGM_POST_LR_CHECK = 2
SGM_POST_ADAPTIVE_P2 = 4
SGM_DISP16_INVALID = 0xFFFF
SGM_SCHED_V_THEN_H = 0
SGM_SCHED_H_THEN_V = 1
SGM_SCHED_PAIRS = 2
SGM_MAX_D = 256
SGM_MAX_PENALTY = 224

_vp = ctypes.c_void_p
_i = ctypes.c_int


class sgm_pair(ctypes.Structure):
    _fields_ = [("left", _vp), ("right", _vp), ("disp_out", _vp), ("W", ctypes.c_int32), ("H", ctypes.c_int32),
                ("D", ctypes.c_int32), ("P1", ctypes.c_int32), ("P2", ctypes.c_int32),
                ("n_paths", ctypes.c_int32)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("sgm_create", _i, [ctypes.POINTER(_vp), _i, ctypes.c_size_t, ctypes.c_uint])
_sig("sgm_destroy", _i, [_vp])
_sig("sgm_last_error", ctypes.c_char_p, [_vp])
_sig("sgm_set_stream", _i, [_vp, _vp])
_sig("sgm_compute", _i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp])
_sig("sgm_compute_async", _i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp])
_sig("sgm_compute_ex", _i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, ctypes.c_uint, _vp])
_sig("sgm_compute_ex_async", _i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, ctypes.c_uint, _vp])
_sig("sgm_compute_batch", _i, [_vp, _i, ctypes.POINTER(sgm_pair)])
_sig("sgm_submit", _i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp, ctypes.POINTER(ctypes.c_uint64)])
_sig("sgm_poll", _i, [_vp, ctypes.c_uint64, ctypes.c_int64])
_sig("sgm_served_stats", _i, [_vp, ctypes.POINTER(ctypes.c_double), _i])
_sig("sgm_served_reset_stats", _i, [_vp])
_sig("sgm_set_admission_bound", _i, [_vp, ctypes.c_int64])
_sig("sgm_save_tuning", _i, [_vp, ctypes.c_char_p])
_sig("sgm_bounds_checked", _i, [])
_sig("sgm_bounds_fault", ctypes.c_uint, [])
_sig("sgm_load_tuning", _i, [_vp, ctypes.c_char_p])
_sig("sgm_debug_stages", _i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp])
_sig("sgm_kernel_launches", ctypes.c_uint64, [_vp])
_sig("sgm_stage_times", _i, [_vp, ctypes.POINTER(ctypes.c_float), _i])
_sig("sgm_stage_name", ctypes.c_char_p, [_i, _i])
_sig("sgm_stage_paths", _i, [_vp])
_sig("sgm_stage_label", ctypes.c_char_p, [_vp, _i])
_sig("sgm_set_schedule", _i, [_vp, _i])
_sig("sgm_schedule_for", _i, [_vp, _i, _i, _i, _i, _i, _i])
_sig("sgm_version", ctypes.c_char_p, [])
_sig("sgm_compute_static", _i, [_vp, _vp, _i, _i, _i, _i, _i, _i, _vp, _vp])


class SgmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def addr(x) -> Optional[int]:
    """Address of a numpy array, torch tensor or integer (None stays None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _check(ctx, rc: int, allow=(SGM_OK,)) -> int:
    if rc not in allow:
        raise SgmError(rc, last_error(ctx))
    return rc


def last_error(ctx) -> str:
    s = _lib.sgm_last_error(ctx)
    return s.decode() if s else ""


def sgm_version() -> str:
    return _lib.sgm_version().decode()


def sgm_create(device: int = 0, mem_cap_bytes: int = 0, flags: int = 0) -> int:
    out = _vp()
    _check(None, _lib.sgm_create(ctypes.byref(out), device, mem_cap_bytes, flags))
    return out.value


def sgm_destroy(ctx) -> None:
    _lib.sgm_destroy(ctx)


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream as an explicit handle


def sgm_set_stream(ctx, stream) -> None:
    """`stream`: a torch.cuda.Stream, an integer cudaStream_t, or None (the
    context's own stream).  torch's default stream has the handle 0, which
    the library reads as None, so it is passed as cudaStreamLegacy."""
    handle = getattr(stream, "cuda_stream", stream)
    if handle == 0 and stream is not None and hasattr(stream, "cuda_stream"):
        handle = CUDA_STREAM_LEGACY
    _check(ctx, _lib.sgm_set_stream(ctx, handle))


def sgm_compute(ctx, left, right, W, H, D, P1, P2, n_paths, disp_out) -> None:
    _check(ctx, _lib.sgm_compute(ctx, addr(left), addr(right), W, H, D, P1, P2, n_paths, addr(disp_out)))


def sgm_compute_ex(ctx, left, right, W, H, D, P1, P2, n_paths, post, disp16_out) -> None:
    _check(ctx, _lib.sgm_compute_ex(ctx, addr(left), addr(right), W, H, D, P1, P2, n_paths, post,
                                    addr(disp16_out)))


def sgm_compute_ex_async(ctx, left, right, W, H, D, P1, P2, n_paths, post, disp16_out) -> None:
    _check(ctx, _lib.sgm_compute_ex_async(ctx, addr(left), addr(right), W, H, D, P1, P2, n_paths, post,
                                          addr(disp16_out)))


def sgm_compute_async(ctx, left, right, W, H, D, P1, P2, n_paths, disp_out) -> None:
    _check(ctx, _lib.sgm_compute_async(ctx, addr(left), addr(right), W, H, D, P1, P2, n_paths, addr(disp_out)))


def sgm_compute_batch(ctx, pairs: Sequence[tuple]) -> None:
    """pairs: (left, right, disp_out, W, H, D, P1, P2, n_paths) tuples."""
    arr = (sgm_pair * max(1, len(pairs)))()
    for i, (l, r, o, W, H, D, P1, P2, npth) in enumerate(pairs):
        arr[i] = sgm_pair(addr(l), addr(r), addr(o), W, H, D, P1, P2, npth)
    _check(ctx, _lib.sgm_compute_batch(ctx, len(pairs), arr))


def sgm_submit(ctx, left, right, W, H, D, P1, P2, n_paths, disp_out) -> Optional[int]:
    """The request's ticket, or None when the admission bound shed it (SGM_EAGAIN)."""
    t = ctypes.c_uint64()
    rc = _check(ctx, _lib.sgm_submit(ctx, addr(left), addr(right), W, H, D, P1, P2, n_paths, addr(disp_out),
                                     ctypes.byref(t)), allow=(SGM_OK, SGM_EAGAIN))
    return t.value if rc == SGM_OK else None


def sgm_bounds_checked() -> bool:
    return _lib.sgm_bounds_checked() == 1


def sgm_bounds_fault() -> int:
    return int(_lib.sgm_bounds_fault())


def sgm_set_admission_bound(ctx, max_wait_us: int) -> None:
    _check(ctx, _lib.sgm_set_admission_bound(ctx, max_wait_us))


def sgm_save_tuning(ctx, path: str) -> None:
    _check(ctx, _lib.sgm_save_tuning(ctx, os.fsencode(path)))


def sgm_load_tuning(ctx, path: str) -> None:
    _check(ctx, _lib.sgm_load_tuning(ctx, os.fsencode(path)))


def sgm_poll(ctx, ticket: int, timeout_us: int = -1) -> int:
    """Returns SGM_OK, SGM_EAGAIN or SGM_ETIMEDOUT; raises on errors."""
    return _check(ctx, _lib.sgm_poll(ctx, ticket, timeout_us), allow=(SGM_OK, SGM_EAGAIN, SGM_ETIMEDOUT))


def sgm_served_stats(ctx) -> dict:
    out = (ctypes.c_double * 13)()
    _check(ctx, _lib.sgm_served_stats(ctx, out, 13))
    return {"completed": int(out[0]), "p50_us": out[1], "p99_us": out[2], "max_us": out[3], "batches": int(out[4]),
            "mean_batch": out[5], "max_in_flight": int(out[6]), "de": out[7], "shed": int(out[8]),
            "service_de_per_s": out[9], "queued": int(out[10]), "in_flight": int(out[11]),
            "pool_bytes": int(out[12])}


def sgm_served_reset_stats(ctx) -> None:
    _check(ctx, _lib.sgm_served_reset_stats(ctx))


def sgm_debug_stages(ctx, left, right, W, H, D, P1, P2, n_paths, Fb=None, Fm=None, MC=None, S=None, raw=None,
                     disp=None) -> None:
    _check(ctx, _lib.sgm_debug_stages(ctx, addr(left), addr(right), W, H, D, P1, P2, n_paths, addr(Fb), addr(Fm),
                                      addr(MC), addr(S), addr(raw), addr(disp)))


def sgm_stage_times(ctx) -> dict:
    """Per-kernel device milliseconds of the last enqueued path, by stage name."""
    buf = (ctypes.c_float * 10)()
    n = _lib.sgm_stage_times(ctx, buf, 10)
    if n < 0:
        raise SgmError(n, last_error(ctx))
    return {_lib.sgm_stage_label(ctx, i).decode(): float(buf[i]) for i in range(n)}


def sgm_set_schedule(ctx, schedule: int) -> None:
    """Force a 4-path sweep schedule (SGM_SCHED_*), or -1 to autotune."""
    _check(ctx, _lib.sgm_set_schedule(ctx, schedule))


def sgm_schedule_for(ctx, W, H, D, P1, P2, n_paths) -> int:
    """The schedule used for this problem, or -1 when not tuned yet."""
    return _lib.sgm_schedule_for(ctx, W, H, D, P1, P2, n_paths)


def sgm_compute_static(left, right, W, H, D, P1, P2, n_paths, disp_out, stream=None) -> None:
    """Allocation-free path on device buffers; enqueued on `stream` (not waited for)."""
    handle = getattr(stream, "cuda_stream", stream)
    _check(None, _lib.sgm_compute_static(addr(left), addr(right), W, H, D, P1, P2, n_paths, addr(disp_out), handle))


def sgm_kernel_launches(ctx) -> int:
    return int(_lib.sgm_kernel_launches(ctx))


class Context:
    """Owns one sgm_ctx; a convenience over the functions above."""

    def __init__(self, device: int = 0, mem_cap_bytes: int = 0, flags: int = 0):
        self.flags = flags
        self.handle = sgm_create(device, mem_cap_bytes, flags)

    def close(self):
        if self.handle:
            sgm_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def compute(self, left, right, D, P1, P2, n_paths, out=None):
        """Disparity of one pair; numpy in -> numpy out, torch in -> torch out."""
        H, W = left.shape
        if out is None:
            out = _empty_like_u8(left)
        sgm_compute(self.handle, left, right, W, H, D, P1, P2, n_paths, out)
        return out

    def compute_ex(self, left, right, D, P1, P2, n_paths, post=0, out=None):
        """Disparity in 1/16 pixel with post-filters: numpy in -> uint16 out;
        torch in -> an int16 tensor holding the uint16 values (SGM_DISP16_INVALID
        reads as -1; view it as uint16 through numpy)."""
        H, W = left.shape
        if out is None:
            if hasattr(left, "data_ptr") and hasattr(left, "device"):
                import torch

                out = torch.empty((H, W), dtype=torch.int16, device=left.device)
            else:
                import numpy as np

                out = np.empty((H, W), np.uint16)
        sgm_compute_ex(self.handle, left, right, W, H, D, P1, P2, n_paths, post, out)
        return out

    def debug(self, left, right, D, P1, P2, n_paths):
        import numpy as np

        H, W = left.shape
        ft = np.uint64 if self.flags & SGM_FLAG_CENSUS_FULL else np.uint32
        r = {"Fb": np.zeros((H, W), ft), "Fm": np.zeros((H, W), ft),
             "MC": np.zeros((H, W, D), np.uint8), "S": np.zeros((H, W, D), np.uint16),
             "raw": np.zeros((H, W), np.uint8), "disp": np.zeros((H, W), np.uint8)}
        sgm_debug_stages(self.handle, np.ascontiguousarray(left), np.ascontiguousarray(right), W, H, D, P1, P2,
                         n_paths, r["Fb"], r["Fm"], r["MC"], r["S"], r["raw"], r["disp"])
        return r

    @property
    def launches(self) -> int:
        return sgm_kernel_launches(self.handle)


def _empty_like_u8(x):
    if hasattr(x, "data_ptr") and hasattr(x, "device"):
        import torch

        return torch.empty(tuple(x.shape), dtype=torch.uint8, device=x.device)
    import numpy as np

    return np.empty(x.shape, dtype=np.uint8)


def header_functions(header_path: Optional[str] = None) -> Iterable[str]:
    """Names of the functions declared in include/sgm.h."""
    import re

    header_path = header_path or os.path.join(_build.INCLUDE, "sgm.h")
    text = open(header_path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgm_[a-z_0-9]+)\s*\(", text)))

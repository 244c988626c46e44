"""ctypes loader for the C oracle (test infrastructure only).

Each wrapper names the equation of the paper (arXiv 1610.04121) that the C
function states; see ``sgm_oracle.c`` for the readings where the paper is
silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u16p = ctypes.POINTER(ctypes.c_uint16)

# post-filter flags of sgm_ex (values of the C ABI's SGM_POST_* flags)
POST_SUBPIXEL = 1
POST_LR_CHECK = 2
POST_ADAPTIVE_P2 = 4
DISP16_INVALID = 0xFFFF


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared", "-fPIC", "-pthread", "-o", tmp,
                        _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_csct_at.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_csct_at.restype = ctypes.c_uint32
            lib.oracle_csct.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, _u32p]
            lib.oracle_csct.restype = None
            lib.oracle_bitcount.argtypes = [ctypes.c_uint32]
            lib.oracle_bitcount.restype = ctypes.c_int
            lib.oracle_cost.argtypes = [_u32p, _u32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p]
            lib.oracle_cost.restype = None
            lib.oracle_aggregate.argtypes = [_u8p] + [ctypes.c_int] * 7 + [_i32p]
            lib.oracle_aggregate.restype = None
            lib.oracle_directions.argtypes = [ctypes.c_int, _i32p, _i32p]
            lib.oracle_directions.restype = ctypes.c_int
            lib.oracle_wta.argtypes = [_i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p]
            lib.oracle_wta.restype = None
            lib.oracle_median3x3.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, _u8p]
            lib.oracle_median3x3.restype = None
            lib.oracle_sgm.argtypes = [_u8p, _u8p] + [ctypes.c_int] * 6 + [_u8p, _u8p, _u32p, _u32p, _i32p]
            lib.oracle_sgm.restype = ctypes.c_int
            lib.oracle_pixel.argtypes = [_u8p, _u8p] + [ctypes.c_int] * 8 + [_i32p]
            lib.oracle_pixel.restype = ctypes.c_int
            lib.oracle_ct62_at.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.oracle_ct62_at.restype = ctypes.c_uint64
            lib.oracle_ct62.argtypes = [_u8p, ctypes.c_int, ctypes.c_int, _u64p]
            lib.oracle_ct62.restype = None
            lib.oracle_bitcount64.argtypes = [ctypes.c_uint64]
            lib.oracle_bitcount64.restype = ctypes.c_int
            lib.oracle_cost64.argtypes = [_u64p, _u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u8p]
            lib.oracle_cost64.restype = None
            lib.oracle_sgm_ct62.argtypes = [_u8p, _u8p] + [ctypes.c_int] * 6 + [_u8p, _u8p, _u64p, _u64p, _i32p]
            lib.oracle_sgm_ct62.restype = ctypes.c_int
            lib.oracle_aggregate_ex.argtypes = [_u8p, _u8p] + [ctypes.c_int] * 7 + [_i32p]
            lib.oracle_aggregate_ex.restype = None
            lib.oracle_subpixel.argtypes = [_i32p, ctypes.c_int, ctypes.c_int]
            lib.oracle_subpixel.restype = ctypes.c_int
            lib.oracle_median3x3_u16.argtypes = [_u16p, ctypes.c_int, ctypes.c_int, _u16p]
            lib.oracle_median3x3_u16.restype = None
            lib.oracle_sgm_ex.argtypes = [_u8p, _u8p] + [ctypes.c_int] * 7 + [ctypes.c_uint, _u16p, _u8p, _u8p]
            lib.oracle_sgm_ex.restype = ctypes.c_int
            lib.oracle_sgm_threads.argtypes = [_u8p, _u8p] + [ctypes.c_int] * 6 + [_u8p, ctypes.c_int]
            lib.oracle_sgm_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, t):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(t)


def _img(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint8)
    assert a.ndim == 2
    return a


def csct_at(img: np.ndarray, x: int, y: int) -> int:
    """Eq. 1 at one pixel."""
    img = _img(img)
    H, W = img.shape
    return int(load().oracle_csct_at(_ptr(img, _u8p), W, H, x, y))


def csct(img: np.ndarray) -> np.ndarray:
    """Eq. 1 over an image -> uint32 [H, W]."""
    img = _img(img)
    H, W = img.shape
    F = np.zeros((H, W), dtype=np.uint32)
    load().oracle_csct(_ptr(img, _u8p), W, H, _ptr(F, _u32p))
    return F


def bitcount(v: int) -> int:
    return int(load().oracle_bitcount(v & 0xFFFFFFFF))


def ct62_at(img: np.ndarray, x: int, y: int) -> int:
    """The full 9x7 Census transform (62 bits) at one pixel."""
    img = _img(img)
    H, W = img.shape
    return int(load().oracle_ct62_at(_ptr(img, _u8p), W, H, x, y))


def ct62(img: np.ndarray) -> np.ndarray:
    """The full 9x7 Census transform over an image -> uint64 [H, W]."""
    img = _img(img)
    H, W = img.shape
    F = np.zeros((H, W), dtype=np.uint64)
    load().oracle_ct62(_ptr(img, _u8p), W, H, _ptr(F, _u64p))
    return F


def bitcount64(v: int) -> int:
    return int(load().oracle_bitcount64(v & 0xFFFFFFFFFFFFFFFF))


def cost64(Fb: np.ndarray, Fm: np.ndarray, D: int) -> np.ndarray:
    """Eq. 2 on 62-bit Census features -> uint8 [H, W, D]."""
    Fb = np.ascontiguousarray(Fb, dtype=np.uint64)
    Fm = np.ascontiguousarray(Fm, dtype=np.uint64)
    H, W = Fb.shape
    MC = np.zeros((H, W, D), dtype=np.uint8)
    load().oracle_cost64(_ptr(Fb, _u64p), _ptr(Fm, _u64p), W, H, D, _ptr(MC, _u8p))
    return MC


def cost(Fb: np.ndarray, Fm: np.ndarray, D: int) -> np.ndarray:
    """Eq. 2 -> uint8 [H, W, D]."""
    Fb = np.ascontiguousarray(Fb, dtype=np.uint32)
    Fm = np.ascontiguousarray(Fm, dtype=np.uint32)
    H, W = Fb.shape
    MC = np.zeros((H, W, D), dtype=np.uint8)
    load().oracle_cost(_ptr(Fb, _u32p), _ptr(Fm, _u32p), W, H, D, _ptr(MC, _u8p))
    return MC


def aggregate(MC: np.ndarray, P1: int, P2: int, rx: int, ry: int) -> np.ndarray:
    """Eq. 3 along r = (rx, ry) -> int32 [H, W, D]."""
    MC = np.ascontiguousarray(MC, dtype=np.uint8)
    H, W, D = MC.shape
    L = np.zeros((H, W, D), dtype=np.int32)
    load().oracle_aggregate(_ptr(MC, _u8p), W, H, D, P1, P2, rx, ry, _ptr(L, _i32p))
    return L


def aggregate_ex(MC: np.ndarray, Ib: Optional[np.ndarray], P1: int, P2: int, rx: int, ry: int) -> np.ndarray:
    """Eq. 3 along r with adaptive P2 from the base image Ib (None: constant P2)."""
    MC = np.ascontiguousarray(MC, dtype=np.uint8)
    H, W, D = MC.shape
    L = np.zeros((H, W, D), dtype=np.int32)
    ib = ctypes.cast(None, _u8p) if Ib is None else _ptr(_img(Ib), _u8p)
    load().oracle_aggregate_ex(_ptr(MC, _u8p), ib, W, H, D, P1, P2, rx, ry, _ptr(L, _i32p))
    return L


def subpixel(S: np.ndarray, d: int) -> int:
    """Sub-pixel disparity (1/16 pixel) at the winner d of one pixel's S."""
    S = np.ascontiguousarray(S, dtype=np.int32)
    return int(load().oracle_subpixel(_ptr(S, _i32p), S.shape[0], d))


def median3x3_u16(v: np.ndarray) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.uint16)
    H, W = v.shape
    out = np.zeros_like(v)
    load().oracle_median3x3_u16(_ptr(v, _u16p), W, H, _ptr(out, _u16p))
    return out


def sgm_ex(left: np.ndarray, right: np.ndarray, D: int, P1: int, P2: int, n_paths: int, post: int = 0,
           census: str = "csct", debug: bool = False):
    """The path with the post-filters (sub-pixel, LR check, adaptive P2).

    Returns uint16 [H, W] in 1/16 pixel, DISP16_INVALID where the LR check
    fails; with ``debug`` a dict with ``out``, ``dL`` and ``dR`` (the integer
    winner-take-all disparities of the left and right passes).
    """
    if census not in ("csct", "ct62"):
        raise ValueError(f"unknown census {census!r}")
    left, right = _img(left), _img(right)
    H, W = left.shape
    out = np.zeros((H, W), dtype=np.uint16)
    dL = np.zeros((H, W), dtype=np.uint8)
    dR = np.zeros((H, W), dtype=np.uint8)
    rc = load().oracle_sgm_ex(_ptr(left, _u8p), _ptr(right, _u8p), W, H, D, P1, P2, n_paths,
                              1 if census == "ct62" else 0, post, _ptr(out, _u16p), _ptr(dL, _u8p), _ptr(dR, _u8p))
    if rc != 0:
        raise ValueError(f"oracle sgm_ex failed with {rc}")
    if debug:
        return {"out": out, "dL": dL, "dR": dR}
    return out


def directions(n_paths: int):
    rx = np.zeros(8, dtype=np.int32)
    ry = np.zeros(8, dtype=np.int32)
    n = load().oracle_directions(n_paths, _ptr(rx, _i32p), _ptr(ry, _i32p))
    return [(int(rx[i]), int(ry[i])) for i in range(n)]


def wta(S: np.ndarray) -> np.ndarray:
    """Eq. 4 -> uint8 [H, W]."""
    S = np.ascontiguousarray(S, dtype=np.int32)
    H, W, D = S.shape
    out = np.zeros((H, W), dtype=np.uint8)
    load().oracle_wta(_ptr(S, _i32p), W, H, D, _ptr(out, _u8p))
    return out


def median3x3(raw: np.ndarray) -> np.ndarray:
    raw = _img(raw)
    H, W = raw.shape
    out = np.zeros_like(raw)
    load().oracle_median3x3(_ptr(raw, _u8p), W, H, _ptr(out, _u8p))
    return out


def sgm(left: np.ndarray, right: np.ndarray, D: int, P1: int, P2: int, n_paths: int,
        debug: bool = False, census: str = "csct"):
    """Stages 2-4 of Section 2 on one pair.

    ``census`` is ``"csct"`` (Eq. 1, 31-bit features) or ``"ct62"`` (the full
    9x7 Census, 62-bit features).  Returns the final disparity (uint8 [H, W]);
    with ``debug`` a dict with ``disp``, ``raw``, ``Fb``, ``Fm`` (uint32 or
    uint64 [H, W]) and ``S`` (int32 [H, W, D]).
    """
    if census not in ("csct", "ct62"):
        raise ValueError(f"unknown census {census!r}")
    left, right = _img(left), _img(right)
    H, W = left.shape
    disp = np.zeros((H, W), dtype=np.uint8)
    null = lambda t: ctypes.cast(None, t)  # noqa: E731
    ftype, fptr = (np.uint32, _u32p) if census == "csct" else (np.uint64, _u64p)
    fn = load().oracle_sgm if census == "csct" else load().oracle_sgm_ct62
    if debug:
        raw = np.zeros((H, W), dtype=np.uint8)
        Fb = np.zeros((H, W), dtype=ftype)
        Fm = np.zeros((H, W), dtype=ftype)
        S = np.zeros((H, W, D), dtype=np.int32)
        rc = fn(_ptr(left, _u8p), _ptr(right, _u8p), W, H, D, P1, P2, n_paths, _ptr(disp, _u8p), _ptr(raw, _u8p),
                _ptr(Fb, fptr), _ptr(Fm, fptr), _ptr(S, _i32p))
    else:
        rc = fn(_ptr(left, _u8p), _ptr(right, _u8p), W, H, D, P1, P2, n_paths, _ptr(disp, _u8p), null(_u8p),
                null(fptr), null(fptr), null(_i32p))
    if rc != 0:
        raise ValueError(f"oracle sgm failed with {rc}")
    if debug:
        return {"disp": disp, "raw": raw, "Fb": Fb, "Fm": Fm, "S": S}
    return disp


def sgm_threads(left: np.ndarray, right: np.ndarray, D: int, P1: int, P2: int, n_paths: int,
                nthreads: int) -> np.ndarray:
    """oracle_sgm's disparity with its independent parts on ``nthreads`` threads
    (the CPU baseline's all-core timing; ``sgm`` stays the parity reference)."""
    left, right = _img(left), _img(right)
    H, W = left.shape
    out = np.zeros((H, W), dtype=np.uint8)
    rc = load().oracle_sgm_threads(_ptr(left, _u8p), _ptr(right, _u8p), W, H, D, P1, P2, n_paths, _ptr(out, _u8p),
                                   nthreads)
    if rc != 0:
        raise RuntimeError(f"oracle_sgm_threads failed ({rc})")
    return out


def pixel(left: np.ndarray, right: np.ndarray, D: int, P1: int, P2: int, n_paths: int, x: int, y: int
          ) -> Tuple[int, np.ndarray]:
    """Raw disparity and S(p, .) at one pixel, evaluated path by path."""
    left, right = _img(left), _img(right)
    H, W = left.shape
    S = np.zeros(D, dtype=np.int32)
    d = load().oracle_pixel(_ptr(left, _u8p), _ptr(right, _u8p), W, H, D, P1, P2, n_paths, x, y, _ptr(S, _i32p))
    if d < 0:
        raise ValueError(f"oracle_pixel failed with {d}")
    return int(d), S


def disp_at(left: np.ndarray, right: np.ndarray, D: int, P1: int, P2: int, n_paths: int,
            points, cache: Optional[Dict[Tuple[int, int], int]] = None) -> Dict[Tuple[int, int], int]:
    """Final (median-filtered) disparity at sampled points, via oracle_pixel.

    The median of an interior point needs the raw disparity of its 3x3
    neighbourhood; border points copy their raw value (the median reading).
    """
    left, right = _img(left), _img(right)
    H, W = left.shape
    cache = {} if cache is None else cache

    def raw(px, py):
        k = (px, py)
        if k not in cache:
            cache[k] = pixel(left, right, D, P1, P2, n_paths, px, py)[0]
        return cache[k]

    out = {}
    for (x, y) in points:
        if x == 0 or y == 0 or x == W - 1 or y == H - 1 or W < 3 or H < 3:
            out[(x, y)] = raw(x, y)
        else:
            v = sorted(raw(x + i, y + j) for j in (-1, 0, 1) for i in (-1, 0, 1))
            out[(x, y)] = v[4]
    return out

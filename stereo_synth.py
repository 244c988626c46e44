"""Seeded synthetic stereo pairs for the SGM hot path.

This module only makes inputs.  It holds none of the matching arithmetic
(no Census, no cost, no aggregation): both the CPU oracle and the CUDA path
consume the identical byte images it returns.

The paper measures on "multiple images" at 640x480 (Section 4) and reports
accuracy on KITTI; neither is available here, so rectified pairs are
synthesised with a known disparity field:

* left image: uniform random bytes smoothed by a 3x3 box filter,
  ``(sum + 4) // 9`` with clamp-to-edge sampling;
* ground-truth disparity on left coordinates: a background value (or a
  horizontal ramp) overwritten by random axis-aligned rectangles;
* right image: forward warp ``right[y, x - d] = left[y, x]`` (larger d wins a
  collision, as a nearer surface occludes), uncovered pixels filled with
  uniform random bytes, then Gaussian noise ``v + round(sigma * z)`` on the
  right image only, clamped to [0, 255].

Random numbers come from a counter-based generator: value ``i`` of stream
``s`` is the SplitMix64 output function applied to
``key(seed, s) + (i + 1) * 0x9E3779B97F4A7C15`` (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014).  Being
counter-based it vectorises in numpy and reproduces bit-for-bit on any host.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 161004121

# stream ids inside one pair
_S_TEXTURE, _S_RECT, _S_FILL, _S_NOISE, _S_META = 1, 2, 3, 4, 5


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        a = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        b = np.uint64(stream) * np.uint64(0xD1B54A32D192ED03)
        return _mix64(np.array([a ^ b], dtype=np.uint64))[0]


def stream_u64(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Values ``offset .. offset+n-1`` of counter stream ``stream``."""
    k = _key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _mix64(k + ctr * GOLDEN)


def uniform_int(u: np.ndarray, lo: int, hi: int) -> np.ndarray:
    """Map uint64 draws onto integers in [lo, hi] (inclusive) by modulo."""
    span = np.uint64(hi - lo + 1)
    return (u % span).astype(np.int64) + lo


def uniform_open01(u: np.ndarray) -> np.ndarray:
    """Map uint64 draws onto doubles in (0, 1]: ((u >> 11) + 1) * 2**-53."""
    return ((u >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


@dataclasses.dataclass(frozen=True)
class PairSpec:
    """Recipe for one synthetic pair (sizes, disparity field, noise)."""

    W: int
    H: int
    D: int
    n_rects: int
    d_lo: int
    d_hi: int
    background: int = 10
    ramp: Optional[Tuple[int, int]] = None  # (d at x=0, d at x=W-1)
    sigma: float = 2.0


@dataclasses.dataclass
class StereoPair:
    left: np.ndarray  # uint8 [H, W], base image
    right: np.ndarray  # uint8 [H, W], match image
    gt: np.ndarray  # int32 [H, W], disparity on left coordinates
    spec: PairSpec
    seed: int


def box3(img: np.ndarray) -> np.ndarray:
    """3x3 box filter with clamp-to-edge, rounded as (sum + 4) // 9."""
    p = np.pad(img.astype(np.int32), 1, mode="edge")
    H, W = img.shape
    s = np.zeros((H, W), dtype=np.int32)
    for dy in range(3):
        for dx in range(3):
            s += p[dy:dy + H, dx:dx + W]
    return ((s + 4) // 9).astype(np.uint8)


def disparity_field(spec: PairSpec, seed: int) -> np.ndarray:
    W, H = spec.W, spec.H
    if spec.ramp is not None:
        a, b = spec.ramp
        xs = np.arange(W, dtype=np.float64)
        row = np.floor(a + (b - a) * xs / max(W - 1, 1) + 0.5).astype(np.int32)
        gt = np.broadcast_to(row, (H, W)).copy()
    else:
        gt = np.full((H, W), spec.background, dtype=np.int32)
    u = stream_u64(seed, _S_RECT, 5 * spec.n_rects)
    for k in range(spec.n_rects):
        uw, uh, ux, uy, ud = (u[5 * k + i:5 * k + i + 1] for i in range(5))
        rw = int(uniform_int(uw, max(1, W // 10), max(1, W // 3))[0])
        rh = int(uniform_int(uh, max(1, H // 10), max(1, H // 3))[0])
        x0 = int(uniform_int(ux, 0, W - rw)[0])
        y0 = int(uniform_int(uy, 0, H - rh)[0])
        d = int(uniform_int(ud, spec.d_lo, spec.d_hi)[0])
        gt[y0:y0 + rh, x0:x0 + rw] = d
    return gt


def forward_warp(left: np.ndarray, gt: np.ndarray, fill: np.ndarray) -> np.ndarray:
    """right[y, x - d] = left[y, x]; larger d wins; holes take ``fill``."""
    H, W = left.shape
    ys, xs = np.mgrid[0:H, 0:W]
    xt = xs - gt
    ok = xt >= 0
    ys, xs, xt, d = ys[ok], xs[ok], xt[ok], gt[ok]
    # sort by target then by d, keep the last (largest d) per target
    tgt = ys.astype(np.int64) * W + xt
    order = np.lexsort((d, tgt))
    tgt_s = tgt[order]
    last = np.ones(tgt_s.size, dtype=bool)
    last[:-1] = tgt_s[1:] != tgt_s[:-1]
    sel = order[last]
    right = fill.reshape(-1).copy()
    right[tgt[sel]] = left[ys[sel], xs[sel]]
    return right.reshape(H, W)


def make_pair(spec: PairSpec, seed: int) -> StereoPair:
    W, H = spec.W, spec.H
    tex = uniform_int(stream_u64(seed, _S_TEXTURE, W * H), 0, 255).astype(np.uint8).reshape(H, W)
    left = box3(tex)
    gt = disparity_field(spec, seed)
    fill = uniform_int(stream_u64(seed, _S_FILL, W * H), 0, 255).astype(np.uint8).reshape(H, W)
    right = forward_warp(left, gt, fill).astype(np.int32)
    if spec.sigma > 0:
        u = stream_u64(seed, _S_NOISE, 2 * W * H)
        u1 = uniform_open01(u[0::2])
        u2 = uniform_open01(u[1::2])
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
        right = right + np.floor(spec.sigma * z + 0.5).astype(np.int32).reshape(H, W)
    right = np.clip(right, 0, 255).astype(np.uint8)
    return StereoPair(left=np.ascontiguousarray(left), right=np.ascontiguousarray(right), gt=gt, spec=spec, seed=seed)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One SGM invocation: a pair recipe plus the method's parameters."""

    name: str
    spec: PairSpec
    P1: int
    P2: int
    n_paths: int


# The three single-pair workloads: the small case, the paper's headline shape
# (640x480, D=128, 4 paths, Section 4) and a KITTI-like 1242x375 8-path case.
WORKLOADS = {
    "sgm_320x240_d64_p4": Workload("sgm_320x240_d64_p4", PairSpec(320, 240, 64, 6, 4, 48, background=10, sigma=2.0), 7, 84, 4),
    "sgm_640x480_d128_p4": Workload("sgm_640x480_d128_p4", PairSpec(640, 480, 128, 12, 2, 120, background=10, sigma=2.0), 7, 84, 4),
    "sgm_1242x375_d128_p8": Workload("sgm_1242x375_d128_p8", PairSpec(1242, 375, 128, 20, 5, 100, ramp=(5, 100), sigma=3.0), 10, 120, 8),
}
WORKLOAD_INDEX = {"sgm_320x240_d64_p4": 0, "sgm_640x480_d128_p4": 1, "sgm_1242x375_d128_p8": 2}

BATCH_SIZES = ((320, 240), (640, 480), (1242, 375), (1920, 1080))
BATCH_DS = (64, 128, 256)
BATCH_PATHS = (4, 8)


def workload_pair(name: str) -> StereoPair:
    return make_pair(WORKLOADS[name].spec, BASE_SEED + WORKLOAD_INDEX[name])


def batch_recipe(n: int = 64, config: int = 3, paths: Optional[Sequence[int]] = None,
                 sizes: Sequence[Tuple[int, int]] = BATCH_SIZES, Ds: Sequence[int] = BATCH_DS,
                 P1: int = 7, P2: int = 84) -> List[Workload]:
    """Uneven batch: size, D and path count drawn per pair with a seed."""
    paths = tuple(paths) if paths is not None else BATCH_PATHS
    u = stream_u64(BASE_SEED + 1000 * config, _S_META, 3 * n)
    out = []
    for i in range(n):
        W, H = sizes[int(u[3 * i] % np.uint64(len(sizes)))]
        D = Ds[int(u[3 * i + 1] % np.uint64(len(Ds)))]
        npaths = paths[int(u[3 * i + 2] % np.uint64(len(paths)))]
        spec = PairSpec(W, H, D, 6, 4, min(48, D - 1), background=10, sigma=2.0)
        out.append(Workload(f"pair{i}_{W}x{H}_d{D}_p{npaths}", spec, P1, P2, npaths))
    return out


def batch_pairs(recipe: Sequence[Workload], config: int = 3) -> List[StereoPair]:
    return [make_pair(w.spec, BASE_SEED + 1000 * config + i) for i, w in enumerate(recipe)]


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream: exponential gaps."""
    n_max = int(rate_hz * duration_s * 1.5) + 64
    gaps = -np.log(uniform_open01(stream_u64(seed, _S_META, n_max))) / rate_hz
    t = np.cumsum(gaps)
    return t[t < duration_s]

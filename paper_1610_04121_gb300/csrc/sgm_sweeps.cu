// Path aggregation (Eq. 3), the sum S and the winner-take-all disparity
// (Eq. 4) of the SGM path in arXiv 1610.04121, for sm_103a.
//
// Parallel scheme (Section 3.2, with the paper's CTA-to-warp conversion): one
// warp carries one path, disparities packed two per 32-bit register; the
// neighbours d-1 / d+1 cross lanes with shuffles and the step minimum m(q) is
// one redux.sync.  Opposite directions of an axis run at the same time and
// meet in the middle: each sweeps its first half of the path storing L_r (u8)
// in a scratch cube, and in its second half adds the other direction's stored
// L_r to its own.
//
// Each warp streams its inputs through a private shared-memory ring filled by
// cp.async a few chunks ahead, keeps its step loop on shared memory only, and
// writes each chunk's outputs back with 16-byte stores.
//
//   sweep_h : left-to-right and right-to-left, one row per warp pair;
//             writes S = L_LR + L_RL (packed u16x2).
//   sweep_v : top-to-bottom and bottom-to-top along columns (rx = 0) or along
//             the wrapped diagonals of Section 3.2 (rx = +1 / -1); either adds
//             its pair sum into S or, for the last axis, finishes with Eq. 4.
#include "sgm_device.cuh"
#include "sgm_internal.h"

namespace sgm {

// Per-warp shared-memory staging for K words per lane (DP = 64 K disparities).
template <int K>
struct Stage {
    static constexpr int DP = 64 * K;
    static constexpr int CH = (16 / K) >= 4 ? (16 / K) : 4;  // pixels per chunk
    static constexpr int NSLOT = 3;                          // chunks in flight + 1
    static constexpr int MC_RING = NSLOT * CH * DP;
    static constexpr int LO_RING = NSLOT * CH * DP;
    static constexpr int S_RING = NSLOT * CH * 2 * DP;
    static constexpr int OUT = CH * 2 * DP;
    static constexpr int BYTES = MC_RING + LO_RING + S_RING + OUT;
};

enum WalkMode {
    kStoreL = 0,    // phase 1 of a pair: store L_r
    kSumH = 1,      // phase 2 of the horizontal pair: S = L + stored L
    kAcc = 2,       // phase 2 of a diagonal pair: S += L + stored L
    kWta2 = 3,      // phase 2 of the vertical pair: raw = argmin_d (S + L + stored L)
    kSingleH = 4,   // 2-path mode, left-to-right: S = L
    kSingleWta = 5  // 2-path mode, top-to-bottom: raw = argmin_d (S + L)
};

// Pixels of a row walk: x = x0 + dx * i.
struct RowGeo {
    size_t rowbase;
    int x0, dx;
    static constexpr bool kResets = false;
    __device__ __forceinline__ size_t pix(int i) const { return rowbase + static_cast<size_t>(x0 + dx * i); }
};

// Pixels of a column / wrapped-diagonal walk: y = y0 + dy * i, x = (c + rx*y) mod W.
struct ColGeo {
    int W, H, c, rx, y0, dy;
    static constexpr bool kResets = true;
    __device__ __forceinline__ int x_at(int y) const {
        if (rx == 0) return c;
        int v = (c + rx * y) % W;
        return v < 0 ? v + W : v;
    }
    __device__ __forceinline__ size_t pix(int i) const {
        const int y = y0 + dy * i;
        return static_cast<size_t>(y) * W + x_at(y);
    }
    // the previous pixel of the path at (x, y) lies outside the image
    __device__ __forceinline__ bool starts(int y, int x) const {
        if (dy > 0) return y == 0 || (rx == 1 && x == 0) || (rx == -1 && x == W - 1);
        return y == H - 1 || (rx == 1 && x == W - 1) || (rx == -1 && x == 0);
    }
};

template <int K, int MODE, class Geo>
__device__ __forceinline__ void walk(Chain<K>& ch, const Geo& g, int n, const SweepArgs& a, uint8_t* ws, int lane) {
    using St = Stage<K>;
    constexpr int DP = St::DP, CH = St::CH, NS = St::NSLOT;
    constexpr bool IN_LO = MODE == kSumH || MODE == kAcc || MODE == kWta2;
    constexpr bool IN_S = MODE == kAcc || MODE == kWta2 || MODE == kSingleWta;
    constexpr bool OUT_LX = MODE == kStoreL;
    constexpr bool OUT_S = MODE == kSumH || MODE == kAcc || MODE == kSingleH;
    constexpr bool WTA = MODE == kWta2 || MODE == kSingleWta;
    constexpr int PM = DP / 16;      // 16-byte pieces per pixel of u8 pairs
    constexpr int PS = 2 * DP / 16;  // 16-byte pieces per pixel of packed sums
    uint8_t* mc_ring = ws;
    uint8_t* lo_ring = mc_ring + St::MC_RING;
    uint8_t* s_ring = lo_ring + St::LO_RING;
    uint8_t* out = s_ring + St::S_RING;
    const uint8_t* Sb = reinterpret_cast<const uint8_t*>(a.S);
    const int nch = (n + CH - 1) / CH;

    auto issue = [&](int c) {
        if (c < nch) {
            const int i0 = c * CH, np = min(CH, n - i0), slot = c % NS;
            for (int q = lane; q < np * PM; q += 32) {
                const int pi = q / PM, off = (q % PM) * 16;
                const size_t p = g.pix(i0 + pi);
                cp16(mc_ring + (slot * CH + pi) * DP + off, a.MC + p * DP + off);
                if (IN_LO) cp16(lo_ring + (slot * CH + pi) * DP + off, a.Lx + p * DP + off);
            }
            if (IN_S) {
                for (int q = lane; q < np * PS; q += 32) {
                    const int pi = q / PS, off = (q % PS) * 16;
                    const size_t p = g.pix(i0 + pi);
                    cp16(s_ring + (slot * CH + pi) * 2 * DP + off, Sb + p * 2 * DP + off);
                }
            }
        }
        cp_commit();
    };

    int y_body = 0, x_body = 0;
    if constexpr (Geo::kResets) {
        y_body = g.y0;
        x_body = g.x_at(g.y0);
    }
    for (int c = 0; c < NS - 1; ++c) issue(c);
    for (int c = 0; c < nch; ++c) {
        issue(c + NS - 1);
        cp_wait<NS - 1>();
        __syncwarp();
        const int i0 = c * CH, np = min(CH, n - i0), slot = c % NS;
#pragma unroll
        for (int pi = 0; pi < CH; ++pi) {
            if (pi < np) {
                if constexpr (Geo::kResets) {
                    if (g.starts(y_body, x_body)) ch.reset();
                }
                uint32_t mc[K], L[K];
                unpack_pairs<K>(ld_pairs<K>(mc_ring + (slot * CH + pi) * DP + lane * 2 * K), mc);
                ch.step(mc, a.P1x2, a.P2x2, L);
                if constexpr (OUT_LX) {
                    st_pairs<K>(out + pi * DP + lane * 2 * K, pack_pairs<K>(L));
                } else {
                    uint32_t s[K];
#pragma unroll
                    for (int j = 0; j < K; ++j) s[j] = L[j];
                    if constexpr (IN_LO) {
                        uint32_t lo[K];
                        unpack_pairs<K>(ld_pairs<K>(lo_ring + (slot * CH + pi) * DP + lane * 2 * K), lo);
#pragma unroll
                        for (int j = 0; j < K; ++j) s[j] += lo[j];
                    }
                    if constexpr (IN_S) {
                        uint32_t t[K];
                        ld_words<K>(reinterpret_cast<const uint32_t*>(s_ring + (slot * CH + pi) * 2 * DP) + lane * K, t);
#pragma unroll
                        for (int j = 0; j < K; ++j) s[j] += t[j];
                    }
                    if constexpr (OUT_S) st_words<K>(reinterpret_cast<uint32_t*>(out + pi * 2 * DP) + lane * K, s);
                    if constexpr (WTA) {
                        uint32_t key = wta_key<K>(s, lane, DP / 2, a.D);
                        key = redux_min(key, 0xffffffffu);
                        const size_t p = g.pix(i0 + pi);
                        if (lane == 0) a.raw[p] = static_cast<uint8_t>(key & 0xffu);
                        if (a.Sdbg) {
#pragma unroll
                            for (int j = 0; j < K; ++j) {
                                const int i = lane * K + j;
                                if (i < a.D) a.Sdbg[p * a.D + i] = static_cast<uint16_t>(s[j] & 0xffffu);
                                if (i + DP / 2 < a.D) a.Sdbg[p * a.D + i + DP / 2] = static_cast<uint16_t>(s[j] >> 16);
                            }
                        }
                    }
                }
                if constexpr (Geo::kResets) {
                    y_body += g.dy;
                    x_body += g.rx * g.dy;
                    x_body = x_body >= g.W ? x_body - g.W : (x_body < 0 ? x_body + g.W : x_body);
                }
            }
        }
        __syncwarp();
        if constexpr (OUT_LX || OUT_S) {
            constexpr int P = OUT_LX ? PM : PS;
            constexpr int BPP = OUT_LX ? DP : 2 * DP;  // bytes per pixel
            uint8_t* dst = OUT_LX ? a.Lx : reinterpret_cast<uint8_t*>(a.S);
            for (int q = lane; q < np * P; q += 32) {
                const int pi = q / P, off = (q % P) * 16;
                const size_t p = g.pix(i0 + pi);
                *reinterpret_cast<uint4*>(dst + p * BPP + off) = *reinterpret_cast<const uint4*>(out + pi * BPP + off);
            }
            __syncwarp();
        }
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// Horizontal axis.  Block = 2 rows x 2 warps; warp 2r walks row r left to
// right, warp 2r+1 right to left.  Phase 1: LR covers x < W/2 and RL covers
// x >= W/2, both storing L in Lx.  Phase 2: each covers the other half and
// writes S = own L + stored L.  Without `pair` (2-path mode) LR covers the
// whole row and writes S = L_LR.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(128) sweep_h_kernel(SweepArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y = blockIdx.x * 2 + (warp >> 1);
    const bool rev = (warp & 1) != 0;
    const bool active = (y < a.H) && (!rev || a.pair);
    uint8_t* ws = smem + warp * Stage<K>::BYTES;
    const int W = a.W;
    const int Wm = a.pair ? W / 2 : W;
    const size_t rowbase = static_cast<size_t>(y < a.H ? y : 0) * W;
    Chain<K> ch;
    ch.init(lane);
    if (active) {
        const RowGeo g{rowbase, rev ? W - 1 : 0, rev ? -1 : 1};
        const int n1 = rev ? (W - Wm) : Wm;
        if (a.pair)
            walk<K, kStoreL>(ch, g, n1, a, ws, lane);
        else
            walk<K, kSingleH>(ch, g, n1, a, ws, lane);
    }
    if (!a.pair) return;  // uniform over the launch
    __syncthreads();
    if (active) {
        const RowGeo g{rowbase, rev ? Wm - 1 : Wm, rev ? -1 : 1};
        const int n2 = rev ? Wm : (W - Wm);
        walk<K, kSumH>(ch, g, n2, a, ws, lane);
    }
}

// ---------------------------------------------------------------------------
// Vertical-type axis.  Block = 2 chains x 2 warps; warp 2c walks chain c
// downward (rows 0 .. H-1), warp 2c+1 upward.  Chain c visits pixel
// x(y) = (c + rx*y) mod W in row y: a column for rx = 0, and for rx = +1/-1 a
// diagonal that wraps to the other border, restarting its path there
// (Section 3.2).  Phase 1: down covers y < H/2, up covers y >= H/2, storing L.
// Phase 2: each covers the other half and combines its L with the stored L
// and S: S += both (wta = 0) or raw = argmin_d (S + both) (wta = 1).
// Without `pair` the downward warp covers all rows (2-path mode, wta = 1).
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(128) sweep_v_kernel(SweepArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 2 + (warp >> 1);
    const bool upward = (warp & 1) != 0;
    const bool active = (c < a.W) && (!upward || a.pair);
    uint8_t* ws = smem + warp * Stage<K>::BYTES;
    const int H = a.H;
    const int Hm = a.pair ? H / 2 : H;
    Chain<K> ch;
    ch.init(lane);
    if (active) {
        const ColGeo g{a.W, H, c, a.rx, upward ? H - 1 : 0, upward ? -1 : 1};
        const int n1 = upward ? (H - Hm) : Hm;
        if (a.pair)
            walk<K, kStoreL>(ch, g, n1, a, ws, lane);
        else
            walk<K, kSingleWta>(ch, g, n1, a, ws, lane);
    }
    if (!a.pair) return;  // uniform over the launch
    __syncthreads();
    if (active) {
        const ColGeo g{a.W, H, c, a.rx, upward ? Hm - 1 : Hm, upward ? -1 : 1};
        const int n2 = upward ? Hm : (H - Hm);
        if (a.wta)
            walk<K, kWta2>(ch, g, n2, a, ws, lane);
        else
            walk<K, kAcc>(ch, g, n2, a, ws, lane);
    }
}

template <int K>
static cudaError_t set_attrs_t() {
    constexpr int smem = 4 * Stage<K>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(sweep_h_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_v_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t init_kernel_attributes() {
    cudaError_t e;
    if ((e = set_attrs_t<1>()) != cudaSuccess) return e;
    if ((e = set_attrs_t<2>()) != cudaSuccess) return e;
    if ((e = set_attrs_t<3>()) != cudaSuccess) return e;
    return set_attrs_t<4>();
}

template <int K>
static cudaError_t launch_h_t(const SweepArgs& a, cudaStream_t stream) {
    sweep_h_kernel<K><<<(a.H + 1) / 2, 128, 4 * Stage<K>::BYTES, stream>>>(a);
    return cudaGetLastError();
}

template <int K>
static cudaError_t launch_v_t(const SweepArgs& a, cudaStream_t stream) {
    sweep_v_kernel<K><<<(a.W + 1) / 2, 128, 4 * Stage<K>::BYTES, stream>>>(a);
    return cudaGetLastError();
}

// K words per lane: DP = 64 K disparities (D rounded up to a multiple of 64).
#define SGM_DISPATCH_K(FN, a, s)               \
    switch (padded_D((a).D) / 64) {            \
        case 1: return FN<1>(a, s);            \
        case 2: return FN<2>(a, s);            \
        case 3: return FN<3>(a, s);            \
        case 4: return FN<4>(a, s);            \
        default: return cudaErrorInvalidValue; \
    }

cudaError_t launch_sweep_h(const SweepArgs& a, cudaStream_t stream) { SGM_DISPATCH_K(launch_h_t, a, stream) }

cudaError_t launch_sweep_v(const SweepArgs& a, cudaStream_t stream) { SGM_DISPATCH_K(launch_v_t, a, stream) }

}  // namespace sgm

// Path aggregation (Eq. 3), the sum S and the winner-take-all disparity
// (Eq. 4) of the SGM path in arXiv 1610.04121, for sm_103a.
//
// Parallel scheme (Section 3.2, with the paper's CTA-to-warp conversion taken
// one step further): one group of G lanes (a warp or a half-warp) carries one
// path, disparities packed two per 32-bit register; neighbours d-1 / d+1 cross
// lanes with shuffles and the step minimum m(q) is one redux.sync.  Opposite
// directions of an axis run at the same time and meet in the middle: each
// sweeps its first half of the path storing L_r (u8) in a scratch cube, and
// in its second half adds the other direction's stored L_r to its own.
//
//   sweep_h : left-to-right and right-to-left, one row per group pair;
//             writes S = L_LR + L_RL (packed u16x2).
//   sweep_v : top-to-bottom and bottom-to-top along columns (rx = 0) or along
//             the wrapped diagonals of Section 3.2 (rx = +1 / -1); either adds
//             its pair sum into S or, for the last axis, finishes with Eq. 4.
#include "sgm_device.cuh"
#include "sgm_internal.h"

namespace sgm {

constexpr int kPF = 8;  // loads issued this many steps ahead

template <int K>
struct Item2 {
    U8Pairs<K> mc;
    U8Pairs<K> lo;
};

template <int K>
struct Item3 {
    U8Pairs<K> mc;
    U8Pairs<K> lo;
    uint32_t s[K];
};

template <int K>
struct Item1s {
    U8Pairs<K> mc;
    uint32_t s[K];
};

// ---------------------------------------------------------------------------
// Horizontal axis.  Block = ROWS rows x 2 groups; group 2r walks row r left to
// right, group 2r+1 right to left.  Phase 1: LR covers x < W/2 and RL covers
// x >= W/2, both storing L in Lx.  Phase 2: each covers the other half and
// writes S = own L + stored L.  Without `pair` (2-path mode) LR covers the
// whole row and writes S = L_LR.
// ---------------------------------------------------------------------------
template <int G, int K, int ROWS>
__global__ void __launch_bounds__(ROWS * 2 * G) sweep_h_kernel(SweepArgs a) {
    const int tid = threadIdx.x;
    const int grp = tid / G, lane = tid % G;
    const uint32_t gmask = group_mask<G>(tid & 31);
    const int y = blockIdx.x * ROWS + grp / 2;
    const bool rev = (grp & 1) != 0;
    const bool active = (y < a.H) && (!rev || a.pair);
    const int W = a.W, D = a.D, half = D / 2;
    const int Wm = a.pair ? W / 2 : W;
    const size_t rowpix = static_cast<size_t>(y < a.H ? y : 0) * W;
    const uint8_t* mcrow = a.MC + rowpix * D + lane * 2 * K;
    uint8_t* lxrow = a.Lx + rowpix * D + lane * 2 * K;
    uint32_t* srow = a.S + rowpix * half + lane * K;

    Chain<G, K> ch;
    ch.reset();
    uint32_t L[K];
    if (active) {
        const int n1 = rev ? (W - Wm) : Wm;
        pipelined<kPF, U8Pairs<K>>(
            n1,
            [&](int i) {
                const int x = rev ? W - 1 - i : i;
                return ld_pairs<K>(mcrow + static_cast<size_t>(x) * D);
            },
            [&](int i, const U8Pairs<K>& b) {
                const int x = rev ? W - 1 - i : i;
                uint32_t mc[K];
                unpack_pairs<K>(b, mc);
                ch.step(mc, a.P1x2, a.P2x2, lane, gmask, L);
                if (a.pair)
                    st_pairs<K>(lxrow + static_cast<size_t>(x) * D, pack_pairs<K>(L));
                else
                    st_words<K>(srow + static_cast<size_t>(x) * half, L);
            });
    }
    if (!a.pair) return;  // uniform over the launch
    __syncthreads();
    if (active) {
        const int n2 = rev ? Wm : (W - Wm);
        pipelined<kPF, Item2<K>>(
            n2,
            [&](int i) {
                const int x = rev ? Wm - 1 - i : Wm + i;
                Item2<K> it;
                it.mc = ld_pairs<K>(mcrow + static_cast<size_t>(x) * D);
                it.lo = ld_pairs<K>(lxrow + static_cast<size_t>(x) * D);
                return it;
            },
            [&](int i, const Item2<K>& it) {
                const int x = rev ? Wm - 1 - i : Wm + i;
                uint32_t mc[K], lo[K];
                unpack_pairs<K>(it.mc, mc);
                ch.step(mc, a.P1x2, a.P2x2, lane, gmask, L);
                unpack_pairs<K>(it.lo, lo);
#pragma unroll
                for (int j = 0; j < K; ++j) L[j] += lo[j];
                st_words<K>(srow + static_cast<size_t>(x) * half, L);
            });
    }
}

// ---------------------------------------------------------------------------
// Vertical-type axis.  Block = CH chains x 2 groups; group 2c walks chain c
// downward (rows 0 .. H-1), group 2c+1 upward.  Chain c visits pixel
// x(y) = (c + rx*y) mod W in row y: a column for rx = 0, and for rx = +1/-1 a
// diagonal that wraps to the other border, restarting its path there
// (Section 3.2).  Phase 1: down covers y < H/2, up covers y >= H/2, storing L.
// Phase 2: each covers the other half and combines its L with the stored L
// and S: S += both (wta = 0) or raw = argmin_d (S + both) (wta = 1).
// Without `pair` the downward group covers all rows (2-path mode).
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ int wrap_x(int x, int W) {
    return x >= W ? x - W : (x < 0 ? x + W : x);
}

template <int G, int K, int CH>
__global__ void __launch_bounds__(CH * 2 * G) sweep_v_kernel(SweepArgs a) {
    const int tid = threadIdx.x;
    const int grp = tid / G, lane = tid % G;
    const uint32_t gmask = group_mask<G>(tid & 31);
    const int c = blockIdx.x * CH + grp / 2;
    const bool upward = (grp & 1) != 0;
    const bool active = (c < a.W) && (!upward || a.pair);
    const int W = a.W, H = a.H, D = a.D, half = D / 2, rx = a.rx;
    const int Hm = a.pair ? H / 2 : H;
    const uint8_t* mcb = a.MC + lane * 2 * K;
    uint8_t* lxb = a.Lx + lane * 2 * K;
    uint32_t* sb = a.S + lane * K;
    const int step_dir = upward ? -1 : 1;

    // x of the chain in row y, (c + rx*y) mod W
    auto x_at = [&](int y) {
        long long v = static_cast<long long>(c) + static_cast<long long>(rx) * y;
        v %= W;
        if (v < 0) v += W;
        return static_cast<int>(v);
    };
    // first pixel of the path in this direction: the previous pixel is outside
    auto starts = [&](int y, int x) {
        if (!upward) return y == 0 || (rx == 1 && x == 0) || (rx == -1 && x == W - 1);
        return y == H - 1 || (rx == 1 && x == W - 1) || (rx == -1 && x == 0);
    };

    auto finish = [&](int y, int x, uint32_t (&s)[K]) {
        const size_t p = static_cast<size_t>(y) * W + x;
        if (a.wta) {
            uint32_t key = wta_key<K>(s, lane, half);
            key = redux_min(key, gmask);
            if (lane == 0) a.raw[p] = static_cast<uint8_t>(key & 0xffu);
            if (a.Sdbg) {
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const int i = lane * K + j;
                    a.Sdbg[p * D + i] = static_cast<uint16_t>(s[j] & 0xffffu);
                    a.Sdbg[p * D + i + half] = static_cast<uint16_t>(s[j] >> 16);
                }
            }
        } else {
            st_words<K>(sb + p * half, s);
        }
    };

    Chain<G, K> ch;
    ch.reset();
    uint32_t L[K];
    if (active) {
        const int y0 = upward ? H - 1 : 0;
        const int n1 = upward ? (H - Hm) : Hm;
        // incremental x for the loader and the body (each called in order)
        int xl = x_at(y0), xb = xl;
        if (a.pair) {
            pipelined<kPF, U8Pairs<K>>(
                n1,
                [&](int i) {
                    const int y = y0 + step_dir * i;
                    U8Pairs<K> v = ld_pairs<K>(mcb + (static_cast<size_t>(y) * W + xl) * D);
                    xl = wrap_x<K>(xl + step_dir * rx, W);
                    return v;
                },
                [&](int i, const U8Pairs<K>& b) {
                    const int y = y0 + step_dir * i;
                    const int x = xb;
                    xb = wrap_x<K>(xb + step_dir * rx, W);
                    if (starts(y, x)) ch.reset();
                    uint32_t mc[K];
                    unpack_pairs<K>(b, mc);
                    ch.step(mc, a.P1x2, a.P2x2, lane, gmask, L);
                    st_pairs<K>(lxb + (static_cast<size_t>(y) * W + x) * D, pack_pairs<K>(L));
                });
        } else {
            pipelined<kPF, Item1s<K>>(
                n1,
                [&](int i) {
                    const int y = y0 + step_dir * i;
                    const size_t p = static_cast<size_t>(y) * W + xl;
                    Item1s<K> v;
                    v.mc = ld_pairs<K>(mcb + p * D);
                    ld_words<K>(sb + p * half, v.s);
                    xl = wrap_x<K>(xl + step_dir * rx, W);
                    return v;
                },
                [&](int i, const Item1s<K>& it) {
                    const int y = y0 + step_dir * i;
                    const int x = xb;
                    xb = wrap_x<K>(xb + step_dir * rx, W);
                    if (starts(y, x)) ch.reset();
                    uint32_t mc[K];
                    unpack_pairs<K>(it.mc, mc);
                    ch.step(mc, a.P1x2, a.P2x2, lane, gmask, L);
                    uint32_t s[K];
#pragma unroll
                    for (int j = 0; j < K; ++j) s[j] = it.s[j] + L[j];
                    finish(y, x, s);
                });
        }
    }
    if (!a.pair) return;  // uniform over the launch
    __syncthreads();
    if (active) {
        const int y0 = upward ? Hm - 1 : Hm;
        const int n2 = upward ? Hm : (H - Hm);
        int xl = x_at(y0), xb = xl;
        pipelined<kPF, Item3<K>>(
            n2,
            [&](int i) {
                const int y = y0 + step_dir * i;
                const size_t p = static_cast<size_t>(y) * W + xl;
                Item3<K> v;
                v.mc = ld_pairs<K>(mcb + p * D);
                v.lo = ld_pairs<K>(lxb + p * D);
                ld_words<K>(sb + p * half, v.s);
                xl = wrap_x<K>(xl + step_dir * rx, W);
                return v;
            },
            [&](int i, const Item3<K>& it) {
                const int y = y0 + step_dir * i;
                const int x = xb;
                xb = wrap_x<K>(xb + step_dir * rx, W);
                if (starts(y, x)) ch.reset();
                uint32_t mc[K], lo[K];
                unpack_pairs<K>(it.mc, mc);
                ch.step(mc, a.P1x2, a.P2x2, lane, gmask, L);
                unpack_pairs<K>(it.lo, lo);
                uint32_t s[K];
#pragma unroll
                for (int j = 0; j < K; ++j) s[j] = it.s[j] + L[j] + lo[j];
                finish(y, x, s);
            });
    }
}

template <int G, int K>
static cudaError_t launch_h_t(const SweepArgs& a, cudaStream_t stream) {
    constexpr int ROWS = (G == 32) ? 2 : 4;
    dim3 grid((a.H + ROWS - 1) / ROWS);
    sweep_h_kernel<G, K, ROWS><<<grid, ROWS * 2 * G, 0, stream>>>(a);
    return cudaGetLastError();
}

template <int G, int K>
static cudaError_t launch_v_t(const SweepArgs& a, cudaStream_t stream) {
    constexpr int CH = (G == 32) ? 2 : 4;
    dim3 grid((a.W + CH - 1) / CH);
    sweep_v_kernel<G, K, CH><<<grid, CH * 2 * G, 0, stream>>>(a);
    return cudaGetLastError();
}

// Lane layout per D: G lanes x K words = D/2 words.
#define SGM_DISPATCH_D(FN, a, s)                    \
    switch ((a).D) {                                \
        case 32: return FN<16, 1>(a, s);            \
        case 64: return FN<32, 1>(a, s);            \
        case 96: return FN<16, 3>(a, s);            \
        case 128: return FN<32, 2>(a, s);           \
        case 160: return FN<16, 5>(a, s);           \
        case 192: return FN<32, 3>(a, s);           \
        case 224: return FN<16, 7>(a, s);           \
        case 256: return FN<32, 4>(a, s);           \
        default: return cudaErrorInvalidValue;      \
    }

cudaError_t launch_sweep_h(const SweepArgs& a, cudaStream_t stream) { SGM_DISPATCH_D(launch_h_t, a, stream) }

cudaError_t launch_sweep_v(const SweepArgs& a, cudaStream_t stream) { SGM_DISPATCH_D(launch_v_t, a, stream) }

}  // namespace sgm

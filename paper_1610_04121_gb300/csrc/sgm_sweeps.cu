// Path aggregation (Eq. 3), the sum S and the winner-take-all disparity
// (Eq. 4) of the SGM path in arXiv 1610.04121, for sm_103a.
//
// Parallel scheme (Section 3.2, with the paper's CTA-to-warp conversion): one
// warp carries the two opposite paths of one row or one column, each spread
// over all 32 lanes with disparities packed two per 32-bit register, and the
// two paths' steps interleaved in one instruction stream so that one path's
// latencies are covered by the other's work.  The two paths meet in the
// middle: each sweeps its first half of the line storing L_r (u8) in a
// scratch cube, and in its second half adds the other path's stored L_r to its
// own.  The exchange between the two halves of the line is warp-local, so no
// block barrier is involved.
//
// Each path streams its inputs through a private shared-memory ring filled by
// cp.async a few chunks ahead, keeps its step loop on shared memory only, and
// writes each chunk's outputs back with 16-byte stores.
//
//   sweep_h : left-to-right with right-to-left, one row per warp;
//             writes S = L_LR + L_RL (packed u16x2).
//   sweep_v : top-to-bottom with bottom-to-top along columns (RX = 0) or along
//             the wrapped diagonals of Section 3.2 (RX = +1 / -1); either adds
//             its pair sum into S or, for the last axis, finishes with Eq. 4.
#include "sgm_device.cuh"
#include "sgm_internal.h"

namespace sgm {

constexpr int kWarpsPerBlock = 4;

// Shared-memory staging of one path with K words per lane (DP = 64 K).
template <int K>
struct Stage {
    static constexpr int DP = 64 * K;
    static constexpr int CH = 1024 / DP < 16 ? 1024 / DP : 16;  // pixels per chunk
    static constexpr int NSLOT = 3;                             // chunks in flight + 1
    static constexpr int MC_RING = NSLOT * CH * DP;
    static constexpr int LO_RING = NSLOT * CH * DP;
    static constexpr int S_RING = NSLOT * CH * 2 * DP;
    static constexpr int OUT = CH * 2 * DP;
    static constexpr int BYTES = MC_RING + LO_RING + S_RING + OUT;
    static constexpr int BLOCK_BYTES = 2 * kWarpsPerBlock * BYTES;
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
    __device__ __forceinline__ void origin(int i0, int& xc, int& yc) const {
        xc = x0 + dx * i0;
        yc = 0;
    }
    __device__ __forceinline__ size_t pix(int xc, int /*yc*/, int k) const {
        return rowbase + static_cast<size_t>(xc + dx * k);
    }
};

// Pixels of a column (RX = 0) or wrapped-diagonal (RX = +1/-1) walk:
// y = y0 + dy * i, x = (c + RX * y) mod W.
template <int RX>
struct ColGeo {
    int W, H, c, y0, dy;
    static constexpr bool kResets = RX != 0;
    __device__ __forceinline__ int x_at(int y) const {
        if constexpr (RX == 0) {
            return c;
        } else {
            int v = (c + RX * y) % W;
            return v < 0 ? v + W : v;
        }
    }
    __device__ __forceinline__ void origin(int i0, int& xc, int& yc) const {
        yc = y0 + dy * i0;
        xc = x_at(yc);
    }
    __device__ __forceinline__ size_t pix(int xc, int yc, int k) const {
        int x = xc;
        if constexpr (RX != 0) {
            x = xc + RX * dy * k;
            if (x >= W) x -= W;
            if (x < 0) x += W;
            if (x >= W || x < 0) {  // only when W is smaller than a chunk
                x %= W;
                if (x < 0) x += W;
            }
        }
        return static_cast<size_t>(yc + dy * k) * W + x;
    }
    // x of the next pixel of the walk
    __device__ __forceinline__ int step_x(int x) const {
        x += RX * dy;
        return x >= W ? x - W : (x < 0 ? x + W : x);
    }
    // the previous pixel of the path at (x, y) lies outside the image
    __device__ __forceinline__ bool starts(int y, int x) const {
        if (dy > 0) return y == 0 || (RX == 1 && x == 0) || (RX == -1 && x == W - 1);
        return y == H - 1 || (RX == 1 && x == W - 1) || (RX == -1 && x == 0);
    }
};

// The I/O of one path during one phase: staging ring, cursor for resets.
template <int K, int MODE, class Geo>
struct PathIO {
    using St = Stage<K>;
    static constexpr int DP = St::DP, CH = St::CH, NS = St::NSLOT;
    static constexpr bool IN_LO = MODE == kSumH || MODE == kAcc || MODE == kWta2;
    static constexpr bool IN_S = MODE == kAcc || MODE == kWta2 || MODE == kSingleWta;
    static constexpr bool OUT_LX = MODE == kStoreL;
    static constexpr bool OUT_S = MODE == kSumH || MODE == kAcc || MODE == kSingleH;
    static constexpr bool WTA = MODE == kWta2 || MODE == kSingleWta;
    static constexpr int PM = DP / 16;      // 16-byte pieces per pixel of u8 pairs
    static constexpr int PS = 2 * DP / 16;  // 16-byte pieces per pixel of packed sums

    Geo g;
    int n;
    uint8_t *mc_ring, *lo_ring, *s_ring, *out;
    int yb, xb;        // pixel of the next step (resetting walks only)
    int xc, yc, np;    // current chunk: origin and pixel count
    uint32_t dkeep;    // lane k keeps the disparity key of step k of the chunk

    __device__ __forceinline__ void init(const Geo& g_, int n_, uint8_t* ws) {
        g = g_;
        n = n_;
        mc_ring = ws;
        lo_ring = mc_ring + St::MC_RING;
        s_ring = lo_ring + St::LO_RING;
        out = s_ring + St::S_RING;
        yb = xb = 0;
        if constexpr (Geo::kResets) g.origin(0, xb, yb);
    }

    __device__ __forceinline__ void issue(const SweepArgs& a, int c, int lane) {
        const int i0 = c * CH, np_c = max(0, min(CH, n - i0)), slot = c % NS;
        if (np_c == 0) return;
        int x0, y0;
        g.origin(i0, x0, y0);
        for (int q = lane; q < np_c * PM; q += 32) {
            const int pi = q / PM, off = (q % PM) * 16;
            const size_t p = g.pix(x0, y0, pi);
            cp16(mc_ring + (slot * CH + pi) * DP + off, a.MC + p * DP + off);
            if constexpr (IN_LO) cp16(lo_ring + (slot * CH + pi) * DP + off, a.Lx + p * DP + off);
        }
        if constexpr (IN_S) {
            const uint8_t* Sb = reinterpret_cast<const uint8_t*>(a.S);
            for (int q = lane; q < np_c * PS; q += 32) {
                const int pi = q / PS, off = (q % PS) * 16;
                const size_t p = g.pix(x0, y0, pi);
                cp16(s_ring + (slot * CH + pi) * 2 * DP + off, Sb + p * 2 * DP + off);
            }
        }
    }

    __device__ __forceinline__ void begin_chunk(int c) {
        const int i0 = c * CH;
        np = max(0, min(CH, n - i0));
        xc = yc = 0;
        if (np > 0) g.origin(i0, xc, yc);
        dkeep = 0;
    }

    // one step at chunk position pi of this path
    __device__ __forceinline__ void step(Chain<K>& ch, const LaneConsts& lc, const SweepArgs& a, int slot, int pi,
                                         const uint32_t (&dconst)[K], int lane) {
        if constexpr (Geo::kResets) {
            if (g.starts(yb, xb)) ch.reset();
            yb += g.dy;
            xb = g.step_x(xb);
        }
        uint32_t mc[K], L[K];
        unpack_pairs<K>(ld_pairs<K>(mc_ring + (slot * CH + pi) * DP + lane * 2 * K), mc);
        ch.step(lc, mc, a.P1x2, a.P2x2, L);
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
                const uint32_t key = redux_min(wta_key<K>(s, dconst));
                dkeep = (lane == pi) ? key : dkeep;
                if (a.Sdbg) {  // debug: natural-order S of the real disparities
                    const size_t p = g.pix(xc, yc, pi);
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        const int i = lane * K + j;
                        if (i < a.D) a.Sdbg[p * a.D + i] = static_cast<uint16_t>(s[j] & 0xffffu);
                        if (i + DP / 2 < a.D) a.Sdbg[p * a.D + i + DP / 2] = static_cast<uint16_t>(s[j] >> 16);
                    }
                }
            }
        }
    }

    // after the chunk's steps (and a __syncwarp): disparities and staged outputs to HBM
    __device__ __forceinline__ void finish_chunk(const SweepArgs& a, int lane) {
        if constexpr (WTA) {
            if (lane < np) a.raw[g.pix(xc, yc, lane)] = static_cast<uint8_t>(dkeep & 0xffu);
        }
        if constexpr (OUT_LX || OUT_S) {
            constexpr int P = OUT_LX ? PM : PS;
            constexpr int BPP = OUT_LX ? DP : 2 * DP;  // bytes per pixel
            uint8_t* dst = OUT_LX ? a.Lx : reinterpret_cast<uint8_t*>(a.S);
            for (int q = lane; q < np * P; q += 32) {
                const int pi = q / P, off = (q % P) * 16;
                const size_t p = g.pix(xc, yc, pi);
                *reinterpret_cast<uint4*>(dst + p * BPP + off) = *reinterpret_cast<const uint4*>(out + pi * BPP + off);
            }
        }
    }
};

// One phase of the two paths of a warp (A: nA steps, B: nB steps).
template <int K, int MODE, class Geo>
__device__ __forceinline__ void walk(Chain<K>& cA, Chain<K>& cB, const Geo& gA, const Geo& gB, int nA, int nB,
                                     const SweepArgs& a, uint8_t* wsA, uint8_t* wsB, const LaneConsts& lc,
                                     int lane) {
    using IO = PathIO<K, MODE, Geo>;
    constexpr int CH = IO::CH, NS = IO::NS;
    IO A, B;
    A.init(gA, nA, wsA);
    B.init(gB, nB, wsB);
    uint32_t dconst[K];
    if constexpr (IO::WTA) wta_consts<K>(lane, a.D, dconst);
    const int nmin = min(nA, nB), nmax = max(nA, nB);
    const int nch = (nmax + CH - 1) / CH;
    for (int c = 0; c < NS - 1; ++c) {
        if (c < nch) {
            A.issue(a, c, lane);
            B.issue(a, c, lane);
        }
        cp_commit();
    }
    for (int c = 0; c < nch; ++c) {
        if (c + NS - 1 < nch) {
            A.issue(a, c + NS - 1, lane);
            B.issue(a, c + NS - 1, lane);
        }
        cp_commit();
        cp_wait<NS - 1>();
        __syncwarp();
        const int slot = c % NS;
        A.begin_chunk(c);
        B.begin_chunk(c);
        if (nmin - c * CH >= CH) {
#pragma unroll
            for (int pi = 0; pi < CH; ++pi) {
                A.step(cA, lc, a, slot, pi, dconst, lane);
                B.step(cB, lc, a, slot, pi, dconst, lane);
            }
        } else {
#pragma unroll
            for (int pi = 0; pi < CH; ++pi) {
                if (pi < A.np) A.step(cA, lc, a, slot, pi, dconst, lane);
                if (pi < B.np) B.step(cB, lc, a, slot, pi, dconst, lane);
            }
        }
        __syncwarp();
        A.finish_chunk(a, lane);
        B.finish_chunk(a, lane);
        __syncwarp();
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// Horizontal axis: one row per warp; path A walks left to right, path B right
// to left.  Phase 1: A covers x < W/2, B covers x >= W/2, both storing L in
// Lx.  Phase 2: each covers the other half and writes S = own L + stored L.
// Without `pair` (2-path mode) A covers the whole row and writes S = L_LR.
// ---------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_h_kernel(SweepArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y = blockIdx.x * kWarpsPerBlock + warp;
    if (y >= a.H) return;  // whole warp: every exchange below is warp-local
    uint8_t* wsA = smem + (2 * warp) * Stage<K>::BYTES;
    uint8_t* wsB = wsA + Stage<K>::BYTES;
    const int W = a.W;
    const size_t rowbase = static_cast<size_t>(y) * W;
    LaneConsts lc;
    lc.init(lane);
    Chain<K> cA, cB;
    cA.reset();
    cB.reset();
    if (!a.pair) {
        walk<K, kSingleH>(cA, cB, RowGeo{rowbase, 0, 1}, RowGeo{rowbase, 0, 1}, W, 0, a, wsA, wsB, lc, lane);
        return;
    }
    const int Wm = W / 2;
    walk<K, kStoreL>(cA, cB, RowGeo{rowbase, 0, 1}, RowGeo{rowbase, W - 1, -1}, Wm, W - Wm, a, wsA, wsB, lc, lane);
    __threadfence_block();  // each path's L stores before the other path reads them
    __syncwarp();
    walk<K, kSumH>(cA, cB, RowGeo{rowbase, Wm, 1}, RowGeo{rowbase, Wm - 1, -1}, W - Wm, Wm, a, wsA, wsB, lc, lane);
}

// ---------------------------------------------------------------------------
// Vertical-type axis: one line per warp; path A walks down (rows 0 .. H-1),
// path B up.  Line c visits pixel x(y) = (c + RX*y) mod W in row y: a column
// for RX = 0, and for RX = +1/-1 a diagonal that wraps to the other border,
// restarting its path there (Section 3.2).  Phase 1: A covers y < H/2, B
// covers y >= H/2, storing L.  Phase 2: each covers the other half and
// combines its L with the stored L and S: S += both (wta = 0) or
// raw = argmin_d (S + both) (wta = 1).  Without `pair` path A covers all rows
// (2-path mode, wta = 1).
// ---------------------------------------------------------------------------
template <int K, int RX>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_v_kernel(SweepArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * kWarpsPerBlock + warp;
    if (c >= a.W) return;  // whole warp
    uint8_t* wsA = smem + (2 * warp) * Stage<K>::BYTES;
    uint8_t* wsB = wsA + Stage<K>::BYTES;
    const int W = a.W, H = a.H;
    LaneConsts lc;
    lc.init(lane);
    Chain<K> cA, cB;
    cA.reset();
    cB.reset();
    using G = ColGeo<RX>;
    if (!a.pair) {
        walk<K, kSingleWta>(cA, cB, G{W, H, c, 0, 1}, G{W, H, c, 0, 1}, H, 0, a, wsA, wsB, lc, lane);
        return;
    }
    const int Hm = H / 2;
    walk<K, kStoreL>(cA, cB, G{W, H, c, 0, 1}, G{W, H, c, H - 1, -1}, Hm, H - Hm, a, wsA, wsB, lc, lane);
    __threadfence_block();
    __syncwarp();
    if (a.wta)
        walk<K, kWta2>(cA, cB, G{W, H, c, Hm, 1}, G{W, H, c, Hm - 1, -1}, H - Hm, Hm, a, wsA, wsB, lc, lane);
    else
        walk<K, kAcc>(cA, cB, G{W, H, c, Hm, 1}, G{W, H, c, Hm - 1, -1}, H - Hm, Hm, a, wsA, wsB, lc, lane);
}

template <int K>
static cudaError_t set_attrs_t() {
    constexpr int smem = Stage<K>::BLOCK_BYTES;
    cudaError_t e = cudaFuncSetAttribute(sweep_h_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_v_kernel<K, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_v_kernel<K, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_v_kernel<K, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

cudaError_t init_kernel_attributes() {
    cudaError_t e = set_attrs_t<1>();
    if (e == cudaSuccess) e = set_attrs_t<2>();
    if (e == cudaSuccess) e = set_attrs_t<3>();
    if (e == cudaSuccess) e = set_attrs_t<4>();
    return e;
}

template <int K>
static cudaError_t launch_h_t(const SweepArgs& a, cudaStream_t stream) {
    sweep_h_kernel<K><<<(a.H + kWarpsPerBlock - 1) / kWarpsPerBlock, 32 * kWarpsPerBlock, Stage<K>::BLOCK_BYTES,
                        stream>>>(a);
    return cudaGetLastError();
}

template <int K>
static cudaError_t launch_v_t(const SweepArgs& a, cudaStream_t stream) {
    const dim3 grid((a.W + kWarpsPerBlock - 1) / kWarpsPerBlock), block(32 * kWarpsPerBlock);
    const int smem = Stage<K>::BLOCK_BYTES;
    if (a.rx == 0)
        sweep_v_kernel<K, 0><<<grid, block, smem, stream>>>(a);
    else if (a.rx > 0)
        sweep_v_kernel<K, 1><<<grid, block, smem, stream>>>(a);
    else
        sweep_v_kernel<K, -1><<<grid, block, smem, stream>>>(a);
    return cudaGetLastError();
}

// K = DP / 64 words per lane (32 lanes per path).
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

// Path aggregation (Eq. 3), the sum S and the winner-take-all disparity
// (Eq. 4) of the SGM path in arXiv 1610.04121, for sm_103a.
//
// Parallel scheme (Section 3.2, with the paper's CTA-to-warp conversion taken
// one step further): one warp carries the two opposite paths of one row or one
// column, 16 lanes each, disparities packed two per 32-bit register.  The two
// paths meet in the middle: each sweeps its first half of the line storing
// L_r (u8) in a scratch cube, and in its second half adds the other path's
// stored L_r to its own.  The exchange between the two halves of the line is
// warp-local, so no block barrier is involved.
//
// Each half-warp streams its inputs through a private shared-memory ring
// filled by cp.async a few chunks ahead, keeps its step loop on shared memory
// only, and writes each chunk's outputs back with 16-byte stores.
//
//   sweep_h : left-to-right with right-to-left, one row per warp;
//             writes S = L_LR + L_RL (packed u16x2).
//   sweep_v : top-to-bottom with bottom-to-top along columns (RX = 0) or along
//             the wrapped diagonals of Section 3.2 (RX = +1 / -1); either adds
//             its pair sum into S or, for the last axis, finishes with Eq. 4.
#pragma once

#include "sgm_device.cuh"
#include "sgm_internal.h"

namespace sgm {

constexpr int kWarpsPerBlock = 4;

enum WalkMode {
    kStoreL = 0,    // phase 1 of a pair: store L_r
    kSumH = 1,      // phase 2 of the horizontal pair: S = L + stored L
    kAcc = 2,       // phase 2 of a diagonal pair: S += L + stored L
    kWta2 = 3,      // phase 2 of the vertical pair: raw = argmin_d (S + L + stored L)
    kSingleH = 4,   // 2-path mode, left-to-right: S = L
    kSingleWta = 5  // 2-path mode, top-to-bottom: raw = argmin_d (S + L)
};

// Shared-memory staging of one half-warp (one path) with K words per lane
// during a walk in MODE: a ring of NSLOT chunks per input stream it reads
// (costs; stored L of the other path; sums) and one chunk of outputs.
template <int K, int MODE>
struct Stage {
    static constexpr bool IN_LO = MODE == kSumH || MODE == kAcc || MODE == kWta2;
    static constexpr bool IN_S = MODE == kAcc || MODE == kWta2 || MODE == kSingleWta;
    static constexpr bool OUT_LX = MODE == kStoreL;
    static constexpr bool OUT_S = MODE == kSumH || MODE == kAcc || MODE == kSingleH;
    static constexpr bool WTA = MODE == kWta2 || MODE == kSingleWta;
    static constexpr int D = 32 * K;
    static constexpr int CH = (K <= 2) ? 16 : (K <= 4 ? 8 : 4);  // pixels per chunk
    static constexpr int NSLOT = 3;                              // chunks in flight + 1
    static constexpr int MC_RING = NSLOT * CH * D;
    static constexpr int LO_RING = IN_LO ? NSLOT * CH * D : 0;
    static constexpr int S_RING = IN_S ? NSLOT * CH * 2 * D : 0;
    static constexpr int OUT = OUT_LX ? CH * D : (OUT_S ? CH * 2 * D : 0);
    static constexpr int BYTES = MC_RING + LO_RING + S_RING + OUT;
};

constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Bytes per half-warp and per block of each kernel (the largest of its walks).
template <int K, bool PAIR>
struct HStage {
    static constexpr int HALF = PAIR ? cmax(Stage<K, kStoreL>::BYTES, Stage<K, kSumH>::BYTES) : Stage<K, kSingleH>::BYTES;
    static constexpr int BLOCK = 2 * kWarpsPerBlock * HALF;
};
template <int K, int PH, bool WTA, bool PAIR>
struct VStage {
    static constexpr int SECOND = WTA ? Stage<K, kWta2>::BYTES : Stage<K, kAcc>::BYTES;
    static constexpr int HALF = !PAIR ? Stage<K, kSingleWta>::BYTES
                                      : (PH == 1 ? Stage<K, kStoreL>::BYTES
                                                 : (PH == 2 ? SECOND : cmax(Stage<K, kStoreL>::BYTES, SECOND)));
    static constexpr int BLOCK = 2 * kWarpsPerBlock * HALF;
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

// One phase of both half-warp paths.  g / n_own: this lane's half; n_min /
// n_max: the shorter and the longer of the two halves' step counts.
template <int K, int MODE, class Geo>
__device__ __forceinline__ void walk(Chain2<K>& ch, const Geo& g, int n_own, int n_min, int n_max, const SweepArgs& a,
                                     uint8_t* ws, int hl) {
    using St = Stage<K, MODE>;
    constexpr int D = St::D, CH = St::CH, NS = St::NSLOT;
    constexpr bool IN_LO = St::IN_LO, IN_S = St::IN_S, OUT_LX = St::OUT_LX, OUT_S = St::OUT_S, WTA = St::WTA;
    constexpr int PM = D / 16;      // 16-byte pieces per pixel of u8 pairs
    constexpr int PS = 2 * D / 16;  // 16-byte pieces per pixel of packed sums
    uint8_t* mc_ring = ws;
    uint8_t* lo_ring = mc_ring + St::MC_RING;
    uint8_t* s_ring = lo_ring + St::LO_RING;
    uint8_t* out = s_ring + St::S_RING;
    const uint8_t* Sb = reinterpret_cast<const uint8_t*>(a.S);
    const int nch = (n_max + CH - 1) / CH;

    uint32_t dconst[K];
    if constexpr (WTA) wta_consts<K>(hl, D, dconst);

    auto issue = [&](int c) {
        if (c < nch) {
            const int i0 = c * CH, np = max(0, min(CH, n_own - i0)), slot = c % NS;
            int xc = 0, yc = 0;
            if (np > 0) g.origin(i0, xc, yc);
            for (int q = hl; q < np * PM; q += 16) {
                const int pi = q / PM, off = (q % PM) * 16;
                const size_t p = g.pix(xc, yc, pi);
                cp16(mc_ring + (slot * CH + pi) * D + off, a.MC + p * D + off);
                if constexpr (IN_LO) cp16(lo_ring + (slot * CH + pi) * D + off, a.Lx + p * D + off);
            }
            if constexpr (IN_S) {
                for (int q = hl; q < np * PS; q += 16) {
                    const int pi = q / PS, off = (q % PS) * 16;
                    const size_t p = g.pix(xc, yc, pi);
                    cp16(s_ring + (slot * CH + pi) * 2 * D + off, Sb + p * 2 * D + off);
                }
            }
        }
        cp_commit();
    };

    int y_body = 0, x_body = 0;
    if constexpr (Geo::kResets) g.origin(0, x_body, y_body);

    // one step at chunk position pi; lane pi of each half keeps that step's disparity key
    auto body = [&](int pi, int slot, int xc, int yc, bool active, uint32_t& dkeep) {
        if constexpr (Geo::kResets) {
            if (g.starts(y_body, x_body)) ch.reset();
            y_body += g.dy;
            x_body = g.step_x(x_body);
        }
        uint32_t mc[K], L[K];
        unpack_pairs<K>(ld_pairs<K>(mc_ring + (slot * CH + pi) * D + hl * 2 * K), mc);
        ch.step(mc, a.P1x2, a.P2x2, L);
        if constexpr (OUT_LX) {
            st_pairs<K>(out + pi * D + hl * 2 * K, pack_pairs<K>(L));
        } else {
            uint32_t s[K];
#pragma unroll
            for (int j = 0; j < K; ++j) s[j] = L[j];
            if constexpr (IN_LO) {
                uint32_t lo[K];
                unpack_pairs<K>(ld_pairs<K>(lo_ring + (slot * CH + pi) * D + hl * 2 * K), lo);
#pragma unroll
                for (int j = 0; j < K; ++j) s[j] += lo[j];
            }
            if constexpr (IN_S) {
                uint32_t t[K];
                ld_words<K>(reinterpret_cast<const uint32_t*>(s_ring + (slot * CH + pi) * 2 * D) + hl * K, t);
#pragma unroll
                for (int j = 0; j < K; ++j) s[j] += t[j];
            }
            if constexpr (OUT_S) st_words<K>(reinterpret_cast<uint32_t*>(out + pi * 2 * D) + hl * K, s);
            if constexpr (WTA) {
                const uint32_t key = ch.half_min(wta_key<K>(s, dconst));
                dkeep = (hl == pi) ? key : dkeep;
                if (a.Sdbg && active) {  // debug: natural-order S
                    const size_t p = g.pix(xc, yc, pi);
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        const int i = hl * K + j;
                        a.Sdbg[p * D + i] = static_cast<uint16_t>(s[j] & 0xffffu);
                        a.Sdbg[p * D + i + D / 2] = static_cast<uint16_t>(s[j] >> 16);
                    }
                }
            }
        }
    };

    for (int c = 0; c < NS - 1; ++c) issue(c);
    for (int c = 0; c < nch; ++c) {
        issue(c + NS - 1);
        cp_wait<NS - 1>();
        __syncwarp();
        const int i0 = c * CH, np = max(0, min(CH, n_own - i0)), slot = c % NS;
        int xc = 0, yc = 0;
        if (np > 0) g.origin(i0, xc, yc);
        uint32_t dkeep = 0;
        if (n_min - i0 >= CH) {
#pragma unroll
            for (int pi = 0; pi < CH; ++pi) body(pi, slot, xc, yc, true, dkeep);
        } else {
            // last chunk: a half with fewer steps keeps its state through the extra steps
#pragma unroll
            for (int pi = 0; pi < CH; ++pi) {
                if (i0 + pi < n_max) {
                    const Chain2<K> saved = ch;
                    const int yb = y_body, xb = x_body;
                    body(pi, slot, xc, yc, pi < np, dkeep);
                    if (pi >= np) {
                        ch = saved;
                        y_body = yb;
                        x_body = xb;
                    }
                }
            }
        }
        __syncwarp();
        if constexpr (WTA) {
            if (hl < np) a.raw[g.pix(xc, yc, hl)] = static_cast<uint8_t>(dkeep & 0xffu);
        }
        if constexpr (OUT_LX || OUT_S) {
            constexpr int P = OUT_LX ? PM : PS;
            constexpr int BPP = OUT_LX ? D : 2 * D;  // bytes per pixel
            uint8_t* dst = OUT_LX ? a.Lx : reinterpret_cast<uint8_t*>(a.S);
            for (int q = hl; q < np * P; q += 16) {
                const int pi = q / P, off = (q % P) * 16;
                const size_t p = g.pix(xc, yc, pi);
                *reinterpret_cast<uint4*>(dst + p * BPP + off) = *reinterpret_cast<const uint4*>(out + pi * BPP + off);
            }
            __syncwarp();
        }
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// Horizontal axis: one row per warp, lanes 0-15 walk left to right, lanes
// 16-31 right to left.  Phase 1: LR covers x < W/2, RL covers x >= W/2, both
// storing L in Lx.  Phase 2: each covers the other half and writes
// S = own L + stored L.  Without `pair` (2-path mode) LR covers the whole row
// and writes S = L_LR.
// ---------------------------------------------------------------------------
template <int K, bool PAIR>
__device__ __forceinline__ void sweep_h_body(const SweepArgs& a, int bx) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, hl = lane & 15;
    const bool in_b = lane >= 16;
    const int y = bx * kWarpsPerBlock + warp;
    if (y >= a.H) return;  // whole warp: every exchange below is warp-local
    uint8_t* ws = smem + (2 * warp + (in_b ? 1 : 0)) * HStage<K, PAIR>::HALF;
    const int W = a.W;
    const size_t rowbase = static_cast<size_t>(y) * W;
    Chain2<K> ch;
    ch.init(lane);
    if constexpr (!PAIR) {
        const RowGeo g{rowbase, 0, 1};
        walk<K, kSingleH>(ch, g, in_b ? 0 : W, 0, W, a, ws, hl);
    } else {
        const int Wm = W / 2;
        {
            const RowGeo g = in_b ? RowGeo{rowbase, W - 1, -1} : RowGeo{rowbase, 0, 1};
            const int nA = Wm, nB = W - Wm;
            walk<K, kStoreL>(ch, g, in_b ? nB : nA, min(nA, nB), max(nA, nB), a, ws, hl);
        }
        __threadfence_block();  // this half's L stores before the other half reads them
        __syncwarp();
        {
            const RowGeo g = in_b ? RowGeo{rowbase, Wm - 1, -1} : RowGeo{rowbase, Wm, 1};
            const int nA = W - Wm, nB = Wm;
            walk<K, kSumH>(ch, g, in_b ? nB : nA, min(nA, nB), max(nA, nB), a, ws, hl);
        }
    }
}

template <int K, bool PAIR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_h_kernel(SweepArgs a) {
    sweep_h_body<K, PAIR>(a, blockIdx.x);
}

template <int K, bool PAIR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_h_batch_kernel(const __grid_constant__ JobTable<SweepArgs> t) {
    const int p = find_job(t, blockIdx.x);
    sweep_h_body<K, PAIR>(t.job[p], blockIdx.x - t.start[p]);
}

// ---------------------------------------------------------------------------
// Vertical-type axis: one chain per warp, lanes 0-15 walk down (rows 0 ..
// H-1), lanes 16-31 up.  Chain c visits pixel x(y) = (c + RX*y) mod W in row y:
// a column for RX = 0, and for RX = +1/-1 a diagonal that wraps to the other
// border, restarting its path there (Section 3.2).  Phase 1: down covers
// y < H/2, up covers y >= H/2, storing L.  Phase 2: each covers the other half
// and combines its L with the stored L and S: S += both (wta = 0) or
// raw = argmin_d (S + both) (wta = 1).  Without `pair` the downward half covers
// all rows (2-path mode, wta = 1).
// ---------------------------------------------------------------------------
// PH: 0 = both phases in one launch, 1 = first halves (saving the path state),
// 2 = second halves (restoring it).  WTA: the pair finishes with Eq. 4
// instead of adding into S.  PAIR = false is the 2-path top-to-bottom sweep.
template <int K, int RX, int PH, bool WTA, bool PAIR>
__device__ __forceinline__ void sweep_v_body(const SweepArgs& a, int bx) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, hl = lane & 15;
    const bool in_b = lane >= 16;
    const int c = bx * kWarpsPerBlock + warp;
    if (c >= a.W) return;  // whole warp
    uint8_t* ws = smem + (2 * warp + (in_b ? 1 : 0)) * VStage<K, PH, WTA, PAIR>::HALF;
    const int W = a.W, H = a.H;
    using G = ColGeo<RX>;
    Chain2<K> ch;
    ch.init(lane);
    if constexpr (!PAIR) {
        walk<K, kSingleWta>(ch, G{W, H, c, 0, 1}, in_b ? 0 : H, 0, H, a, ws, hl);
    } else {
        const int Hm = H / 2;
        // saved path state of this lane: K words, the two neighbour words and m
        uint32_t* st = (PH != 0) ? a.state + (static_cast<size_t>(c) * 32 + lane) * (K + 3) : nullptr;
        if constexpr (PH != 2) {
            const G g = in_b ? G{W, H, c, H - 1, -1} : G{W, H, c, 0, 1};
            const int nA = Hm, nB = H - Hm;
            walk<K, kStoreL>(ch, g, in_b ? nB : nA, min(nA, nB), max(nA, nB), a, ws, hl);
        }
        if constexpr (PH == 1) {
#pragma unroll
            for (int j = 0; j < K; ++j) st[j] = ch.w[j];
            st[K] = ch.up;
            st[K + 1] = ch.dn;
            st[K + 2] = ch.mpx2;
            return;
        }
        if constexpr (PH == 2) {
#pragma unroll
            for (int j = 0; j < K; ++j) ch.w[j] = st[j];
            ch.up = st[K];
            ch.dn = st[K + 1];
            ch.mpx2 = st[K + 2];
        }
        if constexpr (PH != 1) {
            __threadfence_block();
            __syncwarp();
            const G g = in_b ? G{W, H, c, Hm - 1, -1} : G{W, H, c, Hm, 1};
            const int nA = H - Hm, nB = Hm;
            walk<K, WTA ? kWta2 : kAcc>(ch, g, in_b ? nB : nA, min(nA, nB), max(nA, nB), a, ws, hl);
        }
    }
}

template <int K, int RX, int PH, bool WTA, bool PAIR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_v_kernel(SweepArgs a) {
    sweep_v_body<K, RX, PH, WTA, PAIR>(a, blockIdx.x);
}

// Batched form: both phases in one launch (PH = 0).
template <int K, int RX, bool WTA, bool PAIR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_v_batch_kernel(const __grid_constant__ JobTable<SweepArgs> t) {
    const int p = find_job(t, blockIdx.x);
    sweep_v_body<K, RX, 0, WTA, PAIR>(t.job[p], blockIdx.x - t.start[p]);
}

// ---------------------------------------------------------------------------
// Per-K entry points, instantiated one K per translation unit.
// ---------------------------------------------------------------------------
template <int K>
struct SweepK {
    template <class Kern>
    static cudaError_t attr(Kern kern, int bytes) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    }

    template <int RX, bool WTA>
    static cudaError_t attrs_rx() {
        cudaError_t e = attr(sweep_v_kernel<K, RX, 0, WTA, true>, VStage<K, 0, WTA, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_kernel<K, RX, 1, false, true>, VStage<K, 1, false, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_kernel<K, RX, 2, WTA, true>, VStage<K, 2, WTA, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_batch_kernel<K, RX, WTA, true>, VStage<K, 0, WTA, true>::BLOCK);
        return e;
    }

    static cudaError_t set_attrs() {
        cudaError_t e = attr(sweep_h_kernel<K, true>, HStage<K, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_h_kernel<K, false>, HStage<K, false>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_h_batch_kernel<K, true>, HStage<K, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_h_batch_kernel<K, false>, HStage<K, false>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_kernel<K, 0, 0, true, false>, VStage<K, 0, true, false>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_batch_kernel<K, 0, true, false>, VStage<K, 0, true, false>::BLOCK);
        if (e == cudaSuccess) e = attrs_rx<0, true>();
        if (e == cudaSuccess) e = attrs_rx<1, false>();
        if (e == cudaSuccess) e = attrs_rx<-1, false>();
        return e;
    }

    static cudaError_t launch_h(const SweepArgs& a, cudaStream_t s) {
        const dim3 grid((a.H + kWarpsPerBlock - 1) / kWarpsPerBlock), block(32 * kWarpsPerBlock);
        if (a.pair)
            sweep_h_kernel<K, true><<<grid, block, HStage<K, true>::BLOCK, s>>>(a);
        else
            sweep_h_kernel<K, false><<<grid, block, HStage<K, false>::BLOCK, s>>>(a);
        return cudaGetLastError();
    }

    template <int RX, bool WTA>
    static void launch_v_rx(const SweepArgs& a, dim3 grid, dim3 block, cudaStream_t s) {
        if (a.phase == 1)
            sweep_v_kernel<K, RX, 1, false, true><<<grid, block, VStage<K, 1, false, true>::BLOCK, s>>>(a);
        else if (a.phase == 2)
            sweep_v_kernel<K, RX, 2, WTA, true><<<grid, block, VStage<K, 2, WTA, true>::BLOCK, s>>>(a);
        else
            sweep_v_kernel<K, RX, 0, WTA, true><<<grid, block, VStage<K, 0, WTA, true>::BLOCK, s>>>(a);
    }

    static cudaError_t launch_h_batch(JobTable<SweepArgs>& t, cudaStream_t s) {
        t.start[0] = 0;
        for (int i = 0; i < t.n; ++i) t.start[i + 1] = t.start[i] + (t.job[i].H + kWarpsPerBlock - 1) / kWarpsPerBlock;
        const dim3 block(32 * kWarpsPerBlock);
        if (t.job[0].pair)
            sweep_h_batch_kernel<K, true><<<t.start[t.n], block, HStage<K, true>::BLOCK, s>>>(t);
        else
            sweep_h_batch_kernel<K, false><<<t.start[t.n], block, HStage<K, false>::BLOCK, s>>>(t);
        return cudaGetLastError();
    }

    static cudaError_t launch_v_batch(JobTable<SweepArgs>& t, cudaStream_t s) {
        t.start[0] = 0;
        for (int i = 0; i < t.n; ++i) t.start[i + 1] = t.start[i] + (t.job[i].W + kWarpsPerBlock - 1) / kWarpsPerBlock;
        const dim3 grid(t.start[t.n]), block(32 * kWarpsPerBlock);
        const SweepArgs& a = t.job[0];
        if (!a.pair)
            sweep_v_batch_kernel<K, 0, true, false><<<grid, block, VStage<K, 0, true, false>::BLOCK, s>>>(t);
        else if (a.rx == 0)
            sweep_v_batch_kernel<K, 0, true, true><<<grid, block, VStage<K, 0, true, true>::BLOCK, s>>>(t);
        else if (a.rx > 0)
            sweep_v_batch_kernel<K, 1, false, true><<<grid, block, VStage<K, 0, false, true>::BLOCK, s>>>(t);
        else
            sweep_v_batch_kernel<K, -1, false, true><<<grid, block, VStage<K, 0, false, true>::BLOCK, s>>>(t);
        return cudaGetLastError();
    }

    static cudaError_t launch_v(const SweepArgs& a, cudaStream_t s) {
        const dim3 grid((a.W + kWarpsPerBlock - 1) / kWarpsPerBlock), block(32 * kWarpsPerBlock);
        if (!a.pair)
            sweep_v_kernel<K, 0, 0, true, false><<<grid, block, VStage<K, 0, true, false>::BLOCK, s>>>(a);
        else if (a.rx == 0)
            launch_v_rx<0, true>(a, grid, block, s);
        else if (a.rx > 0)
            launch_v_rx<1, false>(a, grid, block, s);
        else
            launch_v_rx<-1, false>(a, grid, block, s);
        return cudaGetLastError();
    }
};

// defined in sgm_sweeps_k<K>.cu; internal to the library (not part of the C ABI)
#define SGM_INTERNAL __attribute__((visibility("hidden")))
template <int K>
SGM_INTERNAL cudaError_t sweep_set_attrs();
template <int K>
SGM_INTERNAL cudaError_t sweep_launch_h(const SweepArgs& a, cudaStream_t s);
template <int K>
SGM_INTERNAL cudaError_t sweep_launch_v(const SweepArgs& a, cudaStream_t s);
template <int K>
SGM_INTERNAL cudaError_t sweep_launch_h_batch(JobTable<SweepArgs>& t, cudaStream_t s);
template <int K>
SGM_INTERNAL cudaError_t sweep_launch_v_batch(JobTable<SweepArgs>& t, cudaStream_t s);

#define SGM_INSTANTIATE_SWEEPS(K)                                                                           \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_set_attrs<K>() {                                                         \
        return SweepK<K>::set_attrs();                                                                      \
    }                                                                                                       \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_launch_h<K>(const SweepArgs& a, cudaStream_t s) {                        \
        return SweepK<K>::launch_h(a, s);                                                                   \
    }                                                                                                       \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_launch_v<K>(const SweepArgs& a, cudaStream_t s) {                        \
        return SweepK<K>::launch_v(a, s);                                                                   \
    }                                                                                                       \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_launch_h_batch<K>(JobTable<SweepArgs> & t, cudaStream_t s) {             \
        return SweepK<K>::launch_h_batch(t, s);                                                             \
    }                                                                                                       \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_launch_v_batch<K>(JobTable<SweepArgs> & t, cudaStream_t s) {             \
        return SweepK<K>::launch_v_batch(t, s);                                                             \
    }

}  // namespace sgm

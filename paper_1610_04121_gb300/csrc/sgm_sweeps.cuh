// Path aggregation (Eq. 3), the sum S and the winner-take-all disparity
// (Eq. 4) of the SGM path in arXiv 1610.04121, for sm_103a.
//
// Parallel scheme (Section 3.2, with the paper's CTA-to-warp conversion taken
// further): a path's disparities are spread over G lanes, two per 32-bit
// register.  When D is a multiple of 64, G = 32 and each warp carries one
// direction of a line, the two opposite directions of a line being a pair of
// warps of one block; otherwise G = 16 and one warp carries both directions,
// one per half.  The two directions meet in the middle: each sweeps its
// first half of the line storing L_r (u8) in a scratch cube, and in its
// second half adds the other direction's stored L_r to its own.  The exchange
// is warp-local (G = 16) or through a 64-thread named barrier (G = 32).
//
// Each path streams its inputs through a private shared-memory ring filled
// by cp.async a few chunks ahead, keeps its step loop on shared memory and
// registers, and writes its outputs with coalesced vector stores.
//
//   sweep_h : left-to-right with right-to-left, one row per line;
//             writes S = L_LR + L_RL (packed u16x2).
//   sweep_v : top-to-bottom with bottom-to-top along columns (RX = 0) or along
//             the wrapped diagonals of Section 3.2 (RX = +1 / -1); either adds
//             its pair sum into S or, for the last axis, finishes with Eq. 4.
#pragma once

#include "sgm_device.cuh"
#include "sgm_internal.h"

namespace sgm {

constexpr int kWarpsPerBlock = 4;

// Lanes per path and packed words per lane for D disparities.
template <int D>
struct PathShape {
    static constexpr int G = (D % 64 == 0) ? 32 : 16;
    static constexpr int K = D / (2 * G);
    static constexpr int PPW = 32 / G;  // paths per warp
};

enum WalkMode {
    kStoreL = 0,    // phase 1 of a pair: store L_r
    kSumH = 1,      // phase 2 of the horizontal pair: S = L + stored L
    kAcc = 2,       // phase 2 of a diagonal pair: S += L + stored L
    kWta2 = 3,      // phase 2 of the vertical pair: raw = argmin_d (S + L + stored L)
    kSingleH = 4,   // 2-path mode, left-to-right: S = L
    kSingleWta = 5  // 2-path mode, top-to-bottom: raw = argmin_d (S + L)
};

// Shared-memory staging of one path during a walk in MODE: a ring of NSLOT
// chunks of CH pixels per input stream it reads (costs; stored L of the other
// direction; sums).  Row walks read contiguous pixels and take longer chunks.
template <int D, int MODE, bool ROW>
struct Stage {
    static constexpr bool IN_LO = MODE == kSumH || MODE == kAcc || MODE == kWta2;
    static constexpr bool IN_S = MODE == kAcc || MODE == kWta2 || MODE == kSingleWta;
    static constexpr bool OUT_LX = MODE == kStoreL;
    static constexpr bool OUT_S = MODE == kSumH || MODE == kAcc || MODE == kSingleH;
    static constexpr bool WTA = MODE == kWta2 || MODE == kSingleWta;
    static constexpr int CH = ROW ? (D <= 128 ? 16 : 8) : (D <= 64 ? 16 : (D <= 128 ? 8 : 4));  // pixels per chunk
    static constexpr int NSLOT = 3;                                // chunks in flight + 1
    static constexpr int MC_RING = NSLOT * CH * D;
    static constexpr int LO_RING = IN_LO ? NSLOT * CH * D : 0;
    static constexpr int S_RING = IN_S ? NSLOT * CH * 2 * D : 0;
    static constexpr int BYTES = MC_RING + LO_RING + S_RING;
};

constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Staging bytes per path and per block of each kernel (the largest of its walks).
template <int D, bool PAIR>
struct HStage {
    static constexpr int PATH =
        PAIR ? cmax(Stage<D, kStoreL, true>::BYTES, Stage<D, kSumH, true>::BYTES) : Stage<D, kSingleH, true>::BYTES;
    static constexpr int BLOCK = kWarpsPerBlock * PathShape<D>::PPW * PATH;
};
template <int D, int PH, bool WTA, bool PAIR>
struct VStage {
    static constexpr int SECOND = WTA ? Stage<D, kWta2, false>::BYTES : Stage<D, kAcc, false>::BYTES;
    static constexpr int FIRST = Stage<D, kStoreL, false>::BYTES;
    static constexpr int PATH =
        !PAIR ? Stage<D, kSingleWta, false>::BYTES : (PH == 1 ? FIRST : (PH == 2 ? SECOND : cmax(FIRST, SECOND)));
    static constexpr int BLOCK = kWarpsPerBlock * PathShape<D>::PPW * PATH;
};

// Lines (rows or columns) per block: with G = 32 a pair takes two warps.
template <int D, bool PAIR>
constexpr int lines_per_block() {
    return (PathShape<D>::G == 32 && PAIR) ? kWarpsPerBlock / 2 : kWarpsPerBlock;
}

// Which line and direction this warp (or, for G = 16, this lane's half) walks.
template <int D, bool PAIR>
struct LaneRole {
    int line, dir, pl, slot;  // slot: index of this path's staging area in the block
    __device__ __forceinline__ LaneRole(int bx) {
        constexpr int G = PathShape<D>::G;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        pl = lane & (G - 1);
        if constexpr (G == 16) {
            line = bx * kWarpsPerBlock + warp;
            dir = lane >> 4;
            slot = 2 * warp + dir;
        } else if constexpr (PAIR) {
            line = bx * (kWarpsPerBlock / 2) + (warp >> 1);
            dir = warp & 1;
            slot = warp;
        } else {
            line = bx * kWarpsPerBlock + warp;
            dir = 0;
            slot = warp;
        }
    }
};

// Between the two phases of a pair: the first halves' L stores are visible to
// the other direction's second half.
template <int D>
__device__ __forceinline__ void pair_barrier() {
    __threadfence_block();
    if constexpr (PathShape<D>::G == 16) {
        __syncwarp();
    } else {
        static_assert(kWarpsPerBlock == 4, "two pairs of warps per block");
        // immediate barrier ids keep the kernel's barrier count small
        if ((threadIdx.x >> 6) == 0)
            asm volatile("bar.sync 1, 64;" ::: "memory");
        else
            asm volatile("bar.sync 2, 64;" ::: "memory");
    }
}

// Pixels of a row walk: x = x0 + dx * i.
struct RowGeo {
    size_t rowbase;
    int x0, dx;
    static constexpr bool kResets = false;
    static constexpr bool kRow = true;
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
    static constexpr bool kRow = false;
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

// One phase of this warp's path(s).  g / n_own: this lane's path; n_min /
// n_max: the shorter and the longer step count of the warp's paths (equal to
// n_own when the warp carries one path).  DBG: a winner-take-all walk also
// writes S in natural order to a.Sdbg.
template <int D, int MODE, class Geo, bool DBG = false>
__device__ __forceinline__ void walk(Chain<PathShape<D>::G, PathShape<D>::K>& ch, const Geo& g, int n_own,
                                     int n_min, int n_max, const SweepArgs& a, uint8_t* ws, int pl) {
    constexpr int G = PathShape<D>::G, K = PathShape<D>::K;
    using St = Stage<D, MODE, Geo::kRow>;
    constexpr int CH = St::CH, NS = St::NSLOT;
    constexpr bool IN_LO = St::IN_LO, IN_S = St::IN_S, OUT_LX = St::OUT_LX, OUT_S = St::OUT_S, WTA = St::WTA;
    constexpr int PM = D / 16;      // 16-byte pieces per pixel of u8 pairs
    constexpr int PS = 2 * D / 16;  // 16-byte pieces per pixel of packed sums
    uint8_t* mc_ring = ws;
    uint8_t* lo_ring = mc_ring + St::MC_RING;
    uint8_t* s_ring = lo_ring + St::LO_RING;
    const uint8_t* Sb = reinterpret_cast<const uint8_t*>(a.S);
    const int nch = (n_max + CH - 1) / CH;

    uint32_t dconst[K];
    if constexpr (WTA) wta_consts<K>(pl, D, dconst);

    auto issue = [&](int c) {
        if (c < nch) {
            const int i0 = c * CH, np = max(0, min(CH, n_own - i0)), slot = c % NS;
            int xc = 0, yc = 0;
            if (np > 0) g.origin(i0, xc, yc);
            for (int q = pl; q < np * PM; q += G) {
                const int pi = q / PM, off = (q % PM) * 16;
                const size_t p = g.pix(xc, yc, pi);
                cp16(mc_ring + (slot * CH + pi) * D + off, a.MC + p * D + off);
                if constexpr (IN_LO) cp16(lo_ring + (slot * CH + pi) * D + off, a.Lx + p * D + off);
            }
            if constexpr (IN_S) {
                for (int q = pl; q < np * PS; q += G) {
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

    // one step at chunk position pi; lane pi of each path keeps that step's disparity key
    auto body = [&](int pi, int slot, int xc, int yc, bool active, uint32_t& dkeep) {
        if constexpr (Geo::kResets) {
            if (g.starts(y_body, x_body)) ch.reset();
            y_body += g.dy;
            x_body = g.step_x(x_body);
        }
        uint32_t mc[K], L[K];
        unpack_pairs<K>(ld_pairs<K>(mc_ring + (slot * CH + pi) * D + pl * 2 * K), mc);
        ch.step(mc, a.P1x2, a.P2x2, L);
        if constexpr (OUT_LX) {
            if (active) st_pairs<K>(a.Lx + g.pix(xc, yc, pi) * D + pl * 2 * K, pack_pairs<K>(L));
        } else {
            uint32_t s[K];
#pragma unroll
            for (int j = 0; j < K; ++j) s[j] = L[j];
            if constexpr (IN_LO) {
                uint32_t lo[K];
                unpack_pairs<K>(ld_pairs<K>(lo_ring + (slot * CH + pi) * D + pl * 2 * K), lo);
#pragma unroll
                for (int j = 0; j < K; ++j) s[j] += lo[j];
            }
            if constexpr (IN_S) {
                uint32_t t[K];
                ld_words<K>(reinterpret_cast<const uint32_t*>(s_ring + (slot * CH + pi) * 2 * D) + pl * K, t);
#pragma unroll
                for (int j = 0; j < K; ++j) s[j] += t[j];
            }
            if constexpr (OUT_S) {
                if (active) st_words<K>(a.S + g.pix(xc, yc, pi) * (D / 2) + pl * K, s);
            }
            if constexpr (WTA) {
                const uint32_t key = ch.path_min(wta_key<K>(s, dconst));
                dkeep = (pl == pi) ? key : dkeep;
                if (DBG && active) {  // debug: natural-order S
                    const size_t p = g.pix(xc, yc, pi);
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        const int i = pl * K + j;
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
            // last chunk: a path with fewer steps keeps its state through the extra steps
#pragma unroll
            for (int pi = 0; pi < CH; ++pi) {
                if (i0 + pi < n_max) {
                    const Chain<G, K> saved = ch;
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
        if constexpr (WTA) {
            if (pl < np) a.raw[g.pix(xc, yc, pl)] = static_cast<uint8_t>(dkeep & 0xffu);
        }
        __syncwarp();  // every lane is done with this slot before it is refilled
    }
    cp_wait<0>();
}

// ---------------------------------------------------------------------------
// Horizontal axis: one row per line; direction A walks left to right,
// direction B right to left.  Phase 1: A covers x < W/2, B covers x >= W/2,
// both storing L in Lx.  Phase 2: each covers the other half and writes
// S = own L + stored L.  Without `pair` (2-path mode) A covers the whole row
// and writes S = L_LR.
// ---------------------------------------------------------------------------
template <int D, bool PAIR>
__device__ __forceinline__ void sweep_h_body(const SweepArgs& a, int bx) {
    extern __shared__ __align__(16) uint8_t smem[];
    constexpr int G = PathShape<D>::G, K = PathShape<D>::K;
    const LaneRole<D, PAIR> r(bx);
    const int y = r.line;
    if (y >= a.H) return;  // whole warp (and its pair): every exchange below is local to them
    const bool in_b = r.dir != 0;
    uint8_t* ws = smem + r.slot * HStage<D, PAIR>::PATH;
    const int W = a.W;
    const size_t rowbase = static_cast<size_t>(y) * W;
    Chain<G, K> ch;
    ch.init(threadIdx.x & 31);
    if constexpr (!PAIR) {
        const RowGeo g{rowbase, 0, 1};
        const int n = in_b ? 0 : W;
        walk<D, kSingleH>(ch, g, n, G == 16 ? 0 : n, W, a, ws, r.pl);
    } else {
        const int Wm = W / 2;
        {
            const RowGeo g = in_b ? RowGeo{rowbase, W - 1, -1} : RowGeo{rowbase, 0, 1};
            const int nA = Wm, nB = W - Wm, n = in_b ? nB : nA;
            walk<D, kStoreL>(ch, g, n, G == 16 ? min(nA, nB) : n, G == 16 ? max(nA, nB) : n, a, ws, r.pl);
        }
        pair_barrier<D>();
        {
            const RowGeo g = in_b ? RowGeo{rowbase, Wm - 1, -1} : RowGeo{rowbase, Wm, 1};
            const int nA = W - Wm, nB = Wm, n = in_b ? nB : nA;
            walk<D, kSumH>(ch, g, n, G == 16 ? min(nA, nB) : n, G == 16 ? max(nA, nB) : n, a, ws, r.pl);
        }
    }
}

template <int D, bool PAIR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_h_kernel(SweepArgs a) {
    sweep_h_body<D, PAIR>(a, blockIdx.x);
}

template <int D, bool PAIR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_h_batch_kernel(const __grid_constant__ JobTable<SweepArgs> t) {
    const int p = find_job(t, blockIdx.x);
    sweep_h_body<D, PAIR>(t.job[p], blockIdx.x - t.start[p]);
}

// ---------------------------------------------------------------------------
// Vertical-type axis: one column-type line per pair; direction A walks down
// (rows 0 .. H-1), direction B up.  Line c visits pixel x(y) = (c + RX*y) mod W
// in row y: a column for RX = 0, and for RX = +1/-1 a diagonal that wraps to
// the other border, restarting its path there (Section 3.2).  Phase 1: A
// covers y < H/2, B covers y >= H/2, storing L.  Phase 2: each covers the
// other half and combines its L with the stored L and S: S += both (wta = 0)
// or raw = argmin_d (S + both) (wta = 1).  Without `pair` direction A covers
// all rows (2-path mode, wta = 1).
// ---------------------------------------------------------------------------
// PH: 0 = both phases in one launch, 1 = first halves (saving the path state),
// 2 = second halves (restoring it).  WTA: the pair finishes with Eq. 4
// instead of adding into S.  PAIR = false is the 2-path top-to-bottom sweep.
template <int D, int RX, int PH, bool WTA, bool PAIR, bool DBG = false>
__device__ __forceinline__ void sweep_v_body(const SweepArgs& a, int bx) {
    extern __shared__ __align__(16) uint8_t smem[];
    constexpr int G = PathShape<D>::G, K = PathShape<D>::K;
    const LaneRole<D, PAIR> r(bx);
    const int c = r.line;
    if (c >= a.W) return;  // whole warp (and its pair)
    const bool in_b = r.dir != 0;
    uint8_t* ws = smem + r.slot * VStage<D, PH, WTA, PAIR>::PATH;
    const int W = a.W, H = a.H;
    using Geo = ColGeo<RX>;
    Chain<G, K> ch;
    const int lane = threadIdx.x & 31;
    ch.init(lane);
    if constexpr (!PAIR) {
        const int n = in_b ? 0 : H;
        walk<D, kSingleWta, Geo, DBG>(ch, Geo{W, H, c, 0, 1}, n, G == 16 ? 0 : n, H, a, ws, r.pl);
    } else {
        const int Hm = H / 2;
        // saved path state of this lane: K words, the two neighbour words and m
        uint32_t* st = nullptr;
        if constexpr (PH != 0)
            st = a.state + ((static_cast<size_t>(c) * (2 / PathShape<D>::PPW) + (G == 32 ? r.dir : 0)) * 32 + lane) *
                               (K + 3);
        if constexpr (PH != 2) {
            const Geo g = in_b ? Geo{W, H, c, H - 1, -1} : Geo{W, H, c, 0, 1};
            const int nA = Hm, nB = H - Hm, n = in_b ? nB : nA;
            walk<D, kStoreL>(ch, g, n, G == 16 ? min(nA, nB) : n, G == 16 ? max(nA, nB) : n, a, ws, r.pl);
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
            if constexpr (PH == 0) pair_barrier<D>();
            const Geo g = in_b ? Geo{W, H, c, Hm - 1, -1} : Geo{W, H, c, Hm, 1};
            const int nA = H - Hm, nB = Hm, n = in_b ? nB : nA;
            walk<D, WTA ? kWta2 : kAcc, Geo, DBG>(ch, g, n, G == 16 ? min(nA, nB) : n, G == 16 ? max(nA, nB) : n, a,
                                                  ws, r.pl);
        }
    }
}

template <int D, int RX, int PH, bool WTA, bool PAIR, bool DBG = false>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_v_kernel(SweepArgs a) {
    sweep_v_body<D, RX, PH, WTA, PAIR, DBG>(a, blockIdx.x);
}

// Batched form: both phases in one launch (PH = 0).
template <int D, int RX, bool WTA, bool PAIR>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_v_batch_kernel(const __grid_constant__ JobTable<SweepArgs> t) {
    const int p = find_job(t, blockIdx.x);
    sweep_v_body<D, RX, 0, WTA, PAIR>(t.job[p], blockIdx.x - t.start[p]);
}

// The horizontal pair and the vertical-type first halves in one grid: one
// block distribution over the SMs for all of them (two kernels sharing the
// SMs through concurrent streams ran far slower than either alone).
template <int D>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_first_kernel(const __grid_constant__ FirstStageArgs f) {
    const int b = blockIdx.x;
    if (b < f.start[1]) {
        sweep_h_body<D, true>(f.h, b);
        return;
    }
    for (int k = 0; k < f.nv; ++k) {
        if (b < f.start[k + 2]) {
            const SweepArgs& v = f.v[k];
            const int bx = b - f.start[k + 1];
            if (v.rx == 0)
                sweep_v_body<D, 0, 1, false, true>(v, bx);
            else if (v.rx > 0)
                sweep_v_body<D, 1, 1, false, true>(v, bx);
            else
                sweep_v_body<D, -1, 1, false, true>(v, bx);
            return;
        }
    }
}

template <int D>
struct FirstStage {
    static constexpr int BLOCK = cmax(HStage<D, true>::BLOCK, VStage<D, 1, false, true>::BLOCK);
};

// ---------------------------------------------------------------------------
// Per-D entry points, instantiated one D per translation unit.
// ---------------------------------------------------------------------------
template <int D>
struct SweepD {
    template <class Kern>
    static cudaError_t attr(Kern kern, int bytes) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    }

    template <int RX, bool WTA>
    static cudaError_t attrs_rx() {
        cudaError_t e = attr(sweep_v_kernel<D, RX, 0, WTA, true>, VStage<D, 0, WTA, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_kernel<D, RX, 1, false, true>, VStage<D, 1, false, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_kernel<D, RX, 2, WTA, true>, VStage<D, 2, WTA, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_batch_kernel<D, RX, WTA, true>, VStage<D, 0, WTA, true>::BLOCK);
        return e;
    }

    static cudaError_t set_attrs() {
        cudaError_t e = attr(sweep_first_kernel<D>, FirstStage<D>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_h_kernel<D, true>, HStage<D, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_h_kernel<D, false>, HStage<D, false>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_h_batch_kernel<D, true>, HStage<D, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_h_batch_kernel<D, false>, HStage<D, false>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_kernel<D, 0, 0, true, false>, VStage<D, 0, true, false>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_kernel<D, 0, 0, true, false, true>, VStage<D, 0, true, false>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_kernel<D, 0, 2, true, true, true>, VStage<D, 2, true, true>::BLOCK);
        if (e == cudaSuccess) e = attr(sweep_v_batch_kernel<D, 0, true, false>, VStage<D, 0, true, false>::BLOCK);
        if (e == cudaSuccess) e = attrs_rx<0, true>();
        if (e == cudaSuccess) e = attrs_rx<1, false>();
        if (e == cudaSuccess) e = attrs_rx<-1, false>();
        return e;
    }

    static int blocks(int lines, bool pair) {
        const int per = pair ? lines_per_block<D, true>() : lines_per_block<D, false>();
        return (lines + per - 1) / per;
    }

    static cudaError_t launch_h(const SweepArgs& a, cudaStream_t s) {
        const dim3 grid(blocks(a.H, a.pair)), block(32 * kWarpsPerBlock);
        if (a.pair)
            sweep_h_kernel<D, true><<<grid, block, HStage<D, true>::BLOCK, s>>>(a);
        else
            sweep_h_kernel<D, false><<<grid, block, HStage<D, false>::BLOCK, s>>>(a);
        return cudaGetLastError();
    }

    static cudaError_t launch_first(FirstStageArgs& f, cudaStream_t s) {
        f.start[0] = 0;
        f.start[1] = blocks(f.h.H, true);
        for (int k = 0; k < f.nv; ++k) f.start[k + 2] = f.start[k + 1] + blocks(f.v[k].W, true);
        const dim3 block(32 * kWarpsPerBlock);
        sweep_first_kernel<D><<<f.start[f.nv + 1], block, FirstStage<D>::BLOCK, s>>>(f);
        return cudaGetLastError();
    }

    template <int RX, bool WTA>
    static void launch_v_rx(const SweepArgs& a, dim3 grid, dim3 block, cudaStream_t s) {
        if (WTA && a.Sdbg && a.phase == 2)
            sweep_v_kernel<D, RX, 2, WTA, true, true><<<grid, block, VStage<D, 2, WTA, true>::BLOCK, s>>>(a);
        else if (a.phase == 1)
            sweep_v_kernel<D, RX, 1, false, true><<<grid, block, VStage<D, 1, false, true>::BLOCK, s>>>(a);
        else if (a.phase == 2)
            sweep_v_kernel<D, RX, 2, WTA, true><<<grid, block, VStage<D, 2, WTA, true>::BLOCK, s>>>(a);
        else
            sweep_v_kernel<D, RX, 0, WTA, true><<<grid, block, VStage<D, 0, WTA, true>::BLOCK, s>>>(a);
    }

    static cudaError_t launch_h_batch(JobTable<SweepArgs>& t, cudaStream_t s) {
        t.start[0] = 0;
        for (int i = 0; i < t.n; ++i) t.start[i + 1] = t.start[i] + blocks(t.job[i].H, t.job[i].pair);
        const dim3 block(32 * kWarpsPerBlock);
        if (t.job[0].pair)
            sweep_h_batch_kernel<D, true><<<t.start[t.n], block, HStage<D, true>::BLOCK, s>>>(t);
        else
            sweep_h_batch_kernel<D, false><<<t.start[t.n], block, HStage<D, false>::BLOCK, s>>>(t);
        return cudaGetLastError();
    }

    static cudaError_t launch_v_batch(JobTable<SweepArgs>& t, cudaStream_t s) {
        t.start[0] = 0;
        for (int i = 0; i < t.n; ++i) t.start[i + 1] = t.start[i] + blocks(t.job[i].W, t.job[i].pair);
        const dim3 grid(t.start[t.n]), block(32 * kWarpsPerBlock);
        const SweepArgs& a = t.job[0];
        if (!a.pair)
            sweep_v_batch_kernel<D, 0, true, false><<<grid, block, VStage<D, 0, true, false>::BLOCK, s>>>(t);
        else if (a.rx == 0)
            sweep_v_batch_kernel<D, 0, true, true><<<grid, block, VStage<D, 0, true, true>::BLOCK, s>>>(t);
        else if (a.rx > 0)
            sweep_v_batch_kernel<D, 1, false, true><<<grid, block, VStage<D, 0, false, true>::BLOCK, s>>>(t);
        else
            sweep_v_batch_kernel<D, -1, false, true><<<grid, block, VStage<D, 0, false, true>::BLOCK, s>>>(t);
        return cudaGetLastError();
    }

    static cudaError_t launch_v(const SweepArgs& a, cudaStream_t s) {
        const dim3 grid(blocks(a.W, a.pair)), block(32 * kWarpsPerBlock);
        if (!a.pair && a.Sdbg)
            sweep_v_kernel<D, 0, 0, true, false, true><<<grid, block, VStage<D, 0, true, false>::BLOCK, s>>>(a);
        else if (!a.pair)
            sweep_v_kernel<D, 0, 0, true, false><<<grid, block, VStage<D, 0, true, false>::BLOCK, s>>>(a);
        else if (a.rx == 0)
            launch_v_rx<0, true>(a, grid, block, s);
        else if (a.rx > 0)
            launch_v_rx<1, false>(a, grid, block, s);
        else
            launch_v_rx<-1, false>(a, grid, block, s);
        return cudaGetLastError();
    }
};

// defined in sgm_sweeps_d<D>.cu; internal to the library (not part of the C ABI)
#define SGM_INTERNAL __attribute__((visibility("hidden")))
template <int D>
SGM_INTERNAL cudaError_t sweep_set_attrs();
template <int D>
SGM_INTERNAL cudaError_t sweep_launch_h(const SweepArgs& a, cudaStream_t s);
template <int D>
SGM_INTERNAL cudaError_t sweep_launch_v(const SweepArgs& a, cudaStream_t s);
template <int D>
SGM_INTERNAL cudaError_t sweep_launch_first(FirstStageArgs& f, cudaStream_t s);
template <int D>
SGM_INTERNAL cudaError_t sweep_launch_h_batch(JobTable<SweepArgs>& t, cudaStream_t s);
template <int D>
SGM_INTERNAL cudaError_t sweep_launch_v_batch(JobTable<SweepArgs>& t, cudaStream_t s);

#define SGM_INSTANTIATE_SWEEPS(D)                                                                           \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_set_attrs<D>() {                                                         \
        return SweepD<D>::set_attrs();                                                                      \
    }                                                                                                       \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_launch_h<D>(const SweepArgs& a, cudaStream_t s) {                        \
        return SweepD<D>::launch_h(a, s);                                                                   \
    }                                                                                                       \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_launch_v<D>(const SweepArgs& a, cudaStream_t s) {                        \
        return SweepD<D>::launch_v(a, s);                                                                   \
    }                                                                                                       \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_launch_first<D>(FirstStageArgs & f, cudaStream_t s) {                    \
        return SweepD<D>::launch_first(f, s);                                                               \
    }                                                                                                       \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_launch_h_batch<D>(JobTable<SweepArgs> & t, cudaStream_t s) {             \
        return SweepD<D>::launch_h_batch(t, s);                                                             \
    }                                                                                                       \
    template <>                                                                                             \
    SGM_INTERNAL cudaError_t sweep_launch_v_batch<D>(JobTable<SweepArgs> & t, cudaStream_t s) {             \
        return SweepD<D>::launch_v_batch(t, s);                                                             \
    }

}  // namespace sgm

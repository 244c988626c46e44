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
// Each lane streams its own bytes of every step's inputs (costs, the other
// direction's stored L_r, sums) straight from global memory into registers,
// one chunk of PF steps ahead of the recurrence, and writes its outputs with
// one coalesced store per step; no shared memory is used (but for the post
// form's 256-entry penalty table).  All cubes of a
// pair live in one array of per-pixel records (sgm_internal.h), so a step's
// loads and stores share one 32-bit record offset, widened onto per-lane
// bases with one mad.wide (on the FMA pipe, off the busy integer ALU).
//
//   sweep_h : left-to-right with right-to-left, one row per line;
//             writes S = L_LR + L_RL.
//   sweep_v : top-to-bottom with bottom-to-top along columns (RX = 0) or along
//             the wrapped diagonals of Section 3.2 (RX = +1 / -1); either adds
//             its pair sum into S or, for the last axis, finishes with Eq. 4.
//   sweep_first4 / sweep_h2 : the 4-path schedule that runs the whole
//             vertical pair beside the horizontal first halves, then the
//             horizontal second halves with Eq. 4.
//   post form (POST = 1): every step takes its jump penalty from the base
//             image (adaptive P2), and the winner-take-all walks also write
//             the sums beside the winner for the sub-pixel step.
//
// S is kept either as packed u16x2 words [H][W][D/2] or, when every value it
// holds before the winner-take-all fits a byte (2 or 4 paths with
// 2 * (MC_max + P2) <= 255, see sum_fits_u8), as paired bytes [H][W][D] like
// the costs (template flag S8).
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

template <int MODE>
struct ModeIO {
    static constexpr bool IN_LO = MODE == kSumH || MODE == kAcc || MODE == kWta2;
    static constexpr bool IN_S = MODE == kAcc || MODE == kWta2 || MODE == kSingleWta;
    static constexpr bool OUT_LX = MODE == kStoreL;
    static constexpr bool OUT_S = MODE == kSumH || MODE == kAcc || MODE == kSingleH;
    static constexpr bool WTA = MODE == kWta2 || MODE == kSingleWta;
};

// Register prefetch: a walk proceeds in chunks of PF steps; at the start of a
// chunk the loads of the next chunk are issued, so every load has at least one
// chunk (PF steps of the recurrence) to arrive.  PF is chosen so that the two
// chunks of inputs held in registers stay near 96 registers.
__host__ __device__ constexpr int prefetch_steps(int regs_per_step, int budget = 48) {
    return budget / regs_per_step > 16 ? 16 : (budget / regs_per_step < 4 ? 4 : budget / regs_per_step);
}

template <int N>
struct Regs {
    uint32_t r[N];
};
template <>
struct Regs<0> {};

// Global loads of one lane's share of a step: K paired-byte values (2K bytes
// at byte offset 2K * pl of the pixel) or K packed words.  Costs are read
// through the non-coherent path (written by an earlier kernel); stored L_r
// and sums may have been written earlier in the same kernel or by the other
// warp of the pair, so they bypass L1.
template <int K, bool NC>
__device__ __forceinline__ void ldg_pairs(const uint8_t* p, uint32_t (&r)[(K + 1) / 2]) {
    if constexpr (K == 2) {
        r[0] = NC ? __ldg(reinterpret_cast<const unsigned*>(p)) : __ldcg(reinterpret_cast<const unsigned*>(p));
    } else if constexpr (K == 4) {
        const uint2 v = NC ? __ldg(reinterpret_cast<const uint2*>(p)) : __ldcg(reinterpret_cast<const uint2*>(p));
        r[0] = v.x;
        r[1] = v.y;
    } else if constexpr (K == 8) {
        const uint4 v = NC ? __ldg(reinterpret_cast<const uint4*>(p)) : __ldcg(reinterpret_cast<const uint4*>(p));
        r[0] = v.x;
        r[1] = v.y;
        r[2] = v.z;
        r[3] = v.w;
    } else {
        // odd K (16-lane paths with D = 32, 96, 160, 224): 2-byte aligned
        const unsigned short* h = reinterpret_cast<const unsigned short*>(p);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t v = NC ? __ldg(h + j) : __ldcg(h + j);
            if (j & 1)
                r[j >> 1] |= v << 16;
            else
                r[j >> 1] = v;
        }
    }
}

template <int K>
__device__ __forceinline__ void ldg_words(const uint32_t* p, uint32_t (&w)[K]) {
    if constexpr (K % 4 == 0) {
#pragma unroll
        for (int j = 0; j < K; j += 4) {
            const uint4 v = __ldcg(reinterpret_cast<const uint4*>(p + j));
            w[j] = v.x;
            w[j + 1] = v.y;
            w[j + 2] = v.z;
            w[j + 3] = v.w;
        }
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int j = 0; j < K; j += 2) {
            const uint2 v = __ldcg(reinterpret_cast<const uint2*>(p + j));
            w[j] = v.x;
            w[j + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = __ldcg(p + j);
    }
}

// 64-bit address base + 32-bit offset in one instruction (IMAD.WIDE.U32).
__device__ __forceinline__ const uint8_t* at(const uint8_t* base, uint32_t off) {
    uint64_t r;
    asm("mad.wide.u32 %0, %1, 1, %2;" : "=l"(r) : "r"(off), "l"(reinterpret_cast<uint64_t>(base)));
    return reinterpret_cast<const uint8_t*>(r);
}
__device__ __forceinline__ uint8_t* at(uint8_t* base, uint32_t off) {
    return const_cast<uint8_t*>(at(static_cast<const uint8_t*>(base), off));
}

// A lane's bases into the records: its paired bytes of MC (and, at +D, of
// byte sums), its u16 sum words, and its bytes of the pair's stored L_r.
struct LaneBases {
    uint8_t* pairs;
    uint8_t* words;
    uint8_t* lx;
    const uint8_t *lo, *hi;  // the records' extent (bounds-checked build)
};

template <int D>
__device__ __forceinline__ LaneBases lane_bases(const SweepArgs& a, int pl) {
    constexpr int K = PathShape<D>::K;
    return LaneBases{a.rec + 2 * K * pl, a.rec + D + 4 * K * pl, a.rec + a.lx_off + 2 * K * pl, a.rec,
                     a.rec + static_cast<size_t>(a.W) * a.H * a.RB};
}

// One step's inputs for one lane, loaded from the record at byte offset `off`.
template <int D, int MODE, bool S8>
struct StepIn {
    static constexpr int K = PathShape<D>::K;
    using M = ModeIO<MODE>;
    static constexpr int PW = (K + 1) / 2;
    static constexpr int REGS = PW + (M::IN_LO ? PW : 0) + (M::IN_S ? (S8 ? PW : K) : 0);
    Regs<PW> mc;
    Regs<M::IN_LO ? PW : 0> lo;
    Regs<M::IN_S ? (S8 ? PW : K) : 0> s;

    template <int N>
    static __device__ __forceinline__ void zero(uint32_t (&r)[N]) {
#pragma unroll
        for (int i = 0; i < N; ++i) r[i] = 0u;
    }

    __device__ __forceinline__ void load(const LaneBases& lb, uint32_t off) {
        const uint8_t* p = at(lb.pairs, off);
        if (SGM_GUARD(p, 2 * K, lb.lo, lb.hi, 201))
            ldg_pairs<K, true>(p, mc.r);
        else
            zero(mc.r);
        if constexpr (M::IN_LO) {
            const uint8_t* q = at(lb.lx, off);
            if (SGM_GUARD(q, 2 * K, lb.lo, lb.hi, 202))
                ldg_pairs<K, false>(q, lo.r);
            else
                zero(lo.r);
        }
        if constexpr (M::IN_S) {
            if constexpr (S8) {
                if (SGM_GUARD(p + D, 2 * K, lb.lo, lb.hi, 203))
                    ldg_pairs<K, false>(p + D, s.r);
                else
                    zero(s.r);
            } else {
                const uint8_t* q = at(lb.words, off);
                if (SGM_GUARD(q, 4 * K, lb.lo, lb.hi, 203))
                    ldg_words<K>(reinterpret_cast<const uint32_t*>(q), s.r);
                else
                    zero(s.r);
            }
        }
    }
};

// Jump penalties of the post form, P2x2 by |I(p) - I(q)| (see SweepArgs).
__device__ __forceinline__ uint32_t* post_p2_table() {
    __shared__ uint32_t tab[256];
    return tab;
}

// Fills the table; every thread of the block calls it before any early exit.
template <int POST>
__device__ __forceinline__ void post_init(const SweepArgs& a) {
    if constexpr (POST != 0) {
        uint32_t* tab = post_p2_table();
        const int P1 = static_cast<int>(a.P1x2 & 0xffffu), P2 = static_cast<int>(a.P2x2 & 0xffffu);
        for (int g = threadIdx.x; g < 256; g += blockDim.x) {
            int v = P2;
            if (a.ap2) {
                v = P2 / (1 + g);
                v = v > P1 ? v : P1;
            }
            tab[g] = static_cast<uint32_t>(v) * 0x10001u;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Walk geometry.  A cursor names the pixel of one step; `advance` moves it to
// the next pixel of the walk.
// ---------------------------------------------------------------------------
// Pixels of a row walk: x = x0 + dx * i in row y.
struct RowGeo {
    static constexpr bool kResets = false;
    static constexpr bool kLinear = true;  // consecutive pixels are step_pix() apart
    int rowbase, x0, dx;
    __device__ __forceinline__ int step_pix() const { return dx; }
    struct Cursor {
        int pix;
    };
    __device__ __forceinline__ Cursor start() const { return Cursor{rowbase + x0}; }
    __device__ __forceinline__ void advance(Cursor& c) const { c.pix += dx; }
    // the pixel before the start on the path (unclamped; may lie outside)
    __device__ __forceinline__ int before_start() const { return rowbase + x0 - dx; }
    // the pixel of step i
    __device__ __forceinline__ int pix_at(int i) const { return rowbase + x0 + dx * i; }
};

// Pixels of a column (RX = 0) or wrapped-diagonal (RX = +1/-1) walk:
// y = y0 + dy * i, x = (c + RX * y) mod W.
template <int RX>
struct ColGeo {
    static constexpr bool kResets = RX != 0;
    static constexpr bool kLinear = RX == 0;
    int W, H, c, y0, dy;
    __device__ __forceinline__ int step_pix() const { return dy * W; }
    struct Cursor {
        int pix, x, y;
    };
    __device__ __forceinline__ int x_at(int y) const {
        if constexpr (RX == 0) {
            return c;
        } else {
            int v = (c + RX * y) % W;
            return v < 0 ? v + W : v;
        }
    }
    __device__ __forceinline__ Cursor start() const {
        const int x = x_at(y0);
        return Cursor{y0 * W + x, x, y0};
    }
    // the pixel of step i
    __device__ __forceinline__ int pix_at(int i) const {
        const int y = y0 + dy * i;
        return y * W + x_at(y);
    }
    // the pixel before the start on the path (its row may lie outside)
    __device__ __forceinline__ int before_start() const {
        const int y = y0 - dy;
        if (y < 0 || y >= H) return y0 * W + x_at(y0);  // a path start: any pixel will do
        return y * W + x_at(y);
    }
    __device__ __forceinline__ void advance(Cursor& k) const {
        if constexpr (RX == 0) {
            k.pix += dy * W;
        } else {
            int x = k.x + RX * dy;
            x = x >= W ? x - W : (x < 0 ? x + W : x);
            k.y += dy;
            k.x = x;
            k.pix = k.y * W + x;
        }
    }
    // the previous pixel of the path at the cursor lies outside the image
    __device__ __forceinline__ bool starts(const Cursor& k) const {
        if (dy > 0) return k.y == 0 || (RX == 1 && k.x == 0) || (RX == -1 && k.x == W - 1);
        return k.y == H - 1 || (RX == 1 && k.x == W - 1) || (RX == -1 && k.x == 0);
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

// Lines (rows or columns) per block: with G = 32 a pair takes two warps.
template <int D, bool PAIR>
constexpr int lines_per_block() {
    return PathShape<D>::G == 32 ? (PAIR ? kWarpsPerBlock / 2 : kWarpsPerBlock) : (PAIR ? kWarpsPerBlock : 2 * kWarpsPerBlock);
}

// Which line and direction this warp (or, for G = 16, this lane's half) walks.
template <int D, bool PAIR>
struct LaneRole {
    int line, dir, pl;
    __device__ __forceinline__ LaneRole(int bx) {
        constexpr int G = PathShape<D>::G;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        pl = lane & (G - 1);
        if constexpr (G == 16 && PAIR) {
            line = bx * kWarpsPerBlock + warp;
            dir = lane >> 4;
        } else if constexpr (G == 16) {
            // 2-path mode: the second half-warp carries the next line
            line = (bx * kWarpsPerBlock + warp) * 2 + (lane >> 4);
            dir = 0;
        } else if constexpr (PAIR) {
            line = bx * (kWarpsPerBlock / 2) + (warp >> 1);
            dir = warp & 1;
        } else {
            line = bx * kWarpsPerBlock + warp;
            dir = 0;
        }
    }
};

// One phase of this warp's path(s).  g / n_own: this lane's path and its step
// count; n_other: the step count of the warp's other path (G = 16), else
// n_own.  DBG: a winner-take-all walk also writes S in natural order to
// a.Sdbg.
// PFB: the registers one chunk of prefetched inputs may take (prefetch_steps).
template <int D, int MODE, bool S8, class Geo, bool DBG = false, int POST = 0, int PFB = 48>
__device__ __forceinline__ void walk(Chain<PathShape<D>::G, PathShape<D>::K>& ch, const Geo& g, int n_own,
                                     int n_other, const SweepArgs& a, int pl) {
    constexpr int G = PathShape<D>::G, K = PathShape<D>::K;
    using M = ModeIO<MODE>;
    using In = StepIn<D, MODE, S8>;
    constexpr int PF = prefetch_steps(In::REGS, PFB);
    const int n_min = min(n_own, n_other), n_max = max(n_own, n_other);
    const uint32_t RB = static_cast<uint32_t>(a.RB);
    const LaneBases lb = lane_bases<D>(a, pl);
    // Every load is issued unconditionally: past the end of this lane's path it
    // re-reads the path's first pixel (a predicated load would keep the old
    // register value alive and make the step wait for the load).
    In nxt[PF];
    typename Geo::Cursor ld = g.start(), cur = ld;
    const int pix0 = n_own > 0 ? ld.pix : 0;  // an empty path (W or H of 1) may start outside the image
    // Walks with a constant pixel stride advance 32-bit record offsets
    // directly (one add per step instead of an index update and a multiply).
    const uint32_t off0 = static_cast<uint32_t>(pix0) * RB;
    const uint32_t doff = Geo::kLinear ? static_cast<uint32_t>(g.step_pix()) * RB : 0u;
    uint32_t off_ld = static_cast<uint32_t>(ld.pix) * RB, off_cur = off_ld;
    auto prefetch = [&](In& b, int i, bool clamp) {
        if constexpr (Geo::kLinear) {
            b.load(lb, (clamp && i >= n_own) ? off0 : off_ld);
            off_ld += doff;
        } else {
            const int pix = (clamp && i >= n_own) ? pix0 : ld.pix;
            b.load(lb, static_cast<uint32_t>(pix) * RB);
            g.advance(ld);
        }
    };
    // Post form: the jump penalty of every step comes from the base image.
    // Lane pl of a path loads the intensity of step i0 + pl of each chunk
    // (one chunk ahead, like the records) and turns it into that step's
    // penalty at the chunk's start; step k then takes lane k's penalty with
    // one shuffle.  im_last carries the intensity of the step before the chunk.
    static_assert(PF <= G, "one lane per step of a chunk");
    auto img_at_step = [&](int i) -> uint32_t {
        const int pix = i < n_own ? g.pix_at(i) : pix0;
        return SGM_GUARD_INDEX(pix, static_cast<long long>(a.W) * a.H, 214) ? __ldg(a.img + pix) : 0u;
    };
    uint32_t im_nxt = 0, im_last = 0, p2_lane = 0;
    if constexpr (POST != 0) {
        im_nxt = img_at_step(pl);
        im_last = __ldg(a.img + min(max(g.before_start(), 0), a.W * a.H - 1));
    }
#pragma unroll
    for (int k = 0; k < PF; ++k) prefetch(nxt[k], k, true);
    // 16-bit keys: byte sums of 2 or 4 paths stay below 511, so S * D + d
    // fits 16 bits for D <= 128
    constexpr bool KEY16 = S8 && D <= 128;
    uint32_t dconst[K];
    if constexpr (M::WTA) wta_consts<K, KEY16>(pl, D, dconst);

    // one step of the recurrence at `cur` and its outputs
    auto body = [&](const In& in, bool active, int k) {
        if constexpr (Geo::kResets) {
            if (g.starts(cur)) ch.reset();
        }
        uint32_t mc[K], L[K];
        unpack_regs<K>(in.mc.r, mc);
        const uint32_t p2x2 = POST != 0 ? __shfl_sync(0xffffffffu, p2_lane, k, G) : a.P2x2;
        ch.step(mc, a.P1x2, p2x2, L);
        const uint32_t off = Geo::kLinear ? off_cur : static_cast<uint32_t>(cur.pix) * RB;
        if constexpr (M::OUT_LX) {
            if (active && SGM_GUARD(at(lb.lx, off), 2 * K, lb.lo, lb.hi, 204))
                st_pairs<K>(at(lb.lx, off), pack_pairs<K>(L));
        } else if constexpr (MODE == kSumH && S8) {
            // byte sums: every L_r <= 127 here (sum_fits_u8), so the paired
            // bytes of L and of the stored L_r add without carries
            U8Pairs<K> o = pack_pairs<K>(L);
#pragma unroll
            for (int q = 0; q < (K + 1) / 2; ++q) o.r[q] += in.lo.r[q];
            if (active && SGM_GUARD(at(lb.pairs, off) + D, 2 * K, lb.lo, lb.hi, 205))
                st_pairs<K>(at(lb.pairs, off) + D, o);
        } else {
            uint32_t s[K];
#pragma unroll
            for (int j = 0; j < K; ++j) s[j] = L[j];
            if constexpr (M::IN_LO) {
                uint32_t lo[K];
                unpack_regs<K>(in.lo.r, lo);
#pragma unroll
                for (int j = 0; j < K; ++j) s[j] += lo[j];
            }
            if constexpr (M::IN_S) {
                if constexpr (S8) {
                    uint32_t t[K];
                    unpack_regs<K>(in.s.r, t);
#pragma unroll
                    for (int j = 0; j < K; ++j) s[j] += t[j];
                } else {
#pragma unroll
                    for (int j = 0; j < K; ++j) s[j] += in.s.r[j];
                }
            }
            if constexpr (M::OUT_S) {
                if (active) {
                    if constexpr (S8) {
                        if (SGM_GUARD(at(lb.pairs, off) + D, 2 * K, lb.lo, lb.hi, 206))
                            st_pairs<K>(at(lb.pairs, off) + D, pack_pairs<K>(s));
                    } else {
                        if (SGM_GUARD(at(lb.words, off), 4 * K, lb.lo, lb.hi, 206))
                            st_words<K>(reinterpret_cast<uint32_t*>(at(lb.words, off)), s);
                    }
                }
            }
            if constexpr (M::WTA) {
                const uint32_t key = ch.path_min(wta_key<K, D, KEY16>(s, dconst));
                if (active && pl == 0 && SGM_GUARD_INDEX(cur.pix, static_cast<long long>(a.W) * a.H, 207))
                    a.raw[cur.pix] = wta_disparity<D, KEY16>(key);
                if constexpr (POST != 0) {
                    if (a.sub) {  // uniform: S at the winner's neighbours for the sub-pixel step
                        const int d = wta_disparity<D, KEY16>(key);
                        const uint32_t Sd = KEY16 ? key / static_cast<uint32_t>(D) : key >> 8;
                        // S(e) from the lane holding disparity e: word i = e mod D/2 in
                        // lane i / K, slot i % K, the high half for e >= D/2
                        auto s_at = [&](int e) -> uint32_t {
                            const int i = e < D / 2 ? e : e - D / 2, src = i / K, jj = i - src * K;
                            uint32_t w = s[0];
#pragma unroll
                            for (int j = 1; j < K; ++j) w = (jj == j) ? s[j] : w;
                            w = __shfl_sync(0xffffffffu, w, src, G);
                            return e < D / 2 ? (w & 0xffffu) : (w >> 16);
                        };
                        const uint32_t sm = s_at(d > 0 ? d - 1 : 0), sp = s_at(d + 1 < D ? d + 1 : d);
                        const uint32_t al = d > 0 ? sm - Sd : 0u;
                        const uint32_t ga = d + 1 < D ? sp - Sd : 0u;
                        if (active && pl == 0 && SGM_GUARD_INDEX(cur.pix, static_cast<long long>(a.W) * a.H, 208))
                            a.sub[cur.pix] = al | ga << 16;
                    }
                }
                if (DBG && active) {  // debug: natural-order S
                    const size_t p = static_cast<size_t>(cur.pix);
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        const int i = pl * K + j;
                        if (SGM_GUARD_INDEX(static_cast<long long>(p * D + i + D / 2),
                                            static_cast<long long>(a.W) * a.H * D, 209)) {
                            a.Sdbg[p * D + i] = static_cast<uint16_t>(s[j] & 0xffffu);
                            a.Sdbg[p * D + i + D / 2] = static_cast<uint16_t>(s[j] >> 16);
                        }
                    }
                }
            }
        }
    };

    for (int i0 = 0; i0 < n_max; i0 += PF) {
        In in[PF];
#pragma unroll
        for (int k = 0; k < PF; ++k) in[k] = nxt[k];
        if constexpr (POST != 0) {
            const uint32_t im = im_nxt;
            im_nxt = img_at_step(i0 + PF + pl);
            uint32_t prev = __shfl_up_sync(0xffffffffu, im, 1, G);
            if (pl == 0) prev = im_last;
            p2_lane = post_p2_table()[abs(static_cast<int>(im) - static_cast<int>(prev))];
            im_last = __shfl_sync(0xffffffffu, im, PF - 1, G);
        }
        if (i0 + 2 * PF <= n_min) {
#pragma unroll
            for (int k = 0; k < PF; ++k) prefetch(nxt[k], i0 + PF + k, false);
        } else {
#pragma unroll
            for (int k = 0; k < PF; ++k) prefetch(nxt[k], i0 + PF + k, true);
        }
        if (n_min - i0 >= PF) {
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                body(in[k], true, k);
                g.advance(cur);
                off_cur += doff;
            }
        } else {
            // last steps: a path with fewer steps keeps its state through the extra ones
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const int i = i0 + k;
                if (i < n_max) {  // warp-uniform
                    // every lane runs the step (it holds warp-synchronous
                    // exchanges); a finished path then takes its state back
                    const Chain<G, K> saved = ch;
                    body(in[k], i < n_own, k);
                    if (i >= n_own) ch = saved;
                    g.advance(cur);
                    off_cur += doff;
                }
            }
        }
    }
}

// Path state of one lane between the two phases of a pair that run in
// different launches: its K words, the two neighbour words and m, at
// a.state + ((line * (warps per line) + warp of the line) * 32 + lane) * (K + 3).
template <int D>
__device__ __forceinline__ uint32_t* state_slot(const SweepArgs& a, int line, int dir) {
    constexpr int G = PathShape<D>::G, K = PathShape<D>::K;
    return a.state + ((static_cast<size_t>(line) * (2 / PathShape<D>::PPW) + (G == 32 ? dir : 0)) * 32 +
                      (threadIdx.x & 31)) * (K + 3);
}

template <int G, int K>
__device__ __forceinline__ void save_state(const Chain<G, K>& ch, uint32_t* st) {
#pragma unroll
    for (int j = 0; j < K; ++j) st[j] = ch.w[j];
    st[K] = ch.up;
    st[K + 1] = ch.dn;
    st[K + 2] = ch.mpx2;
}

template <int G, int K>
__device__ __forceinline__ void load_state(Chain<G, K>& ch, const uint32_t* st) {
#pragma unroll
    for (int j = 0; j < K; ++j) ch.w[j] = __ldcg(st + j);
    ch.up = __ldcg(st + K);
    ch.dn = __ldcg(st + K + 1);
    ch.mpx2 = __ldcg(st + K + 2);
}

// ---------------------------------------------------------------------------
// Horizontal axis: one row per line; direction A walks left to right,
// direction B right to left.  Phase 1: A covers x < W/2, B covers x >= W/2,
// both storing L in the stored-L_r field.  Phase 2: each covers the other
// half and writes S = own L + stored L (WTA = false) or finishes with Eq. 4,
// raw = argmin_d (S + own L + stored L), when S already holds the vertical
// pair (WTA = true).  PH: 0 = both phases in one launch, 1 = phase 1 (saving
// the path state), 2 = phase 2 (restoring it).  Without `pair` (2-path mode)
// A covers the whole row and writes S = L_LR.
// ---------------------------------------------------------------------------
template <int D, bool PAIR, bool S8, int PH = 0, bool WTA = false, bool DBG = false, int POST = 0, int PFB = 48>
__device__ __forceinline__ void sweep_h_body(const SweepArgs& a, int bx) {
    constexpr int G = PathShape<D>::G, K = PathShape<D>::K;
    const LaneRole<D, PAIR> r(bx);
    const int y = r.line;
    // whole warp (and its pair): every exchange below is local to them; in
    // 2-path mode with 16-lane paths the warp's lines are y & ~1 and y | 1
    if ((G == 16 && !PAIR ? (y & ~1) : y) >= a.H) return;
    const bool in_b = r.dir != 0;
    const int W = a.W, rowbase = y * W;
    Chain<G, K> ch;
    ch.init(threadIdx.x & 31);
    if constexpr (!PAIR) {
        // a half-warp past the last row walks nothing (it still joins the exchanges)
        const bool valid = y < a.H;
        const RowGeo g{valid ? rowbase : 0, 0, 1};
        const int n = valid ? W : 0;
        walk<D, kSingleH, S8, RowGeo, false, POST, PFB>(ch, g, n, G == 16 ? ((y ^ 1) < a.H ? W : 0) : n, a, r.pl);
    } else {
        const int Wm = W / 2;
        if constexpr (PH != 2) {
            const RowGeo g = in_b ? RowGeo{rowbase, W - 1, -1} : RowGeo{rowbase, 0, 1};
            const int nA = Wm, nB = W - Wm;
            walk<D, kStoreL, S8, RowGeo, false, POST, PFB>(ch, g, in_b ? nB : nA,
                                                           G == 16 ? (in_b ? nA : nB) : (in_b ? nB : nA), a, r.pl);
        }
        if constexpr (PH == 1) {
            uint32_t* st = state_slot<D>(a, y, r.dir);
            if (SGM_GUARD(st, 4 * (K + 3), a.state, a.state_end, 210)) save_state(ch, st);
            return;
        }
        if constexpr (PH == 2) {
            const uint32_t* st = state_slot<D>(a, y, r.dir);
            if (SGM_GUARD(st, 4 * (K + 3), a.state, a.state_end, 211)) load_state(ch, st);
        }
        if constexpr (PH == 0) pair_barrier<D>();
        {
            const RowGeo g = in_b ? RowGeo{rowbase, Wm - 1, -1} : RowGeo{rowbase, Wm, 1};
            const int nA = W - Wm, nB = Wm;
            walk<D, WTA ? kWta2 : kSumH, S8, RowGeo, DBG, POST, PFB>(
                ch, g, in_b ? nB : nA, G == 16 ? (in_b ? nA : nB) : (in_b ? nB : nA), a, r.pl);
        }
    }
}

// Second halves of the horizontal pair with the winner-take-all (4 paths: S
// holds the vertical pair's sums).
template <int D, bool S8, bool DBG, int POST = 0>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_h2_kernel(SweepArgs a) {
    post_init<POST>(a);
    sweep_h_body<D, true, S8, 2, true, DBG, POST>(a, blockIdx.x);
}

template <int D, bool PAIR, bool S8, int POST = 0>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_h_kernel(SweepArgs a) {
    post_init<POST>(a);
    sweep_h_body<D, PAIR, S8, 0, false, false, POST>(a, blockIdx.x);
}

// Work-list forms (batched pairs): many chains in flight, so more warps per
// SM (up to kSweepListMaxPerSM blocks) with half the prefetch registers serve
// better than deep prefetch.  A unit is one block's lines of one pair.
constexpr int kBatchPrefetchBudget = 24;

template <int D, bool PAIR, bool S8>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, kSweepListMaxPerSM)
    sweep_h_list_kernel(const WorkList<SweepArgs>* __restrict__ Lp, uint32_t* __restrict__ next,
                        uint32_t* __restrict__ status) {
    const WorkList<SweepArgs> L = *Lp;
    int p, u;
    while (take_unit(L, next, p, u)) {
        const SweepArgs a = L.job[p];
        if (a.D != D) {
            report_bad_job(status);
            continue;
        }
        sweep_h_body<D, PAIR, S8, 0, false, false, 0, kBatchPrefetchBudget>(a, u);
    }
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
// SUMV: a pair that does not finish with Eq. 4 writes S = L + stored L (the
// first pair to write S) instead of adding into S.
template <int D, int RX, int PH, bool WTA, bool PAIR, bool S8, bool DBG = false, bool SUMV = false, int POST = 0,
          int PFB = 48>
__device__ __forceinline__ void sweep_v_body(const SweepArgs& a, int bx) {
    constexpr int G = PathShape<D>::G, K = PathShape<D>::K;
    const LaneRole<D, PAIR> r(bx);
    const int c = r.line;
    if ((G == 16 && !PAIR ? (c & ~1) : c) >= a.W) return;  // whole warp (and its pair)
    const bool in_b = r.dir != 0;
    const int W = a.W, H = a.H;
    using Geo = ColGeo<RX>;
    Chain<G, K> ch;
    const int lane = threadIdx.x & 31;
    ch.init(lane);
    if constexpr (!PAIR) {
        const bool valid = c < W;
        const int n = valid ? H : 0;
        walk<D, kSingleWta, S8, Geo, DBG, POST, PFB>(ch, Geo{W, H, valid ? c : 0, 0, 1}, n,
                                                     G == 16 ? ((c ^ 1) < W ? H : 0) : n, a, r.pl);
    } else {
        const int Hm = H / 2;
        if constexpr (PH != 2) {
            const Geo g = in_b ? Geo{W, H, c, H - 1, -1} : Geo{W, H, c, 0, 1};
            const int nA = Hm, nB = H - Hm;
            walk<D, kStoreL, S8, Geo, false, POST, PFB>(ch, g, in_b ? nB : nA,
                                                        G == 16 ? (in_b ? nA : nB) : (in_b ? nB : nA), a, r.pl);
        }
        if constexpr (PH == 1) {
            uint32_t* st = state_slot<D>(a, c, r.dir);
            if (SGM_GUARD(st, 4 * (K + 3), a.state, a.state_end, 212)) save_state(ch, st);
            return;
        }
        if constexpr (PH == 2) {
            const uint32_t* st = state_slot<D>(a, c, r.dir);
            if (SGM_GUARD(st, 4 * (K + 3), a.state, a.state_end, 213)) load_state(ch, st);
        }
        if constexpr (PH != 1) {
            if constexpr (PH == 0) pair_barrier<D>();
            const Geo g = in_b ? Geo{W, H, c, Hm - 1, -1} : Geo{W, H, c, Hm, 1};
            const int nA = H - Hm, nB = Hm;
            walk<D, WTA ? kWta2 : (SUMV ? kSumH : kAcc), S8, Geo, DBG, POST, PFB>(
                ch, g, in_b ? nB : nA, G == 16 ? (in_b ? nA : nB) : (in_b ? nB : nA), a, r.pl);
        }
    }
}

template <int D, int RX, int PH, bool WTA, bool PAIR, bool S8, bool DBG = false, int POST = 0>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_v_kernel(SweepArgs a) {
    post_init<POST>(a);
    sweep_v_body<D, RX, PH, WTA, PAIR, S8, DBG, false, POST>(a, blockIdx.x);
}

// Work-list form: both phases in one unit (PH = 0).
template <int D, int RX, bool WTA, bool PAIR, bool S8>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, kSweepListMaxPerSM)
    sweep_v_list_kernel(const WorkList<SweepArgs>* __restrict__ Lp, uint32_t* __restrict__ next,
                        uint32_t* __restrict__ status) {
    const WorkList<SweepArgs> L = *Lp;
    int p, u;
    while (take_unit(L, next, p, u)) {
        const SweepArgs a = L.job[p];
        if (a.D != D) {
            report_bad_job(status);
            continue;
        }
        sweep_v_body<D, RX, 0, WTA, PAIR, S8, false, false, 0, kBatchPrefetchBudget>(a, u);
    }
}

// The horizontal pair and the vertical-type first halves in one grid: one
// block distribution over the SMs for all of them (two kernels sharing the
// SMs through concurrent streams ran far slower than either alone).  NV = 1
// (4 paths: the vertical pair only) keeps the diagonal code out of the kernel.
template <int D, bool S8, int NV, int POST = 0>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_first_kernel(const __grid_constant__ FirstStageArgs f) {
    post_init<POST>(f.h);
    const int b = blockIdx.x;
    if (b < f.start[1]) {
        sweep_h_body<D, true, S8, 0, false, false, POST>(f.h, b);
        return;
    }
    if constexpr (NV == 1) {
        sweep_v_body<D, 0, 1, false, true, S8, false, false, POST>(f.v[0], b - f.start[1]);
    } else {
        for (int k = 0; k < NV; ++k) {
            if (b < f.start[k + 2]) {
                const SweepArgs& v = f.v[k];
                const int bx = b - f.start[k + 1];
                if (v.rx == 0)
                    sweep_v_body<D, 0, 1, false, true, S8, false, false, POST>(v, bx);
                else if (v.rx > 0)
                    sweep_v_body<D, 1, 1, false, true, S8, false, false, POST>(v, bx);
                else
                    sweep_v_body<D, -1, 1, false, true, S8, false, false, POST>(v, bx);
                return;
            }
        }
    }
}

// 4 paths, first stage: the horizontal pair's first halves (saving their
// state) beside the whole vertical pair, which writes S = L_TB + L_BT.  The
// vertical chains (H steps) are longer than the horizontal first halves (W/2
// steps at 640x480), so the grid stays busy to the end of the launch; the
// horizontal second halves then finish with Eq. 4 (sweep_h2_kernel).
template <int D, bool S8, int POST = 0>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) sweep_first4_kernel(const __grid_constant__ FirstStageArgs f) {
    post_init<POST>(f.h);
    const int b = blockIdx.x;
    if (b < f.start[1])
        sweep_h_body<D, true, S8, 1, false, false, POST>(f.h, b);
    else
        sweep_v_body<D, 0, 0, false, true, S8, false, true, POST>(f.v[0], b - f.start[1]);
}

// ---------------------------------------------------------------------------
// Per-D entry points, instantiated one D per translation unit.  The sums are
// bytes (S8) in 2-path mode always and in 4-path mode when SweepArgs::s8 is
// set; 8-path sums are u16 words.
// ---------------------------------------------------------------------------
template <int D>
struct SweepD {
    static int blocks(int lines, bool pair) {
        const int per = pair ? lines_per_block<D, true>() : lines_per_block<D, false>();
        return (lines + per - 1) / per;
    }

    // No kernel needs an attribute (no dynamic shared memory).
    static cudaError_t set_attrs() { return cudaSuccess; }

    static cudaError_t launch_h(const SweepArgs& a, cudaStream_t s) {
        const dim3 grid(blocks(a.H, a.pair)), block(32 * kWarpsPerBlock);
        if (a.post) {  // post form: 2-path left-to-right only
            if (a.pair) return cudaErrorInvalidValue;
            sweep_h_kernel<D, false, true, 1><<<grid, block, 0, s>>>(a);
            return cudaGetLastError();
        }
        if (!a.pair)
            sweep_h_kernel<D, false, true><<<grid, block, 0, s>>>(a);
        else if (a.s8)
            sweep_h_kernel<D, true, true><<<grid, block, 0, s>>>(a);
        else
            sweep_h_kernel<D, true, false><<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }

    static cudaError_t launch_first(FirstStageArgs& f, cudaStream_t s) {
        f.start[0] = 0;
        f.start[1] = blocks(f.h.H, true);
        for (int k = 0; k < f.nv; ++k) f.start[k + 2] = f.start[k + 1] + blocks(f.v[k].W, true);
        const dim3 block(32 * kWarpsPerBlock);
        const int grid = f.start[f.nv + 1];
        if (f.h.post) {  // post form: 8 paths only
            if (f.nv != 3 || f.h.s8) return cudaErrorInvalidValue;
            sweep_first_kernel<D, false, 3, 1><<<grid, block, 0, s>>>(f);
            return cudaGetLastError();
        }
        if (f.nv == 1 && f.h.s8)
            sweep_first_kernel<D, true, 1><<<grid, block, 0, s>>>(f);
        else if (f.nv == 1)
            sweep_first_kernel<D, false, 1><<<grid, block, 0, s>>>(f);
        else
            sweep_first_kernel<D, false, 3><<<grid, block, 0, s>>>(f);
        return cudaGetLastError();
    }

    static cudaError_t launch_first4(FirstStageArgs& f, cudaStream_t s) {
        f.start[0] = 0;
        f.start[1] = blocks(f.h.H, true);
        f.start[2] = f.start[1] + blocks(f.v[0].W, true);
        const dim3 block(32 * kWarpsPerBlock);
        if (f.h.post && f.h.s8)
            sweep_first4_kernel<D, true, 1><<<f.start[2], block, 0, s>>>(f);
        else if (f.h.post)
            sweep_first4_kernel<D, false, 1><<<f.start[2], block, 0, s>>>(f);
        else if (f.h.s8)
            sweep_first4_kernel<D, true><<<f.start[2], block, 0, s>>>(f);
        else
            sweep_first4_kernel<D, false><<<f.start[2], block, 0, s>>>(f);
        return cudaGetLastError();
    }

    static cudaError_t launch_h2(const SweepArgs& a, cudaStream_t s) {
        const dim3 grid(blocks(a.H, true)), block(32 * kWarpsPerBlock);
        if (a.post && a.s8)
            sweep_h2_kernel<D, true, false, 1><<<grid, block, 0, s>>>(a);
        else if (a.post)
            sweep_h2_kernel<D, false, false, 1><<<grid, block, 0, s>>>(a);
        else if (a.s8 && a.Sdbg)
            sweep_h2_kernel<D, true, true><<<grid, block, 0, s>>>(a);
        else if (a.s8)
            sweep_h2_kernel<D, true, false><<<grid, block, 0, s>>>(a);
        else if (a.Sdbg)
            sweep_h2_kernel<D, false, true><<<grid, block, 0, s>>>(a);
        else
            sweep_h2_kernel<D, false, false><<<grid, block, 0, s>>>(a);
        return cudaGetLastError();
    }

    static cudaError_t launch_h_list(const ListLaunch& l, cudaStream_t s) {
        const auto* L = static_cast<const WorkList<SweepArgs>*>(l.list);
        const dim3 block(32 * kWarpsPerBlock);
        if (!l.pair)
            sweep_h_list_kernel<D, false, true><<<l.grid, block, 0, s>>>(L, l.next, l.status);
        else if (l.s8)
            sweep_h_list_kernel<D, true, true><<<l.grid, block, 0, s>>>(L, l.next, l.status);
        else
            sweep_h_list_kernel<D, true, false><<<l.grid, block, 0, s>>>(L, l.next, l.status);
        return cudaGetLastError();
    }

    static cudaError_t launch_v_list(const ListLaunch& l, cudaStream_t s) {
        const auto* L = static_cast<const WorkList<SweepArgs>*>(l.list);
        const dim3 block(32 * kWarpsPerBlock);
        if (!l.pair)
            sweep_v_list_kernel<D, 0, true, false, true><<<l.grid, block, 0, s>>>(L, l.next, l.status);
        else if (l.rx == 0 && l.s8)
            sweep_v_list_kernel<D, 0, true, true, true><<<l.grid, block, 0, s>>>(L, l.next, l.status);
        else if (l.rx == 0)
            sweep_v_list_kernel<D, 0, true, true, false><<<l.grid, block, 0, s>>>(L, l.next, l.status);
        else if (l.rx > 0)
            sweep_v_list_kernel<D, 1, false, true, false><<<l.grid, block, 0, s>>>(L, l.next, l.status);
        else
            sweep_v_list_kernel<D, -1, false, true, false><<<l.grid, block, 0, s>>>(L, l.next, l.status);
        return cudaGetLastError();
    }

    // Vertical-type sweeps of a pair in phase 1 or 2 (or both, phase 0).
    template <int RX, bool WTA, bool S8>
    static void launch_v_rx(const SweepArgs& a, dim3 grid, dim3 block, cudaStream_t s) {
        if (WTA && a.Sdbg && a.phase == 2)
            sweep_v_kernel<D, RX, 2, WTA, true, S8, true><<<grid, block, 0, s>>>(a);
        else if (a.phase == 1)
            sweep_v_kernel<D, RX, 1, false, true, S8><<<grid, block, 0, s>>>(a);
        else if (a.phase == 2)
            sweep_v_kernel<D, RX, 2, WTA, true, S8><<<grid, block, 0, s>>>(a);
        else
            sweep_v_kernel<D, RX, 0, WTA, true, S8><<<grid, block, 0, s>>>(a);
    }

    static cudaError_t launch_v(const SweepArgs& a, cudaStream_t s) {
        const dim3 grid(blocks(a.W, a.pair)), block(32 * kWarpsPerBlock);
        if (a.post) {
            // post form: the 2-path top-to-bottom sweep, and the second halves
            // of the three vertical-type pairs of 8 paths (u16 sums)
            if (!a.pair)
                sweep_v_kernel<D, 0, 0, true, false, true, false, 1><<<grid, block, 0, s>>>(a);
            else if (a.phase != 2 || a.s8)
                return cudaErrorInvalidValue;
            else if (a.rx == 0)
                sweep_v_kernel<D, 0, 2, true, true, false, false, 1><<<grid, block, 0, s>>>(a);
            else if (a.rx > 0)
                sweep_v_kernel<D, 1, 2, false, true, false, false, 1><<<grid, block, 0, s>>>(a);
            else
                sweep_v_kernel<D, -1, 2, false, true, false, false, 1><<<grid, block, 0, s>>>(a);
            return cudaGetLastError();
        }
        if (!a.pair && a.Sdbg)
            sweep_v_kernel<D, 0, 0, true, false, true, true><<<grid, block, 0, s>>>(a);
        else if (!a.pair)
            sweep_v_kernel<D, 0, 0, true, false, true><<<grid, block, 0, s>>>(a);
        else if (a.rx == 0 && a.s8)
            launch_v_rx<0, true, true>(a, grid, block, s);
        else if (a.rx == 0)
            launch_v_rx<0, true, false>(a, grid, block, s);
        else if (a.rx > 0)
            launch_v_rx<1, false, false>(a, grid, block, s);
        else
            launch_v_rx<-1, false, false>(a, grid, block, s);
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
SGM_INTERNAL cudaError_t sweep_launch_h_list(const ListLaunch& l, cudaStream_t s);
template <int D>
SGM_INTERNAL cudaError_t sweep_launch_first4(FirstStageArgs& f, cudaStream_t s);
template <int D>
SGM_INTERNAL cudaError_t sweep_launch_h2(const SweepArgs& a, cudaStream_t s);
template <int D>
SGM_INTERNAL cudaError_t sweep_launch_v_list(const ListLaunch& l, cudaStream_t s);

#define SGM_INSTANTIATE_SWEEPS(D)                                                               \
    template <>                                                                                 \
    SGM_INTERNAL cudaError_t sweep_set_attrs<D>() {                                             \
        return SweepD<D>::set_attrs();                                                          \
    }                                                                                           \
    template <>                                                                                 \
    SGM_INTERNAL cudaError_t sweep_launch_h<D>(const SweepArgs& a, cudaStream_t s) {            \
        return SweepD<D>::launch_h(a, s);                                                       \
    }                                                                                           \
    template <>                                                                                 \
    SGM_INTERNAL cudaError_t sweep_launch_v<D>(const SweepArgs& a, cudaStream_t s) {            \
        return SweepD<D>::launch_v(a, s);                                                       \
    }                                                                                           \
    template <>                                                                                 \
    SGM_INTERNAL cudaError_t sweep_launch_first<D>(FirstStageArgs & f, cudaStream_t s) {        \
        return SweepD<D>::launch_first(f, s);                                                   \
    }                                                                                           \
    template <>                                                                                 \
    SGM_INTERNAL cudaError_t sweep_launch_h_list<D>(const ListLaunch& l, cudaStream_t s) {      \
        return SweepD<D>::launch_h_list(l, s);                                                  \
    }                                                                                           \
    template <>                                                                                 \
    SGM_INTERNAL cudaError_t sweep_launch_v_list<D>(const ListLaunch& l, cudaStream_t s) {      \
        return SweepD<D>::launch_v_list(l, s);                                                  \
    }                                                                                           \
    template <>                                                                                 \
    SGM_INTERNAL cudaError_t sweep_launch_first4<D>(FirstStageArgs & f, cudaStream_t s) {       \
        return SweepD<D>::launch_first4(f, s);                                                  \
    }                                                                                           \
    template <>                                                                                 \
    SGM_INTERNAL cudaError_t sweep_launch_h2<D>(const SweepArgs& a, cudaStream_t s) {           \
        return SweepD<D>::launch_h2(a, s);                                                      \
    }

}  // namespace sgm

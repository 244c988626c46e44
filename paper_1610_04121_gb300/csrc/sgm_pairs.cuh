// Path aggregation (Eq. 3), the sum S and the winner-take-all disparity
// (Eq. 4) of the 4-path SGM of arXiv 1610.04121 with two lines per warp, for
// sm_103a.
//
// Parallel scheme (Section 3.2's CTA-to-warp conversion, with the paper's
// byte-SIMD replaced by packed 16-bit lanes): a warp carries two adjacent
// lines of one direction, line A in the low u16 half of every packed word
// and line B in the high half.  Lane l holds the path costs of disparities
// d = K l + j, j < K = D / 32, of both lines, so word j of lane l is
// (L_A(d), L_B(d)).  The disparity neighbours d - 1 and d + 1 sit in the
// neighbouring words of the lane, or one lane over (two shuffles per step);
// the two per-line minima m(q) are two warp reductions.  No byte of a word
// ever crosses into the other line's half: every value stays below 2^14.
//
// Data layout (sgm_internal.h): every cube lives in quads of 2 x 2 pixels,
// one array per cube, so that a walk in either axis reads one quad (4 K bytes
// per lane) per two steps and writes one quad per two steps of the same walk,
// and the walks of neighbouring line pairs touch neighbouring memory.  Rows and columns
// are padded to even counts; the padding pixels have MC = 0, so a path that
// starts on one (a walk from the bottom or right edge of an odd-sized image)
// passes through it unchanged: from the reset state a zero-cost step leaves
// L = 0 and m = 0, which is the reset state again.
//
// Schedule (4 paths: left-to-right, right-to-left, top-to-bottom,
// bottom-to-top):
//   launch 1  the vertical pair, meeting in the middle (the first halves
//             store L_r, the second halves write S_v = L_TB + L_BT), beside
//             n1 steps of each horizontal direction (storing L_r);
//   launch 2  the rest of each horizontal direction, finishing its pixels
//             with Eq. 4 (S = S_v + L_LR + L_RL), beside a parallel
//             winner-take-all over the columns both horizontal directions
//             passed in launch 1.
// With n1 = min(W, H) the longest chain is max(W, H) steps, against H + W / 2
// for a schedule that finishes one pair before the other starts.
#pragma once

#include "sgm_device.cuh"
#include "sgm_internal.h"

namespace sgm {
namespace pairs {

constexpr uint32_t kInf2 = kInf16 * 0x10001u;
constexpr unsigned kFull = 0xffffffffu;

// Field arrays (sgm_internal.h).
enum Field { kMC = 0, kLV = 1, kLH0 = 2, kLH1 = 3, kSV = 4, kSV1 = 5 };

// One quad register [x0y0, x1y0, x0y1, x1y1] -> the u16x2 word of one step:
// the column pair at row h (vertical walks) or the row pair at column h
// (horizontal walks).
template <bool VERT>
__device__ __forceinline__ uint32_t unq(uint32_t q, int h) {
    return __byte_perm(q, 0u, VERT ? (h ? 0x4342u : 0x4140u) : (h ? 0x4341u : 0x4240u));
}

// The words of half 0 and half 1 of a unit (values below 256) -> one quad register.
template <bool VERT>
__device__ __forceinline__ uint32_t toq(uint32_t w0, uint32_t w1) {
    return __byte_perm(w0, w1, VERT ? 0x6420u : 0x6240u);
}

// N registers from 4N bytes at p (16-byte aligned when N % 4 == 0, 8-byte when N is even).
template <int N, bool NC>
__device__ __forceinline__ void ldv(const uint8_t* p, uint32_t (&r)[N]) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const uint4* q = reinterpret_cast<const uint4*>(p) + i;
            const uint4 v = NC ? __ldg(q) : __ldcg(q);
            r[4 * i] = v.x;
            r[4 * i + 1] = v.y;
            r[4 * i + 2] = v.z;
            r[4 * i + 3] = v.w;
        }
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) {
            const uint2* q = reinterpret_cast<const uint2*>(p) + i;
            const uint2 v = NC ? __ldg(q) : __ldcg(q);
            r[2 * i] = v.x;
            r[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const unsigned* q = reinterpret_cast<const unsigned*>(p) + i;
            r[i] = NC ? __ldg(q) : __ldcg(q);
        }
    }
}

template <int N>
__device__ __forceinline__ void stv(uint8_t* p, const uint32_t (&r)[N]) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i)
            reinterpret_cast<uint4*>(p)[i] = make_uint4(r[4 * i], r[4 * i + 1], r[4 * i + 2], r[4 * i + 3]);
    } else if constexpr (N % 2 == 0) {
#pragma unroll
        for (int i = 0; i < N / 2; ++i) reinterpret_cast<uint2*>(p)[i] = make_uint2(r[2 * i], r[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) reinterpret_cast<unsigned*>(p)[i] = r[i];
    }
}

// 64-bit base + 32-bit record offset in one instruction.
__device__ __forceinline__ uint8_t* at(uint8_t* base, uint32_t off) {
    uint64_t r;
    asm("mad.wide.u32 %0, %1, 1, %2;" : "=l"(r) : "r"(off), "l"(reinterpret_cast<uint64_t>(base)));
    return reinterpret_cast<uint8_t*>(r);
}

// Two chains (lines A and B) of Eq. 3 in one warp.  The first pixel of a path
// starts from the reset state (L = 0, m = 0), which gives L = MC.
template <int K>
struct Chain2 {
    uint32_t w[K];
    uint32_t up, dn;  // word K-1 of lane l-1 and word 0 of lane l+1, exchanged after every step
    uint32_t mpx2;    // (m_A, m_B)
    uint32_t mul_up, add_up, mul_dn, add_dn;

    __device__ __forceinline__ void init(int lane) {
        // d = 0 has no d - 1 (lane 0) and d = D - 1 no d + 1 (lane 31): those
        // neighbours read "infinity" through a multiply-add on the FMA pipe
        mul_up = lane == 0 ? 0u : 1u;
        add_up = lane == 0 ? kInf2 : 0u;
        mul_dn = lane == 31 ? 0u : 1u;
        add_dn = lane == 31 ? kInf2 : 0u;
        reset();
    }

    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = 0u;
        up = dn = 0u;
        mpx2 = 0u;
    }

    __device__ __forceinline__ void exchange() {
        up = __shfl_up_sync(kFull, w[K - 1], 1);
        dn = __shfl_down_sync(kFull, w[0], 1);
    }

    // L(p, d) = MC(p, d) + min(L(q, d), L(q, d-1) + P1, L(q, d+1) + P1, m(q) + P2) - m(q)
    __device__ __forceinline__ void step(const uint32_t (&mc)[K], uint32_t P1x2, uint32_t P2x2) {
        const uint32_t u = up * mul_up + add_up;
        const uint32_t d = dn * mul_dn + add_dn;
        const uint32_t mp2 = mpx2 + P2x2;
        uint32_t L[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t dm1 = j == 0 ? u : w[j - 1];
            const uint32_t dp1 = j == K - 1 ? d : w[j + 1];
            // every candidate is >= m(q) in each half, so the packed subtraction never borrows
            L[j] = vmin2(vmin2(dm1, dp1) + P1x2, vmin2(w[j], mp2)) + mc[j] - mpx2;
        }
        uint32_t r = L[0];
#pragma unroll
        for (int j = 1; j < K; ++j) r = vmin2(r, L[j]);
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = L[j];
        exchange();
        // per-half minima: the 32-bit minimum orders by the high half first
        const uint32_t hi = __reduce_min_sync(kFull, r);
        const uint32_t lo = __reduce_min_sync(kFull, r << 16);
        mpx2 = __byte_perm(lo, hi, 0x7632u);
    }
};

// Winner-take-all (Eq. 4) of two pixels at once: S holds (S_A(d), S_B(d)) for
// the lane's disparities; returns (d_A, d_B) in the two u16 halves, the
// lowest d among equal minima.  KEY16: S * D + d fits 16 bits, so one packed
// multiply-add makes both keys; else 32-bit keys S << 8 | d per pixel.
template <int K, int D, bool KEY16>
__device__ __forceinline__ uint32_t wta2(const uint32_t (&S)[K], const uint32_t (&dc)[K]) {
    if constexpr (KEY16) {
        uint32_t best = S[0] * static_cast<uint32_t>(D) + dc[0];
#pragma unroll
        for (int j = 1; j < K; ++j) best = vmin2(best, S[j] * static_cast<uint32_t>(D) + dc[j]);
        const uint32_t hi = __reduce_min_sync(kFull, best);
        const uint32_t lo = __reduce_min_sync(kFull, best << 16);
        const uint32_t mk = __byte_perm(lo, hi, 0x7632u);
        if constexpr ((D & (D - 1)) == 0) {
            return mk & (static_cast<uint32_t>(D - 1) * 0x10001u);
        } else {
            return ((mk & 0xffffu) % static_cast<uint32_t>(D)) | (((mk >> 16) % static_cast<uint32_t>(D)) << 16);
        }
    } else {
        uint32_t bA = 0xffffffffu, bB = 0xffffffffu;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            bA = min(bA, __byte_perm(S[j], dc[j], 0x5104u));  // [d, S_A.b0, S_A.b1, 0]
            bB = min(bB, __byte_perm(S[j], dc[j], 0x5324u));  // [d, S_B.b0, S_B.b1, 0]
        }
        bA = __reduce_min_sync(kFull, bA);
        bB = __reduce_min_sync(kFull, bB);
        return (bA & 0xffu) | ((bB & 0xffu) << 16);
    }
}

template <int K, bool KEY16>
__device__ __forceinline__ void wta_dconst(int lane, uint32_t (&dc)[K]) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const uint32_t d = static_cast<uint32_t>(K * lane + j);
        dc[j] = KEY16 ? d * 0x10001u : d;
    }
}

enum Mode {
    kStore = 0,  // store L_r in a field (first halves)
    kSumV = 1,   // vertical second halves: S_v = L + the other direction's stored L_r
    kWta = 2     // horizontal last steps: S = L + the other direction's stored L_r + S_v, then Eq. 4
};

// Inputs of one unit (two steps: one quad) of a walk; with u16 sums S_v
// takes K registers from each of its two arrays (s, s1).
template <int D, int MODE, bool S8>
struct UnitIn {
    static constexpr int K = D / 32;
    static constexpr int NO = MODE == kStore ? 0 : K;
    static constexpr int NS = MODE == kWta ? K : 0;
    static constexpr int NS1 = MODE == kWta && !S8 ? K : 0;
    static constexpr int REGS = K + NO + NS + NS1;
    uint32_t mc[K];
    uint32_t o[NO > 0 ? NO : 1];
    uint32_t s[NS > 0 ? NS : 1];
    uint32_t s1[NS1 > 0 ? NS1 : 1];
};

// Per-lane field bases of a walk.
struct Bases {
    uint8_t* mc;   // MC
    uint8_t* o;    // the other direction's stored L_r (kSumV, kWta)
    uint8_t* out;  // this direction's stored L_r (kStore) or S_v (kSumV; u16 sums: row 2qy)
    uint8_t* sv;   // S_v (kWta; u16 sums: row 2qy)
    uint8_t* sv1;  // u16 sums: row 2qy + 1 of S_v (kSumV, kWta)
};

// A walk over `nu` units: unit k at record offset off0 + k * dstride (a
// wrapped negative step for descending walks) and quad column qc0 + k * dqc
// (horizontal walks: raw output and debug).
struct Walk {
    uint32_t off0, dstride;
    int nu;
    int qc0, dqc;  // horizontal walks: quad column of unit 0 and its step
    int r;         // horizontal walks: the row pair
};

// Byte selectors of a walk, held in registers so that one body of code serves
// every axis and direction: the two steps of a unit take halves h0 then h1
// (0 then 1 for ascending rows or columns); un[t] turns a quad register into
// the word of step t, cq turns the words of steps 0 and 1 into a quad, and
// s16[t] picks step t's u16 pair out of a u16 quad (horizontal walks).
struct Sel {
    uint32_t un[2], cq, s16[2];
    int h0;
};

__device__ __forceinline__ Sel walk_sel(bool vert, bool asc) {
    Sel s;
    const uint32_t u_lo = vert ? 0x4140u : 0x4240u, u_hi = vert ? 0x4342u : 0x4341u;
    s.un[0] = asc ? u_lo : u_hi;
    s.un[1] = asc ? u_hi : u_lo;
    // words w0 (half 0), w1 (half 1): vertical [w0.b0, w0.b2, w1.b0, w1.b2],
    // horizontal [w0.b0, w1.b0, w0.b2, w1.b2]; descending walks pass (w1, w0)
    s.cq = vert ? (asc ? 0x6420u : 0x2064u) : (asc ? 0x6240u : 0x2604u);
    s.s16[0] = asc ? 0x5410u : 0x7632u;
    s.s16[1] = asc ? 0x7632u : 0x5410u;
    s.h0 = asc ? 0 : 1;
    return s;
}

// Units prefetched ahead of the recurrence for `regs_per_unit` input registers.
__host__ __device__ constexpr int units_ahead(int regs_per_unit, int budget) {
    return budget / regs_per_unit > 6 ? 6 : (budget / regs_per_unit < 2 ? 2 : budget / regs_per_unit);
}

// One walk.  The inputs of unit k + PU are loaded into unit k's registers as
// soon as unit k is done, so every load has PU units of the recurrence to
// arrive, and the loop body is PU units long.
template <int D, int MODE, bool S8, bool KEY16 = true, bool DBG = false, int PFB = 48>
__device__ __forceinline__ void walk(Chain2<D / 32>& ch, const PairsArgs& a, const Bases& bs, const Walk& wk,
                                     const Sel& sel) {
    constexpr int K = D / 32;
    using In = UnitIn<D, MODE, S8>;
    constexpr int PU = units_ahead(In::REGS, PFB);
    const int nu = wk.nu;
    if (nu <= 0) return;
    const int lane = threadIdx.x & 31;
    // every input goes through L2 only: one 16-byte piece per lane of a 512-byte
    // run is never re-read by the same SM (measured: the L1 path made the
    // first launch 1.7x slower)
    auto load = [&](In& in, uint32_t off) {
        ldv<K, false>(at(bs.mc, off), in.mc);
        if constexpr (MODE != kStore) ldv<K, false>(at(bs.o, off), in.o);
        if constexpr (MODE == kWta) {
            ldv<K, false>(at(bs.sv, off), in.s);
            if constexpr (!S8) ldv<K, false>(at(bs.sv1, off), in.s1);
        }
    };
    uint32_t dc[K];
    if constexpr (MODE == kWta) wta_dconst<K, KEY16>(lane, dc);
    uint32_t off_cur = wk.off0, off_ld = wk.off0;
    int qc = wk.qc0;
    // u16 sums of the vertical pair: step t writes its row's array
    uint8_t* const sv_first = sel.h0 ? bs.sv1 : bs.out;
    uint8_t* const sv_second = sel.h0 ? bs.out : bs.sv1;

    auto unit = [&](const In& in) {
        uint32_t first[K];    // kStore / kSumV with byte sums: L of the unit's first step
        uint32_t dfirst = 0;  // kWta: disparities of the first step
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            uint32_t m[K];
#pragma unroll
            for (int j = 0; j < K; ++j) m[j] = __byte_perm(in.mc[j], 0u, sel.un[t]);
            ch.step(m, a.P1x2, a.P2x2);
            if constexpr (MODE == kStore || (MODE == kSumV && S8)) {
                if (t == 0) {
#pragma unroll
                    for (int j = 0; j < K; ++j) first[j] = ch.w[j];
                } else {
                    uint32_t q[K];
#pragma unroll
                    for (int j = 0; j < K; ++j) {
                        q[j] = __byte_perm(first[j], ch.w[j], sel.cq);
                        // byte sums: both terms and their sum stay below 256 (no carries)
                        if constexpr (MODE == kSumV) q[j] += in.o[j];
                    }
                    stv<K>(at(bs.out, off_cur), q);
                }
            } else if constexpr (MODE == kSumV) {  // vertical, u16 sums: (S(x0, y), S(x1, y)) per row array
                uint32_t s[K];
#pragma unroll
                for (int j = 0; j < K; ++j) s[j] = ch.w[j] + __byte_perm(in.o[j], 0u, sel.un[t]);
                stv<K>(at(t == 0 ? sv_first : sv_second, off_cur), s);
            } else {  // kWta (horizontal)
                uint32_t S[K];
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const uint32_t sv = S8 ? __byte_perm(in.s[j], 0u, sel.un[t])
                                           : __byte_perm(in.s[j], in.s1[j], sel.s16[t]);
                    S[j] = ch.w[j] + __byte_perm(in.o[j], 0u, sel.un[t]) + sv;
                }
                const uint32_t dd = wta2<K, D, KEY16>(S, dc);
                if constexpr (DBG) {
                    const int x = 2 * qc + (t == 0 ? sel.h0 : 1 - sel.h0), y0 = 2 * wk.r;
                    if (x < a.W) {
#pragma unroll
                        for (int j = 0; j < K; ++j) {
                            const size_t d = static_cast<size_t>(K * lane + j);
                            if (y0 < a.H) a.Sdbg[(static_cast<size_t>(y0) * a.W + x) * D + d] = S[j] & 0xffffu;
                            if (y0 + 1 < a.H) a.Sdbg[(static_cast<size_t>(y0 + 1) * a.W + x) * D + d] = S[j] >> 16;
                        }
                    }
                }
                if (t == 0) {
                    dfirst = dd;
                } else if (lane == 0) {
                    *reinterpret_cast<uint32_t*>(a.rawq + (static_cast<size_t>(wk.r) * a.QW + qc) * 4) =
                        __byte_perm(dfirst, dd, sel.cq);
                }
            }
        }
        off_cur += wk.dstride;
        qc += wk.dqc;
    };

    In buf[PU];
#pragma unroll
    for (int i = 0; i < PU; ++i) {
        if (i < nu) load(buf[i], off_ld);
        off_ld += wk.dstride;
    }
    for (int k0 = 0;; k0 += PU) {
#pragma unroll
        for (int i = 0; i < PU; ++i) {
            if (k0 + i >= nu) return;
            unit(buf[i]);
            if (k0 + i + PU < nu) load(buf[i], off_ld);  // refill with unit k0 + i + PU
            off_ld += wk.dstride;
        }
    }
}

// The two warps of a block (the two directions of one line pair).
__device__ __forceinline__ void pair_sync() {
    __threadfence_block();
    asm volatile("bar.sync 1, 64;" ::: "memory");
}

// Horizontal chain state between the launches: the K words and m of each lane.
template <int K>
__device__ __forceinline__ uint32_t* state_slot(const PairsArgs& a, int r, int dir) {
    return a.state + ((static_cast<size_t>(r) * 2 + dir) * 32 + (threadIdx.x & 31)) * (K + 1);
}

// A lane's 4 K bytes of every quad sit at 4 K lane in each field array.
template <int D>
__device__ __forceinline__ Bases lane_bases(const PairsArgs& a, int o_field, int out_field) {
    constexpr int K = D / 32;
    uint8_t* const l = a.rec + 4 * K * (threadIdx.x & 31);
    return Bases{l, l + o_field * a.FS, l + out_field * a.FS, l + kSV * a.FS, l + kSV1 * a.FS};
}

// Launch 1: blocks alternate between vertical line pairs (warp 0 top-to-bottom,
// warp 1 bottom-to-top) and horizontal line pairs (warp 0 left-to-right,
// warp 1 right-to-left) while both last.
template <int D, bool S8>
__global__ void __launch_bounds__(64) pairs_stage1_kernel(const __grid_constant__ PairsArgs a) {
    constexpr int K = D / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x, nmin = min(a.nvb, a.nhb);
    bool vert;
    int idx;
    if (b < 2 * nmin) {
        vert = (b & 1) == 0;
        idx = b >> 1;
    } else {
        vert = a.nvb > a.nhb;
        idx = b - nmin;
    }
    Chain2<K> ch;
    ch.init(lane);
    const uint32_t QB = static_cast<uint32_t>(a.QB);
    if (vert) {
        const int c = idx;  // columns 2c, 2c + 1
        const uint32_t us = static_cast<uint32_t>(a.QW) * QB, off0 = static_cast<uint32_t>(c) * QB;
        const int hu = a.Hm / 2;
        const Bases st = lane_bases<D>(a, 0, kLV);
        const Bases sm = lane_bases<D>(a, kLV, kSV);
        // warp 0 walks down (rows [0, Hm) then [Hm, H2)), warp 1 up
        const bool down = warp == 0;
        const Sel sel = walk_sel(true, down);
        const Walk w1 = down ? Walk{off0, us, hu, 0, 0, 0} : Walk{off0 + (a.QH - 1) * us, 0u - us, a.QH - hu, 0, 0, 0};
        const Walk w2 = down ? Walk{off0 + hu * us, us, a.QH - hu, 0, 0, 0} : Walk{off0 + (hu - 1) * us, 0u - us, hu, 0, 0, 0};
        walk<D, kStore, S8>(ch, a, st, w1, sel);
        pair_sync();
        walk<D, kSumV, S8>(ch, a, sm, w2, sel);
    } else {
        const int r = idx;  // rows 2r, 2r + 1
        const uint32_t off0 = static_cast<uint32_t>(r) * a.QW * QB;
        const int n = a.n1 / 2;
        const bool right = warp == 0;  // warp 0 walks left to right, warp 1 right to left
        walk<D, kStore, S8>(ch, a, lane_bases<D>(a, 0, right ? kLH0 : kLH1),
                            right ? Walk{off0, QB, n, 0, 0, r} : Walk{off0 + (a.QW - 1) * QB, 0u - QB, n, 0, 0, r},
                            walk_sel(false, right));
        if (a.nh2 > 0) {
            uint32_t* st = state_slot<K>(a, r, warp);
#pragma unroll
            for (int j = 0; j < K; ++j) st[j] = ch.w[j];
            st[K] = ch.mpx2;
        }
    }
}

// Launch 2: blocks [0, nh2) finish the horizontal pairs (one row pair per
// block); the others run the parallel winner-take-all over columns [b, a).
template <int D, bool S8, bool KEY16, bool DBG>
__global__ void __launch_bounds__(64) pairs_stage2_kernel(const __grid_constant__ PairsArgs a) {
    constexpr int K = D / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t QB = static_cast<uint32_t>(a.QB);
    if (static_cast<int>(blockIdx.x) < a.nh2) {
        const int r = blockIdx.x;
        Chain2<K> ch;
        ch.init(lane);
        {
            const uint32_t* st = state_slot<K>(a, r, warp);
#pragma unroll
            for (int j = 0; j < K; ++j) ch.w[j] = __ldcg(st + j);
            ch.mpx2 = __ldcg(st + K);
            ch.exchange();
        }
        const uint32_t off0 = static_cast<uint32_t>(r) * a.QW * QB;
        const int n1u = a.n1 / 2, au = a.a / 2, bu = a.b / 2, ru = (a.W2 - a.n1) / 2;
        const bool right = warp == 0;  // warp 0 walks left to right, warp 1 right to left
        const Sel sel = walk_sel(false, right);
        walk<D, kStore, S8>(ch, a, lane_bases<D>(a, 0, right ? kLH0 : kLH1),
                            right ? Walk{off0 + n1u * QB, QB, au - n1u, 0, 0, r}
                                  : Walk{off0 + (ru - 1) * QB, 0u - QB, ru - bu, 0, 0, r},
                            sel);
        if (a.a > a.n1) pair_sync();  // the other direction's stores of this launch
        walk<D, kWta, S8, KEY16, DBG, 72>(ch, a, lane_bases<D>(a, right ? kLH1 : kLH0, 0),
                                          right ? Walk{off0 + au * QB, QB, a.QW - au, au, 1, r}
                                                : Walk{off0 + (bu - 1) * QB, 0u - QB, bu, bu - 1, -1, r},
                                          sel);
        return;
    }
    // parallel winner-take-all: one quad per warp (its loads wait for DRAM
    // once; many warps keep many quads in flight)
    const int cols = (a.a - a.b) / 2, items = cols * a.QH;
    if (cols <= 0) return;
    uint32_t dc[K];
    wta_dconst<K, KEY16>(lane, dc);
    const int nw = 2 * a.npw;
    const int lb = 4 * K * lane;
    for (int it = (blockIdx.x - a.nh2) * 2 + warp; it < items; it += nw) {
        const int r = it / cols, qx = a.b / 2 + it % cols;
        const uint8_t* q = a.rec + (static_cast<size_t>(r) * a.QW + qx) * a.QB + lb;
        uint32_t l0[K], l1[K], sv[K], sv1[K];
        ldv<K, false>(q + kLH0 * a.FS, l0);
        ldv<K, false>(q + kLH1 * a.FS, l1);
        ldv<K, false>(q + kSV * a.FS, sv);
        if constexpr (!S8) ldv<K, false>(q + kSV1 * a.FS, sv1);
        uint32_t dd[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // rows 2r and 2r + 1
            uint32_t S[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if constexpr (S8)  // both stored costs in a byte: l0 + l1 <= 2 (MC_max + P2) <= 255
                    S[j] = unq<true>(l0[j] + l1[j], h) + unq<true>(sv[j], h);
                else
                    S[j] = unq<true>(l0[j], h) + unq<true>(l1[j], h) + (h ? sv1[j] : sv[j]);
            }
            dd[h] = wta2<K, D, KEY16>(S, dc);
            if constexpr (DBG) {
                const int y = 2 * r + h;
                if (y < a.H) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int x = 2 * qx + i;
                        if (x >= a.W) continue;
#pragma unroll
                        for (int j = 0; j < K; ++j)
                            a.Sdbg[(static_cast<size_t>(y) * a.W + x) * D + K * lane + j] =
                                i ? (S[j] >> 16) : (S[j] & 0xffffu);
                    }
                }
            }
        }
        if (lane == 0)
            *reinterpret_cast<uint32_t*>(a.rawq + (static_cast<size_t>(r) * a.QW + qx) * 4) =
                __byte_perm(dd[0], dd[1], 0x6420u);
    }
}

template <int D>
struct PairsD {
    // S * D + d < 2^16 for every sum of 4 paths: 4 (MC_max + P2) * D + D - 1 <= 65535
    static bool key16(const PairsArgs& a) {
        const int P2 = static_cast<int>(a.P2x2 & 0xffffu);
        return 4 * (a.mc_max + P2) * D + D - 1 <= 65535;
    }
    static cudaError_t stage1(const PairsArgs& a, cudaStream_t s) {
        const int grid = a.nvb + a.nhb;
        if (grid <= 0) return cudaSuccess;
        if (a.s8)
            pairs_stage1_kernel<D, true><<<grid, 64, 0, s>>>(a);
        else
            pairs_stage1_kernel<D, false><<<grid, 64, 0, s>>>(a);
        return cudaGetLastError();
    }
    template <bool S8, bool KEY16>
    static void stage2_t(const PairsArgs& a, int grid, cudaStream_t s) {
        if (a.Sdbg)
            pairs_stage2_kernel<D, S8, KEY16, true><<<grid, 64, 0, s>>>(a);
        else
            pairs_stage2_kernel<D, S8, KEY16, false><<<grid, 64, 0, s>>>(a);
    }
    static cudaError_t stage2(const PairsArgs& a, cudaStream_t s) {
        const int grid = a.nh2 + a.npw;
        if (grid <= 0) return cudaSuccess;
        const bool k16 = key16(a);
        if (a.s8 && k16)
            stage2_t<true, true>(a, grid, s);
        else if (a.s8)
            stage2_t<true, false>(a, grid, s);
        else if (k16)
            stage2_t<false, true>(a, grid, s);
        else
            stage2_t<false, false>(a, grid, s);
        return cudaGetLastError();
    }
};

}  // namespace pairs

// defined in sgm_sweeps_d<D>.cu; internal to the library (not part of the C ABI)
#define SGM_INTERNAL_P __attribute__((visibility("hidden")))
template <int D>
SGM_INTERNAL_P cudaError_t pairs_launch1(const PairsArgs& a, cudaStream_t s);
template <int D>
SGM_INTERNAL_P cudaError_t pairs_launch2(const PairsArgs& a, cudaStream_t s);

#define SGM_INSTANTIATE_PAIRS(D)                                                      \
    template <>                                                                       \
    SGM_INTERNAL_P cudaError_t pairs_launch1<D>(const PairsArgs& a, cudaStream_t s) { \
        return pairs::PairsD<D>::stage1(a, s);                                        \
    }                                                                                 \
    template <>                                                                       \
    SGM_INTERNAL_P cudaError_t pairs_launch2<D>(const PairsArgs& a, cudaStream_t s) { \
        return pairs::PairsD<D>::stage2(a, s);                                        \
    }

}  // namespace sgm

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
//   launch 1  every walker stores its own L_r: the vertical pair walks every
//             row, each horizontal direction n1 columns; nothing is read but
//             the costs, so no walker waits for another;
//   launch 2  the rest of each horizontal direction, finishing its pixels
//             with Eq. 4 (S = its own L_r + the three stored ones), beside a
//             parallel winner-take-all over the columns both horizontal
//             directions passed in launch 1.
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
enum Field { kMC = 0, kLVT = 1, kLVB = 2, kLH0 = 3, kLH1 = 4 };

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

// L2 eviction priority of a cube's loads and stores: kL2Normal, or kL2Last
// (kept over normal and first lines; the costs, read by four walkers) or
// kL2First (streamed through; stored costs read much later).
enum L2Hint { kL2Normal = 0, kL2Last = 1, kL2First = 2 };

template <int HINT>
__device__ __forceinline__ uint64_t l2_policy() {
    uint64_t pol;
    if constexpr (HINT == kL2Last)
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else
        asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// N registers from 4N bytes at p (16-byte aligned when N % 4 == 0, 8-byte when
// N is even), through L2 only.
template <int N, bool NC, int HINT = kL2Normal>
__device__ __forceinline__ void ldv(const uint8_t* p, uint32_t (&r)[N]) {
    if constexpr (N % 4 == 0 && HINT != kL2Normal) {
        const uint64_t pol = l2_policy<HINT>();
#pragma unroll
        for (int i = 0; i < N / 4; ++i)
            asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                         : "=r"(r[4 * i]), "=r"(r[4 * i + 1]), "=r"(r[4 * i + 2]), "=r"(r[4 * i + 3])
                         : "l"(p + 16 * i), "l"(pol));
    } else if constexpr (N % 4 == 0) {
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

template <int N, int HINT = kL2Normal>
__device__ __forceinline__ void stv(uint8_t* p, const uint32_t (&r)[N]) {
    if constexpr (N % 4 == 0 && HINT != kL2Normal) {
        const uint64_t pol = l2_policy<HINT>();
#pragma unroll
        for (int i = 0; i < N / 4; ++i)
            asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p + 16 * i),
                         "r"(r[4 * i]), "r"(r[4 * i + 1]), "r"(r[4 * i + 2]), "r"(r[4 * i + 3]), "l"(pol)
                         : "memory");
    } else if constexpr (N % 4 == 0) {
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

// Launch 2: input registers of the chains' prefetch, and quads per warp of the
// parallel winner-take-all.
constexpr int kChainPrefetchRegs = 192, kParItems = 4;

// Cache policy of the walks' traffic (measured on the 640x480 D=128 frame):
// the stored costs, written in the first launch and read in the second, go
// through L2 as evict-first, so that they do not push out the costs the other
// walkers are about to read (first launch 51 -> 43 us, second 41 -> 35 us).
constexpr int kHintMcLoad = kL2Normal, kHintLStore = kL2First, kHintLLoad = kL2First;

// Extents for the bounds-checked build: the field arrays, the quad raw
// disparity, the chains' state and the debug sums.
__device__ __forceinline__ const uint8_t* cubes_end(const PairsArgs& a) {
    return a.rec + kPairsFields * a.FS - a.check_shrink;
}
__device__ __forceinline__ size_t state_words(const PairsArgs& a) {
    return static_cast<size_t>(a.QH) * 2 * 32 * (a.D / 32 + 1);
}

template <int N, int HINT>
__device__ __forceinline__ void ldv_checked(const PairsArgs& a, const uint8_t* p, uint32_t (&r)[N], unsigned site) {
    if (SGM_GUARD(p, 4 * N, a.rec, cubes_end(a), site)) {
        ldv<N, false, HINT>(p, r);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) r[i] = 0u;
    }
}

template <int N, int HINT>
__device__ __forceinline__ void stv_checked(const PairsArgs& a, uint8_t* p, const uint32_t (&r)[N], unsigned site) {
    if (SGM_GUARD(p, 4 * N, a.rec, cubes_end(a), site)) stv<N, HINT>(p, r);
}

__device__ __forceinline__ void raw_quad_store(const PairsArgs& a, size_t q, uint32_t v, unsigned site) {
    if (SGM_GUARD_INDEX(static_cast<long long>(q), static_cast<long long>(a.QW) * a.QH, site))
        reinterpret_cast<uint32_t*>(a.rawq)[q] = v;
}

__device__ __forceinline__ void sdbg_store(const PairsArgs& a, size_t i, uint32_t v, unsigned site) {
    if (SGM_GUARD_INDEX(static_cast<long long>(i), static_cast<long long>(a.W) * a.H * a.D, site))
        a.Sdbg[i] = static_cast<uint16_t>(v);
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
    kStore = 0,  // store L_r in this direction's field
    kWta = 1     // horizontal last steps: S = L + the three stored L_r, then Eq. 4
};

// Inputs of one unit (two steps: one quad) of a walk: MC, and for kWta the
// other horizontal direction's stored L_r and the two vertical ones.
template <int D, int MODE>
struct UnitIn {
    static constexpr int K = D / 32;
    static constexpr int NO = MODE == kWta ? K : 0;
    static constexpr int REGS = K + 3 * NO;
    uint32_t mc[K];
    uint32_t o[NO > 0 ? NO : 1];
    uint32_t v0[NO > 0 ? NO : 1];
    uint32_t v1[NO > 0 ? NO : 1];
};

// Per-lane field bases of a walk.
struct Bases {
    uint8_t* mc;   // MC
    uint8_t* out;  // this direction's stored L_r (kStore)
    uint8_t* o;    // the other horizontal direction's stored L_r (kWta)
    uint8_t* v0;   // top-to-bottom stored L_r (kWta)
    uint8_t* v1;   // bottom-to-top stored L_r (kWta)
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
// the word of step t and cq turns the words of steps 0 and 1 into a quad.
struct Sel {
    uint32_t un[2], cq;
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
    s.h0 = asc ? 0 : 1;
    return s;
}

// Units prefetched ahead of the recurrence for `regs_per_unit` input registers.
__host__ __device__ constexpr int units_ahead(int regs_per_unit, int budget) {
    return budget / regs_per_unit > 12 ? 12 : (budget / regs_per_unit < 2 ? 2 : budget / regs_per_unit);
}

// Sum of the three stored L_r of a pixel pair in one step's u16 words: the
// other horizontal direction (o) and the two vertical ones (v0, v1).  S8:
// the two vertical costs add as bytes (L_TB + L_BT <= 2 (MC_max + P2) <= 255).
template <bool S8>
__device__ __forceinline__ uint32_t stored3(uint32_t o, uint32_t v0, uint32_t v1, uint32_t sel) {
    if constexpr (S8)
        return __byte_perm(o, 0u, sel) + __byte_perm(v0 + v1, 0u, sel);
    else
        return __byte_perm(o, 0u, sel) + __byte_perm(v0, 0u, sel) + __byte_perm(v1, 0u, sel);
}

// One walk.  The inputs of unit k + PU are loaded into unit k's registers as
// soon as unit k is done, so every load has PU units of the recurrence to
// arrive, and the loop body is PU units long.
template <int D, int MODE, bool S8 = true, bool KEY16 = true, bool DBG = false, int PFB = 48>
__device__ __forceinline__ void walk(Chain2<D / 32>& ch, const PairsArgs& a, const Bases& bs, const Walk& wk,
                                     const Sel& sel) {
    constexpr int K = D / 32;
    using In = UnitIn<D, MODE>;
    constexpr int PU = units_ahead(In::REGS, PFB);
    const int nu = wk.nu;
    if (nu <= 0) return;
    const int lane = threadIdx.x & 31;
    // every input goes through L2 only: one 16-byte piece per lane of a 512-byte
    // run is never re-read by the same SM (measured: the L1 path made the
    // first launch 1.7x slower)
    auto load = [&](In& in, uint32_t off) {
        ldv_checked<K, kHintMcLoad>(a, at(bs.mc, off), in.mc, 101);
        if constexpr (MODE == kWta) {
            ldv_checked<K, kHintLLoad>(a, at(bs.o, off), in.o, 102);
            ldv_checked<K, kHintLLoad>(a, at(bs.v0, off), in.v0, 103);
            ldv_checked<K, kHintLLoad>(a, at(bs.v1, off), in.v1, 104);
        }
    };
    uint32_t dc[K];
    if constexpr (MODE == kWta) wta_dconst<K, KEY16>(lane, dc);
    uint32_t off_cur = wk.off0, off_ld = wk.off0;
    int qc = wk.qc0;

    auto unit = [&](const In& in) {
        uint32_t first[K];    // kStore: L of the unit's first step
        uint32_t dfirst = 0;  // kWta: disparities of the first step
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            uint32_t m[K];
#pragma unroll
            for (int j = 0; j < K; ++j) m[j] = __byte_perm(in.mc[j], 0u, sel.un[t]);
            ch.step(m, a.P1x2, a.P2x2);
            if constexpr (MODE == kStore) {
                if (t == 0) {
#pragma unroll
                    for (int j = 0; j < K; ++j) first[j] = ch.w[j];
                } else {
                    uint32_t q[K];
#pragma unroll
                    for (int j = 0; j < K; ++j) q[j] = __byte_perm(first[j], ch.w[j], sel.cq);
                    stv_checked<K, kHintLStore>(a, at(bs.out, off_cur), q, 105);
                }
            } else {  // kWta (horizontal)
                uint32_t S[K];
#pragma unroll
                for (int j = 0; j < K; ++j) S[j] = ch.w[j] + stored3<S8>(in.o[j], in.v0[j], in.v1[j], sel.un[t]);
                const uint32_t dd = wta2<K, D, KEY16>(S, dc);
                if constexpr (DBG) {
                    const int x = 2 * qc + (t == 0 ? sel.h0 : 1 - sel.h0), y0 = 2 * wk.r;
                    if (x < a.W) {
#pragma unroll
                        for (int j = 0; j < K; ++j) {
                            const size_t d = static_cast<size_t>(K * lane + j);
                            if (y0 < a.H) sdbg_store(a, (static_cast<size_t>(y0) * a.W + x) * D + d, S[j] & 0xffffu, 106);
                            if (y0 + 1 < a.H)
                                sdbg_store(a, (static_cast<size_t>(y0 + 1) * a.W + x) * D + d, S[j] >> 16, 106);
                        }
                    }
                }
                if (t == 0) {
                    dfirst = dd;
                } else if (lane == 0) {
                    raw_quad_store(a, static_cast<size_t>(wk.r) * a.QW + qc, __byte_perm(dfirst, dd, sel.cq), 107);
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
__device__ __forceinline__ Bases lane_bases(const PairsArgs& a, int out_field, int o_field = kMC) {
    constexpr int K = D / 32;
    uint8_t* const l = a.rec + 4 * K * (threadIdx.x & 31);
    return Bases{l, l + out_field * a.FS, l + o_field * a.FS, l + kLVT * a.FS, l + kLVB * a.FS};
}

// Launch 1: every walker stores its own L_r.  Blocks alternate between
// vertical line pairs (warp 0 top-to-bottom, warp 1 bottom-to-top, every row)
// and horizontal line pairs (warp 0 left-to-right over columns [0, n1),
// warp 1 right-to-left over [W2 - n1, W2)) while both last.
template <int D>
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
        const bool down = warp == 0;
        walk<D, kStore>(ch, a, lane_bases<D>(a, down ? kLVT : kLVB),
                        down ? Walk{off0, us, a.QH, 0, 0, 0} : Walk{off0 + (a.QH - 1) * us, 0u - us, a.QH, 0, 0, 0},
                        walk_sel(true, down));
    } else {
        const int r = idx;  // rows 2r, 2r + 1
        const uint32_t off0 = static_cast<uint32_t>(r) * a.QW * QB;
        const int n = a.n1 / 2;
        const bool right = warp == 0;  // warp 0 walks left to right, warp 1 right to left
        walk<D, kStore>(ch, a, lane_bases<D>(a, right ? kLH0 : kLH1),
                        right ? Walk{off0, QB, n, 0, 0, r} : Walk{off0 + (a.QW - 1) * QB, 0u - QB, n, 0, 0, r},
                        walk_sel(false, right));
        if (a.nh2 > 0) {
            uint32_t* st = state_slot<K>(a, r, warp);
            if (SGM_GUARD(st, 4 * (K + 1), a.state, a.state + state_words(a), 108)) {
#pragma unroll
                for (int j = 0; j < K; ++j) st[j] = ch.w[j];
                st[K] = ch.mpx2;
            }
        }
    }
}

// Launch 2a: the rest of the horizontal pairs, one row pair per block (warp 0
// left to right, warp 1 right to left), finishing their pixels with Eq. 4.
// Few warps walk long chains here, so they prefetch deep.
template <int D, bool S8, bool KEY16, bool DBG>
__global__ void __launch_bounds__(64) pairs_chain2_kernel(const __grid_constant__ PairsArgs a) {
    constexpr int K = D / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t QB = static_cast<uint32_t>(a.QB);
    const int r = blockIdx.x;
    Chain2<K> ch;
    ch.init(lane);
    {
        const uint32_t* st = state_slot<K>(a, r, warp);
        if (SGM_GUARD(st, 4 * (K + 1), a.state, a.state + state_words(a), 109)) {
#pragma unroll
            for (int j = 0; j < K; ++j) ch.w[j] = __ldcg(st + j);
            ch.mpx2 = __ldcg(st + K);
        }
        ch.exchange();
    }
    const uint32_t off0 = static_cast<uint32_t>(r) * a.QW * QB;
    const int n1u = a.n1 / 2, au = a.a / 2, bu = a.b / 2, ru = (a.W2 - a.n1) / 2;
    const bool right = warp == 0;
    const Sel sel = walk_sel(false, right);
    walk<D, kStore>(ch, a, lane_bases<D>(a, right ? kLH0 : kLH1),
                    right ? Walk{off0 + n1u * QB, QB, au - n1u, 0, 0, r}
                          : Walk{off0 + (ru - 1) * QB, 0u - QB, ru - bu, 0, 0, r},
                    sel);
    // when the pair meets in the middle each direction stores columns the other
    // finishes in this launch (also when a == n1: then only right to left does)
    if (a.W2 > 2 * a.n1) pair_sync();
    walk<D, kWta, S8, KEY16, DBG, kChainPrefetchRegs>(ch, a, lane_bases<D>(a, kMC, right ? kLH1 : kLH0),
                                                      right ? Walk{off0 + au * QB, QB, a.QW - au, au, 1, r}
                                                            : Walk{off0 + (bu - 1) * QB, 0u - QB, bu, bu - 1, -1, r},
                                                      sel);
}

// Launch 2b (beside 2a): the winner-take-all of the quads in columns [b, a),
// which both horizontal directions passed in launch 1.  Each warp takes
// kParItems quads and issues all their loads before the first sum, so many
// quads are in flight.
template <int D, bool S8, bool KEY16, bool DBG>
__global__ void __launch_bounds__(64) pairs_par_kernel(const __grid_constant__ PairsArgs a) {
    constexpr int K = D / 32, NI = kParItems;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cols = (a.a - a.b) / 2, items = cols * a.QH;
    uint32_t dc[K];
    wta_dconst<K, KEY16>(lane, dc);
    const int lb = 4 * K * lane;
    const int it0 = (blockIdx.x * 2 + warp) * NI;
    uint32_t l0[NI][K], l1[NI][K], v0[NI][K], v1[NI][K];
#pragma unroll
    for (int n = 0; n < NI; ++n) {
        const int it = min(it0 + n, items - 1);  // past the end: re-read the last quad
        const uint8_t* q = a.rec + (static_cast<size_t>(it / cols) * a.QW + a.b / 2 + it % cols) * a.QB + lb;
        ldv_checked<K, kHintLLoad>(a, q + kLH0 * a.FS, l0[n], 110);
        ldv_checked<K, kHintLLoad>(a, q + kLH1 * a.FS, l1[n], 110);
        ldv_checked<K, kHintLLoad>(a, q + kLVT * a.FS, v0[n], 110);
        ldv_checked<K, kHintLLoad>(a, q + kLVB * a.FS, v1[n], 110);
    }
#pragma unroll
    for (int n = 0; n < NI; ++n) {
        const int it = it0 + n;
        if (it >= items) return;
        const int r = it / cols, qx = a.b / 2 + it % cols;
        uint32_t dd[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // rows 2r and 2r + 1
            uint32_t S[K];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if constexpr (S8)  // pairs of stored costs in a byte: each pair <= 2 (MC_max + P2) <= 255
                    S[j] = unq<true>(l0[n][j] + l1[n][j], h) + unq<true>(v0[n][j] + v1[n][j], h);
                else
                    S[j] = unq<true>(l0[n][j], h) + unq<true>(l1[n][j], h) + unq<true>(v0[n][j], h) +
                           unq<true>(v1[n][j], h);
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
                            sdbg_store(a, (static_cast<size_t>(y) * a.W + x) * D + K * lane + j,
                                       i ? (S[j] >> 16) : (S[j] & 0xffffu), 111);
                    }
                }
            }
        }
        if (lane == 0) raw_quad_store(a, static_cast<size_t>(r) * a.QW + qx, __byte_perm(dd[0], dd[1], 0x6420u), 112);
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
        pairs_stage1_kernel<D><<<grid, 64, 0, s>>>(a);
        return cudaGetLastError();
    }
    template <bool S8, bool KEY16>
    static void chain_t(const PairsArgs& a, cudaStream_t s) {
        if (a.Sdbg)
            pairs_chain2_kernel<D, S8, KEY16, true><<<a.nh2, 64, 0, s>>>(a);
        else
            pairs_chain2_kernel<D, S8, KEY16, false><<<a.nh2, 64, 0, s>>>(a);
    }
    template <bool S8, bool KEY16>
    static void par_t(const PairsArgs& a, cudaStream_t s) {
        if (a.Sdbg)
            pairs_par_kernel<D, S8, KEY16, true><<<a.npw, 64, 0, s>>>(a);
        else
            pairs_par_kernel<D, S8, KEY16, false><<<a.npw, 64, 0, s>>>(a);
    }
    static cudaError_t chain2(const PairsArgs& a, cudaStream_t s) {
        if (a.nh2 <= 0) return cudaSuccess;
        const bool k16 = key16(a);
        if (a.s8 && k16)
            chain_t<true, true>(a, s);
        else if (a.s8)
            chain_t<true, false>(a, s);
        else if (k16)
            chain_t<false, true>(a, s);
        else
            chain_t<false, false>(a, s);
        return cudaGetLastError();
    }
    static cudaError_t par(const PairsArgs& a, cudaStream_t s) {
        if (a.npw <= 0) return cudaSuccess;
        const bool k16 = key16(a);
        if (a.s8 && k16)
            par_t<true, true>(a, s);
        else if (a.s8)
            par_t<true, false>(a, s);
        else if (k16)
            par_t<false, true>(a, s);
        else
            par_t<false, false>(a, s);
        return cudaGetLastError();
    }
};

}  // namespace pairs

// defined in sgm_sweeps_d<D>.cu; internal to the library (not part of the C ABI)
#define SGM_INTERNAL_P __attribute__((visibility("hidden")))
template <int D>
SGM_INTERNAL_P cudaError_t pairs_launch1(const PairsArgs& a, cudaStream_t s);
template <int D>
SGM_INTERNAL_P cudaError_t pairs_launch_chain2(const PairsArgs& a, cudaStream_t s);
template <int D>
SGM_INTERNAL_P cudaError_t pairs_launch_par(const PairsArgs& a, cudaStream_t s);

#define SGM_INSTANTIATE_PAIRS(D)                                                            \
    template <>                                                                             \
    SGM_INTERNAL_P cudaError_t pairs_launch1<D>(const PairsArgs& a, cudaStream_t s) {       \
        return pairs::PairsD<D>::stage1(a, s);                                              \
    }                                                                                       \
    template <>                                                                             \
    SGM_INTERNAL_P cudaError_t pairs_launch_chain2<D>(const PairsArgs& a, cudaStream_t s) { \
        return pairs::PairsD<D>::chain2(a, s);                                              \
    }                                                                                       \
    template <>                                                                             \
    SGM_INTERNAL_P cudaError_t pairs_launch_par<D>(const PairsArgs& a, cudaStream_t s) {    \
        return pairs::PairsD<D>::par(a, s);                                                 \
    }

}  // namespace sgm

// Device-side building blocks of the SGM path (arXiv 1610.04121) for sm_103a.
//
// Data layouts in HBM (all row-major, y outermost):
//   image      uint8  [H][W]
//   feature    uint32 [H][W]              CSCT of Eq. 1, 31 bits
//   cost       uint8  [H][W][D]           "paired" order: for word i in [0, D/2)
//                                         bytes 2i, 2i+1 hold MC(i), MC(i + D/2)
//   path cost  uint8  [H][W][D]           L_r in the same paired order (L_r <= 255)
//   sum        uint32 [H][W][D/2]         packed u16x2 word i = (S(i), S(i + D/2))
//   disparity  uint8  [H][W]
//
// The paired order makes the disparity neighbours d-1 / d+1 of both halves of
// word i live in words i-1 / i+1, so the Eq. 3 step needs no byte shuffling
// inside a word; only the two seams (d = 0 and d = D/2) need a permute.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sgm_check.cuh"
#include "sgm_internal.h"

namespace sgm {

// "+infinity" in one u16 lane: adding a penalty (<= 224) stays below 0x10000,
// so packed 32-bit adds never carry across lanes.
constexpr uint32_t kInf16 = 0x3FFFu;

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t redux_min(uint32_t v) { return __reduce_min_sync(0xffffffffu, v); }

__device__ __forceinline__ uint32_t shfl_idx(uint32_t v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Paired bytes held in registers -> packed u16x2 words.
template <int K>
__device__ __forceinline__ void unpack_regs(const uint32_t (&b)[(K + 1) / 2], uint32_t (&w)[K]) {
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = __byte_perm(b[j >> 1], 0u, (j & 1) ? 0x4342u : 0x4140u);
}

// ---------------------------------------------------------------------------
// Paired-byte and packed-word loads / stores for one lane's K words.
// ---------------------------------------------------------------------------
template <int K>
struct U8Pairs {
    uint32_t r[(K + 1) / 2];
};

// Packed u16x2 words (each lane <= 255) -> paired bytes.
template <int K>
__device__ __forceinline__ U8Pairs<K> pack_pairs(const uint32_t (&w)[K]) {
    U8Pairs<K> o;
#pragma unroll
    for (int j = 0; j < K; j += 2) {
        if (j + 1 < K)
            o.r[j >> 1] = __byte_perm(w[j], w[j + 1], 0x6420u);
        else
            o.r[j >> 1] = __byte_perm(w[j], 0u, 0x4420u);
    }
    return o;
}

template <int K>
__device__ __forceinline__ void st_pairs(uint8_t* p, const U8Pairs<K>& o) {
    if constexpr (K == 1) {
        *reinterpret_cast<uint16_t*>(p) = static_cast<uint16_t>(o.r[0]);
    } else if constexpr (K == 2) {
        *reinterpret_cast<uint32_t*>(p) = o.r[0];
    } else if constexpr (K == 4) {
        *reinterpret_cast<uint2*>(p) = make_uint2(o.r[0], o.r[1]);
    } else if constexpr (K == 8) {
        *reinterpret_cast<uint4*>(p) = make_uint4(o.r[0], o.r[1], o.r[2], o.r[3]);
    } else if constexpr (K == 6) {
        uint32_t* q = reinterpret_cast<uint32_t*>(p);
        q[0] = o.r[0];
        q[1] = o.r[1];
        q[2] = o.r[2];
    } else {
        uint16_t* h = reinterpret_cast<uint16_t*>(p);
#pragma unroll
        for (int j = 0; j < K; ++j) h[j] = static_cast<uint16_t>((j & 1) ? (o.r[j >> 1] >> 16) : o.r[j >> 1]);
    }
}

template <int K>
__device__ __forceinline__ void st_words(uint32_t* p, const uint32_t (&w)[K]) {
    if constexpr (K == 1) {
        p[0] = w[0];
    } else if constexpr (K % 4 == 0) {
#pragma unroll
        for (int j = 0; j < K; j += 4) *reinterpret_cast<uint4*>(p + j) = make_uint4(w[j], w[j + 1], w[j + 2], w[j + 3]);
    } else if constexpr (K % 2 == 0) {
#pragma unroll
        for (int j = 0; j < K; j += 2) *reinterpret_cast<uint2*>(p + j) = make_uint2(w[j], w[j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) p[j] = w[j];
    }
}

// ---------------------------------------------------------------------------
// Aggregation chains (Eq. 3, Section 3.2) with G lanes per path: G = 32 puts
// one path in a warp; G = 16 puts two in it, lanes 0-15 carrying chain A and
// lanes 16-31 chain B (the two opposite directions of one row or one column).
// Every cross-lane operation is a full-warp instruction; with G = 16 each
// half shuffles within itself and the two step minima are two masked
// reductions.
//
// Lane l of a path holds words i = (l mod G)*K + j, j < K, of the path cost
// of the previous pixel; word i packs L(i) (low half) and L(i + D/2) (high
// half), D = 2*G*K.  Each step computes, for every d,
//   L(p, d) = MC(p, d) + min(L(q, d), L(q, d-1) + P1, L(q, d+1) + P1, m(q) + P2) - m(q)
// with q the previous pixel and m(q) = min_k L(q, k).  Starting a path with
// L(q, .) = 0 and m(q) = 0 yields L(p, .) = MC(p, .), the reading used for the
// first pixel of every path.  `up` / `dn` hold the neighbour words across the
// lane boundary, already exchanged at the end of the previous step.
// ---------------------------------------------------------------------------
template <int G, int K>
struct Chain {
    static_assert(G == 16 || G == 32, "16 or 32 lanes per path");
    uint32_t w[K];
    uint32_t up, dn;  // word pl*K-1 from lane pl-1, word pl*K+K from lane pl+1 (wrapping in the path)
    uint32_t mpx2;    // m(q) in both u16 halves
    uint32_t mul_up, add_up, sel_dn, mask_a, mask_b;
    int src_up, src_dn;
    bool in_b;

    __device__ __forceinline__ void init(int lane) {
        const int pl = lane & (G - 1), base = lane & (32 - G);
        src_up = base | ((pl + G - 1) & (G - 1));
        src_dn = base | ((pl + 1) & (G - 1));
        // first lane of a path: d-1 of d=0 is absent, d-1 of d=D/2 is the low
        // half of word D/2-1, so up -> [inf, up.lo] = up * 2^16 + inf (one
        // multiply-add on the FMA pipe); other lanes take up * 1 + 0
        mul_up = (pl == 0) ? 0x10000u : 1u;
        add_up = (pl == 0) ? kInf16 : 0u;
        // last lane of a path: d+1 of d=D-1 is absent, d+1 of d=D/2-1 is the high half of word 0
        sel_dn = (pl == G - 1) ? 0x5432u : 0x3210u;
        in_b = G == 16 && lane >= 16;
        mask_a = in_b ? 0xffffffffu : 0u;
        mask_b = ~mask_a;
        reset();
    }

    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = 0u;
        up = dn = 0u;
        mpx2 = 0u;
    }

    // the minimum of v over this lane's path
    __device__ __forceinline__ uint32_t path_min(uint32_t v) const {
        if constexpr (G == 32) {
            return redux_min(v);
        } else {
            const uint32_t a = redux_min(v | mask_a);
            const uint32_t b = redux_min(v | mask_b);
            return in_b ? b : a;
        }
    }

    __device__ __forceinline__ void step(const uint32_t (&mc)[K], uint32_t P1x2, uint32_t P2x2, uint32_t (&L)[K]) {
        const uint32_t inf2 = kInf16 * 0x10001u;
        const uint32_t u = up * mul_up + add_up;
        const uint32_t d = __byte_perm(dn, inf2, sel_dn);
        const uint32_t mp2 = mpx2 + P2x2;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t dm1 = (j == 0) ? u : w[j - 1];
            const uint32_t dp1 = (j == K - 1) ? d : w[j + 1];
            // every candidate is >= m(q) lane-wise, so the packed subtraction never borrows
            L[j] = vmin2(vmin2(dm1, dp1) + P1x2, vmin2(w[j], mp2)) + mc[j] - mpx2;
        }
        uint32_t r = L[0];
#pragma unroll
        for (int j = 1; j < K; ++j) r = vmin2(r, L[j]);
        r = vmin2(r, __byte_perm(r, 0u, 0x1032u));  // both u16 halves = lane minimum
        up = shfl_idx(L[K - 1], src_up);
        dn = shfl_idx(L[0], src_dn);
        mpx2 = path_min(r);
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = L[j];
    }
};

// Winner-take-all over one lane's words (Eq. 4).  The key orders by S, then
// by d, so its minimum over the path is the smallest S with, among equal S,
// the lowest d.
//
// KEY16 (every S below 65536 / D - 1): both u16 halves of word j become
// S * D + d in one multiply-add on the FMA pipe, d from dconst[j] = [i, i + D/2]
// for word i = pl*K + j; the lane's minimum key ends in the low half.
// Otherwise key = S << 8 | d in a u32, built with byte permutes, dconst[j]
// holding the bytes [i, i + D/2, 0, 0].
template <int K, bool KEY16>
__device__ __forceinline__ void wta_consts(int pl, int D, uint32_t (&dconst)[K]) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const uint32_t i = static_cast<uint32_t>(pl * K + j);
        dconst[j] = i | ((i + static_cast<uint32_t>(D / 2)) << (KEY16 ? 16 : 8));
    }
}

template <int K, int D, bool KEY16>
__device__ __forceinline__ uint32_t wta_key(const uint32_t (&s)[K], const uint32_t (&dconst)[K]) {
    if constexpr (KEY16) {
        uint32_t best = s[0] * static_cast<uint32_t>(D) + dconst[0];
#pragma unroll
        for (int j = 1; j < K; ++j) best = vmin2(best, s[j] * static_cast<uint32_t>(D) + dconst[j]);
        return vmin2(best, __umulhi(best, 0x10000u));
    } else {
        uint32_t best = 0xffffffffu;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t klo = __byte_perm(s[j], dconst[j], 0x6104u);  // [d_lo, S_lo.b0, S_lo.b1, 0]
            const uint32_t khi = __byte_perm(s[j], dconst[j], 0x6325u);  // [d_hi, S_hi.b0, S_hi.b1, 0]
            best = min(best, min(klo, khi));
        }
        return best;
    }
}

// The disparity of a path's minimum key.
template <int D, bool KEY16>
__device__ __forceinline__ uint8_t wta_disparity(uint32_t key) {
    return static_cast<uint8_t>(KEY16 ? key % static_cast<uint32_t>(D) : key & 0xffu);
}

// The next unit of a work list for this block (job index and unit within
// the job): thread 0 takes it with an atomic on the list's counter and
// shares it.  False once the list is exhausted.  Every thread of the block
// calls it (it synchronises the block, which also orders the reuse of the
// block's shared memory between units).
template <class Job>
__device__ __forceinline__ bool take_unit(const WorkList<Job>& L, uint32_t* next, int& job, int& unit) {
    __shared__ uint32_t s_unit;
    if (threadIdx.x == 0) s_unit = atomicAdd(next, 1u);
    __syncthreads();
    const uint32_t i = s_unit;
    __syncthreads();
    if (L.n <= 0 || i >= L.start[L.n]) return false;
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.start[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    job = lo;
    unit = static_cast<int>(i - L.start[lo]);
    return true;
}

// A descriptor the kernel cannot run: recorded in the device status word.
__device__ __forceinline__ void report_bad_job(uint32_t* status) {
    if (threadIdx.x == 0) atomicOr(status, 1u);
}

}  // namespace sgm

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

namespace sgm {

// "+infinity" in one u16 lane: adding a penalty (<= 224) stays below 0x10000,
// so packed 32-bit adds never carry across lanes.
constexpr uint32_t kInf16 = 0x3FFFu;

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t redux_min(uint32_t v, uint32_t mask) {
    uint32_t d;
    asm volatile("redux.sync.min.u32 %0, %1, %2;" : "=r"(d) : "r"(v), "r"(mask));
    return d;
}

// Lanes [g*G, g*G + G) of the warp that form one chain group.
template <int G>
__device__ __forceinline__ uint32_t group_mask(int lane_in_warp) {
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        return ((1u << G) - 1u) << ((lane_in_warp / G) * G);
    }
}

// ---------------------------------------------------------------------------
// Paired-byte and packed-word loads / stores for one lane's K words.
// ---------------------------------------------------------------------------
template <int K>
struct U8Pairs {
    uint32_t r[(K + 1) / 2];
};

template <int K>
__device__ __forceinline__ U8Pairs<K> ld_pairs(const uint8_t* p) {
    U8Pairs<K> o;
    if constexpr (K == 1) {
        o.r[0] = *reinterpret_cast<const uint16_t*>(p);
    } else if constexpr (K == 2) {
        o.r[0] = *reinterpret_cast<const uint32_t*>(p);
    } else if constexpr (K == 4) {
        uint2 v = *reinterpret_cast<const uint2*>(p);
        o.r[0] = v.x;
        o.r[1] = v.y;
    } else if constexpr (K == 8) {
        uint4 v = *reinterpret_cast<const uint4*>(p);
        o.r[0] = v.x;
        o.r[1] = v.y;
        o.r[2] = v.z;
        o.r[3] = v.w;
    } else {
        const uint16_t* h = reinterpret_cast<const uint16_t*>(p);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            uint32_t v = h[j];
            if (j & 1)
                o.r[j >> 1] |= v << 16;
            else
                o.r[j >> 1] = v;
        }
    }
    return o;
}

// Paired bytes -> packed u16x2 words.
template <int K>
__device__ __forceinline__ void unpack_pairs(const U8Pairs<K>& b, uint32_t (&w)[K]) {
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = __byte_perm(b.r[j >> 1], 0u, (j & 1) ? 0x4342u : 0x4140u);
}

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
    } else {
        uint16_t* h = reinterpret_cast<uint16_t*>(p);
#pragma unroll
        for (int j = 0; j < K; ++j) h[j] = static_cast<uint16_t>((j & 1) ? (o.r[j >> 1] >> 16) : o.r[j >> 1]);
    }
}

template <int K>
__device__ __forceinline__ void ld_words(const uint32_t* p, uint32_t (&w)[K]) {
    if constexpr (K == 1) {
        w[0] = p[0];
    } else if constexpr (K == 2) {
        uint2 v = *reinterpret_cast<const uint2*>(p);
        w[0] = v.x;
        w[1] = v.y;
    } else if constexpr (K % 4 == 0) {
#pragma unroll
        for (int j = 0; j < K; j += 4) {
            uint4 v = *reinterpret_cast<const uint4*>(p + j);
            w[j] = v.x;
            w[j + 1] = v.y;
            w[j + 2] = v.z;
            w[j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = p[j];
    }
}

template <int K>
__device__ __forceinline__ void st_words(uint32_t* p, const uint32_t (&w)[K]) {
    if constexpr (K == 1) {
        p[0] = w[0];
    } else if constexpr (K == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    } else if constexpr (K % 4 == 0) {
#pragma unroll
        for (int j = 0; j < K; j += 4) *reinterpret_cast<uint4*>(p + j) = make_uint4(w[j], w[j + 1], w[j + 2], w[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) p[j] = w[j];
    }
}

// ---------------------------------------------------------------------------
// One aggregation chain (Eq. 3, Section 3.2) held by a group of G lanes.
//
// Lane l of the group holds words i = l*K + j, j < K, of the path cost of the
// previous pixel; word i packs L(i) (low half) and L(i + D/2) (high half).
// Each step computes, for every d,
//   L(p, d) = MC(p, d) + min(L(q, d), L(q, d-1) + P1, L(q, d+1) + P1, m(q) + P2) - m(q)
// with q the previous pixel and m(q) = min_k L(q, k).  Starting a path with
// L(q, .) = 0 and m(q) = 0 yields L(p, .) = MC(p, .), the reading used for the
// first pixel of every path.
// ---------------------------------------------------------------------------
template <int G, int K>
struct Chain {
    uint32_t w[K];
    uint32_t mpx2;  // m(q) in both halves

    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = 0u;
        mpx2 = 0u;
    }

    // mc: packed costs of this lane's words at the new pixel.  Returns the new
    // path costs in L (also kept as the state for the next step).
    __device__ __forceinline__ void step(const uint32_t (&mc)[K], uint32_t P1x2, uint32_t P2x2, int lane,
                                         uint32_t gmask, uint32_t (&L)[K]) {
        // neighbours across lane boundaries; the group wraps so that lane 0 sees
        // word D/2 - 1 (for d = D/2 - 1) and lane G-1 sees word 0 (for d = D/2)
        uint32_t up = __shfl_sync(gmask, w[K - 1], (lane + G - 1) % G, G);
        uint32_t dn = __shfl_sync(gmask, w[0], (lane + 1) % G, G);
        if (lane == 0) up = (up << 16) | kInf16;            // d-1 of d=0 is absent
        if (lane == G - 1) dn = (dn >> 16) | (kInf16 << 16);  // d+1 of d=D-1 is absent
        const uint32_t mp2 = mpx2 + P2x2;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const uint32_t dm1 = (j == 0) ? up : w[j - 1];
            const uint32_t dp1 = (j == K - 1) ? dn : w[j + 1];
            const uint32_t a = vmin2(dm1, dp1) + P1x2;
            const uint32_t b = vmin2(w[j], mp2);
            // every candidate is >= m(q) lane-wise, so this never borrows
            L[j] = vmin2(a, b) + mc[j] - mpx2;
        }
        uint32_t r = L[0];
#pragma unroll
        for (int j = 1; j < K; ++j) r = vmin2(r, L[j]);
        r = vmin2(r, __byte_perm(r, 0u, 0x1032u));  // both halves = lane minimum
        mpx2 = redux_min(r, gmask);
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = L[j];
    }
};

// Winner-take-all over one lane's words (Eq. 4): key = S << 8 | d, so the
// u32 minimum is the smallest S and, among equal S, the lowest d.
template <int K>
__device__ __forceinline__ uint32_t wta_key(const uint32_t (&s)[K], int lane, int half) {
    uint32_t best = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const uint32_t i = static_cast<uint32_t>(lane * K + j);
        const uint32_t dconst = i | ((i + static_cast<uint32_t>(half)) << 8);
        const uint32_t klo = __byte_perm(s[j], dconst, 0x6104u);  // [d_lo, S_lo.b0, S_lo.b1, 0]
        const uint32_t khi = __byte_perm(s[j], dconst, 0x6325u);  // [d_hi, S_hi.b0, S_hi.b1, 0]
        best = min(best, min(klo, khi));
    }
    return best;
}

// Iterate i = 0 .. n-1 with loads issued PF iterations ahead (register ring).
template <int PF, class T, class LoadF, class BodyF>
__device__ __forceinline__ void pipelined(int n, LoadF&& load, BodyF&& body) {
    T buf[PF];
#pragma unroll
    for (int s = 0; s < PF; ++s)
        if (s < n) buf[s] = load(s);
    for (int i0 = 0; i0 < n; i0 += PF) {
#pragma unroll
        for (int s = 0; s < PF; ++s) {
            const int i = i0 + s;
            if (i < n) {
                T v = buf[s];
                if (i + PF < n) buf[s] = load(i + PF);
                body(i, v);
            }
        }
    }
}

}  // namespace sgm

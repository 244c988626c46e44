// Census (Eq. 1), matching cost (Eq. 2) and the 3x3 median (Section 2,
// stage 4) of the SGM path in arXiv 1610.04121, for sm_103a.
#include <algorithm>
#include <type_traits>

#include "sgm_device.cuh"
#include "sgm_internal.h"

namespace sgm {

// ---------------------------------------------------------------------------
// Eq. 1: 9x7 center-symmetric Census transform.  A CTA of kCtT threads covers
// a kCtW x kCtH tile (kCtW = 2 kCtT): the (kCtW+8) x (kCtH+6) bytes around it
// are staged in shared memory (the read-cooperative 2D tiling of Section 3.1)
// and each thread walks two adjacent columns of the tile downwards with the
// 7 x 10 window they share in registers, loading one new row of 10 bytes per
// pair of pixels; blockIdx.z picks the image.  The feature is 0 where the 9x7
// window leaves the image.
// Bit k follows the printed order of Eq. 1: i = 1..4, j = -3..3 give bit
// (i-1)*7 + j+3; the i = 0 pairs j = 1..3 give bits 28..30; s(u,v) = u >= v.
// Each bit costs two instructions: for bytes u, v the value v + ~u = v - u - 1
// is negative exactly when u >= v, and a funnel shift moves its sign bit in
// below the bits already collected (highest bit first).  The 31 bits are
// gathered as four independent 8-bit chains joined by byte permutes, which
// keeps the dependent chain per pixel short.
// ---------------------------------------------------------------------------
constexpr int kCtT = 32, kCtW = 2 * kCtT, kCtH = 4;

// Census feature of the pixel whose 9 window columns start at column c0 of
// the window rows; row k of the window (image y - 3 + k) is win[(r + k) % 7].
template <int NC>
__device__ __forceinline__ uint32_t census_feature(const uint32_t (&win)[7][NC], int r, int c0) {
    auto diff = [&](int b) -> uint32_t {
        int i, j;
        if (b >= 28) {
            i = 0;
            j = b - 27;  // bits 28..30: i = 0, j = 1..3
        } else {
            i = b / 7 + 1;
            j = b % 7 - 3;  // bit (i-1)*7 + j+3
        }
        // sign bit set when I(x+i, y+j) >= I(x-i, y-j)
        return win[(r + 3 - j) % 7][c0 + 4 - i] + ~win[(r + 3 + j) % 7][c0 + 4 + i];
    };
    uint32_t c[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int b = q * 8 + 7; b >= q * 8; --b)  // highest bit of the byte first
            if (b < 31) c[q] = __funnelshift_l(diff(b), c[q], 1);
    return __byte_perm(__byte_perm(c[0], c[1], 0x0040u), __byte_perm(c[2], c[3], 0x0040u), 0x5410u);
}

// The full 9x7 Census (the CT Section 2 contrasts CSCT with): bit k compares
// the k-th window pixel in row-major order (rows j = -3..3, columns
// i = -4..4, the centre skipped) with the centre, s(I(x+i, y+j), I(x, y));
// 62 bits gathered as eight 8-bit chains (the sign of I(x, y) + ~I(x+i, y+j)
// is set exactly when I(x+i, y+j) >= I(x, y)).
template <int NC>
__device__ __forceinline__ uint64_t census62_feature(const uint32_t (&win)[7][NC], int r, int c0) {
    auto diff = [&](int b) -> uint32_t {
        const int idx = b < 31 ? b : b + 1;  // window position, the centre (31) skipped
        const int j = idx / 9 - 3, i = idx % 9 - 4;
        return win[(r + 3) % 7][c0 + 4] + ~win[(r + 3 + j) % 7][c0 + 4 + i];
    };
    uint32_t c[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int b = q * 8 + 7; b >= q * 8; --b)  // highest bit of the byte first
            if (b < 62) c[q] = __funnelshift_l(diff(b), c[q], 1);
    const uint32_t lo =
        __byte_perm(__byte_perm(c[0], c[1], 0x0040u), __byte_perm(c[2], c[3], 0x0040u), 0x5410u);
    const uint32_t hi =
        __byte_perm(__byte_perm(c[4], c[5], 0x0040u), __byte_perm(c[6], c[7], 0x0040u), 0x5410u);
    return static_cast<uint64_t>(hi) << 32 | lo;
}

// CT = false: the CSCT of Eq. 1 into uint32 features; CT = true: the full
// 9x7 Census into uint64 features.
template <bool CT>
__device__ __forceinline__ void census_body(const uint8_t* __restrict__ left, const uint8_t* __restrict__ right,
                                            void* __restrict__ Fb, void* __restrict__ Fm, int W, int H, int bx,
                                            int by, int bz) {
    using FT = typename std::conditional<CT, uint64_t, uint32_t>::type;
    constexpr int TW = kCtW + 8, TH = kCtH + 6, NS = (TW + kCtT - 1) / kCtT;
    __shared__ uint8_t tile[TH][TW];
    const uint8_t* img = bz ? right : left;
    FT* F = static_cast<FT*>(bz ? Fm : Fb);
    const int x0 = bx * kCtW, y0 = by * kCtH;
    // Thread t stages tile columns t, t + kCtT, ...: all loads are issued
    // before the first shared-memory store.
    {
        uint8_t v[NS][TH];
#pragma unroll
        for (int h = 0; h < NS; ++h) {
            const int tx = threadIdx.x + h * kCtT, gx = x0 - 4 + tx;
            const bool xin = tx < TW && gx >= 0 && gx < W;
#pragma unroll
            for (int ty = 0; ty < TH; ++ty) {
                const int gy = y0 - 3 + ty;
                v[h][ty] = (xin && gy >= 0 && gy < H &&
                            SGM_GUARD_INDEX((long long)gy * W + gx, (long long)W * H, 301))
                               ? __ldg(img + (size_t)gy * W + gx)
                               : uint8_t(0);
            }
        }
#pragma unroll
        for (int h = 0; h < NS; ++h) {
            const int tx = threadIdx.x + h * kCtT;
            if (tx < TW) {
#pragma unroll
                for (int ty = 0; ty < TH; ++ty) tile[ty][tx] = v[h][ty];
            }
        }
    }
    __syncthreads();
    const int lx = 2 * threadIdx.x, x = x0 + lx;
    if (x >= W) return;
    const bool ok0 = x >= 4 && x <= W - 5, ok1 = x + 1 >= 4 && x + 1 <= W - 5, has1 = x + 1 < W;
    uint32_t win[7][10];  // win[r % 7][c]: tile row r, tile column lx + c (image x - 4 + c)
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 10; ++c) win[r][c] = tile[r][lx + c];
#pragma unroll
    for (int r = 0; r < kCtH; ++r) {
#pragma unroll
        for (int c = 0; c < 10; ++c) win[(r + 6) % 7][c] = tile[r + 6][lx + c];
        const int y = y0 + r;
        if (y >= H) break;
        const bool yok = y >= 3 && y <= H - 4;
        FT f0, f1;
        if constexpr (CT) {
            f0 = census62_feature(win, r, 0);
            f1 = census62_feature(win, r, 1);
        } else {
            f0 = census_feature(win, r, 0);
            f1 = census_feature(win, r, 1);
        }
        FT* row = F + (size_t)y * W + x;
        if (SGM_GUARD_INDEX((long long)y * W + x + (has1 ? 1 : 0), (long long)W * H, 302)) {
            row[0] = (ok0 && yok) ? f0 : FT(0);
            if (has1) row[1] = (ok1 && yok) ? f1 : FT(0);
        }
    }
}

template <bool CT>
__global__ void __launch_bounds__(kCtT) census_kernel(const uint8_t* __restrict__ left, const uint8_t* __restrict__ right,
                                                      void* __restrict__ Fb, void* __restrict__ Fm, int W, int H) {
    census_body<CT>(left, right, Fb, Fm, W, H, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <bool CT>
__global__ void __launch_bounds__(kCtT) census_list_kernel(const WorkList<CensusJob>* __restrict__ Lp,
                                                           uint32_t* __restrict__ next, uint32_t* __restrict__ status) {
    const WorkList<CensusJob> L = *Lp;
    int p, u;
    while (take_unit(L, next, p, u)) {
        const CensusJob j = L.job[p];
        const int tx = (j.W + kCtW - 1) / kCtW, ty = (j.H + kCtH - 1) / kCtH;
        census_body<CT>(j.left, j.right, j.Fb, j.Fm, j.W, j.H, u % tx, (u / tx) % ty, u / (tx * ty));
    }
}

int census_units(int W, int H) { return 2 * ((W + kCtW - 1) / kCtW) * ((H + kCtH - 1) / kCtH); }

cudaError_t launch_census_list(const ListLaunch& l, cudaStream_t stream) {
    const auto* L = static_cast<const WorkList<CensusJob>*>(l.list);
    if (l.ct62)
        census_list_kernel<true><<<l.grid, kCtT, 0, stream>>>(L, l.next, l.status);
    else
        census_list_kernel<false><<<l.grid, kCtT, 0, stream>>>(L, l.next, l.status);
    return cudaGetLastError();
}

cudaError_t launch_census(const uint8_t* left, const uint8_t* right, void* Fb, void* Fm, int W, int H, bool ct62,
                          cudaStream_t stream) {
    dim3 grid((W + kCtW - 1) / kCtW, (H + kCtH - 1) / kCtH, 2);
    if (ct62)
        census_kernel<true><<<grid, kCtT, 0, stream>>>(left, right, Fb, Fm, W, H);
    else
        census_kernel<false><<<grid, kCtT, 0, stream>>>(left, right, Fb, Fm, W, H);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Eq. 2: MC(x, y, d) = bitcount(F_base(x, y) XOR F_match(x - d, y)), with the
// match feature 0 left of the image.  A CTA covers kMcSeg pixels of one row;
// the match features x0-D+1 .. x0+kMcSeg-1 and the base features are staged in
// shared memory (the 1D tiling of Section 3.1).  A thread computes one output
// word (paired words i0 = 2*wi and i0 + 1, i.e. d = i0, i0 + D/2, i0 + 1,
// i0 + 1 + D/2) for kMcPix consecutive pixels, so that the match features it
// loads are shared between neighbouring pixels; consecutive threads take
// consecutive words, which keeps the stores coalesced.  The kernel is bound by
// the bit-count pipe.
// ---------------------------------------------------------------------------
constexpr int kMcSeg = 128, kMcPix = 4, kMcThreads = 128;

// Two consecutive staged features.
__device__ __forceinline__ void ld2(const uint32_t* p, uint32_t& a, uint32_t& b) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld2(const uint64_t* p, uint64_t& a, uint64_t& b) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ uint32_t bitcount(uint32_t v) { return __popc(v); }
__device__ __forceinline__ uint32_t bitcount(uint64_t v) { return __popcll(v); }

// FT: uint32_t (CSCT features) or uint64_t (full Census features).
template <int D, class FT>
__device__ __forceinline__ void cost_body(const FT* __restrict__ Fb, const FT* __restrict__ Fm,
                                          uint8_t* __restrict__ rec, int RB, int W, int H, int seg, int y) {
    constexpr int Q = D / 4, half = D / 2, NF = kMcSeg + D;  // words per pixel; staged match features (even)
    __shared__ __align__(16) FT fm[NF];  // fm[k] = F_match(x0 - D + k)
    __shared__ __align__(16) FT fb[kMcSeg];
    const int x0 = seg * kMcSeg;
    const FT* fmrow = Fm + (size_t)y * W;
    {
        // every load is issued before the first shared-memory store
        constexpr int NI = (NF + kMcThreads - 1) / kMcThreads, NB = kMcSeg / kMcThreads;
        FT vm[NI], vb[NB];
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int i = threadIdx.x + it * kMcThreads, gx = x0 - D + i;
            vm[it] = (i < NF && gx >= 0 && gx < W) ? __ldg(fmrow + gx) : FT(0);
        }
#pragma unroll
        for (int it = 0; it < NB; ++it) {
            const int i = threadIdx.x + it * kMcThreads;
            vb[it] = (x0 + i < W) ? __ldg(Fb + (size_t)y * W + x0 + i) : FT(0);
        }
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int i = threadIdx.x + it * kMcThreads;
            if (i < NF) fm[i] = vm[it];
        }
#pragma unroll
        for (int it = 0; it < NB; ++it) fb[threadIdx.x + it * kMcThreads] = vb[it];
    }
    __syncthreads();
    const int npx = min(kMcSeg, W - x0);
    const int items = ((npx + kMcPix - 1) / kMcPix) * Q;
    uint8_t* out = rec + ((size_t)y * W + x0) * RB;  // MC at offset 0 of each record
    for (int t = threadIdx.x; t < items; t += kMcThreads) {
        const int g = t / Q, wi = t - g * Q, i0 = 2 * wi, px = g * kMcPix;
        // F_match(x - d) for x = x0 + px + p lives at fm[px + p + D - d]
        const int ba = px + D - i0 - 2;  // d = i0 + 1 - p' ... : fm[ba + p + 1] is d = i0 + 1, fm[ba + p + 2] is d = i0
        const int bb = ba - half;
        FT ra[kMcPix + 2], rb[kMcPix + 2], b4[kMcPix];
        if (!SGM_GUARD_INDEX(bb, NF, 303) || !SGM_GUARD_INDEX(ba + kMcPix + 1, NF, 303)) continue;
#pragma unroll
        for (int k = 0; k < kMcPix + 2; k += 2) {
            ld2(fm + ba + k, ra[k], ra[k + 1]);
            ld2(fm + bb + k, rb[k], rb[k + 1]);
        }
#pragma unroll
        for (int k = 0; k < kMcPix; k += 2) ld2(fb + px + k, b4[k], b4[k + 1]);
#pragma unroll
        for (int p = 0; p < kMcPix; ++p) {
            if (px + p >= npx) break;
            const FT b = b4[p];
            const uint32_t c0 = bitcount(b ^ ra[p + 2]);  // d = i0
            const uint32_t c1 = bitcount(b ^ rb[p + 2]);  // d = i0 + D/2
            const uint32_t c2 = bitcount(b ^ ra[p + 1]);  // d = i0 + 1
            const uint32_t c3 = bitcount(b ^ rb[p + 1]);  // d = i0 + 1 + D/2
            if (SGM_GUARD_INDEX(((long long)y * W + x0 + px + p) * RB + 4 * wi + 3, (long long)W * H * RB, 304))
                reinterpret_cast<uint32_t*>(out + (size_t)(px + p) * RB)[wi] =
                    __byte_perm(c0 | (c2 << 16), c1 | (c3 << 16), 0x6240u);  // [c0, c1, c2, c3]
        }
    }
}

template <int D, class FT>
__global__ void __launch_bounds__(kMcThreads) cost_kernel(const FT* __restrict__ Fb, const FT* __restrict__ Fm,
                                                          uint8_t* __restrict__ rec, int RB, int W, int H) {
    cost_body<D, FT>(Fb, Fm, rec, RB, W, H, blockIdx.x, blockIdx.y);
}

template <int D, class FT>
__global__ void __launch_bounds__(kMcThreads) cost_list_kernel(const WorkList<CostJob>* __restrict__ Lp,
                                                               uint32_t* __restrict__ next, uint32_t* __restrict__ status) {
    const WorkList<CostJob> L = *Lp;
    int p, u;
    while (take_unit(L, next, p, u)) {
        const CostJob j = L.job[p];
        if (j.D != D) {
            report_bad_job(status);
            continue;
        }
        const int segs = (j.W + kMcSeg - 1) / kMcSeg;
        cost_body<D, FT>(static_cast<const FT*>(j.Fb), static_cast<const FT*>(j.Fm), j.rec, j.RB, j.W, j.H,
                         u % segs, u / segs);
    }
}

int cost_units(int W, int H) { return ((W + kMcSeg - 1) / kMcSeg) * H; }

template <int D>
static cudaError_t launch_cost_list_t(const ListLaunch& l, cudaStream_t s) {
    const auto* L = static_cast<const WorkList<CostJob>*>(l.list);
    if (l.ct62)
        cost_list_kernel<D, uint64_t><<<l.grid, kMcThreads, 0, s>>>(L, l.next, l.status);
    else
        cost_list_kernel<D, uint32_t><<<l.grid, kMcThreads, 0, s>>>(L, l.next, l.status);
    return cudaGetLastError();
}

cudaError_t launch_cost_list(const ListLaunch& l, cudaStream_t stream) {
    switch (l.D) {
        case 32: return launch_cost_list_t<32>(l, stream);
        case 64: return launch_cost_list_t<64>(l, stream);
        case 96: return launch_cost_list_t<96>(l, stream);
        case 128: return launch_cost_list_t<128>(l, stream);
        case 160: return launch_cost_list_t<160>(l, stream);
        case 192: return launch_cost_list_t<192>(l, stream);
        case 224: return launch_cost_list_t<224>(l, stream);
        case 256: return launch_cost_list_t<256>(l, stream);
        default: return cudaErrorInvalidValue;
    }
}

template <int D>
static cudaError_t launch_cost_t(const void* Fb, const void* Fm, uint8_t* rec, int RB, int W, int H, bool ct62,
                                 cudaStream_t s) {
    const dim3 grid((W + kMcSeg - 1) / kMcSeg, H);
    if (ct62)
        cost_kernel<D, uint64_t><<<grid, kMcThreads, 0, s>>>(static_cast<const uint64_t*>(Fb),
                                                             static_cast<const uint64_t*>(Fm), rec, RB, W, H);
    else
        cost_kernel<D, uint32_t><<<grid, kMcThreads, 0, s>>>(static_cast<const uint32_t*>(Fb),
                                                             static_cast<const uint32_t*>(Fm), rec, RB, W, H);
    return cudaGetLastError();
}

cudaError_t launch_cost(const void* Fb, const void* Fm, uint8_t* rec, int RB, int W, int H, int D, bool ct62,
                        cudaStream_t stream) {
    switch (D) {
        case 32: return launch_cost_t<32>(Fb, Fm, rec, RB, W, H, ct62, stream);
        case 64: return launch_cost_t<64>(Fb, Fm, rec, RB, W, H, ct62, stream);
        case 96: return launch_cost_t<96>(Fb, Fm, rec, RB, W, H, ct62, stream);
        case 128: return launch_cost_t<128>(Fb, Fm, rec, RB, W, H, ct62, stream);
        case 160: return launch_cost_t<160>(Fb, Fm, rec, RB, W, H, ct62, stream);
        case 192: return launch_cost_t<192>(Fb, Fm, rec, RB, W, H, ct62, stream);
        case 224: return launch_cost_t<224>(Fb, Fm, rec, RB, W, H, ct62, stream);
        case 256: return launch_cost_t<256>(Fb, Fm, rec, RB, W, H, ct62, stream);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Eq. 2 into the quad cube of the paired-line schedule (sgm_internal.h): per
// quad of 2 x 2 pixels and disparity d, the four costs at byte i + 2j of a
// 32-bit word (pixel (2qx + i, 2qy + j)); padding pixels (x >= W or y >= H)
// get MC = 0.  A CTA covers kQcSeg quads of one quad row: the two rows' base
// features and the match features x0 - D .. x0 + 2 kQcSeg - 1 are staged in
// shared memory.  A thread computes kQcDisp = 8 consecutive disparities of
// one quad (one 32-byte store; the quad cube is 256-byte aligned and a quad
// takes 4D bytes) from nine match features of each row; the 32 threads of a
// warp take 8 quads x 4 disparity groups.
// ---------------------------------------------------------------------------
constexpr int kQcSeg = 32, kQcThreads = 128, kQcDisp = 8;

template <int D, class FT>
__device__ __forceinline__ void cost_quads_body(const FT* __restrict__ Fb, const FT* __restrict__ Fm,
                                                uint8_t* __restrict__ mc, int QB, int W, int H, int bx, int qy) {
    constexpr int NG = D / kQcDisp, SW = 2 * kQcSeg, NF = SW + D;
    __shared__ __align__(16) FT fm[2][NF];  // fm[j][k] = F_match(x0 - D + k, 2 qy + j)
    __shared__ __align__(16) FT fb[2][SW];  // fb[j][k] = F_base(x0 + k, 2 qy + j)
    const int qx0 = bx * kQcSeg, x0 = 2 * qx0, QW = (W + 1) / 2;
    {
        constexpr int NI = (2 * NF + kQcThreads - 1) / kQcThreads, NB = (2 * SW + kQcThreads - 1) / kQcThreads;
        FT vm[NI], vb[NB];
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int i = threadIdx.x + it * kQcThreads, j = i / NF, k = i - j * NF, gx = x0 - D + k, y = 2 * qy + j;
            vm[it] = (i < 2 * NF && gx >= 0 && gx < W && y < H) ? __ldg(Fm + (size_t)y * W + gx) : FT(0);
        }
#pragma unroll
        for (int it = 0; it < NB; ++it) {
            const int i = threadIdx.x + it * kQcThreads, j = i / SW, k = i - j * SW, gx = x0 + k, y = 2 * qy + j;
            vb[it] = (i < 2 * SW && gx < W && y < H) ? __ldg(Fb + (size_t)y * W + gx) : FT(0);
        }
#pragma unroll
        for (int it = 0; it < NI; ++it) {
            const int i = threadIdx.x + it * kQcThreads;
            if (i < 2 * NF) fm[i / NF][i % NF] = vm[it];
        }
#pragma unroll
        for (int it = 0; it < NB; ++it) {
            const int i = threadIdx.x + it * kQcThreads;
            if (i < 2 * SW) fb[i / SW][i % SW] = vb[it];
        }
    }
    __syncthreads();
    const int nq = min(kQcSeg, QW - qx0);
    // a warp takes 8 quads x 4 disparity groups: its feature loads span 40
    // words of shared memory (few bank conflicts) and its stores 8 runs of
    // 128 contiguous bytes
    const int items = ((nq + 7) / 8) * 8 * NG;
    // padding: column 2qx + 1 beyond the image only in the last quad column
    // (odd W), row 2qy + 1 only in the last quad row (odd H)
    const bool row1 = 2 * qy + 1 < H;
    for (int t = threadIdx.x; t < items; t += kQcThreads) {
        const int lane = t % 32, blk = t / 32, go = blk % (NG / 4), qo = blk / (NG / 4);
        const int ql = 8 * qo + lane % 8, g = 4 * go + lane / 8, xl = 2 * ql, d0 = kQcDisp * g;
        if (ql >= nq) continue;
        const bool col1 = x0 + xl + 1 < W;
        // byte weights of pixels (1, 0), (0, 1), (1, 1) in a quad word (0 at
        // padding pixels): the word is built by multiply-adds
        const uint32_t w10 = col1 ? 0x100u : 0u, w01 = row1 ? 0x10000u : 0u, w11 = (row1 && col1) ? 0x1000000u : 0u;
        uint32_t q[kQcDisp];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            // match features of pixels xl, xl + 1 at d0 .. d0 + kQcDisp - 1:
            // fm[j][xl + i - d + D] = m[kQcDisp + i - e] for d = d0 + e
            const int kb = xl + D - d0 - kQcDisp;  // even
            if (!SGM_GUARD_INDEX(kb, 2 * kQcSeg + D, 305) || !SGM_GUARD_INDEX(kb + kQcDisp + 1, 2 * kQcSeg + D, 305) ||
                !SGM_GUARD_INDEX(xl + 1, 2 * kQcSeg, 305))
                continue;
            FT m[kQcDisp + 2];
#pragma unroll
            for (int k = 0; k < kQcDisp + 2; k += 2) ld2(&fm[j][kb + k], m[k], m[k + 1]);
            FT b0, b1;
            ld2(&fb[j][xl], b0, b1);
#pragma unroll
            for (int e = 0; e < kQcDisp; ++e) {
                const uint32_t c0 = bitcount(b0 ^ m[kQcDisp - e]), c1 = bitcount(b1 ^ m[kQcDisp + 1 - e]);
                q[e] = j == 0 ? c0 + c1 * w10 : q[e] + c0 * w01 + c1 * w11;
            }
        }
        // one 32-byte store
        uint8_t* dst = mc + ((size_t)qy * QW + qx0 + ql) * QB + 4 * d0;
        if (!SGM_GUARD_INDEX(((long long)qy * QW + qx0 + ql) * QB + 4 * d0 + 31, (long long)QW * ((H + 1) / 2) * QB, 306))
            continue;
        asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(dst), "r"(q[0]), "r"(q[1]),
                     "r"(q[2]), "r"(q[3]), "r"(q[4]), "r"(q[5]), "r"(q[6]), "r"(q[7])
                     : "memory");
    }
}

template <int D, class FT>
__global__ void __launch_bounds__(kQcThreads) cost_quads_kernel(const FT* __restrict__ Fb, const FT* __restrict__ Fm,
                                                                uint8_t* __restrict__ mc, int QB, int W, int H) {
    cost_quads_body<D, FT>(Fb, Fm, mc, QB, W, H, blockIdx.x, blockIdx.y);
}

template <int D>
static cudaError_t launch_cost_quads_t(const void* Fb, const void* Fm, uint8_t* mc, int QB, int W, int H, bool ct62,
                                       cudaStream_t s) {
    const int QW = (W + 1) / 2, QH = (H + 1) / 2;
    const dim3 grid((QW + kQcSeg - 1) / kQcSeg, QH);
    if (ct62)
        cost_quads_kernel<D, uint64_t><<<grid, kQcThreads, 0, s>>>(static_cast<const uint64_t*>(Fb),
                                                                   static_cast<const uint64_t*>(Fm), mc, QB, W, H);
    else
        cost_quads_kernel<D, uint32_t><<<grid, kQcThreads, 0, s>>>(static_cast<const uint32_t*>(Fb),
                                                                   static_cast<const uint32_t*>(Fm), mc, QB, W, H);
    return cudaGetLastError();
}

cudaError_t launch_cost_quads(const void* Fb, const void* Fm, uint8_t* mc, int QB, int W, int H, int D, bool ct62,
                              cudaStream_t stream) {
    switch (D) {
        case 32: return launch_cost_quads_t<32>(Fb, Fm, mc, QB, W, H, ct62, stream);
        case 64: return launch_cost_quads_t<64>(Fb, Fm, mc, QB, W, H, ct62, stream);
        case 96: return launch_cost_quads_t<96>(Fb, Fm, mc, QB, W, H, ct62, stream);
        case 128: return launch_cost_quads_t<128>(Fb, Fm, mc, QB, W, H, ct62, stream);
        case 160: return launch_cost_quads_t<160>(Fb, Fm, mc, QB, W, H, ct62, stream);
        case 192: return launch_cost_quads_t<192>(Fb, Fm, mc, QB, W, H, ct62, stream);
        case 224: return launch_cost_quads_t<224>(Fb, Fm, mc, QB, W, H, ct62, stream);
        case 256: return launch_cost_quads_t<256>(Fb, Fm, mc, QB, W, H, ct62, stream);
        default: return cudaErrorInvalidValue;
    }
}

// A quad-layout cube -> natural order [H][W][D] (debug only).
__global__ void unquad_kernel(const uint8_t* __restrict__ cube, int QB, uint8_t* __restrict__ out, int W, int H, int D) {
    const size_t n = (size_t)W * H * D;
    const int QW = (W + 1) / 2;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const size_t p = t / D;
        const int d = static_cast<int>(t % D), x = static_cast<int>(p % W), y = static_cast<int>(p / W);
        out[t] = cube[((size_t)(y >> 1) * QW + (x >> 1)) * QB + 4 * d + (x & 1) + 2 * (y & 1)];
    }
}

cudaError_t launch_unquad_cost(const uint8_t* cube, int QB, uint8_t* out, int W, int H, int D, cudaStream_t stream) {
    unquad_kernel<<<1024, 256, 0, stream>>>(cube, QB, out, W, H, D);
    return cudaGetLastError();
}

// Paired order in RB-byte records -> natural order [H][W][D] (debug only).
__global__ void unpair_kernel(const uint8_t* __restrict__ rec, int RB, uint8_t* __restrict__ out, size_t npix, int D) {
    const size_t n = npix * D;
    const int half = D / 2;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const size_t p = t / D;
        const int d = static_cast<int>(t % D);
        const int src = (d < half) ? 2 * d : 2 * (d - half) + 1;
        out[t] = rec[p * RB + src];
    }
}

cudaError_t launch_unpair_cost(const uint8_t* rec, int RB, uint8_t* out, int W, int H, int D, cudaStream_t stream) {
    unpair_kernel<<<1024, 256, 0, stream>>>(rec, RB, out, (size_t)W * H, D);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 3x3 median of the winner-take-all disparity (Section 2, stage 4).  The
// one-pixel border ring copies the raw value.  With each row of the window
// sorted (lo <= mid <= hi), the median of the nine values is the median of
// {max of the lows, median of the mids, min of the highs}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sort3(int& a, int& b, int& c) {
    const int lo = min(a, b), hi = max(a, b);
    a = min(lo, c);
    const int m = max(lo, c);
    b = min(m, hi);
    c = max(m, hi);
}

__device__ __forceinline__ int med3(int a, int b, int c) { return max(min(a, b), min(max(a, b), c)); }

// A CTA of 128 threads covers a 128 x 8 tile: thread t walks column x0 + t
// down the tile with its three columns of the 3 x 10 neighbourhood loaded
// (clamped to the image) into registers up front; each row's three values are
// sorted once and shared by the three windows that contain the row.
constexpr int kMedW = 128, kMedH = 4;

// QUAD: raw in quads of 2 x 2 pixels ([ceil(H/2)][ceil(W/2)][4], pixel (x, y)
// at byte (x & 1) + 2 (y & 1) of its quad), else row-major [H][W].
template <bool QUAD = false>
__device__ __forceinline__ int raw_at(const uint8_t* __restrict__ raw, int W, int x, int y) {
    if constexpr (QUAD)
        return __ldg(raw + ((size_t)(y >> 1) * ((W + 1) >> 1) + (x >> 1)) * 4 + (x & 1) + 2 * (y & 1));
    else
        return SGM_GUARD_INDEX(x, W, 307) ? __ldg(raw + (size_t)y * W + x) : 0;
}

template <bool QUAD = false>
__device__ __forceinline__ void median_body(const uint8_t* __restrict__ raw, uint8_t* __restrict__ out, int W, int H,
                                            int bx, int by) {
    const int x = bx * kMedW + threadIdx.x, y0 = by * kMedH;
    if (x >= W) return;
    const int xl = max(x - 1, 0), xr = min(x + 1, W - 1);
    int lo[kMedH + 2], mid[kMedH + 2], hi[kMedH + 2];
#pragma unroll
    for (int r = 0; r < kMedH + 2; ++r) {
        const int gy = min(max(y0 - 1 + r, 0), H - 1);
        lo[r] = raw_at<QUAD>(raw, W, xl, gy);
        mid[r] = raw_at<QUAD>(raw, W, x, gy);
        hi[r] = raw_at<QUAD>(raw, W, xr, gy);
    }
    int c[kMedH];  // raw centre values: the border ring keeps them
#pragma unroll
    for (int k = 0; k < kMedH; ++k) c[k] = mid[k + 1];
#pragma unroll
    for (int r = 0; r < kMedH + 2; ++r) sort3(lo[r], mid[r], hi[r]);
    const bool x_inner = x > 0 && x < W - 1;
#pragma unroll
    for (int k = 0; k < kMedH; ++k) {
        const int y = y0 + k;
        if (y >= H) break;
        int v = c[k];
        if (x_inner && y > 0 && y < H - 1) {
            const int l = max(max(lo[k], lo[k + 1]), lo[k + 2]);
            const int m = med3(mid[k], mid[k + 1], mid[k + 2]);
            const int h = min(min(hi[k], hi[k + 1]), hi[k + 2]);
            v = med3(l, m, h);
        }
        if (SGM_GUARD_INDEX(x, W, 308)) out[(size_t)y * W + x] = static_cast<uint8_t>(v);
    }
}

__global__ void __launch_bounds__(kMedW) median_kernel(const uint8_t* __restrict__ raw, uint8_t* __restrict__ out,
                                                     int W, int H) {
    median_body(raw, out, W, H, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(kMedW) median_list_kernel(const WorkList<MedianJob>* __restrict__ Lp,
                                                             uint32_t* __restrict__ next) {
    const WorkList<MedianJob> L = *Lp;
    int p, u;
    while (take_unit(L, next, p, u)) {
        const MedianJob j = L.job[p];
        const int tx = (j.W + kMedW - 1) / kMedW;
        median_body(j.raw, j.out, j.W, j.H, u % tx, u / tx);
    }
}

int median_units(int W, int H) { return ((W + kMedW - 1) / kMedW) * ((H + kMedH - 1) / kMedH); }

cudaError_t launch_median_list(const ListLaunch& l, cudaStream_t stream) {
    median_list_kernel<<<l.grid, kMedW, 0, stream>>>(static_cast<const WorkList<MedianJob>*>(l.list), l.next);
    return cudaGetLastError();
}

cudaError_t launch_median(const uint8_t* raw, uint8_t* disp, int W, int H, cudaStream_t stream) {
    dim3 grid((W + kMedW - 1) / kMedW, (H + kMedH - 1) / kMedH);
    median_kernel<<<grid, kMedW, 0, stream>>>(raw, disp, W, H);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kMedW) median_quads_kernel(const uint8_t* __restrict__ rawq,
                                                           uint8_t* __restrict__ out, int W, int H) {
    median_body<true>(rawq, out, W, H, blockIdx.x, blockIdx.y);
}

cudaError_t launch_median_quads(const uint8_t* rawq, uint8_t* disp, int W, int H, cudaStream_t stream) {
    dim3 grid((W + kMedW - 1) / kMedW, (H + kMedH - 1) / kMedH);
    median_quads_kernel<<<grid, kMedW, 0, stream>>>(rawq, disp, W, H);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Copies between pinned host buffers and the work arena: few wide requests
// (16 bytes per thread when both sides and the size allow it), so that the
// host link carries each byte once.  Up to two buffers per launch
// (blockIdx.y; src[1] may be null).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) stage_kernel(const uint8_t* __restrict__ src0, uint8_t* __restrict__ dst0,
                                                    const uint8_t* __restrict__ src1, uint8_t* __restrict__ dst1,
                                                    size_t n) {
    const uint8_t* src = blockIdx.y ? src1 : src0;
    uint8_t* dst = blockIdx.y ? dst1 : dst0;
    if (!src) return;
    const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
    const size_t t0 = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n % 16 == 0 && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        for (size_t i = t0; i < n / 16; i += stride) d4[i] = s4[i];
    } else {
        for (size_t i = t0; i < n; i += stride) dst[i] = src[i];
    }
}

cudaError_t launch_stage(const uint8_t* src0, uint8_t* dst0, const uint8_t* src1, uint8_t* dst1, size_t n,
                         cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    constexpr size_t kPer = 256 * 16;        // bytes one block moves per pass
    constexpr size_t kMaxBlocks = 4 * 152;   // four per SM of a GB300: enough requests in flight
    const unsigned blocks = static_cast<unsigned>(std::min<size_t>(kMaxBlocks, (n + kPer - 1) / kPer));
    stage_kernel<<<dim3(blocks, src1 ? 2 : 1), 256, 0, stream>>>(src0, dst0, src1, dst1, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Post-filters (announced in Section 5; the readings are those of
// sgm_compute_ex in sgm.h).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) mirror_kernel(const uint8_t* __restrict__ left,
                                                     const uint8_t* __restrict__ right, uint8_t* __restrict__ ml,
                                                     uint8_t* __restrict__ mr, int W, int H) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const size_t src = static_cast<size_t>(y) * W + (W - 1 - x), dst = static_cast<size_t>(y) * W + x;
    ml[dst] = __ldg(left + src);
    mr[dst] = __ldg(right + src);
}

cudaError_t launch_mirror(const uint8_t* left, const uint8_t* right, uint8_t* ml, uint8_t* mr, int W, int H,
                          cudaStream_t stream) {
    dim3 grid((W + 255) / 256, H);
    mirror_kernel<<<grid, 256, 0, stream>>>(left, right, ml, mr, W, H);
    return cudaGetLastError();
}

// The value in 1/16 pixel at one pixel: 16 d, plus the rounded vertex offset
// of the parabola through S(d-1), S(d), S(d+1) (alpha = S(d-1) - S(d) > 0,
// gamma = S(d+1) - S(d) >= 0): floor((16 (alpha - gamma) + (alpha + gamma)) /
// (2 (alpha + gamma))), none at d = 0 or D-1.
__device__ __forceinline__ int subpixel_value(int d, uint32_t ag, int D) {
    if (d <= 0 || d >= D - 1) return 16 * d;
    const int al = static_cast<int>(ag & 0xffffu), ga = static_cast<int>(ag >> 16);
    const int n = 16 * (al - ga) + (al + ga), den = 2 * (al + ga);
    int q = n / den;
    if (n % den != 0 && n < 0) --q;  // floor
    return 16 * d + q;
}

constexpr int kPostW = 32, kPostH = 8;

// v = the sub-pixel (or 16 d) value of each pixel of a 34 x 10 tile in shared
// memory, then the 3x3 median (border ring copied), then the left-right check.
__global__ void __launch_bounds__(kPostW* kPostH) post_kernel(const uint8_t* __restrict__ rawL,
                                                              const uint32_t* __restrict__ sub,
                                                              const uint8_t* __restrict__ rawRm,
                                                              uint16_t* __restrict__ out16, int W, int H, int D) {
    __shared__ int v[kPostH + 2][kPostW + 2];
    const int x0 = blockIdx.x * kPostW, y0 = blockIdx.y * kPostH;
    const int t = threadIdx.y * kPostW + threadIdx.x;
    for (int c = t; c < (kPostH + 2) * (kPostW + 2); c += kPostW * kPostH) {
        const int cy = c / (kPostW + 2), cx = c - cy * (kPostW + 2);
        const int gx = x0 - 1 + cx, gy = y0 - 1 + cy;
        int val = 0;
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) {
            const size_t p = static_cast<size_t>(gy) * W + gx;
            const int d = rawL[p];
            val = sub ? subpixel_value(d, sub[p], D) : 16 * d;
        }
        v[cy][cx] = val;
    }
    __syncthreads();
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    if (x >= W || y >= H) return;
    const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
    int out;
    if (x == 0 || y == 0 || x == W - 1 || y == H - 1) {
        out = v[ty][tx];
    } else {
        // median of 9: sort each row, then the median of (largest row
        // minimum, median of the row medians, smallest row maximum)
        int a0 = v[ty - 1][tx - 1], a1 = v[ty - 1][tx], a2 = v[ty - 1][tx + 1];
        int b0 = v[ty][tx - 1], b1 = v[ty][tx], b2 = v[ty][tx + 1];
        int c0 = v[ty + 1][tx - 1], c1 = v[ty + 1][tx], c2 = v[ty + 1][tx + 1];
        sort3(a0, a1, a2);
        sort3(b0, b1, b2);
        sort3(c0, c1, c2);
        out = med3(max(max(a0, b0), c0), med3(a1, b1, c1), min(min(a2, b2), c2));
    }
    const size_t p = static_cast<size_t>(y) * W + x;
    if (rawRm) {
        const int d = rawL[p], xr = x - d;
        bool ok = xr >= 0;
        if (ok) {
            const int dr = rawRm[static_cast<size_t>(y) * W + (W - 1 - xr)];
            ok = d - dr <= 1 && dr - d <= 1;
        }
        if (!ok) out = 0xffff;
    }
    out16[p] = static_cast<uint16_t>(out);
}

cudaError_t launch_post(const uint8_t* rawL, const uint32_t* sub, const uint8_t* rawRm, uint16_t* out16, int W,
                        int H, int D, cudaStream_t stream) {
    dim3 grid((W + kPostW - 1) / kPostW, (H + kPostH - 1) / kPostH), block(kPostW, kPostH);
    post_kernel<<<grid, block, 0, stream>>>(rawL, sub, rawRm, out16, W, H, D);
    return cudaGetLastError();
}

bool supported_D(int D) { return D >= 32 && D <= 256 && D % 32 == 0; }

}  // namespace sgm

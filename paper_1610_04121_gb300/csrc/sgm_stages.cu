// Census (Eq. 1), matching cost (Eq. 2) and the 3x3 median (Section 2,
// stage 4) of the SGM path in arXiv 1610.04121, for sm_103a.
#include "sgm_device.cuh"
#include "sgm_internal.h"

namespace sgm {

// ---------------------------------------------------------------------------
// Eq. 1: 9x7 center-symmetric Census transform.  A CTA of kCtW threads covers
// a kCtW x kCtH tile: the (kCtW+8) x (kCtH+6) bytes around it are staged in
// shared memory (the read-cooperative 2D tiling of Section 3.1) and each
// thread walks one column of the tile downwards with the 7 x 9 window in
// registers, loading one new row of 9 bytes per pixel; blockIdx.z picks the
// image.  The feature is 0 where the 9x7 window leaves the image.
// Bit k follows the printed order of Eq. 1: i = 1..4, j = -3..3 give bit
// (i-1)*7 + j+3; the i = 0 pairs j = 1..3 give bits 28..30; s(u,v) = u >= v.
// Each bit costs two instructions: for bytes u, v the value v + ~u = v - u - 1
// is negative exactly when u >= v, and a funnel shift moves its sign bit in
// below the bits already collected (highest bit first).
// ---------------------------------------------------------------------------
constexpr int kCtW = 64, kCtH = 16;

__device__ __forceinline__ void census_body(const uint8_t* __restrict__ left, const uint8_t* __restrict__ right,
                                            uint32_t* __restrict__ Fb, uint32_t* __restrict__ Fm, int W, int H,
                                            int bx, int by, int bz) {
    __shared__ uint8_t tile[kCtH + 6][kCtW + 8];
    const uint8_t* img = bz ? right : left;
    uint32_t* F = bz ? Fm : Fb;
    const int x0 = bx * kCtW, y0 = by * kCtH;
    for (int i = threadIdx.x; i < (kCtH + 6) * (kCtW + 8); i += kCtW) {
        const int ty = i / (kCtW + 8), tx = i % (kCtW + 8);
        const int gx = x0 - 4 + tx, gy = y0 - 3 + ty;
        tile[ty][tx] = (gx >= 0 && gx < W && gy >= 0 && gy < H) ? img[(size_t)gy * W + gx] : 0;
    }
    __syncthreads();
    const int lx = threadIdx.x, x = x0 + lx;
    if (x >= W) return;
    const bool x_ok = x >= 4 && x <= W - 5;
    uint32_t win[7][9];  // win[r % 7][c]: tile row r, tile column lx + c (image x - 4 + c)
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 9; ++c) win[r][c] = tile[r][lx + c];
#pragma unroll
    for (int r = 0; r < kCtH; ++r) {
#pragma unroll
        for (int c = 0; c < 9; ++c) win[(r + 6) % 7][c] = tile[r + 6][lx + c];
        const int y = y0 + r;
        if (y >= H) break;
        // window row k (image y - 3 + k) is win[(r + k) % 7]
        uint32_t f = 0;
#pragma unroll
        for (int j = 3; j >= 1; --j)  // bits 30..28: i = 0
            f = __funnelshift_l(win[(r + 3 - j) % 7][4] + ~win[(r + 3 + j) % 7][4], f, 1);
#pragma unroll
        for (int i = 4; i >= 1; --i)
#pragma unroll
            for (int j = 3; j >= -3; --j)  // bits (i-1)*7 + j+3, highest first
                f = __funnelshift_l(win[(r + 3 - j) % 7][4 - i] + ~win[(r + 3 + j) % 7][4 + i], f, 1);
        const bool ok = x_ok && y >= 3 && y <= H - 4;
        F[(size_t)y * W + x] = ok ? f : 0u;
    }
}

__global__ void __launch_bounds__(kCtW) census_kernel(const uint8_t* __restrict__ left, const uint8_t* __restrict__ right,
                                                      uint32_t* __restrict__ Fb, uint32_t* __restrict__ Fm, int W,
                                                      int H) {
    census_body(left, right, Fb, Fm, W, H, blockIdx.x, blockIdx.y, blockIdx.z);
}

__global__ void __launch_bounds__(kCtW) census_batch_kernel(const __grid_constant__ JobTable<CensusJob> t) {
    const int p = find_job(t, blockIdx.x);
    const CensusJob& j = t.job[p];
    const int b = blockIdx.x - t.start[p];
    const int tx = (j.W + kCtW - 1) / kCtW, ty = (j.H + kCtH - 1) / kCtH;
    census_body(j.left, j.right, j.Fb, j.Fm, j.W, j.H, b % tx, (b / tx) % ty, b / (tx * ty));
}

cudaError_t launch_census_batch(JobTable<CensusJob>& t, cudaStream_t stream) {
    t.start[0] = 0;
    for (int i = 0; i < t.n; ++i)
        t.start[i + 1] = t.start[i] + 2 * ((t.job[i].W + kCtW - 1) / kCtW) * ((t.job[i].H + kCtH - 1) / kCtH);
    census_batch_kernel<<<t.start[t.n], kCtW, 0, stream>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_census(const uint8_t* left, const uint8_t* right, uint32_t* Fb, uint32_t* Fm, int W, int H,
                          cudaStream_t stream) {
    dim3 grid((W + kCtW - 1) / kCtW, (H + kCtH - 1) / kCtH, 2);
    census_kernel<<<grid, kCtW, 0, stream>>>(left, right, Fb, Fm, W, H);
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

template <int D>
__device__ __forceinline__ void cost_body(const uint32_t* __restrict__ Fb, const uint32_t* __restrict__ Fm,
                                          uint8_t* __restrict__ MC, int W, int seg, int y) {
    constexpr int Q = D / 4, half = D / 2, NF = kMcSeg + D;  // words per pixel; staged match features (even)
    __shared__ __align__(16) uint32_t fm[NF];  // fm[k] = F_match(x0 - D + k)
    __shared__ __align__(16) uint32_t fb[kMcSeg];
    const int x0 = seg * kMcSeg;
    const uint32_t* fmrow = Fm + (size_t)y * W;
    for (int i = threadIdx.x; i < NF; i += kMcThreads) {
        const int gx = x0 - D + i;
        fm[i] = (gx >= 0 && gx < W) ? fmrow[gx] : 0u;
    }
    for (int i = threadIdx.x; i < kMcSeg; i += kMcThreads) fb[i] = (x0 + i < W) ? Fb[(size_t)y * W + x0 + i] : 0u;
    __syncthreads();
    const int npx = min(kMcSeg, W - x0);
    const int items = ((npx + kMcPix - 1) / kMcPix) * Q;
    uint32_t* out = reinterpret_cast<uint32_t*>(MC + ((size_t)y * W + x0) * D);
    for (int t = threadIdx.x; t < items; t += kMcThreads) {
        const int g = t / Q, wi = t - g * Q, i0 = 2 * wi, px = g * kMcPix;
        // F_match(x - d) for x = x0 + px + p lives at fm[px + p + D - d]
        const int ba = px + D - i0 - 2;  // d = i0 + 1 - p' ... : fm[ba + p + 1] is d = i0 + 1, fm[ba + p + 2] is d = i0
        const int bb = ba - half;
        uint32_t ra[kMcPix + 2], rb[kMcPix + 2];
#pragma unroll
        for (int k = 0; k < kMcPix + 2; k += 2) {
            const uint2 va = *reinterpret_cast<const uint2*>(fm + ba + k);
            const uint2 vb = *reinterpret_cast<const uint2*>(fm + bb + k);
            ra[k] = va.x;
            ra[k + 1] = va.y;
            rb[k] = vb.x;
            rb[k + 1] = vb.y;
        }
        const uint4 vb4 = *reinterpret_cast<const uint4*>(fb + px);
        const uint32_t b4[4] = {vb4.x, vb4.y, vb4.z, vb4.w};
#pragma unroll
        for (int p = 0; p < kMcPix; ++p) {
            if (px + p >= npx) break;
            const uint32_t b = b4[p];
            const uint32_t c0 = __popc(b ^ ra[p + 2]);  // d = i0
            const uint32_t c1 = __popc(b ^ rb[p + 2]);  // d = i0 + D/2
            const uint32_t c2 = __popc(b ^ ra[p + 1]);  // d = i0 + 1
            const uint32_t c3 = __popc(b ^ rb[p + 1]);  // d = i0 + 1 + D/2
            out[(px + p) * Q + wi] = __byte_perm(c0 | (c2 << 16), c1 | (c3 << 16), 0x6240u);  // [c0, c1, c2, c3]
        }
    }
}

template <int D>
__global__ void __launch_bounds__(kMcThreads) cost_kernel(const uint32_t* __restrict__ Fb,
                                                          const uint32_t* __restrict__ Fm, uint8_t* __restrict__ MC,
                                                          int W) {
    cost_body<D>(Fb, Fm, MC, W, blockIdx.x, blockIdx.y);
}

template <int D>
__global__ void __launch_bounds__(kMcThreads) cost_batch_kernel(const __grid_constant__ JobTable<CostJob> t) {
    const int p = find_job(t, blockIdx.x);
    const CostJob& j = t.job[p];
    const int b = blockIdx.x - t.start[p];
    const int segs = (j.W + kMcSeg - 1) / kMcSeg;
    cost_body<D>(j.Fb, j.Fm, j.MC, j.W, b % segs, b / segs);
}

template <int D>
static cudaError_t launch_cost_batch_t(JobTable<CostJob>& t, cudaStream_t s) {
    t.start[0] = 0;
    for (int i = 0; i < t.n; ++i) t.start[i + 1] = t.start[i] + ((t.job[i].W + kMcSeg - 1) / kMcSeg) * t.job[i].H;
    cost_batch_kernel<D><<<t.start[t.n], kMcThreads, 0, s>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_cost_batch(JobTable<CostJob>& t, int D, cudaStream_t stream) {
    switch (D) {
        case 32: return launch_cost_batch_t<32>(t, stream);
        case 64: return launch_cost_batch_t<64>(t, stream);
        case 96: return launch_cost_batch_t<96>(t, stream);
        case 128: return launch_cost_batch_t<128>(t, stream);
        case 160: return launch_cost_batch_t<160>(t, stream);
        case 192: return launch_cost_batch_t<192>(t, stream);
        case 224: return launch_cost_batch_t<224>(t, stream);
        case 256: return launch_cost_batch_t<256>(t, stream);
        default: return cudaErrorInvalidValue;
    }
}

template <int D>
static cudaError_t launch_cost_t(const uint32_t* Fb, const uint32_t* Fm, uint8_t* MC, int W, int H, cudaStream_t s) {
    const dim3 grid((W + kMcSeg - 1) / kMcSeg, H);
    cost_kernel<D><<<grid, kMcThreads, 0, s>>>(Fb, Fm, MC, W);
    return cudaGetLastError();
}

cudaError_t launch_cost(const uint32_t* Fb, const uint32_t* Fm, uint8_t* MC, int W, int H, int D,
                        cudaStream_t stream) {
    switch (D) {
        case 32: return launch_cost_t<32>(Fb, Fm, MC, W, H, stream);
        case 64: return launch_cost_t<64>(Fb, Fm, MC, W, H, stream);
        case 96: return launch_cost_t<96>(Fb, Fm, MC, W, H, stream);
        case 128: return launch_cost_t<128>(Fb, Fm, MC, W, H, stream);
        case 160: return launch_cost_t<160>(Fb, Fm, MC, W, H, stream);
        case 192: return launch_cost_t<192>(Fb, Fm, MC, W, H, stream);
        case 224: return launch_cost_t<224>(Fb, Fm, MC, W, H, stream);
        case 256: return launch_cost_t<256>(Fb, Fm, MC, W, H, stream);
        default: return cudaErrorInvalidValue;
    }
}

// Paired order -> natural order [H][W][D] (debug only).
__global__ void unpair_kernel(const uint8_t* __restrict__ MC, uint8_t* __restrict__ out, size_t npix, int D) {
    const size_t n = npix * D;
    const int half = D / 2;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const size_t p = t / D;
        const int d = static_cast<int>(t % D);
        const int src = (d < half) ? 2 * d : 2 * (d - half) + 1;
        out[t] = MC[p * D + src];
    }
}

cudaError_t launch_unpair_cost(const uint8_t* MC, uint8_t* out, int W, int H, int D, cudaStream_t stream) {
    unpair_kernel<<<1024, 256, 0, stream>>>(MC, out, (size_t)W * H, D);
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

// A CTA covers a 128 x 8 tile (4 pixels per thread along x) staged with its
// one-pixel halo in shared memory.
__device__ __forceinline__ void median_body(const uint8_t* __restrict__ raw, uint8_t* __restrict__ out, int W, int H,
                                            int bx, int by) {
    __shared__ uint8_t t[10][136];
    const int x0 = bx * 128, y0 = by * 8;
    for (int i = threadIdx.y * 32 + threadIdx.x; i < 10 * 130; i += 256) {
        const int ty = i / 130, tx = i % 130;
        const int gx = min(max(x0 - 1 + tx, 0), W - 1), gy = min(max(y0 - 1 + ty, 0), H - 1);
        t[ty][tx] = raw[(size_t)gy * W + gx];
    }
    __syncthreads();
    const int y = y0 + threadIdx.y;
    if (y >= H) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int lx = threadIdx.x + 32 * k, x = x0 + lx;
        if (x >= W) continue;
        const int cx = lx + 1, cy = threadIdx.y + 1;
        const size_t p = (size_t)y * W + x;
        if (x == 0 || y == 0 || x == W - 1 || y == H - 1) {
            out[p] = t[cy][cx];
            continue;
        }
        int a0 = t[cy - 1][cx - 1], b0 = t[cy - 1][cx], c0 = t[cy - 1][cx + 1];
        int a1 = t[cy][cx - 1], b1 = t[cy][cx], c1 = t[cy][cx + 1];
        int a2 = t[cy + 1][cx - 1], b2 = t[cy + 1][cx], c2 = t[cy + 1][cx + 1];
        sort3(a0, b0, c0);
        sort3(a1, b1, c1);
        sort3(a2, b2, c2);
        const int lo = max(max(a0, a1), a2);
        const int mid = med3(b0, b1, b2);
        const int hi = min(min(c0, c1), c2);
        out[p] = static_cast<uint8_t>(med3(lo, mid, hi));
    }
}

__global__ void __launch_bounds__(256) median_kernel(const uint8_t* __restrict__ raw, uint8_t* __restrict__ out,
                                                     int W, int H) {
    median_body(raw, out, W, H, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(256) median_batch_kernel(const __grid_constant__ JobTable<MedianJob> t) {
    const int p = find_job(t, blockIdx.x);
    const MedianJob& j = t.job[p];
    const int b = blockIdx.x - t.start[p];
    const int tx = (j.W + 127) / 128;
    median_body(j.raw, j.out, j.W, j.H, b % tx, b / tx);
}

cudaError_t launch_median_batch(JobTable<MedianJob>& t, cudaStream_t stream) {
    t.start[0] = 0;
    for (int i = 0; i < t.n; ++i) t.start[i + 1] = t.start[i] + ((t.job[i].W + 127) / 128) * ((t.job[i].H + 7) / 8);
    median_batch_kernel<<<t.start[t.n], dim3(32, 8), 0, stream>>>(t);
    return cudaGetLastError();
}

cudaError_t launch_median(const uint8_t* raw, uint8_t* disp, int W, int H, cudaStream_t stream) {
    dim3 grid((W + 127) / 128, (H + 7) / 8);
    median_kernel<<<grid, dim3(32, 8), 0, stream>>>(raw, disp, W, H);
    return cudaGetLastError();
}

bool supported_D(int D) { return D >= 32 && D <= 256 && D % 32 == 0; }

}  // namespace sgm

// Dispatch of the aggregation sweeps (Eq. 3, Eq. 4) by disparity count; the
// kernels themselves are in sgm_sweeps.cuh, instantiated per D in
// sgm_sweeps_d<D>.cu so that the translation units compile in parallel.
#include <algorithm>

#include "sgm_pairs.cuh"
#include "sgm_sweeps.cuh"

namespace sgm {

cudaError_t init_kernel_attributes() {
    cudaError_t e = sweep_set_attrs<32>();
    if (e == cudaSuccess) e = sweep_set_attrs<64>();
    if (e == cudaSuccess) e = sweep_set_attrs<96>();
    if (e == cudaSuccess) e = sweep_set_attrs<128>();
    if (e == cudaSuccess) e = sweep_set_attrs<160>();
    if (e == cudaSuccess) e = sweep_set_attrs<192>();
    if (e == cudaSuccess) e = sweep_set_attrs<224>();
    if (e == cudaSuccess) e = sweep_set_attrs<256>();
    return e;
}

#define SGM_DISPATCH_D(FN, D, arg, s)          \
    switch (D) {                               \
        case 32: return FN<32>(arg, s);        \
        case 64: return FN<64>(arg, s);        \
        case 96: return FN<96>(arg, s);        \
        case 128: return FN<128>(arg, s);      \
        case 160: return FN<160>(arg, s);      \
        case 192: return FN<192>(arg, s);      \
        case 224: return FN<224>(arg, s);      \
        case 256: return FN<256>(arg, s);      \
        default: return cudaErrorInvalidValue; \
    }

cudaError_t launch_sweep_h(const SweepArgs& a, cudaStream_t stream) { SGM_DISPATCH_D(sweep_launch_h, a.D, a, stream) }

cudaError_t launch_sweep_v(const SweepArgs& a, cudaStream_t stream) { SGM_DISPATCH_D(sweep_launch_v, a.D, a, stream) }

cudaError_t launch_sweep_first(FirstStageArgs& f, cudaStream_t stream) {
    SGM_DISPATCH_D(sweep_launch_first, f.h.D, f, stream)
}

cudaError_t launch_sweep_first4(FirstStageArgs& f, cudaStream_t stream) {
    SGM_DISPATCH_D(sweep_launch_first4, f.h.D, f, stream)
}

cudaError_t launch_sweep_h2(const SweepArgs& a, cudaStream_t stream) { SGM_DISPATCH_D(sweep_launch_h2, a.D, a, stream) }

cudaError_t launch_sweep_h_list(const ListLaunch& l, cudaStream_t stream) {
    SGM_DISPATCH_D(sweep_launch_h_list, l.D, l, stream)
}

cudaError_t launch_sweep_v_list(const ListLaunch& l, cudaStream_t stream) {
    SGM_DISPATCH_D(sweep_launch_v_list, l.D, l, stream)
}

int sweep_units(int lines, int D, bool pair) {
    // lines per block: a path takes G = 32 lanes (D % 64 == 0) or 16, a pair two paths
    const int G = (D % 64 == 0) ? 32 : 16, per_warp = 32 / G, per = kWarpsPerBlock * per_warp / (pair ? 2 : 1);
    return (lines + per - 1) / per;
}

// The paired-line 4-path schedule: n1 steps of each horizontal direction
// beside the vertical pair in the first launch (default min(W2, H2), which
// ends both at the same step).
PairsArgs pairs_geometry(int W, int H, int D, int n1_req) {
    PairsArgs a{};
    a.W = W;
    a.H = H;
    a.D = D;
    a.W2 = W + (W & 1);
    a.H2 = H + (H & 1);
    a.QW = a.W2 / 2;
    a.QH = a.H2 / 2;
    int n1 = n1_req < 0 ? std::min(a.W2, a.H2) : n1_req;
    a.n1 = std::max(0, std::min(a.W2, n1 & ~1));
    if (a.W2 > 2 * a.n1) {
        a.a = a.b = (a.W2 / 2) & ~1;  // the horizontal pair meets in the middle in the second launch
    } else {
        a.a = a.n1;  // columns [W2 - n1, n1) were passed by both directions in the first launch
        a.b = a.W2 - a.n1;
    }
    a.nvb = a.QW;
    a.nhb = a.QH;
    a.nh2 = a.W2 > a.n1 ? a.QH : 0;
    const int par = (a.a - a.b) / 2 * a.QH;  // quads of the parallel winner-take-all
    const int per_block = 2 * pairs::kParItems;
    a.npw = par > 0 ? (par + per_block - 1) / per_block : 0;
    return a;
}

cudaError_t launch_pairs_stage1(const PairsArgs& a, cudaStream_t stream) {
    SGM_DISPATCH_D(pairs_launch1, a.D, a, stream)
}

cudaError_t launch_pairs_chain2(const PairsArgs& a, cudaStream_t stream) {
    SGM_DISPATCH_D(pairs_launch_chain2, a.D, a, stream)
}

cudaError_t launch_pairs_par(const PairsArgs& a, cudaStream_t stream) {
    SGM_DISPATCH_D(pairs_launch_par, a.D, a, stream)
}

}  // namespace sgm

// Dispatch of the aggregation sweeps (Eq. 3, Eq. 4) by disparity count; the
// kernels themselves are in sgm_sweeps.cuh, instantiated per K in
// sgm_sweeps_k<K>.cu so that the translation units compile in parallel.
#include "sgm_sweeps.cuh"

namespace sgm {

cudaError_t init_kernel_attributes() {
    cudaError_t e = sweep_set_attrs<1>();
    if (e == cudaSuccess) e = sweep_set_attrs<2>();
    if (e == cudaSuccess) e = sweep_set_attrs<3>();
    if (e == cudaSuccess) e = sweep_set_attrs<4>();
    if (e == cudaSuccess) e = sweep_set_attrs<5>();
    if (e == cudaSuccess) e = sweep_set_attrs<6>();
    if (e == cudaSuccess) e = sweep_set_attrs<7>();
    if (e == cudaSuccess) e = sweep_set_attrs<8>();
    return e;
}

// K = D / 32 words per lane (16 lanes per path).
#define SGM_DISPATCH_K(FN, a, s)               \
    switch ((a).D / 32) {                      \
        case 1: return FN<1>(a, s);            \
        case 2: return FN<2>(a, s);            \
        case 3: return FN<3>(a, s);            \
        case 4: return FN<4>(a, s);            \
        case 5: return FN<5>(a, s);            \
        case 6: return FN<6>(a, s);            \
        case 7: return FN<7>(a, s);            \
        case 8: return FN<8>(a, s);            \
        default: return cudaErrorInvalidValue; \
    }

cudaError_t launch_sweep_h(const SweepArgs& a, cudaStream_t stream) { SGM_DISPATCH_K(sweep_launch_h, a, stream) }

cudaError_t launch_sweep_v(const SweepArgs& a, cudaStream_t stream) { SGM_DISPATCH_K(sweep_launch_v, a, stream) }

#define SGM_DISPATCH_K_TABLE(FN, t, s)         \
    switch ((t).job[0].D / 32) {               \
        case 1: return FN<1>(t, s);            \
        case 2: return FN<2>(t, s);            \
        case 3: return FN<3>(t, s);            \
        case 4: return FN<4>(t, s);            \
        case 5: return FN<5>(t, s);            \
        case 6: return FN<6>(t, s);            \
        case 7: return FN<7>(t, s);            \
        case 8: return FN<8>(t, s);            \
        default: return cudaErrorInvalidValue; \
    }

cudaError_t launch_sweep_h_batch(JobTable<SweepArgs>& t, cudaStream_t stream) {
    if (t.n < 1) return cudaSuccess;
    SGM_DISPATCH_K_TABLE(sweep_launch_h_batch, t, stream)
}

cudaError_t launch_sweep_v_batch(JobTable<SweepArgs>& t, cudaStream_t stream) {
    if (t.n < 1) return cudaSuccess;
    SGM_DISPATCH_K_TABLE(sweep_launch_v_batch, t, stream)
}

}  // namespace sgm

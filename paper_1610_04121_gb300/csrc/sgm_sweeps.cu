// Dispatch of the aggregation sweeps (Eq. 3, Eq. 4) by disparity count; the
// kernels themselves are in sgm_sweeps.cuh, instantiated per D in
// sgm_sweeps_d<D>.cu so that the translation units compile in parallel.
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

cudaError_t launch_sweep_h_batch(JobTable<SweepArgs>& t, cudaStream_t stream) {
    if (t.n < 1) return cudaSuccess;
    SGM_DISPATCH_D(sweep_launch_h_batch, t.job[0].D, t, stream)
}

cudaError_t launch_sweep_v_batch(JobTable<SweepArgs>& t, cudaStream_t stream) {
    if (t.n < 1) return cudaSuccess;
    SGM_DISPATCH_D(sweep_launch_v_batch, t.job[0].D, t, stream)
}

}  // namespace sgm

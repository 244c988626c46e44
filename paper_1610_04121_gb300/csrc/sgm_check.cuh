// The bounds-checked build (-DSGM_BOUNDS_CHECK).  Every global access of the
// sweeps and stages (and the shared-memory feature indices of the cost
// kernels) is tested against the extent of the array it belongs to; the
// first violation records its site number in the translation unit's fault
// word and the access is skipped (a load yields zeros).  Nothing traps.  The
// host reads and clears the fault words after every synchronous call and
// reports SGM_EDEVICE.  In the ordinary build every guard is the constant
// true and compiles away.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace sgm {

// Host: collect the fault words of every translation unit (first site found
// wins, all words are cleared); 0 when none fired.
void register_bounds_reader(unsigned (*reader)());
unsigned take_bounds_fault();

#ifdef SGM_BOUNDS_CHECK
static __device__ unsigned int g_bounds_fault = 0;

__device__ __forceinline__ bool bounds_guard(const void* p, size_t n, const void* lo, const void* hi, unsigned site) {
    const char* q = static_cast<const char*>(p);
    if (q >= static_cast<const char*>(lo) && q + n <= static_cast<const char*>(hi)) return true;
    atomicCAS(&g_bounds_fault, 0u, site);
    return false;
}

__device__ __forceinline__ bool bounds_guard_index(long long i, long long n, unsigned site) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_bounds_fault, 0u, site);
    return false;
}

namespace {
unsigned take_bounds_fault_here() {
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_fault, sizeof v) != cudaSuccess) return 0;
    if (v != 0) cudaMemcpyToSymbol(g_bounds_fault, &z, sizeof z);
    return v;
}
struct BoundsReaderRegistrar {
    BoundsReaderRegistrar() { register_bounds_reader(&take_bounds_fault_here); }
};
const BoundsReaderRegistrar g_bounds_registrar;
}  // namespace

#define SGM_GUARD(p, n, lo, hi, site) ::sgm::bounds_guard((p), (n), (lo), (hi), (site))
#define SGM_GUARD_INDEX(i, n, site) ::sgm::bounds_guard_index((i), (n), (site))
#else
#define SGM_GUARD(p, n, lo, hi, site) true
#define SGM_GUARD_INDEX(i, n, site) true
#endif

}  // namespace sgm

// Aggregation sweeps for D = 64 (32 lanes per path, 1 packed word per lane).
#include "sgm_pairs.cuh"
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(64)
SGM_INSTANTIATE_PAIRS(64)
}  // namespace sgm

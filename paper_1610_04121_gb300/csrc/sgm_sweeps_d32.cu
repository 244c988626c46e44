// Aggregation sweeps for D = 32 (16 lanes per path, 1 packed word per lane).
#include "sgm_pairs.cuh"
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(32)
SGM_INSTANTIATE_PAIRS(32)
}  // namespace sgm

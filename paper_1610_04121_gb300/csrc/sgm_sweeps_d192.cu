// Aggregation sweeps for D = 192 (32 lanes per path, 3 packed words per lane).
#include "sgm_pairs.cuh"
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(192)
SGM_INSTANTIATE_PAIRS(192)
}  // namespace sgm

// Aggregation sweeps for D = 128 (32 lanes per path, 2 packed words per lane).
#include "sgm_pairs.cuh"
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(128)
SGM_INSTANTIATE_PAIRS(128)
}  // namespace sgm

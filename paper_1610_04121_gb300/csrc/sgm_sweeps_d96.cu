// Aggregation sweeps for D = 96 (16 lanes per path, 3 packed words per lane).
#include "sgm_pairs.cuh"
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(96)
SGM_INSTANTIATE_PAIRS(96)
}  // namespace sgm

// Aggregation sweeps for D = 160 (16 lanes per path, 5 packed words per lane).
#include "sgm_pairs.cuh"
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(160)
SGM_INSTANTIATE_PAIRS(160)
}  // namespace sgm

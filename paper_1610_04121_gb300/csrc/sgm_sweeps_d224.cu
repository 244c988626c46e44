// Aggregation sweeps for D = 224 (16 lanes per path, 7 packed words per lane).
#include "sgm_pairs.cuh"
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(224)
SGM_INSTANTIATE_PAIRS(224)
}  // namespace sgm

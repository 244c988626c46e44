// Aggregation sweeps for D = 256 (32 lanes per path, 4 packed words per lane).
#include "sgm_pairs.cuh"
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(256)
SGM_INSTANTIATE_PAIRS(256)
}  // namespace sgm

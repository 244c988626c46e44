// Aggregation sweeps for D = 96 (16 lanes per path, 3 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(96)
}  // namespace sgm

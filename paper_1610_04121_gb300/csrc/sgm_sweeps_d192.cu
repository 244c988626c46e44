// Aggregation sweeps for D = 192 (32 lanes per path, 3 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(192)
}  // namespace sgm

// Aggregation sweeps for D = 32 (1 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(1)
}  // namespace sgm

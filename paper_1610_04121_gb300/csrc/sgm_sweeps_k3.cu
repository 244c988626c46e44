// Aggregation sweeps for D = 96 (3 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(3)
}  // namespace sgm

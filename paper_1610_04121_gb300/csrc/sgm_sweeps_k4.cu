// Aggregation sweeps for D = 128 (4 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(4)
}  // namespace sgm

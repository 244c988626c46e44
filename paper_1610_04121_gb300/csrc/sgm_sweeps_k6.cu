// Aggregation sweeps for D = 192 (6 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(6)
}  // namespace sgm

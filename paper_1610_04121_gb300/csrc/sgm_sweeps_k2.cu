// Aggregation sweeps for D = 64 (2 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(2)
}  // namespace sgm

// Aggregation sweeps for D = 256 (8 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(8)
}  // namespace sgm

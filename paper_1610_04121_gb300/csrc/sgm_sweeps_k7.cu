// Aggregation sweeps for D = 224 (7 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(7)
}  // namespace sgm

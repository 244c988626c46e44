// Aggregation sweeps for D = 160 (5 packed words per lane).
#include "sgm_sweeps.cuh"

namespace sgm {
SGM_INSTANTIATE_SWEEPS(5)
}  // namespace sgm

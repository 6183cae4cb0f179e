// Instantiations of the (sub-)warp row-major kernel for FP32 and FP64.
#include "pull_warp.cuh"

namespace asv {
ASV_INSTANTIATE_PULL_WARP(float)
ASV_INSTANTIATE_PULL_WARP(double)
}  // namespace asv

// Kernels of the 3-D mesh (all degrees).
#include "kernels.cuh"

namespace dgsrhd {
template cudaError_t dispatch_stage<3>(int N, const StageArgs& a);
}  // namespace dgsrhd

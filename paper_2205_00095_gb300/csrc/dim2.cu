// Kernels of the 2-D mesh (all degrees).
#include "kernels.cuh"

namespace dgsrhd {
template cudaError_t dispatch_stage<2>(int N, const StageArgs& a);
}  // namespace dgsrhd

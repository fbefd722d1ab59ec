// Kernels of the 1-D mesh (all degrees).
#include "kernels.cuh"

namespace dgsrhd {
template cudaError_t dispatch_stage<1>(int N, const StageArgs& a);
}  // namespace dgsrhd

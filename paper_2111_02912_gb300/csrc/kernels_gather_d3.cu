// Interpolation kernels for 3-dimensional images (template in interp.cuh).
#include "interp.cuh"

namespace nj {

cudaError_t launch_gather_d3(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s) {
    return gather_dim<3>(mode, a, cpl, s);
}

}  // namespace nj

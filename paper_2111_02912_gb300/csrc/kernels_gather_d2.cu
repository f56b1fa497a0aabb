// Interpolation kernels for 2-dimensional images (template in interp.cuh).
#include "interp.cuh"

namespace nj {

cudaError_t launch_gather_d2(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s) {
    return gather_dim<2>(mode, a, cpl, s);
}

}  // namespace nj

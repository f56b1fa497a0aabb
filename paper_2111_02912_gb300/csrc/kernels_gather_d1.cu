// Interpolation kernels for 1-dimensional images (template in interp.cuh).
#include "interp.cuh"

namespace nj {

cudaError_t launch_gather_d1(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s) {
    return gather_dim<1>(mode, a, cpl, s);
}

}  // namespace nj

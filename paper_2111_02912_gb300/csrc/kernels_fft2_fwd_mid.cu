// Register-resident two-phase line FFT, pass kind PASS_FWD_MID (one translation
// unit per pass kind so that the kernels compile in parallel).
#include "fft_twostep.cuh"

namespace nj {
template cudaError_t launch_fft2_kind<PASS_FWD_MID>(int, int, const LinePass&, dim3, int, size_t, cudaStream_t);
}  // namespace nj

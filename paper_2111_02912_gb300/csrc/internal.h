// Host-side launcher declarations shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace nj {

// ---------------------------------------------------------------- sorting
struct SortArgs {
    const float* omega;   // [D][M]
    int64_t m;
    int D, J;
    int K[kMaxDim];
    int B[kMaxDim], nb[kMaxDim];
    int nbins, P;
    float c_hi[kMaxDim], c_lo[kMaxDim];  // K/(2 pi) as a float pair
    int* count;       // [nbins]
    int* local;       // [M]
    int* binid;       // [M]
    int* offsets;     // [nbins + 1]
    int* subp_off;    // [nbins + 1]
    int4* subp;       // [nbins + M/P + 1]
    int* nsubp;       // [1]
    int4* pidx;       // [M]
    float4* pfrac;    // [M]
};
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s);
cudaError_t launch_bin_count(const SortArgs& a, cudaStream_t s);
cudaError_t launch_bin_scan(const SortArgs& a, cudaStream_t s);
cudaError_t launch_bin_scatter(const SortArgs& a, cudaStream_t s);
cudaError_t launch_bin_subprob(const SortArgs& a, cudaStream_t s);

// -------------------------------------------------------------------- FFT
struct ImageSide {
    const float2* x;       // image(s), [N] or [C][N]
    const float2* smaps;   // [C][N] or null
    float2* xout;          // adjoint image output
    int C;                 // coils
    int has_plain;         // forward side: channel block 0 is the unweighted image
    int D;
    int N[kMaxDim];
    const float* deap[kMaxDim];   // per-dim scaling factors s_d[n]
    int64_t nimg;          // prod N
};

struct LinePass {
    FftAxis ax;
    int n_in, n_out;       // elements along the axis on input / output side
    int64_t B, S;          // outer lines, inner stride (complex elements)
    int TB, TS, lgTS, lgTL, TLP;
    int nchunks;           // coil-sum epilogue: channel chunks looped in one block
    int coil_sum;
    const float2* in;
    float2* out;
    ImageSide im;
    uint32_t magic_L;      // ceil(2^32 / L)
    uint32_t magic_n;      // ceil(2^32 / n) for the axis length used in index maps
};
enum PassKind { PASS_FWD_FIRST, PASS_FWD_MID, PASS_INV_MID, PASS_INV_LAST };
cudaError_t launch_line_pass(PassKind kind, const LinePass& a, dim3 grid, int threads, size_t smem,
                             cudaStream_t s);

// ---------------------------------------------------------- interpolation
enum GatherMode { GM_FWD = 0, GM_JVP = 1, GM_VJP = 2 };
struct GatherArgs {
    PointsView pts;
    int D, J;
    int K[kMaxDim];
    const float2* grid;   // [K...][ch], ch = nd * C, channel = dblock * C + c
    int C, nd, has_plain;
    int G, lgG;           // lanes per point (power of two <= 32)
    KbPoly kb;
    int64_t M;
    float2* y;            // [C][M]
    float2* dy;           // [C][M]
    const float* domega;  // [D][M]
    const float2* v;      // [C][M]
    float* grad;          // [D][M]
};
cudaError_t launch_gather(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s);

struct SpreadArgs {
    PointsView pts;
    int D, J;
    int K[kMaxDim];
    int B[kMaxDim], nb[kMaxDim], T[kMaxDim];   // bin edge, bins per dim, tile extent B+J-1
    const int4* subp;
    const int* nsubp;
    int max_subp;
    const float2* y;      // [C][M]
    int64_t M;
    int C, CC;            // coils, coils per block
    int G, lgG;
    KbPoly kb;
    float2* grid;         // [K...][C]
};
cudaError_t launch_spread(const SpreadArgs& a, int cpl, cudaStream_t s, size_t smem);

}  // namespace nj

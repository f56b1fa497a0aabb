// Shared types and device helpers of the NUFFT-Jacobian kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace nj {

constexpr int kMaxDim = 3;
constexpr int kMaxStages = 12;
constexpr int kKbTerms = 32;   // Horner terms of the Kaiser-Bessel power series
constexpr int kJMin = 4;       // smallest interpolation width
constexpr int kJMax = 8;       // largest interpolation width
constexpr int kFftEpt = 16;    // complex elements held per thread in an FFT pass

// ---------------------------------------------------------------- kernel psi
// psi(u) = I0(beta sqrt(1 - (2u/J)^2)) on |u| < J/2 (open support).  With
// z = 1 - (2u/J)^2 the power series of I0 gives psi = sum_k a_k z^k,
// a_k = (beta^2/4)^k / (k!)^2: all terms positive on z in (0, 1].
struct KbPoly {
    float a[kKbTerms];   // a_k, zero-padded past the needed degree
    float two_over_j;    // 2/J
};

__device__ __forceinline__ float kb_psi(const float* __restrict__ a, float two_over_j, float u) {
    const float s = u * two_over_j;
    const float z = fmaf(-s, s, 1.0f);
    float acc = a[kKbTerms - 1];
#pragma unroll
    for (int k = kKbTerms - 2; k >= 0; --k) acc = fmaf(acc, z, a[k]);
    return z > 0.f ? acc : 0.f;
}

// psi read from a table of psi(l / L), l = 0 .. n + 1, zero from l = n = L J / 2 on, by linear
// interpolation in |u| L: the table interpolator the paper's baseline uses (Sec. II-B, Sec. IV-A).
__device__ __forceinline__ float kb_table(const float* __restrict__ tab, float L, int n, float u) {
    const float au = fabsf(u) * L;
    const float lf = floorf(au);
    const int l = min((int)lf, n);
    const float a = au - lf;
    return fmaf(a, __ldg(tab + l + 1) - __ldg(tab + l), __ldg(tab + l));
}

// ---------------------------------------------------------- sorted points
// Per point, per dim: wrapped window start k0 in [0, K) and the offset of the
// first tap u0 = t - k0_unwrapped in [J/2 - 1, J/2); tap j has offset u0 - j.
// idx.w holds the caller's point index.  w holds the D*J kernel weights of
// each sorted point, psi(u0_d - j) at w[i * ws + d * wd + j] (wd = J and ws =
// D*J rounded up to a multiple of 4; for the strip spread wd = 8, ws = 8 D, the
// pads zero), evaluated once per omega by the sort.
struct PointsView {
    const int4* idx;     // {k0_0, k0_1, k0_2, original index}, sorted by bin
    const float4* frac;  // {u0_0, u0_1, u0_2, 0}
    int64_t m;
    const float* w;      // [m][ws] kernel weights
    int ws;
    int wd;              // weights per dimension in a row: J, or 8 (strip layout, zero padded)
};

// ------------------------------------------------------------- FFT plans
struct FftStage {
    int R;          // radix
    int Ns;         // product of the radices of the earlier stages
    int tw_step;    // L / (Ns R): twiddle table stride
    uint32_t magic; // ceil(2^32 / Ns) for Ns > 1 (division j / Ns)
};

struct FftAxis {
    int L;
    int nstages;
    FftStage st[kMaxStages];
    const float2* tw;   // exp(-2 pi i t / L), t < L (device)
    const float2* tw2;  // two-phase kernels, L = L1 L2: exp(-2 pi i n2 k1 / L) at n2 L1 + k1 (device)
};

__device__ __forceinline__ uint32_t div_magic(uint32_t n, uint32_t d, uint32_t magic) {
    return d == 1 ? n : __umulhi(n, magic);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Raise a kernel's dynamic shared-memory limit once per device (not on every
// launch), so that launches recorded into a CUDA graph make no attribute call.
template <auto KERNEL>
inline void ensure_smem(size_t bytes) {
    static std::atomic<size_t> done[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (bytes > done[dev].load(std::memory_order_relaxed)) {
        cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        done[dev].store(bytes, std::memory_order_relaxed);
    }
}


// Programmatic dependent launch (sm_90 and later).  Kernels are launched with programmatic stream
// serialization, so the launch of a kernel is processed while the kernel before it in the stream
// still runs, and every kernel starts with pdl_wait(): griddepcontrol.wait blocks until that
// previous kernel has completed and its memory operations are visible (at once for a kernel
// launched without the attribute).  Every global access thus still follows the previous kernel's
// completion; only the launch gap between them shrinks.  No kernel signals its dependents early
// (griddepcontrol.launch_dependents): blocks parked on the wait held SM slots that a concurrent
// stream's kernels needed (measured: replayed radial320 step 0.2895 -> 0.3037 ms with an early
// signal, 0.2857 ms without; eager step 0.3126 -> 0.2887 ms).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// Launches kernel<<<grid, block, smem, s>>>(args...) with programmatic stream serialization.
template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace nj

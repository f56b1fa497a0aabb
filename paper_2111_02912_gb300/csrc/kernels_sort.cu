// Bin sort of the sample locations (done once per omega update).
//
// For every point and dimension the window of the J-tap interpolator (Appendix:
// offsets k_m and coefficients u_j(omega_m)) is fixed by t = omega K / (2 pi):
// taps k = floor(t - J/2) + 1 + j, j = 0..J-1, with offsets t - k.  t is formed
// as an unevaluated float pair (an FMA recovers the rounding error of the
// product omega * c_hi, Dekker / Ogita-Rump-Oishi error-free product), so the
// integer window start and the fractional offset keep ~2^-40 relative accuracy
// of the FP64 value although all arithmetic is FP32.
#include <algorithm>

#include "internal.h"

namespace nj {

__device__ __forceinline__ void window_of(float w, float c_hi, float c_lo, int K, int J, int& k0, float& u0) {
    const float p = w * c_hi;
    float e = fmaf(w, c_hi, -p);       // exact rounding error of the product
    e = fmaf(w, c_lo, e);
    float fl = floorf(p);
    float fr = (p - fl) + e;           // p - fl is exact
    if (fr < 0.f) { fr += 1.f; fl -= 1.f; }
    else if (fr >= 1.f) { fr -= 1.f; fl += 1.f; }
    const int hq = J >> 1;
    const float hf = (J & 1) ? 0.5f : 0.f;
    long long start;
    if (fr < hf) { start = (long long)fl - hq;     u0 = fr + (float)hq; }
    else         { start = (long long)fl - hq + 1; u0 = fr + (float)(hq - 1); }
    long long s = start % K;
    if (s < 0) s += K;
    k0 = (int)s;
}

__device__ __forceinline__ void point_record(const SortArgs& a, int64_t i, int4& ix, float4& fr, int& bin) {
    int k0[3] = {0, 0, 0};
    float u0[3] = {0.f, 0.f, 0.f};
    bin = 0;
    for (int d = 0; d < a.D; ++d) {
        window_of(a.omega[(int64_t)d * a.m + i], a.c_hi[d], a.c_lo[d], a.K[d], a.J, k0[d], u0[d]);
        bin = bin * a.nb[d] + k0[d] / a.B[d];
    }
    ix = make_int4(k0[0], k0[1], k0[2], (int)i);
    fr = make_float4(u0[0], u0[1], u0[2], 0.f);
}

__global__ void k_zero(float4* p, int64_t n4, int* tail, int64_t ntail) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (blockIdx.x == 0 && threadIdx.x < ntail) tail[threadIdx.x] = 0;
}

__global__ void k_bin_count(SortArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    int4 ix;
    float4 fr;
    int bin;
    point_record(a, i, ix, fr, bin);
    a.binid[i] = bin;
    a.local[i] = atomicAdd(&a.count[bin], 1);
}

// One block: exclusive scans of the bin counts and of the per-bin numbers of
// sub-problems (ceil(count / P)).
__global__ void k_bin_scan(SortArgs a) {
    __shared__ int s_pts[1024];
    __shared__ int s_sub[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const int per = (a.nbins + nt - 1) / nt;
    const int lo = min(a.nbins, t * per), hi = min(a.nbins, lo + per);
    int sp = 0, ss = 0;
    for (int b = lo; b < hi; ++b) {
        const int c = a.count[b];
        sp += c;
        ss += (c + a.P - 1) / a.P;
    }
    s_pts[t] = sp;
    s_sub[t] = ss;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {   // Hillis-Steele inclusive scan
        int vp = 0, vs = 0;
        if (t >= off) { vp = s_pts[t - off]; vs = s_sub[t - off]; }
        __syncthreads();
        s_pts[t] += vp;
        s_sub[t] += vs;
        __syncthreads();
    }
    int rp = t ? s_pts[t - 1] : 0, rs = t ? s_sub[t - 1] : 0;
    for (int b = lo; b < hi; ++b) {
        const int c = a.count[b];
        a.offsets[b] = rp;
        a.subp_off[b] = rs;
        rp += c;
        rs += (c + a.P - 1) / a.P;
    }
    if (t == nt - 1) {
        a.offsets[a.nbins] = s_pts[t];
        a.subp_off[a.nbins] = s_sub[t];
        a.nsubp[0] = s_sub[t];
    }
}

__global__ void k_bin_scatter(SortArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    int4 ix;
    float4 fr;
    int bin;
    point_record(a, i, ix, fr, bin);
    const int dst = a.offsets[a.binid[i]] + a.local[i];
    a.pidx[dst] = ix;
    a.pfrac[dst] = fr;
}

__global__ void k_bin_subprob(SortArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.nbins) return;
    const int start = a.offsets[b], cnt = a.offsets[b + 1] - start;
    const int base = a.subp_off[b];
    for (int s = 0; s * a.P < cnt; ++s)
        a.subp[base + s] = make_int4(b, start + s * a.P, min(a.P, cnt - s * a.P), 0);
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s) {
    const int64_t n4 = (int64_t)(bytes / 16);
    const int64_t ntail = (int64_t)((bytes - n4 * 16) / 4);
    int blocks = (int)std::min<int64_t>((n4 + 255) / 256, 152 * 16);
    if (blocks < 1) blocks = 1;
    k_zero<<<blocks, 256, 0, s>>>((float4*)p, n4, (int*)((char*)p + n4 * 16), ntail);
    return cudaGetLastError();
}
cudaError_t launch_bin_count(const SortArgs& a, cudaStream_t s) {
    if (a.m == 0) return cudaSuccess;
    k_bin_count<<<(unsigned)((a.m + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_bin_scan(const SortArgs& a, cudaStream_t s) {
    k_bin_scan<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_bin_scatter(const SortArgs& a, cudaStream_t s) {
    if (a.m == 0) return cudaSuccess;
    k_bin_scatter<<<(unsigned)((a.m + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_bin_subprob(const SortArgs& a, cudaStream_t s) {
    k_bin_subprob<<<(a.nbins + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace nj

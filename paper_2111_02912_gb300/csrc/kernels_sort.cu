// Bin sort of the sample locations (done once per omega update).
//
// For every point and dimension the window of the J-tap interpolator (Appendix:
// offsets k_m and coefficients u_j(omega_m)) is fixed by t = omega K / (2 pi):
// taps k = floor(t - J/2) + 1 + j, j = 0..J-1, with offsets t - k.  t is formed
// as an unevaluated float pair (an FMA recovers the rounding error of the
// product omega * c_hi, Dekker / Ogita-Rump-Oishi error-free product), so the
// integer window start and the fractional offset keep ~2^-40 relative accuracy
// of the FP64 value although all arithmetic is FP32.
//
// Counting sort by key = (bin, cell of the window start): bins are tiles of
// B_d cells per axis; inside a bin, points are ordered by the cell their
// window starts in, so points that share a window are adjacent.  The spread
// (the adjoint interpolation) is output-driven: tile t owns its cells and
// takes contributions from the points of the bins that can reach it, so the
// sort also lists the spread's work items (candidate ranges of <= P points).
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

__device__ __forceinline__ void point_record(const SortArgs& a, int64_t i, int4& ix, float4& fr, int64_t& key) {
    int k0[3] = {0, 0, 0};
    float u0[3] = {0.f, 0.f, 0.f};
    int64_t bin = 0, cell = 0;
    for (int d = 0; d < a.D; ++d) {
        window_of(a.omega[(int64_t)d * a.m + i], a.c_hi[d], a.c_lo[d], a.K[d], a.J, k0[d], u0[d]);
        bin = bin * a.nb[d] + k0[d] / a.B[d];
        cell = cell * a.B[d] + k0[d] % a.B[d];
    }
    key = bin * a.cpb + cell;
    ix = make_int4(k0[0], k0[1], k0[2], (int)i);
    fr = make_float4(u0[0], u0[1], u0[2], 0.f);
}

__global__ void k_zero(float4* p, int64_t n4, int* tail, int64_t ntail) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (blockIdx.x == 0 && threadIdx.x < ntail) tail[threadIdx.x] = 0;
}

__global__ void k_key_count(SortArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    int4 ix;
    float4 fr;
    int64_t key;
    point_record(a, i, ix, fr, key);
    a.keyid[i] = (int)key;
    a.local[i] = atomicAdd(&a.kcount[key], 1);
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int* sh, int& excl) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sh[lane] = w;
    }
    __syncthreads();
    const int total = sh[nw - 1];
    excl = x - v + (wid ? sh[wid - 1] : 0);
    __syncthreads();
    return total;
}

// Pass 1: each block scans kScanPerBlock keys in place (exclusive, block-local).
__global__ void __launch_bounds__(1024) k_scan_local(SortArgs a) {
    __shared__ int sh[32];
    constexpr int per = kScanPerBlock / 1024;
    const int64_t base = (int64_t)blockIdx.x * kScanPerBlock + (int64_t)threadIdx.x * per;
    int v[per], s = 0;
#pragma unroll
    for (int q = 0; q < per; ++q) {
        v[q] = base + q < a.nkeys ? a.kcount[base + q] : 0;
        s += v[q];
    }
    int excl;
    const int total = block_exclusive_scan(s, sh, excl);
#pragma unroll
    for (int q = 0; q < per; ++q) {
        if (base + q < a.nkeys) a.kcount[base + q] = excl;
        excl += v[q];
    }
    if (threadIdx.x == 0) a.bsum[blockIdx.x] = total;
}

// Pass 2 (one block): exclusive scan of the block totals.
__global__ void __launch_bounds__(1024) k_scan_bsum(SortArgs a, int nblk) {
    __shared__ int sh[32];
    const int per = (nblk + 1023) / 1024;
    const int lo = min(nblk, (int)threadIdx.x * per), hi = min(nblk, lo + per);
    int s = 0;
    for (int b = lo; b < hi; ++b) s += a.bsum[b];
    int excl;
    block_exclusive_scan(s, sh, excl);
    for (int b = lo; b < hi; ++b) {
        const int v = a.bsum[b];
        a.bsum[b] = excl;
        excl += v;
    }
}

// Pass 3: add the block offsets; record the first position of every bin.
__global__ void k_scan_add(SortArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= a.nkeys) return;
    const int v = a.kcount[k] + a.bsum[k / kScanPerBlock];
    a.kcount[k] = v;
    if (k % a.cpb == 0) a.offsets[k / a.cpb] = v;
    if (k == a.nkeys - 1) a.offsets[a.nbins] = (int)a.m;
}

// One block: spread work items per tile (candidates = points of the bins that
// can reach the tile, at most 3^D bins), and their exclusive scan.
__global__ void __launch_bounds__(1024) k_tile_scan(SortArgs a) {
    __shared__ int sh[32];
    const int per = (a.nbins + 1023) / 1024;
    const int lo = min(a.nbins, (int)threadIdx.x * per), hi = min(a.nbins, lo + per);
    int nbr[27];
    int si = 0;
    for (int b = lo; b < hi; ++b) {
        const int nn = neighbour_bins(a.D, a.nb, a.B, a.K, a.J, b, nbr);
        int* tn = a.tile_nbr + (int64_t)b * kNbrStride;
        tn[0] = nn;
        int cand = 0;
        for (int q = 0; q < nn; ++q) {
            const int st = a.offsets[nbr[q]];
            tn[1 + 2 * q] = st;
            tn[2 + 2 * q] = cand;
            cand += a.offsets[nbr[q] + 1] - st;
        }
        tn[1 + 2 * nn] = 0;
        tn[2 + 2 * nn] = cand;
        const int parts = max(1, (cand + a.P - 1) / a.P);
        a.tile_parts[b] = parts;
        si += parts;
    }
    int excl;
    const int total = block_exclusive_scan(si, sh, excl);
    for (int b = lo; b < hi; ++b) {
        a.item_off[b] = excl;
        excl += a.tile_parts[b];
    }
    if (threadIdx.x == 0) {
        a.item_off[a.nbins] = total;
        a.nitems[0] = total;
    }
}

__global__ void k_bin_scatter(SortArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    int4 ix;
    float4 fr;
    int64_t key;
    point_record(a, i, ix, fr, key);
    const int dst = a.kcount[a.keyid[i]] + a.local[i];
    a.pidx[dst] = ix;
    a.pfrac[dst] = fr;
    // the D*J kernel weights, evaluated once here and read by every gather and spread
    float* w = a.pw + (int64_t)dst * a.ws;
    for (int d = 0; d < a.D; ++d) {
        const float u0 = d == 0 ? fr.x : (d == 1 ? fr.y : fr.z);
        for (int j = 0; j < a.J; ++j) w[d * a.J + j] = kb_psi(a.kb.a, a.kb.two_over_j, u0 - (float)j);
    }
}

__global__ void k_bin_items(SortArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.nbins) return;
    const int parts = a.tile_parts[b], base = a.item_off[b];
    for (int k = 0; k < parts; ++k) a.items[base + k] = make_int4(b, k, parts, 0);
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s) {
    const int64_t n4 = (int64_t)(bytes / 16);
    const int64_t ntail = (int64_t)((bytes - n4 * 16) / 4);
    int blocks = (int)std::min<int64_t>((n4 + 255) / 256, 152 * 16);
    if (blocks < 1) blocks = 1;
    k_zero<<<blocks, 256, 0, s>>>((float4*)p, n4, (int*)((char*)p + n4 * 16), ntail);
    return cudaGetLastError();
}
cudaError_t launch_key_count(const SortArgs& a, cudaStream_t s) {
    if (a.m == 0) return cudaSuccess;
    k_key_count<<<(unsigned)((a.m + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_key_scan(const SortArgs& a, cudaStream_t s) {
    const int nblk = (int)((a.nkeys + kScanPerBlock - 1) / kScanPerBlock);
    k_scan_local<<<nblk, 1024, 0, s>>>(a);
    k_scan_bsum<<<1, 1024, 0, s>>>(a, nblk);
    k_scan_add<<<(unsigned)((a.nkeys + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_tile_scan(const SortArgs& a, cudaStream_t s) {
    k_tile_scan<<<1, 1024, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_bin_scatter(const SortArgs& a, cudaStream_t s) {
    if (a.m == 0) return cudaSuccess;
    k_bin_scatter<<<(unsigned)((a.m + 255) / 256), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_bin_items(const SortArgs& a, cudaStream_t s) {
    k_bin_items<<<(a.nbins + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace nj

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
// Counting sort by the bin of the window start (bins are tiles of B_d cells
// per axis): a histogram with atomics, one block's exclusive scan (which also
// clears the histogram for the next sort), and a scatter that writes the
// point records and their D*J kernel weights in bin order.  The spread (the
// adjoint interpolation) is output-driven: tile t owns its cells and takes
// contributions from the points of the bins that can reach it, so the sort
// also lists, per tile, those bins and the spread's work items (candidate
// ranges of <= P points).
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
    int64_t bin = 0;
    for (int d = 0; d < a.D; ++d) {
        window_of(a.omega[(int64_t)d * a.m + i], a.c_hi[d], a.c_lo[d], a.K[d], a.J, k0[d], u0[d]);
        bin = bin * a.nb[d] + k0[d] / a.B[d];
    }
    key = bin;
    ix = make_int4(k0[0], k0[1], k0[2], (int)i);
    fr = make_float4(u0[0], u0[1], u0[2], 0.f);
}

__global__ void k_zero(float4* p, int64_t n4, int* tail, int64_t ntail) {
    pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (blockIdx.x == 0 && threadIdx.x < ntail) tail[threadIdx.x] = 0;
}

// Histogram of bins and each point's rank within its bin.  Consecutive samples
// (a trajectory's readout) usually share a bin, so the lanes of a warp with the
// same bin take one atomic between them: the group leader adds the group size
// and the others offset from the returned base by their rank in the group.
__global__ void k_key_count(SortArgs a) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i < a.m;
    int key = -1;
    if (live) {
        int4 ix;
        float4 fr;
        int64_t k64;
        point_record(a, i, ix, fr, k64);
        key = (int)k64;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (!live) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(&a.kcount[key], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    a.keyid[i] = key;
    a.local[i] = base + rank;
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

// One block: exclusive scan of the bin counts into offsets (offsets[nbins] = m).
// Each thread scans a contiguous chunk; the counts are cleared on the way, so
// the next sort needs no clearing pass.
__global__ void __launch_bounds__(1024) k_bin_scan(SortArgs a) {
    pdl_wait();
    __shared__ int sh[32];
    const int n = a.nbins;
    const int per = (n + 1023) / 1024;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    int s = 0;
    for (int b = lo; b < hi; ++b) s += a.kcount[b];
    int excl;
    block_exclusive_scan(s, sh, excl);
    for (int b = lo; b < hi; ++b) {
        const int v = a.kcount[b];
        a.offsets[b] = excl;
        a.kcount[b] = 0;
        excl += v;
    }
    if (threadIdx.x == 0) {
        a.offsets[n] = (int)a.m;
        a.heavy[0] = 0;
    }
}

// Per tile: the bins that can reach it (its own and those holding the J-1
// cells before it, at most 3^D), their point ranges as one candidate list, and
// the number of spread work items (candidates / P, at least one).
__global__ void k_tile_lists(SortArgs a) {
    pdl_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.nbins) return;
    const int cand = tile_bin_list(a.D, a.nb, a.B, a.K, a.J, b, a.offsets, a.tile_nbr + b, a.nbins);
    a.tile_parts[b] = max(1, (cand + a.P - 1) / a.P);
}

// One block: exclusive scan of the work items per tile, and the item list
// {tile, part, parts, 0}.
__global__ void __launch_bounds__(1024) k_item_scan(SortArgs a) {
    pdl_wait();
    __shared__ int sh[32];
    const int n = a.nbins;
    const int per = (n + 1023) / 1024;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    int s = 0;
    for (int b = lo; b < hi; ++b) s += a.tile_parts[b];
    int excl;
    const int total = block_exclusive_scan(s, sh, excl);
    for (int b = lo; b < hi; ++b) {
        const int parts = a.tile_parts[b];
        a.item_off[b] = excl;
        for (int k = 0; k < parts; ++k) a.items[excl + k] = make_int4(b, k, parts, 0);
        if (parts > 1) a.heavy[1 + atomicAdd(a.heavy, 1)] = b;
        excl += parts;
    }
    if (threadIdx.x == 0) {
        a.item_off[n] = total;
        a.nitems[0] = total;
    }
}

// All three tables in one block when the bins are few (one launch instead of
// three): bin offsets, the tiles' reaching bins and parts, item offsets and list.
__global__ void __launch_bounds__(1024) k_sort_tables(SortArgs a) {
    pdl_wait();
    __shared__ int sh[32];
    const int n = a.nbins, t = threadIdx.x;
    const int per = (n + 1023) / 1024;
    const int lo = min(n, t * per), hi = min(n, lo + per);
    int s = 0;
    for (int b = lo; b < hi; ++b) s += a.kcount[b];
    int excl;
    block_exclusive_scan(s, sh, excl);
    for (int b = lo; b < hi; ++b) {
        const int v = a.kcount[b];
        a.offsets[b] = excl;
        a.kcount[b] = 0;
        excl += v;
    }
    if (t == 0) {
        a.offsets[n] = (int)a.m;
        a.heavy[0] = 0;
    }
    __syncthreads();   // offsets are read by other threads below (global, same block)
    int parts_sum = 0;
    for (int b = lo; b < hi; ++b) {
        const int cand = tile_bin_list(a.D, a.nb, a.B, a.K, a.J, b, a.offsets, a.tile_nbr + b, a.nbins);
        const int parts = max(1, (cand + a.P - 1) / a.P);
        a.tile_parts[b] = parts;
        parts_sum += parts;
    }
    const int total = block_exclusive_scan(parts_sum, sh, excl);
    for (int b = lo; b < hi; ++b) {
        const int parts = a.tile_parts[b];
        a.item_off[b] = excl;
        for (int k = 0; k < parts; ++k) a.items[excl + k] = make_int4(b, k, parts, 0);
        if (parts > 1) a.heavy[1 + atomicAdd(a.heavy, 1)] = b;
        excl += parts;
    }
    if (t == 0) {
        a.item_off[n] = total;
        a.nitems[0] = total;
    }
}

// Deterministic order (nufft_opts.deterministic): the histogram's ranks within a bin follow the
// order in which the atomics arrived.  k_det_place writes every point's original index at that
// position (into the scratch `tmp`, [M]); k_det_rank then gives each point the rank of its original
// index among the points of its bin, so the scatter orders each bin by original index.
__global__ void k_det_place(SortArgs a, int* tmp) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    tmp[a.offsets[a.keyid[i]] + a.local[i]] = (int)i;
}

__global__ void k_det_rank(SortArgs a, const int* tmp) {
    pdl_wait();
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.m) return;
    const int i = tmp[j];
    const int key = a.keyid[i];
    const int lo = a.offsets[key], hi = a.offsets[key + 1];
    int rank = 0;
    for (int t = lo; t < hi; ++t) rank += tmp[t] < i;
    a.local[i] = rank;
}

cudaError_t launch_det_ranks(const SortArgs& a, int step, int* tmp, cudaStream_t s) {
    if (a.m == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((a.m + 255) / 256);
    if (step == 0) (void)launch_pdl(k_det_place, blocks, 256, 0, s, a, tmp);
    else (void)launch_pdl(k_det_rank, blocks, 256, 0, s, a, (const int*)tmp);
    return cudaGetLastError();
}

__global__ void k_bin_scatter(SortArgs a) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.m) return;
    int4 ix;
    float4 fr;
    int64_t key;
    point_record(a, i, ix, fr, key);
    const int dst = a.offsets[a.keyid[i]] + a.local[i];
    a.local[i] = dst;   // the inverse of the sort permutation, for reordering coil values
    a.pidx[dst] = ix;
    a.pfrac[dst] = fr;
    // the D*J kernel weights, evaluated once here and read by every gather and spread
    float* w = a.pw + (int64_t)dst * a.ws;
    for (int d = 0; d < a.D; ++d) {
        const float u0 = d == 0 ? fr.x : (d == 1 ? fr.y : fr.z);
        if (a.kbtab)
            for (int j = 0; j < a.J; ++j) w[d * a.wd + j] = kb_table(a.kbtab, a.tab_L, a.tab_n, u0 - (float)j);
        else
            for (int j = 0; j < a.J; ++j) w[d * a.wd + j] = kb_psi(a.kb.a, a.kb.two_over_j, u0 - (float)j);
        for (int j = a.J; j < a.wd; ++j) w[d * a.wd + j] = 0.f;
    }
    // strips: count the point as a hit of every unit its window reaches
    if (a.strip) strip_point_units(a.sg, ix, [&](int u, int, int, int) { atomicAdd(a.st.hcount + u, 1); });
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s) {
    const int64_t n4 = (int64_t)(bytes / 16);
    const int64_t ntail = (int64_t)((bytes - n4 * 16) / 4);
    int blocks = (int)std::min<int64_t>((n4 + 255) / 256, 152 * 16);
    if (blocks < 1) blocks = 1;
    (void)launch_pdl(k_zero, blocks, 256, 0, s, (float4*)p, n4, (int*)((char*)p + n4 * 16), ntail);
    return cudaGetLastError();
}
cudaError_t launch_key_count(const SortArgs& a, cudaStream_t s) {
    if (a.m == 0) return cudaSuccess;
    (void)launch_pdl(k_key_count, (unsigned)((a.m + 255) / 256), 256, 0, s, a);
    return cudaGetLastError();
}
cudaError_t launch_bin_scan(const SortArgs& a, cudaStream_t s) {
    (void)launch_pdl(k_bin_scan, 1, 1024, 0, s, a);
    return cudaGetLastError();
}
cudaError_t launch_sort_tables(const SortArgs& a, cudaStream_t s) {
    (void)launch_pdl(k_sort_tables, 1, 1024, 0, s, a);
    return cudaGetLastError();
}
cudaError_t launch_tile_lists(const SortArgs& a, cudaStream_t s) {
    (void)launch_pdl(k_tile_lists, (a.nbins + 127) / 128, 128, 0, s, a);
    return cudaGetLastError();
}
cudaError_t launch_item_scan(const SortArgs& a, cudaStream_t s) {
    (void)launch_pdl(k_item_scan, 1, 1024, 0, s, a);
    return cudaGetLastError();
}
cudaError_t launch_bin_scatter(const SortArgs& a, cudaStream_t s) {
    if (a.m == 0) return cudaSuccess;
    (void)launch_pdl(k_bin_scatter, (unsigned)((a.m + 255) / 256), 256, 0, s, a);
    return cudaGetLastError();
}

}  // namespace nj

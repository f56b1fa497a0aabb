// Adjoint interpolation (spread), Sec. II-D: G[k] = sum_i psi(t_i - k) y_i, the transpose of
// the gather, onto the oversampled grid [K0][K1]([K2])[C], on strip units (2-D and 3-D).
//
// A strip unit is NSL grid rows x kStripW columns of the last axis (a row is a k0 index in 2-D,
// a (k0, k1) pair of an R0 x R1 block in 3-D).  A warp owns one unit (or one part of a unit) for a
// coil group of CPW = 64 / NSL coils: lane (s, p) holds row s of the unit, coils 2p and 2p + 1 of
// the group, all kStripW columns, in registers.
//
// Sort time (once per omega, read by every adjoint of the same points).  The
// scatter counts every point as a hit of each unit its window reaches
// (strip_point_units); the plan turns the counts into hit offsets and work items (a
// unit with more than P hits is split into parts of P hits, and the parts of split
// units are listed first, so they start in the first wave); the fill has every
// point append {sorted point, packed window start} to the hit lists of its units.
//
// Spread.  Persistent blocks own every gridDim.x-th work item and their warps take
// them in turn from a shared counter, loading the next item's descriptor and hit
// records while the current one is processed.  A warp takes its item's hits 32 at
// a time: each lane copies
// one hit's kernel weights and CPW coil values into the warp's shared staging area
// with asynchronous copies (cp.async), and then every hit is added to the accumulators
// of all lanes at once: the lane's row tap comes from its row slot, and the column
// taps land on compile-time register indices through a warp-uniform jump table on
// the window's start column (strip_cases.inc, generated by gen_strip_cases.py); in 3-D the row
// weight is the product of the lane's taps along dims 0 and 1.
// There is no shared-memory read-modify-write and no block barrier.
//
// Each grid cell belongs to exactly one unit, whose owner writes it (zeros
// included), so the grid needs no clearing and no atomics.  The parts of a split
// unit store their partial sums in their own slots and count themselves done on
// the unit's counter; the part that finishes last adds all the slots in part order
// and writes the cells (no part ever waits), then resets the counter for the next
// call.  Hits are summed in hit-list order and parts in part order, so the result
// depends on the sort's order of the points only.
#include <algorithm>
#include <atomic>

#include "internal.h"
#include "strip_cases.inc"

namespace nj {

constexpr int kStripWarps = 4;
constexpr int kStripBatch = 32;

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ int warp_inclusive_scan(int x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += v;
    }
    return x;
}

// Exclusive scan of V values per element over n elements, 1024 threads: tiles of 8192 elements,
// warp w of a tile takes 256 consecutive elements as 8 rows of 32 (coalesced loads, shuffle scans).
// get(i, v) loads element i (v[q] = 0 past n); put(i, excl, v) receives its exclusive prefixes.
template <int V, typename Get, typename Put>
__device__ __forceinline__ void block_scan_tiles(int n, int (&carry)[V], Get get, Put put) {
    __shared__ int sh[V][32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    for (int base = 0; base < n; base += 8192) {
        int v[8][V], incl[8][V], run[V];
#pragma unroll
        for (int q = 0; q < V; ++q) run[q] = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = base + w * 256 + k * 32 + lane;
            get(i, v[k]);
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const int x = warp_inclusive_scan(v[k][q], lane);
                incl[k][q] = x + run[q];
                run[q] += __shfl_sync(0xffffffffu, x, 31);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < V; ++q) sh[q][w] = run[q];
        }
        __syncthreads();
        int woff[V], tot[V];
#pragma unroll
        for (int q = 0; q < V; ++q) {
            const int x = warp_inclusive_scan(sh[q][lane], lane);
            woff[q] = __shfl_sync(0xffffffffu, x, w) - sh[q][w];
            tot[q] = __shfl_sync(0xffffffffu, x, 31);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int i = base + w * 256 + k * 32 + lane;
            int ex[V];
#pragma unroll
            for (int q = 0; q < V; ++q) ex[q] = carry[q] + woff[q] + incl[k][q] - v[k][q];
            if (i < n) put(i, ex, v[k]);
        }
#pragma unroll
        for (int q = 0; q < V; ++q) carry[q] += tot[q];
        __syncthreads();   // sh is refilled by the next tile
    }
}

// --------------------------------------------------------------- sort tables
// Packed window start of a hit: column sd in [-(J-1), 15] and start-row offsets dr0, dr1 in
// [-(R-1), J-1] (dr1 = 0 in 2-D).
__device__ __forceinline__ int strip_meta(int sd, int dr0, int dr1) {
    return (sd + 8) | ((dr0 + 32) << 8) | ((dr1 + 32) << 16);
}

// The plan in two launches of 256-thread blocks (unit b * 256 + t in block b, thread t).  Split
// parts are counted for P * 2^L, L = 0..7: the smallest level whose split parts fit the partial
// slots is used.  (a) Per block and level: hits, split parts and whole units.  (b) Every block sums
// the totals of the blocks before it, picks the level, scans its own units and writes their hit
// offsets and items (split parts first: they start in the first wave), clearing the hit counts
// (the next sort's scatter counts into them) and the fill cursors.
constexpr int kPlanThreads = 256;
constexpr int kPlanLevels = 8;
constexpr int kPlanVals = 1 + 2 * kPlanLevels;   // hits, then split parts and whole units per level

__device__ __forceinline__ int plan_parts(int h, int lgP) { return max(1, (int)(((int64_t)h + (1 << lgP) - 1) >> lgP)); }

__global__ void __launch_bounds__(kPlanThreads) k_strip_plan_a(SortArgs a) {
    pdl_wait();
    __shared__ int sh[kPlanVals][kPlanThreads / 32];
    const StripTables& T = a.st;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int u = blockIdx.x * kPlanThreads + t;
    const int h = u < a.nunits ? T.hcount[u] : 0;
    const int lgP = 31 - __clz(T.P);
    int v[kPlanVals];
    v[0] = h;
#pragma unroll
    for (int L = 0; L < kPlanLevels; ++L) {
        const int parts = plan_parts(h, lgP + L);
        v[1 + 2 * L] = u < a.nunits && parts > 1 ? parts : 0;
        v[2 + 2 * L] = u < a.nunits && parts == 1 ? 1 : 0;
    }
#pragma unroll
    for (int q = 0; q < kPlanVals; ++q) {
        int x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[q][w] = x;
    }
    __syncthreads();
    if (t < kPlanVals) {
        int x = 0;
        for (int k = 0; k < kPlanThreads / 32; ++k) x += sh[t][k];
        T.partial_sums[blockIdx.x * kPlanVals + t] = x;
    }
}

__global__ void __launch_bounds__(kPlanThreads) k_strip_plan_b(SortArgs a) {
    pdl_wait();
    __shared__ int s_tot[kPlanVals], s_pre[kPlanVals];
    __shared__ int sh[3][kPlanThreads / 32];
    const StripTables& T = a.st;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int nblk = (int)gridDim.x, b = blockIdx.x;
    if (t < kPlanVals) {
        int tot = 0, pre = 0;
        for (int k = 0; k < nblk; ++k) {
            const int x = T.partial_sums[k * kPlanVals + t];
            tot += x;
            if (k < b) pre += x;
        }
        s_tot[t] = tot;
        s_pre[t] = pre;
    }
    __syncthreads();
    int L = 0;
    while (L < kPlanLevels - 1 && s_tot[1 + 2 * L] > T.slots) ++L;
    const bool fits = s_tot[1 + 2 * L] <= T.slots;
    const int lgP = (31 - __clz(T.P)) + L;
    const int H = fits ? s_tot[1 + 2 * L] : 0;   // split parts (items of split units come first)
    const int u = b * kPlanThreads + t;
    const bool live = u < a.nunits;
    const int h = live ? T.hcount[u] : 0;
    const int parts = fits ? plan_parts(h, lgP) : 1;
    int v[3] = {h, live && parts > 1 ? parts : 0, live && parts == 1 ? 1 : 0};
    int incl[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        int x = v[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        incl[q] = x;
        if (lane == 31) sh[q][w] = x;
    }
    __syncthreads();
    // prefixes of the blocks before this one (with no split anywhere every unit is one item, and
    // the blocks before hold kPlanThreads units each)
    const int base[3] = {s_pre[0], fits ? s_pre[1 + 2 * L] : 0, fits ? H + s_pre[2 + 2 * L] : b * kPlanThreads};
    int ex[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        int wo = 0;
        for (int k = 0; k < w; ++k) wo += sh[q][k];
        ex[q] = base[q] + wo + incl[q] - v[q];
    }
    if (live) {
        T.hoff[u] = ex[0];
        T.hcount[u] = 0;
        T.hcur[u] = 0;
        if (v[1] > 0) {
            for (int k = 0; k < parts; ++k) {
                const int hb = ex[0] + (k << lgP);
                T.items[ex[1] + k] = make_int4(u, hb, min(hb + (1 << lgP), ex[0] + h), ex[1] + k);
                T.splits[ex[1] + k] = make_int4(k, parts, ex[1], 0);
            }
        } else {
            T.items[ex[2]] = make_int4(u, ex[0], ex[0] + h, -1);
        }
    }
    if (b == 0 && t == 0) {
        T.hoff[a.nunits] = s_tot[0];
        T.nitems[0] = fits ? H + s_tot[2 + 2 * L] : a.nunits;
        T.nitems[1] = 1 << lgP;
    }
}

// One thread per sorted point: the point joins the hit list of every unit its window reaches.
__global__ void k_strip_fill(SortArgs a) {
    pdl_wait();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.m) return;
    const int4 ix = a.pidx[p];
    const StripTables& T = a.st;
    strip_point_units(a.sg, ix, [&](int u, int sd, int dr0, int dr1) {
        const int64_t pos = (int64_t)T.hoff[u] + atomicAdd(T.hcur + u, 1);
        if (pos < T.hit_cap) T.fill_to[pos] = make_int2((int)p, strip_meta(sd, dr0, dr1));
    });
}

// Deterministic order: one warp per unit ranks each of its hits by sorted point index (the indices
// of a unit are distinct) and writes it at that rank; the fill's order followed its atomics.
__global__ void k_strip_order(SortArgs a, const int2* __restrict__ tmp) {
    pdl_wait();
    const int u = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (u >= a.nunits) return;   // warp-uniform
    const int lane = threadIdx.x & 31;
    const int lo = a.st.hoff[u], hi = a.st.hoff[u + 1];
    for (int h = lo + lane; h < hi; h += 32) {
        const int2 e = tmp[h];
        int rank = 0;
        for (int t = lo; t < hi; ++t) rank += tmp[t].x < e.x;
        a.st.hits[lo + rank] = e;
    }
}

cudaError_t launch_strip_order(const SortArgs& a, const int2* hits_tmp, cudaStream_t s) {
    (void)launch_pdl(k_strip_order, (unsigned)((a.nunits + 7) / 8), 256, 0, s, a, hits_tmp);
    return cudaGetLastError();
}

cudaError_t launch_strip_plan(const SortArgs& a, int step, cudaStream_t s) {
    const unsigned nblk = (unsigned)((a.nunits + kPlanThreads - 1) / kPlanThreads);
    if (step == 0) (void)launch_pdl(k_strip_plan_a, nblk, kPlanThreads, 0, s, a);
    else (void)launch_pdl(k_strip_plan_b, nblk, kPlanThreads, 0, s, a);
    return cudaGetLastError();
}

int strip_plan_blocks(int nunits) { return (nunits + kPlanThreads - 1) / kPlanThreads; }
int strip_plan_vals() { return kPlanVals; }

cudaError_t launch_strip_fill(const SortArgs& a, cudaStream_t s) {
    if (a.m == 0) return cudaSuccess;
    (void)launch_pdl(k_strip_fill, (unsigned)((a.m + 255) / 256), 256, 0, s, a);
    return cudaGetLastError();
}

// -------------------------------------------------------------------- spread
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Staging rows hold a hit's 16-byte chunks in order.  Lane h copies the chunks of hit h in an order
// rotated by h (coil-pair chunk (q + h) mod NQ, weight chunk (q + h / 2) mod 4 at step q), so that
// the asynchronous copies of the eight lanes of a wavefront fall on distinct banks; the reads of
// one hit by all lanes are broadcasts or distinct chunks of one row.
template <int D, int J, int NSL>
__global__ void __launch_bounds__(kStripWarps * 32, 4) k_spread_strips(StripArgs a) {
    pdl_wait();
    constexpr int CPW = 64 / NSL;     // coils per warp (a coil pair per lane)
    constexpr int NQ = CPW / 2;       // coil pairs = 16-byte chunks per staged hit
    constexpr int R1 = D == 3 ? strip_rows1(NSL) : 1, R0 = NSL / R1;   // rows of a unit per row axis
    constexpr int WS = 8 * D;         // staged weights per hit: 8 per axis, the column taps last
    constexpr int WQ = WS / 4;        // ... in 16-byte chunks
    __shared__ __align__(16) float4 s_y[kStripWarps][kStripBatch][NQ];
    __shared__ __align__(16) float s_w[kStripWarps][kStripBatch][WS];
    __shared__ int4 s_m[kStripWarps][kStripBatch];                      // {start column, row offsets dr0, dr1}
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cg = blockIdx.y;
    const StripGeom g = a.g;
    const int s = lane / NQ, pc = lane - s * NQ;      // row slot, coil pair
    const int s0 = s / R1, s1 = s - s0 * R1;          // the slot's row along dims 0 and 1
    const int coil = cg * CPW + 2 * pc;
    const int C = a.C;
    const float4* yg = (const float4*)(a.y + (int64_t)cg * a.pts.m * CPW);   // [M][NQ] pairs of this group
    const int nitems = a.t.nitems[0];
    // Block b owns items b, b + gridDim.x, ... (split parts, first in the list, spread over the
    // blocks); its warps take them in turn from a shared counter, so a warp that drew a heavy item
    // takes fewer.  The next item's descriptor and first hit records are loaded while the current
    // item is processed.
    __shared__ int s_next;
    if (threadIdx.x == 0) s_next = kStripWarps;
    __syncthreads();   // the only block barrier: the counter is set before any warp takes from it
    const int nb = (int)gridDim.x;
    int it = (int)blockIdx.x + warp * nb;
    int4 item = make_int4(0, 0, 0, -1);
    int2 hit = make_int2(0, 0);
    if (it < nitems) {
        item = a.t.items[it];
        if (lane < item.z - item.y) hit = a.t.hits[item.y + lane];
    }
    while (it < nitems) {
        int k = 0;
        if (lane == 0) k = atomicAdd(&s_next, 1);
        const int itn = (int)blockIdx.x + __shfl_sync(0xffffffffu, k, 0) * nb;
        int4 itemn = make_int4(0, 0, 0, -1);
        if (itn < nitems) itemn = a.t.items[itn];
        const int u = item.x;
        const int r = u / g.nbl, tc = u - r * g.nbl;
        const int g0 = D == 3 ? r / g.ng1 : r, g1 = D == 3 ? r - g0 * g.ng1 : 0;
        const int row0 = g0 * R0 + s0, row1 = g1 * R1 + s1;   // this lane's row (row1: 3-D only)
        const int org1 = tc * kStripW;
        const int Bt1 = min(kStripW, g.KL - org1);

        float acc[4 * kStripW];   // column k: acc[4k .. 4k+3] = re, im of coil 2 pc, then of coil 2 pc + 1
#pragma unroll
        for (int q = 0; q < 4 * kStripW; ++q) acc[q] = 0.f;
        for (int b = item.y; b < item.z; b += kStripBatch) {
            const int nh = min(kStripBatch, item.z - b);
            if (b != item.y && lane < nh) hit = a.t.hits[b + lane];   // later batches of a split part
            if (lane < nh) {
                const float* pw = a.pts.w + (int64_t)hit.x * WS;
#pragma unroll
                for (int q = 0; q < WQ; ++q) {   // rotated: 8 lanes of 64- or 96-byte rows on distinct banks
                    const int qq = D == 2 ? (q + (lane >> 1)) & 3 : (q + (lane >> 2)) % WQ;
                    cp_async16(&s_w[warp][lane][4 * qq], pw + 4 * qq);
                }
                const float4* py = yg + (int64_t)hit.x * NQ;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const int qq = (q + lane) & (NQ - 1);
                    cp_async16(&s_y[warp][lane][qq], py + qq);
                }
                s_m[warp][lane] = make_int4((hit.y & 255) - 8, ((hit.y >> 8) & 255) - 32, ((hit.y >> 16) & 255) - 32, 0);
            }
            cp_async_wait_all();
            __syncwarp();
#pragma unroll 2
            for (int h = 0; h < nh; ++h) {
                const int4 m = s_m[warp][h];
                const float* w = s_w[warp][h];
                const int ta = m.y + s0;   // this lane's row tap along dim 0 (taps 0..7, zero past J)
                float wo = (unsigned)ta < (unsigned)J ? w[ta & 7] : 0.f;
                if (D == 3) {              // times its row tap along dim 1
                    const int tb = m.z + s1;
                    wo = (unsigned)tb < (unsigned)J ? wo * w[8 + (tb & 7)] : 0.f;
                }
                const float4 yv = s_y[warp][h][pc];
                const float4 wa = *(const float4*)(w + 8 * (D - 1));
                const float4 wb = *(const float4*)(w + 8 * (D - 1) + 4);
                const float wx[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
                const float yw[4] = {wo * yv.x, wo * yv.y, wo * yv.z, wo * yv.w};
                strip_add_J<J>(acc, m.x, wx, yw);
            }
            __syncwarp();   // the staging area is refilled by the next batch
        }
        // the next item's first hit records (its descriptor has arrived during the batches above)
        int2 hitn = make_int2(0, 0);
        if (itn < nitems && lane < itemn.z - itemn.y) hitn = a.t.hits[itemn.y + lane];

        const bool rok = row0 < g.K0 && (D == 2 || row1 < g.K1);
        bool write = item.w < 0;
        if (!write) {   // split unit: deposit this part, count it; the last part adds all parts in order
            const int4 sp = a.t.splits[item.w];
            const int part = sp.x, nparts = sp.y, slot0 = sp.z;
            float4* pp = (float4*)a.partial + ((int64_t)(slot0 + part) * a.ncg + cg) * (kStripW * 32);
#pragma unroll
            for (int q = 0; q < kStripW; ++q)
                pp[q * 32 + lane] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
            __threadfence();
            __syncwarp();
            int old = 0;
            if (lane == 0) old = atomicAdd(a.counters + (int64_t)slot0 * a.ncg + cg, 1);
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old == nparts - 1) {
                __threadfence();
#pragma unroll
                for (int q = 0; q < 4 * kStripW; ++q) acc[q] = 0.f;
                for (int q2 = 0; q2 < nparts; ++q2) {
                    const float4* src = (const float4*)a.partial + ((int64_t)(slot0 + q2) * a.ncg + cg) * (kStripW * 32);
#pragma unroll
                    for (int q = 0; q < kStripW; ++q) {
                        const float4 v = __ldcg(src + q * 32 + lane);
                        acc[4 * q] += v.x;
                        acc[4 * q + 1] += v.y;
                        acc[4 * q + 2] += v.z;
                        acc[4 * q + 3] += v.w;
                    }
                }
                if (lane == 0) a.counters[(int64_t)slot0 * a.ncg + cg] = 0;
                write = true;
            }
        }
        if (write && rok && coil < C) {
            const int64_t cell = D == 3 ? ((int64_t)row0 * g.K1 + row1) * g.KL + org1 : (int64_t)row0 * g.KL + org1;
            float2* dst = a.grid + cell * C + coil;
            if (coil + 1 < C && (C & 1) == 0) {   // both coils, one 16-byte store per column
#pragma unroll
                for (int q = 0; q < kStripW; ++q)
                    if (q < Bt1)
                        *(float4*)(dst + (int64_t)q * C) = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
            } else {
                const bool two = coil + 1 < C;
#pragma unroll
                for (int q = 0; q < kStripW; ++q)
                    if (q < Bt1) {
                        dst[(int64_t)q * C] = make_float2(acc[4 * q], acc[4 * q + 1]);
                        if (two) dst[(int64_t)q * C + 1] = make_float2(acc[4 * q + 2], acc[4 * q + 3]);
                    }
            }
        }
        it = itn;
        item = itemn;
        hit = hitn;
    }
}

// Resident blocks of a persistent kernel on the current device (queried once per kernel and device).
template <auto KERNEL>
static int resident_blocks(int threads) {
    static std::atomic<int> n[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int v = n[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, KERNEL, threads, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        cudaGetLastError();
        v = per_sm * sms;
        n[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

template <int D, int J, int NSL>
static void strips_launch(const StripArgs& a, cudaStream_t s) {
    constexpr int threads = kStripWarps * 32;
    const int need = (a.max_items + kStripWarps - 1) / kStripWarps;
    const int blocks = std::max(1, std::min(need, resident_blocks<k_spread_strips<D, J, NSL>>(threads)));
    (void)launch_pdl(k_spread_strips<D, J, NSL>, dim3((unsigned)blocks, (unsigned)a.ncg), threads, 0, s, a);
}

template <int D, int J>
static cudaError_t strips_j(const StripArgs& a, cudaStream_t s) {
    switch (a.g.NSL) {
        case 4: strips_launch<D, J, 4>(a, s); break;
        case 8: strips_launch<D, J, 8>(a, s); break;
        case 16: strips_launch<D, J, 16>(a, s); break;
        default: strips_launch<D, J, 32>(a, s); break;
    }
    return cudaGetLastError();
}

template <int D>
static cudaError_t strips_d(const StripArgs& a, cudaStream_t s) {
    switch (a.g.J) {
        case 4: return strips_j<D, 4>(a, s);
        case 5: return strips_j<D, 5>(a, s);
        case 6: return strips_j<D, 6>(a, s);
        case 7: return strips_j<D, 7>(a, s);
        default: return strips_j<D, 8>(a, s);
    }
}

cudaError_t launch_spread_strips(const StripArgs& a, cudaStream_t s) {
    if (a.max_items == 0) return cudaSuccess;
    return a.g.D == 3 ? strips_d<3>(a, s) : strips_d<2>(a, s);
}

// Coil values in sorted point order, in the strip layout [C / cpt][M][cpt], from y [C][M] in the
// caller's point order.  A block takes kPermPts consecutive points of the caller's order: it reads
// each coil's values of those points as one coalesced row segment into shared memory, then writes
// every point's coil values as contiguous runs at the point's sorted position pos[o] (the bin
// scatter leaves it there).  Both the reads and the writes are whole sectors.
constexpr int kPermPts = 32;
__global__ void __launch_bounds__(256) k_permute_y_strips(const int* __restrict__ pos, const float2* __restrict__ y,
                                                          float2* __restrict__ ys, int64_t M, int C, int cpt) {
    pdl_wait();
    extern __shared__ float2 tp[];   // [C][kPermPts + 1]
    const int64_t o0 = (int64_t)blockIdx.x * kPermPts;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int np = (int)(M - o0 < kPermPts ? M - o0 : kPermPts);
    for (int c = warp; c < C; c += nwarps)
        if (lane < np) tp[c * (kPermPts + 1) + lane] = __ldg(y + (int64_t)c * M + o0 + lane);
    __syncthreads();
    for (int f = threadIdx.x; f < np * C; f += blockDim.x) {
        const int q = f / C, c = f - q * C;   // consecutive threads: consecutive coils of one point
        const int64_t i = __ldg(pos + o0 + q);
        const int grp = c / cpt;
        ys[((int64_t)grp * M + i) * cpt + (c - grp * cpt)] = tp[c * (kPermPts + 1) + q];
    }
}

cudaError_t launch_permute_y_strips(const int* pos, const float2* y, float2* ys, int64_t M, int C, int cpt,
                                    cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    const size_t smem = (size_t)C * (kPermPts + 1) * sizeof(float2);
    (void)launch_pdl(k_permute_y_strips, (unsigned)((M + kPermPts - 1) / kPermPts), 256, smem, s, pos, y, ys, M, C,
                     cpt);
    return cudaGetLastError();
}

}  // namespace nj

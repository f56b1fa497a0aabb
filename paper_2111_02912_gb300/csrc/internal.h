// Host-side launcher declarations shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace nj {

// ---------------------------------------------------------------- sorting
// Points are ordered by the bin (a tile of B_d cells per axis) of their window
// start; each bin is a contiguous range.
constexpr int kNbrStride = 64;        // entries per tile in tile_nbr: n, then 27 (start, prefix) pairs, total

// ---------------------------------------------------------- strip geometry
// The adjoint spread of the strip kernel runs on strip units: NSL grid "rows" by kStripW
// consecutive cells of the last axis (the columns), all coils of a coil group.  In 2-D a row is a
// k0 index and a unit holds NSL consecutive rows; in 3-D a row is a (k0, k1) pair and a unit
// holds R0 x R1 of them (R0 R1 = NSL), R0 consecutive k0 by R1 consecutive k1.  Unit
// u = (g0 ng1 + g1) nbl + t covers rows g0 R0 .., g1 R1 .. (g1 = 0, R1 = 1 in 2-D) and columns
// t kStripW .. + kStripW - 1.
constexpr int kStripW = 16;           // columns of a strip unit (the accumulators of one lane)
// 3-D: rows of a unit along dim 1 for NSL rows in all (R0 = NSL / R1 along dim 0), near square
__host__ __device__ constexpr int strip_rows1(int nsl) { return nsl >= 32 ? 8 : (nsl >= 8 ? 4 : 2); }
struct StripGeom {
    int D;
    int K0, K1, KL;     // grid edges: dims 0 and 1, and the last (column) axis (KL = K1 in 2-D)
    int R0, R1;         // rows of a unit along dim 0 and (3-D) dim 1; R1 = 1 in 2-D
    int ng1, nbl;       // row groups along dim 1 (1 in 2-D), column tiles
    int J, NSL;
};

// Distinct groups of R cells (mod K) holding the J cells k .. k + J - 1 of one axis, at most 5:
// calls f(group, offset) with offset = group start - k (+ K past the wrap), in [-(R-1), J-1].
template <typename F>
__device__ __forceinline__ void strip_axis_groups(int k, int K, int R, int J, F f) {
    int prev = -1;
    for (int j = 0; j < J; ++j) {
        int c = k + j;
        if (c >= K) c -= K;
        const int grp = c / R;
        if (grp == prev) continue;
        prev = grp;
        f(grp, grp * R - k + (c < k ? K : 0));
    }
}

// Strip units reached by the window starting at cell ix (k0, k1 and, in 3-D, k2): the row groups
// holding its J rows of every row axis (mod K) times the column tiles holding its J columns (mod
// KL), at most 3 tiles.  Calls unit(u, sd, dr0, dr1) once per unit, with the window's start
// column relative to the unit, sd in [-(J-1), kStripW), and its start-row offsets (group start -
// k) along dim 0 and (3-D) dim 1, in [-(R-1), J-1] (dr1 = 0 in 2-D).
template <typename F>
__device__ __forceinline__ void strip_point_units(const StripGeom& g, int4 ix, F unit) {
    const int kl = g.D == 3 ? ix.z : ix.y;
    int tiles[3], sds[3], nt = 0;
    for (int j = 0; j < g.J; ++j) {
        int col = kl + j;
        if (col >= g.KL) col -= g.KL;
        const int t = col / kStripW;
        if (nt == 0 || t != tiles[nt - 1]) {
            if (nt < 3) {
                tiles[nt] = t;
                sds[nt] = kl - t * kStripW - (col < kl ? g.KL : 0);   // past the wrap: start lies left
            }
            ++nt;
        }
    }
    if (nt > 3) nt = 3;
    strip_axis_groups(ix.x, g.K0, g.R0, g.J, [&](int g0, int dr0) {
        if (g.D == 3) {
            strip_axis_groups(ix.y, g.K1, g.R1, g.J, [&](int g1, int dr1) {
                for (int q = 0; q < nt; ++q) unit((g0 * g.ng1 + g1) * g.nbl + tiles[q], sds[q], dr0, dr1);
            });
        } else {
            for (int q = 0; q < nt; ++q) unit(g0 * g.nbl + tiles[q], sds[q], dr0, 0);
        }
    });
}

// Sort-time tables of the strip spread (once per omega, read by every adjoint of those points).
// A hit is a point whose window reaches a unit: {sorted point index, packed window start}, the
// start column relative to the unit in bits 0..7 (biased by 8) and the start-row offsets along
// dim 0 in bits 8..15 and (3-D) dim 1 in bits 16..23 (biased by 32).  The hits of unit u are hits[hoff[u] .. hoff[u + 1]).  Work items are
// {unit, first hit, end hit, split index} (split index -1: the unit is one item; else
// splits[split index] = {part, parts, first partial slot, 0}); the parts of split units come first.
struct StripTables {
    int* hcount;      // [nunits]   hits per unit (counted by the scatter; zeroed before it)
    int* hcur;        // [nunits]   fill cursors (zeroed by the plan)
    int* hoff;        // [nunits+1] first hit of each unit
    int2* hits;       // [hit_cap]
    int2* fill_to;    // where the fill writes: hits, or a scratch list reordered into hits
    int64_t hit_cap;
    int4* items;      // [nunits + slots]
    int4* splits;     // [slots]
    int* nitems;      // [0] items, [1] hits per part
    int P;            // hits per part (doubled until the split parts fit the slots), a power of two
    int slots;        // partial-sum slots
    int* partial_sums;  // [plan blocks][plan values] per-block totals of the plan
};

struct SortArgs {
    const float* omega;   // [D][M]
    int64_t m;
    int D, J;
    int K[kMaxDim];
    int B[kMaxDim], nb[kMaxDim];
    int nbins, P;         // P: spread candidates per work item
    float c_hi[kMaxDim], c_lo[kMaxDim];  // K/(2 pi) as a float pair
    int* kcount;      // [nbins]      points per bin; zero before the sort, cleared again by the bin scan
    int* local;       // [M]          rank among the points of the same bin; the bin scatter then
                      //              replaces it by the point's sorted position
    int* keyid;       // [M]
    int* offsets;     // [nbins + 1]  first sorted point of each bin
    int* item_off;    // [nbins + 1]  first spread work item of each tile
    int* tile_parts;  // [nbins]      spread work items of each tile
    int* heavy;       // [nbins + 1]  count, then the tiles with more than one work item (any order)
    int* tile_nbr;    // [kNbrStride][nbins]  bins that reach the tile: count, then (start, prefix) pairs
                      //                      (entry-major: the stores of neighbouring tiles coalesce)
    int4* items;      // [max_items]  {tile, part, nparts, 0}
    int* nitems;      // [1]
    int4* pidx;       // [M]
    float4* pfrac;    // [M]
    float* pw;        // [M][ws]   kernel weights psi(u0_d - j) of the sorted points, at d * wd + j
    int ws, wd;
    KbPoly kb;
    const float* kbtab;   // table mode: psi(l / tab_L) for l = 0 .. tab_n + 1 (zero from tab_n on), else null
    float tab_L;
    int tab_n;
    // strip mode: the scatter also counts the strip units' hits, then the plan and fill
    int strip, nunits;
    StripGeom sg;
    StripTables st;
};
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s);
cudaError_t launch_key_count(const SortArgs& a, cudaStream_t s);     // histogram of bins, rank within bin
cudaError_t launch_bin_scan(const SortArgs& a, cudaStream_t s);      // offsets; clears the histogram
cudaError_t launch_tile_lists(const SortArgs& a, cudaStream_t s);    // reaching bins, parts per tile
cudaError_t launch_item_scan(const SortArgs& a, cudaStream_t s);     // item offsets and list
constexpr int kFusedTablesMaxBins = 8192;
cudaError_t launch_sort_tables(const SortArgs& a, cudaStream_t s);   // the three above in one block
cudaError_t launch_bin_scatter(const SortArgs& a, cudaStream_t s);   // records and weights in bin order
// Deterministic order: ranks within each bin by original index (before the scatter; tmp is [M]
// scratch).  Step 0 places the original indices, step 1 ranks them.
cudaError_t launch_det_ranks(const SortArgs& a, int step, int* tmp, cudaStream_t s);
// Strip tables (kernels_strip.cu), after the scatter (which counts the hits per unit):
cudaError_t launch_strip_plan(const SortArgs& a, int step, cudaStream_t s);   // step 0: block totals; 1: offsets, items
int strip_plan_blocks(int nunits);   // blocks of the plan launches
int strip_plan_vals();               // per-block totals the plan keeps
cudaError_t launch_strip_fill(const SortArgs& a, cudaStream_t s);    // hit lists
// Deterministic order: the fill writes into hits_tmp, then each unit's hits are ranked by sorted
// point index into hits.
cudaError_t launch_strip_order(const SortArgs& a, const int2* hits_tmp, cudaStream_t s);

// Bins whose points can reach tile `bin` (tiles are the bins).  A window
// covers J cells to the right of its start, so along each axis these are the
// tile's own bin and the bins holding the J-1 cells before its first cell
// (periodic; at most three, without repeats).  Writes the tile's list entry,
// tn[0] = count, then (first point, candidate prefix) pairs and the total, entry
// k at tn[k * stride], and returns the candidate count.  Every array index is fixed after unrolling, so
// nothing goes to local memory.
__device__ __forceinline__ int tile_bin_list(int D, const int* nb, const int* B, const int* K, int J, int bin,
                                             const int* offsets, int* tn, int stride) {
    int x[kMaxDim][3], n[kMaxDim];
    int r = bin;
#pragma unroll
    for (int d = kMaxDim - 1; d >= 0; --d) {
        x[d][0] = x[d][1] = x[d][2] = 0;
        n[d] = 1;
        if (d < D) {
            const int bc = r % nb[d];
            r /= nb[d];
            const int org = bc * B[d];
            int c1 = org - 1, c2 = org - (J - 1);
            if (c1 < 0) c1 += K[d];
            if (c2 < 0) c2 += K[d];
            const int b1 = c1 / B[d], b2 = c2 / B[d];
            x[d][0] = bc;   // own bin, then those of cells org-1 and org-(J-1), in order, no repeats
            if (b1 != bc) {
                x[d][1] = b1;
                n[d] = 2;
                if (b2 != bc && b2 != b1) {
                    x[d][2] = b2;
                    n[d] = 3;
                }
            } else if (b2 != bc) {
                x[d][1] = b2;
                n[d] = 2;
            }
        }
    }
    int q = 0, cand = 0;
#pragma unroll
    for (int i0 = 0; i0 < 3; ++i0)
#pragma unroll
        for (int i1 = 0; i1 < 3; ++i1)
#pragma unroll
            for (int i2 = 0; i2 < 3; ++i2) {
                if (i0 < n[0] && i1 < n[1] && i2 < n[2]) {
                    int id = x[0][i0];
                    if (D > 1) id = id * nb[1] + x[1][i1];
                    if (D > 2) id = id * nb[2] + x[2][i2];
                    const int st = offsets[id];
                    tn[(int64_t)(1 + 2 * q) * stride] = st;
                    tn[(int64_t)(2 + 2 * q) * stride] = cand;
                    cand += offsets[id + 1] - st;
                    ++q;
                }
            }
    tn[0] = q;
    tn[(int64_t)(1 + 2 * q) * stride] = 0;
    tn[(int64_t)(2 + 2 * q) * stride] = cand;
    return cand;
}

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
    int64_t xout_stride;   // coil-sum pass: partial image of channel chunk y at xout + y * xout_stride
};

struct LinePass {
    FftAxis ax;
    int n_in, n_out;       // elements along the axis on input / output side
    int64_t B, S;          // outer lines, inner stride (complex elements)
    int TB, TS, lgTS, lgTL, TLP;
    int nchunks;           // coil-sum epilogue: channel chunks looped in one block
    int64_t ntiles_s;      // channel tiles per row tile (see line_grid)
    int coil_sum;
    int pair_add;          // coil-sum epilogue with two channel chunks: both add into xout, which the
                           // pass before cleared (two additions onto zero: the order cannot matter)
    float2* clear;         // INV_MID: image for the next pass's pair_add, cleared here (or null)
    int64_t nclear;
    const float2* in;
    float2* out;
    ImageSide im;
    uint32_t magic_L;      // ceil(2^32 / L)
    uint32_t magic_n;      // ceil(2^32 / n) for the axis length used in index maps
};
enum PassKind { PASS_FWD_FIRST, PASS_FWD_MID, PASS_INV_MID, PASS_INV_LAST };
// Launch grid of a line pass: (row tile, channel tile) as blockIdx (x, y) when the channel tiles fit
// gridDim.y, else one flat index with channel tiles fastest (then the row tiles fit gridDim.y: the
// product is at most 2^31 - 1).  line_tile inverts it without 64-bit division.
constexpr int64_t kGridYMax = 65535;
inline dim3 line_grid(int64_t ntiles_b, int64_t ntiles_s) {
    return ntiles_s <= kGridYMax ? dim3((unsigned)ntiles_b, (unsigned)ntiles_s) : dim3((unsigned)(ntiles_b * ntiles_s));
}
#ifdef __CUDACC__
__device__ __forceinline__ void line_tile(int64_t ntiles_s, uint32_t& tile_b, uint32_t& tile_s) {
    if (ntiles_s <= kGridYMax) {
        tile_b = blockIdx.x;
        tile_s = blockIdx.y;
    } else {
        const uint32_t n = (uint32_t)ntiles_s;
        tile_b = blockIdx.x / n;
        tile_s = blockIdx.x - tile_b * n;
    }
}
#endif
cudaError_t launch_line_pass(PassKind kind, const LinePass& a, dim3 grid, int threads, size_t smem,
                             cudaStream_t s);
// Register-resident two-phase passes (k_line_fft2): factorisations L = L1 L2
// with a compiled kernel, X(L1, L2), L1 <= L2 <= 32.  Launch with TL lines per
// block (power of two, TL L2 threads, a multiple of 32, at most 512) and
// TL (L + 1) complex of dynamic shared memory.
#define NJ_FFT2_SIZES(X) \
    X(8, 8) X(8, 10) X(8, 12) X(8, 16) X(10, 16) X(12, 16) X(12, 20) X(16, 16) \
    X(16, 20) X(16, 24) X(20, 20) X(20, 24) X(16, 32) X(20, 32) X(24, 32) X(32, 32)
template <PassKind KIND>
cudaError_t launch_fft2_kind(int L1, int L2, const LinePass& a, dim3 grid, int threads, size_t smem, cudaStream_t s);
inline bool fft2_factor(int L, int& L1, int& L2) {
#define NJ_FFT2_MATCH(A, B) \
    if (L == (A) * (B)) {   \
        L1 = A;             \
        L2 = B;             \
        return true;        \
    }
    NJ_FFT2_SIZES(NJ_FFT2_MATCH)
#undef NJ_FFT2_MATCH
    return false;
}
// x[i] = sum_k part[k * n + i] for k < nparts, in order (the coil-sum chunks of PASS_INV_LAST).
cudaError_t launch_sum_chunks(const float2* part, int nparts, int64_t n, float2* x, cudaStream_t s);

// ---------------------------------------------------------- interpolation
enum GatherMode { GM_FWD = 0, GM_JVP = 1, GM_VJP = 2 };
struct GatherArgs {
    PointsView pts;
    int D, J;
    int K[kMaxDim];
    const float2* grid;   // [K...][ch], ch = nd * C, channel = dblock * C + c
    int C, nd, has_plain;
    int G, lgG;           // lanes per point (power of two <= 32)
    int W;                // coils per lane slot (1, 2 or 4: single coils, pairs, quads), host dispatch
    KbPoly kb;
    int64_t M;
    float2* y;            // [C][M]
    float2* dy;           // [C][M]
    const float* domega;  // [D][M]
    const float2* v;      // [C][M]
    float* grad;          // [D][M]
    float2* v_sorted;     // VJP: if set, v is also written here in sorted point order, [C][M]
    int v_sorted_cpt;     // ... in the strip layout [C / cpt][M][cpt] instead, when > 0
};
// cpl: lane slots per lane (coils l + k G), or 0 for coil pairs, kGatherQuads for coil quads
constexpr int kGatherQuads = -4;
cudaError_t launch_gather_d1(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s);
cudaError_t launch_gather_d2(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s);
cudaError_t launch_gather_d3(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s);
// cpl: 0 = coil pairs (C even, C <= 64, G >= C / 2), 1 = one coil per lane (C <= G), else 4.
inline cudaError_t launch_gather(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s) {
    return a.D == 1 ? launch_gather_d1(mode, a, cpl, s)
                    : (a.D == 2 ? launch_gather_d2(mode, a, cpl, s) : launch_gather_d3(mode, a, cpl, s));
}

struct SpreadArgs {
    PointsView pts;
    int D, J;
    int K[kMaxDim];
    int B[kMaxDim], nb[kMaxDim];   // tile (= bin) edge, tiles per dim
    int nbins;
    const int* offsets;   // [nbins + 1]
    const int* tile_nbr;  // [kNbrStride][nbins], entry-major
    const int4* items;    // spread work items {tile, part, nparts, candidates}
    const int* nitems;
    const int* tile_parts;
    const int* heavy;     // [nbins + 1]: count, then the tiles split over several work items
    int max_items, P;
    const float2* y;      // [C][M], by original index, or by sorted position when y_sorted
    int y_sorted;
    int64_t M;
    int C, CC;            // coils, coils per block
    int G, lgG;           // tap slots per warp (lanes = G slots x 32/G coils)
    KbPoly kb;
    float2* grid;         // [K...][C]
};
// Strip spread (kernels_strip.cu, 2-D and 3-D): one warp per work item (a strip unit or a part of one).
struct StripArgs {
    PointsView pts;
    StripGeom g;
    StripTables t;
    int max_items;
    const float2* y;      // sorted coil values, [ncg][M][CPW] (coil c: group c / CPW, slot c % CPW)
    int C, ncg;           // coils, coil groups of CPW = 64 / NSL coils (a coil pair per lane)
    float2* grid;         // [K0][K1][C]
    float2* partial;      // [slots][ncg][kStripW][32] coil pairs (float4)
    int* counters;        // [slots][ncg], zero between calls
};
cudaError_t launch_spread_strips(const StripArgs& a, cudaStream_t s);
// ys[sorted position pos[o] of point o] = y[c][o], in the strip layout [ncg][M][cpt].
cudaError_t launch_permute_y_strips(const int* pos, const float2* y, float2* ys, int64_t M, int C, int cpt,
                                    cudaStream_t s);
cudaError_t launch_spread(const SpreadArgs& a, int cpl, cudaStream_t s, size_t smem);
cudaError_t launch_zero_heavy_tiles(const SpreadArgs& a, cudaStream_t s);
// ys[c][i] = y[c][idx[i].w]: the coil values in sorted point order (coalesced reads in the spread).
cudaError_t launch_permute_y(const int4* idx, const float2* y, float2* ys, int64_t M, int C, cudaStream_t s);
int spread_min_slots(int D, int J);   // fewest tap slots per warp the spread kernel supports
// Tile spread (row owners in 2-D, cell owners in 3-D): D in {2, 3}, every tile edge <= K - J + 1 and >= J - 1, prod B <= 512,
// a.CC = coils per block (4, 8 or 16), a.P candidates per work item (<= prod B).
cudaError_t launch_spread_cells(const SpreadArgs& a, cudaStream_t s);

}  // namespace nj

// Adjoint interpolation (spread), Sec. II-D: G[k] = sum_i psi(t_i - k) y_i, the
// transpose of the gather, onto the oversampled grid [K...][C].
//
// Output-driven tiles.  The grid is cut into tiles (the bins of the sort); a
// work item owns one tile and visits the points of the bins that can reach
// it: its own bin and the bins holding the J-1 cells before it (a window
// covers J cells to the right of its start).  A tile with few candidates is
// one work item and is stored with plain coalesced writes, zeros included, so
// the grid needs no clearing and no global atomics.  A tile with many
// candidates (the k-space centre of radial trajectories) is split over several
// work items; it is cleared first and each item adds its partial tile with
// float2 vector atomics, skipping cells it did not touch.
//
// Inside a work item the warps take batches of 32 consecutive candidates in
// turn and stage them one per lane (record, window test, the J*D kernel
// weights and the y values go to shared memory).  It then walks the staged
// candidates in order with its 32 lanes split into NS row slots x (32 / NS)
// coils: lane (s, c) owns the window rows s, s + NS, ... for coil c, so no
// two lanes of a warp ever address the same tile cell.  Consecutive points
// that share a window (dense sampling near the k-space centre) are summed in
// registers and added to the shared tile once per run.
#include <algorithm>

#include "interp.cuh"

namespace nj {

template <int D, int J>
struct SpreadShape {
    // A window is JO outer rows (all axes but the last) of JI taps (the last axis);
    // 1-D windows are J rows of one tap.
    static constexpr int JO = D == 1 ? J : (D == 2 ? J : J * J);
    static constexpr int JI = D == 1 ? 1 : J;
    static constexpr int NT_CAP = 18;   // accumulators per lane
    static constexpr int ns_for(int n) { return n >= 32 ? 32 : (((JO + n - 1) / n) * JI <= NT_CAP ? n : ns_for(2 * n)); }
    static constexpr int NS_MIN = ns_for(1);          // fewest row slots keeping NR * JI <= NT_CAP
    static constexpr int NR = (JO + NS_MIN - 1) / NS_MIN;
};

constexpr int kSpreadWarps = 8;
constexpr int kSpreadCoilsPerWarp = 16;   // y staging per warp: 32 candidates x up to 16 coils

template <int D, int J>
__global__ void __launch_bounds__(256, 2) k_spread(SpreadArgs a) {
    pdl_wait();
    using SH = SpreadShape<D, J>;
    constexpr int JO = SH::JO, JI = SH::JI, NR = SH::NR;
    extern __shared__ float4 smem4[];
    __shared__ int s_start[27], s_pref[28], s_nn;
    __shared__ float s_w[kSpreadWarps][32][D * J + 1];                 // kernel weights per staged candidate
    __shared__ int4 s_ix[kSpreadWarps][32];                            // window start, original index
    __shared__ float2 s_y[kSpreadWarps][32][kSpreadCoilsPerWarp + 1];  // y of the staged candidates
    const int it = blockIdx.x;
    if (it >= a.nitems[0]) return;     // block-uniform
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int4 item = a.items[it];
    const int tile = item.x, part = item.y, nparts = item.z;
    int nb[kMaxDim] = {a.nb[0], a.nb[1], a.nb[2]};
    int org[kMaxDim] = {0, 0, 0}, Bt[kMaxDim] = {1, 1, 1}, Kd[kMaxDim] = {1, 1, 1};
    {
        int r = tile;
        for (int d = D - 1; d >= 0; --d) {
            const int bc = r % nb[d];
            r /= nb[d];
            Kd[d] = a.K[d];
            org[d] = bc * a.B[d];
            Bt[d] = min(a.B[d], Kd[d] - org[d]);
        }
    }
    const int c0 = blockIdx.y * a.CC;
    const int ncc = min(a.CC, a.C - c0);
    const int CC = a.CC;
    const int tcells = Bt[0] * Bt[1] * Bt[2];
    float2* tl = (float2*)smem4;   // [tcells][CC]

    {   // bins that reach this tile (listed by the sort)
        const int* tn = a.tile_nbr + tile;
        const int64_t st = a.nbins;
        if (tid == 0) s_nn = tn[0];
        if (tid < 27) s_start[tid] = tn[(1 + 2 * tid) * st];      // entries past the count are never used
        if (tid < 28) s_pref[tid] = tn[(2 + 2 * tid) * st];
    }
    {   // clear the tile
        float4* t4 = (float4*)tl;
        const int n4 = tcells * CC / 2;
        for (int i = tid; i < n4; i += blockDim.x) t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((tcells * CC) & 1 && tid == 0) tl[tcells * CC - 1] = make_float2(0.f, 0.f);
    }
    __syncthreads();

    // lane roles: NS row slots x CCW coils; slot s owns rows s, s + NS, ...
    const int NS = a.G;
    const int CCW = 32 / NS;
    const int slot = lane / CCW, cw = lane - slot * CCW;
    const int nn = s_nn;
    const int lo = part * a.P, hi = min(s_pref[nn], lo + a.P);
    int q = 0;   // neighbour-bin cursor of this lane's staged candidate

    for (int cp = 0; cp < ncc; cp += CCW) {
        const int c = cp + cw;
        const bool cok = c < ncc;
        const int nyc = min(CCW, ncc - cp);   // coils staged per candidate in this pass
        float2 acc[NR][JI];
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int j = 0; j < JI; ++j) acc[r][j] = make_float2(0.f, 0.f);
        int rk0 = -1, rk1 = 0, rk2 = 0;   // window start of the open run (rk0 < 0: none)
        bool run_in = false;             // the open run's window lies wholly inside the tile

        auto flush = [&]() {
            if (rk0 < 0) return;
            if (cok) {
                int ls[kMaxDim] = {rk0 - org[0], rk1 - org[1], rk2 - org[2]};
#pragma unroll
                for (int d = 0; d < D; ++d)
                    if (ls[d] < 0) ls[d] += Kd[d];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int o = slot + NS * r;   // outer row: (j0) in 2-D, (j0, j1) in 3-D, tap in 1-D
                    if (o >= JO) continue;
                    int rowcell;
                    bool rin = true;
                    if (D == 1) {
                        int l = ls[0] + o;
                        if (l >= Kd[0]) l -= Kd[0];
                        rin = l < Bt[0];
                        rowcell = l;
                    } else if (D == 2) {
                        int l = ls[0] + o;
                        if (l >= Kd[0]) l -= Kd[0];
                        rin = l < Bt[0];
                        rowcell = l * Bt[1];
                    } else {
                        int l0 = ls[0] + o / J, l1 = ls[1] + o % J;
                        if (l0 >= Kd[0]) l0 -= Kd[0];
                        if (l1 >= Kd[1]) l1 -= Kd[1];
                        rin = l0 < Bt[0] && l1 < Bt[1];
                        rowcell = (l0 * Bt[1] + l1) * Bt[2];
                    }
                    if (!rin) continue;
                    const int li0 = D == 1 ? 0 : ls[D - 1];
                    const int Kl = Kd[D - 1], Bl = Bt[D - 1];
#pragma unroll
                    for (int j = 0; j < JI; ++j) {
                        if (acc[r][j].x == 0.f && acc[r][j].y == 0.f) continue;
                        int l = li0 + j;
                        if (D > 1 && !run_in) {
                            if (l >= Kl) l -= Kl;
                            if (l >= Bl) continue;
                        }
                        float2* tp = tl + (size_t)(rowcell + (D > 1 ? l : 0)) * CC + c;
                        atomicAdd(&tp->x, acc[r][j].x);
                        atomicAdd(&tp->y, acc[r][j].y);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int j = 0; j < JI; ++j) acc[r][j] = make_float2(0.f, 0.f);
            rk0 = -1;
        };

        q = 0;
        // batches of 32 consecutive candidates, dealt to the warps in turn
        for (int bb = lo + 32 * warp; bb < hi; bb += 32 * kSpreadWarps) {
            // stage 32 candidates, one per lane: record, hit test, weights, y
            const int cand = bb + lane;
            bool hit = false, inside = false;
            if (cand < hi) {
                while (q + 1 < nn && s_pref[q + 1] <= cand) ++q;
                const int64_t p = s_start[q] + (cand - s_pref[q]);
                const int4 ix = a.pts.idx[p];
                hit = true;
                inside = true;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    int ls = (d == 0 ? ix.x : (d == 1 ? ix.y : ix.z)) - org[d];
                    if (ls < 0) ls += Kd[d];
                    const int lend = ls + J - 1;   // last tap, unwrapped
                    hit = hit && (ls < Bt[d] || lend >= Kd[d]);
                    inside = inside && lend < Bt[d];
                }
                if (hit) {
                    const float* pw = a.pts.w + (int64_t)p * a.pts.ws;
#pragma unroll
                    for (int q = 0; q < D * J; ++q) s_w[warp][lane][q] = __ldg(pw + q);
                    for (int cc = 0; cc < nyc; ++cc)
                        s_y[warp][lane][cc] = __ldg(a.y + (int64_t)(c0 + cp + cc) * a.M + ix.w);
                    s_ix[warp][lane] = make_int4(ix.x, ix.y, ix.z, inside ? 1 : 0);
                }
            }
            unsigned hits = __ballot_sync(0xffffffffu, hit);
            __syncwarp();
            while (hits) {
                const int b = __ffs(hits) - 1;
                hits &= hits - 1;
                const int4 rec = s_ix[warp][b];
                if (rec.x != rk0 || (D > 1 && rec.y != rk1) || (D > 2 && rec.z != rk2)) {
                    flush();
                    rk0 = rec.x;
                    rk1 = rec.y;
                    rk2 = rec.z;
                    run_in = rec.w != 0;
                }
                const float* wv = s_w[warp][b];
                const float2 yv = cok ? s_y[warp][b][cw] : make_float2(0.f, 0.f);
                float wi[JI];
#pragma unroll
                for (int j = 0; j < JI; ++j) wi[j] = D == 1 ? 1.f : wv[(D - 1) * J + j];
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int o = slot + NS * r;
                    if (o >= JO) continue;
                    const float wo = D == 3 ? wv[o / J] * wv[J + o % J] : wv[o];
                    const float2 yw = make_float2(wo * yv.x, wo * yv.y);
#pragma unroll
                    for (int j = 0; j < JI; ++j) {
                        acc[r][j].x = fmaf(wi[j], yw.x, acc[r][j].x);
                        acc[r][j].y = fmaf(wi[j], yw.y, acc[r][j].y);
                    }
                }
            }
            __syncwarp();
        }
        flush();
    }
    __syncthreads();

    // write the tile row by row: a row (all axes but the last fixed) is Bt_last cells,
    // contiguous in the grid; element i of a row is cell i / ncc, coil i % ncc
    const int K1 = D > 1 ? Kd[1] : 1, K2 = D > 2 ? Kd[2] : 1;
    const int Bl = Bt[D - 1];
    const int rowlen = Bl * ncc;
    const int nrows = tcells / Bl;
    const uint32_t mg = ncc > 1 ? (uint32_t)((((uint64_t)1 << 32) + ncc - 1) / ncc) : 0u;
    for (int f = tid; f < nrows * rowlen; f += blockDim.x) {
        const int row = f / rowlen, i = f - row * rowlen;   // rowlen: block-uniform
        const int cell_in_row = (int)div_magic((uint32_t)i, (uint32_t)ncc, mg);
        const int cl = i - cell_in_row * ncc;
        int r0 = row, r1 = 0;
        if (D == 3) { r1 = row % Bt[1]; r0 = row / Bt[1]; }
        int64_t gcell;
        if (D == 1) gcell = org[0] + cell_in_row;
        else if (D == 2) gcell = (int64_t)(org[0] + r0) * K1 + org[1] + cell_in_row;
        else gcell = ((int64_t)(org[0] + r0) * K1 + (org[1] + r1)) * K2 + org[2] + cell_in_row;
        const float2 v = tl[(size_t)(row * Bl + cell_in_row) * CC + cl];
        float2* dst = a.grid + gcell * a.C + c0 + cl;
        if (nparts == 1) *dst = v;
        else if (v.x != 0.f || v.y != 0.f) atomicAdd(dst, v);
    }
}

// ---------------------------------------------------------------------------
// Cell-owner spread (fast path in 3-D).  Used when no window can cover a tile twice
// (every tile edge Bt_d <= K_d - J + 1) and tiles are at least J - 1 wide.
// The block stages the work item's candidates (one per thread), keeps those
// whose window reaches the tile, and counting-sorts them in shared memory by
// window-start row, in coordinates e_d = start_d - org_d + J - 1 in
// [0, Bt_d + J - 1) (the row is e_0 in 2-D, (e_0, e_1) in 3-D).  Thread t then
// owns tile cell t for CPT coils: the points covering cell l are those with
// e_d in [l_d, l_d + J - 1] for every axis, with tap j_d = l_d + J - 1 - e_d,
// so it visits the J (2-D) or J^2 (3-D) rows around it, keeps the points whose
// last coordinate fits, and sums w * y in registers.  No atomics on the tile;
// within a row the points are summed in original-index order, so a tile that
// is one work item is bitwise reproducible.  Heavy tiles (several work items)
// are cleared first and receive float2 vector atomics (rounding-level order
// differences).
template <int D, int J, int CPT>
__global__ void __launch_bounds__(512) k_spread_cells(SpreadArgs a) {
    pdl_wait();
    extern __shared__ float4 smem4[];
    __shared__ int s_start[27], s_pref[28], s_nn, s_nh;
    const int it = blockIdx.x;
    if (it >= a.nitems[0]) return;     // block-uniform
    const int tid = threadIdx.x, nt = blockDim.x;
    const int4 item = a.items[it];
    const int tile = item.x, part = item.y, nparts = item.z;
    int org[kMaxDim] = {0, 0, 0}, Bt[kMaxDim] = {1, 1, 1}, Kd[kMaxDim] = {1, 1, 1}, E[kMaxDim] = {1, 1, 1};
    {
        int r = tile;
        for (int d = D - 1; d >= 0; --d) {
            const int nbd = a.nb[d];
            const int bc = r % nbd;
            r /= nbd;
            Kd[d] = a.K[d];
            org[d] = bc * a.B[d];
            Bt[d] = min(a.B[d], Kd[d] - org[d]);
            E[d] = Bt[d] + J - 1;
        }
    }
    // row bins: all start coordinates but the last (E0 in 2-D, E0 * E1 in 3-D); hits are
    // bucketed by their full window-start cell, key = row * El + e_last
    const int NR = D == 2 ? E[0] : E[0] * E[1];
    const int El = E[D - 1];
    const int NK = NR * El;
    const int P = a.P;
    const int c0 = blockIdx.y * CPT;
    const int ncc = min(CPT, a.C - c0);
    // shared layout: weights [P][D*J], y [P][CPT+1], last start coordinate and original index
    // per hit [P] each, sorted hits [P], row starts/ends [NR+1], cursors [NR], arrival list [P]
    float* s_w = (float*)smem4;
    float2* s_y = (float2*)(s_w + P * D * J + ((P * D * J) & 1));
    int* s_el = (int*)(s_y + (size_t)P * (CPT + 1));
    int* s_orig = s_el + P;
    int* s_list = s_orig + P;
    int* s_cnt = s_list + P;       // [NK + 1] first slot of each start cell
    int* s_cur = s_cnt + NK + 1;   // [NK]
    int* s_tmp = s_cur + NK;       // [P] hits in arrival order within their start cells

    {
        const int* tn = a.tile_nbr + tile;
        const int64_t st = a.nbins;
        if (tid == 0) { s_nn = tn[0]; s_nh = 0; }
        if (tid < 27) s_start[tid] = tn[(1 + 2 * tid) * st];      // entries past the count are never used
        if (tid < 28) s_pref[tid] = tn[(2 + 2 * tid) * st];
    }
    for (int i = tid; i <= NK; i += nt) s_cnt[i] = 0;
    __syncthreads();

    // stage: thread t takes candidate lo + t
    const int nn = s_nn;
    const int lo = part * P, hi = min(s_pref[nn], lo + P);
    const int cand = lo + tid;
    int my_row = -1, my_slot = -1, my_orig = 0;
    if (tid < P && cand < hi) {
        int q = 0;
        while (q + 1 < nn && s_pref[q + 1] <= cand) ++q;
        const int64_t p = s_start[q] + (cand - s_pref[q]);
        const int4 ix = a.pts.idx[p];
        bool hit = true;
        int e[kMaxDim] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < D; ++d) {
            int sd = (d == 0 ? ix.x : (d == 1 ? ix.y : ix.z)) - org[d];
            if (sd < 0) sd += Kd[d];
            if (sd > Kd[d] - J) sd -= Kd[d];           // starts up to J-1 cells before the tile
            hit = hit && sd >= -(J - 1) && sd < Bt[d];
            e[d] = sd + J - 1;
        }
        if (hit) {
            my_slot = atomicAdd(&s_nh, 1);
            my_row = (D == 2 ? e[0] : e[0] * E[1] + e[1]) * El + e[D - 1];   // start-cell key
            my_orig = ix.w;
            s_el[my_slot] = e[D - 1];
            s_orig[my_slot] = my_orig;
            const float* pw = a.pts.w + p * a.pts.ws;
            float* w = s_w + my_slot * (D * J);
#pragma unroll
            for (int q = 0; q < D * J; ++q) w[q] = __ldg(pw + q);
            float2* yv = s_y + (size_t)my_slot * (CPT + 1);
            float2 yl[CPT];   // all coil loads in flight at once (clamped coil, zero past the chunk)
#pragma unroll
            for (int c = 0; c < CPT; ++c)
                yl[c] = __ldg(a.y + (int64_t)(c0 + min(c, ncc - 1)) * a.M + (a.y_sorted ? p : (int64_t)ix.w));
#pragma unroll
            for (int c = 0; c < CPT; ++c) yv[c] = c < ncc ? yl[c] : make_float2(0.f, 0.f);
            atomicAdd(&s_cnt[my_row], 1);
        }
    }
    __syncthreads();
    // exclusive scan of the row counts: each thread a chunk, then a two-level shuffle scan of
    // the chunk sums; s_cnt[r] = first slot of row r, s_cur[r] a copy used as placement cursor
    {
        __shared__ int s_wsum[32];
        const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
        const int per = (NK + nt - 1) / nt;
        const int b0 = min(NK, tid * per), b1 = min(NK, b0 + per);
        int sum = 0;
        for (int b = b0; b < b1; ++b) sum += s_cnt[b];
        int x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int w = lane < nw ? s_wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nw) s_wsum[lane] = w;
        }
        __syncthreads();
        int run = x - sum + (wid ? s_wsum[wid - 1] : 0);
        for (int b = b0; b < b1; ++b) {
            const int c = s_cnt[b];
            s_cnt[b] = run;
            s_cur[b] = run;
            run += c;
        }
        if (tid == nt - 1) s_cnt[NK] = run;
    }
    __syncthreads();
    // place hits in a fixed order: first in arrival order inside their start cell's range, then
    // each hit ranks itself by original point index among the hits of its own start cell (few),
    // so the sums below do not depend on the order in which threads arrived.
    if (my_slot >= 0) s_tmp[atomicAdd(&s_cur[my_row], 1)] = my_slot;
    __syncthreads();
    if (my_slot >= 0) {
        const int r0 = s_cnt[my_row], r1 = s_cur[my_row];
        int rank = 0;
        for (int k = r0; k < r1; ++k) rank += s_orig[s_tmp[k]] < my_orig;
        s_list[r0 + rank] = my_slot;
    }
    __syncthreads();

    // gather: thread t owns cell t (one thread per tile cell).  The points covering cell l
    // start in rows l_0 .. l_0 + J - 1 (and l_1 .. l_1 + J - 1 in 3-D) and have
    // e_last - l_last in [0, J); tap j_d = J - 1 - (e_d - l_d).
    const int tcells = Bt[0] * Bt[1] * Bt[2];
    const int cell = tid;
    float2 acc[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[c] = make_float2(0.f, 0.f);
    if (cell < tcells) {
        int l[kMaxDim] = {0, 0, 0};
        {
            int r = cell;
            for (int d = D - 1; d >= 0; --d) {
                l[d] = r % Bt[d];
                r /= Bt[d];
            }
        }
        const int ll = l[D - 1];
#pragma unroll 1
        for (int a0 = 0; a0 < J; ++a0) {
#pragma unroll 1
            for (int a1 = 0; a1 < (D > 2 ? J : 1); ++a1) {
                const int row = D == 2 ? l[0] + a0 : (l[0] + a0) * E[1] + (l[1] + a1);
                // start cells (row, ll .. ll + J - 1): one contiguous range of the sorted hits
                const int h0 = s_cnt[row * El + ll], h1 = s_cnt[row * El + ll + J];
                for (int hh = h0; hh < h1; ++hh) {
                    const int h = s_list[hh];
                    const int al = s_el[h] - ll;
                    const float* w = s_w + h * (D * J);
                    float wt = w[J - 1 - a0] * w[(D - 1) * J + J - 1 - al];
                    if (D > 2) wt *= w[J + J - 1 - a1];
                    const float2* yv = s_y + (size_t)h * (CPT + 1);
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        acc[c].x = fmaf(wt, yv[c].x, acc[c].x);
                        acc[c].y = fmaf(wt, yv[c].y, acc[c].y);
                    }
                }
            }
        }
    }
    __syncthreads();   // every staged y has been read
    if (cell < tcells) {
        float2* o = s_y + (size_t)cell * (CPT + 1);
#pragma unroll
        for (int c = 0; c < CPT; ++c) o[c] = acc[c];
    }
    __syncthreads();
    // write the tile coil-fastest: a tile row is Bt_last cells, contiguous in the grid
    const int K1 = D > 1 ? Kd[1] : 1, K2 = D > 2 ? Kd[2] : 1;
    const int Bl = Bt[D - 1];
    const int rowlen = Bl * ncc;
    const int nrows = tcells / Bl;
    const uint32_t mg = ncc > 1 ? (uint32_t)((((uint64_t)1 << 32) + ncc - 1) / ncc) : 0u;
    for (int f = tid; f < nrows * rowlen; f += nt) {
        const int row = f / rowlen, i = f - row * rowlen;
        const int cr = (int)div_magic((uint32_t)i, (uint32_t)ncc, mg);
        const int c = i - cr * ncc;
        int r0 = row, r1 = 0;
        if (D == 3) { r1 = row % Bt[1]; r0 = row / Bt[1]; }
        const int64_t gcell = D == 2 ? (int64_t)(org[0] + r0) * K1 + org[1] + cr
                                     : ((int64_t)(org[0] + r0) * K1 + (org[1] + r1)) * K2 + org[2] + cr;
        const float2 v = s_y[(size_t)(row * Bl + cr) * (CPT + 1) + c];
        float2* dst = a.grid + gcell * a.C + c0 + c;
        if (nparts == 1) *dst = v;
        else if (v.x != 0.f || v.y != 0.f) atomicAdd(dst, v);
    }
}

template <int D, int J>
static cudaError_t spread_cells_cpt(const SpreadArgs& a, cudaStream_t s, int threads) {
    const int cpt = a.CC;
    int E = 1;   // start-cell buckets
    for (int d = 0; d < D; ++d) E *= a.B[d] + J - 1;
    const size_t smem = (size_t)a.P * D * J * sizeof(float) + sizeof(float) + (size_t)a.P * (cpt + 1) * sizeof(float2) +
                        4 * (size_t)a.P * sizeof(int) + (size_t)(2 * E + 1) * sizeof(int);
    dim3 grid((unsigned)a.max_items, (unsigned)((a.C + cpt - 1) / cpt));
    if (cpt <= 4) {
        ensure_smem<k_spread_cells<D, J, 4>>(smem);
        (void)launch_pdl(k_spread_cells<D, J, 4>, grid, threads, smem, s, a);
    } else if (cpt <= 8) {
        ensure_smem<k_spread_cells<D, J, 8>>(smem);
        (void)launch_pdl(k_spread_cells<D, J, 8>, grid, threads, smem, s, a);
    } else {
        ensure_smem<k_spread_cells<D, J, 16>>(smem);
        (void)launch_pdl(k_spread_cells<D, J, 16>, grid, threads, smem, s, a);
    }
    return cudaGetLastError();
}

template <int D>
static cudaError_t spread_cells_d(const SpreadArgs& a, cudaStream_t s, int threads) {
    switch (a.J) {
        case 4: return spread_cells_cpt<D, 4>(a, s, threads);
        case 5: return spread_cells_cpt<D, 5>(a, s, threads);
        case 6: return spread_cells_cpt<D, 6>(a, s, threads);
        case 7: return spread_cells_cpt<D, 7>(a, s, threads);
        default: return spread_cells_cpt<D, 8>(a, s, threads);
    }
}

static cudaError_t launch_spread_cells_3d(const SpreadArgs& a, cudaStream_t s) {
    if (a.max_items == 0) return cudaSuccess;
    int threads = 1;
    for (int d = 0; d < a.D; ++d) threads *= a.B[d];
    return spread_cells_d<3>(a, s, threads);
}

// ---------------------------------------------------------------------------
// Row-owner spread (fast path in 2-D).  Used when no window can cover a tile twice
// (every tile edge Bt_d <= K_d - J + 1) and tiles are at least J - 1 wide.
// The block stages the work item's candidates (one per thread), keeps those
// whose window reaches the tile and counting-sorts them in shared memory by
// the outer coordinates of their window start, e_d = start_d - org_d + J - 1
// in [0, Bt_d + J - 1) (bucket e_0 in 2-D, (e_0, e_1) in 3-D).
//
// The tile (all coils of the block's chunk) is accumulated in shared memory.
// Its rows (all axes but the last) are cut into units of a row segment, and
// warp w owns the units u = w mod (warps): the points covering row l are those
// of the J (2-D) or J^2 (3-D) buckets with e_d in [l_d, l_d + J - 1], with
// outer taps j_d = l_d + J - 1 - e_d.  For each such point the warp's lanes
// take (last-axis tap, coil) pairs and add w * y to the cells of the row that
// fall inside the unit: no two lanes of a warp, and no two warps, ever write
// the same cell, so the tile needs no atomics.  Heavy tiles (several work
// items) are cleared first and receive float2 vector atomics; the order of the
// sums follows the (arrival-ordered) hit list, so results agree to rounding.
template <int D, int J, int CPT>
__global__ void __launch_bounds__(512) k_spread_rows(SpreadArgs a) {
    pdl_wait();
    extern __shared__ float4 smem4[];
    __shared__ int s_start[27], s_pref[28], s_nn, s_nh;
    const int nitems = a.nitems[0];
    int it = blockIdx.x;
    if (it >= nitems) return;     // block-uniform
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, NW = nt >> 5;
    // Persistent: the block walks items it, it + gridDim.x, ...  The next item's descriptor and
    // its tile's bin list are loaded while the current item is processed (two dependent global
    // round trips that would otherwise open every item).
    int4 item = a.items[it];
    int tn0 = 0, tn1 = 0, tn2 = 0;   // this thread's entries of the tile's bin list
    {
        const int* tn = a.tile_nbr + item.x;
        const int64_t st = a.nbins;
        if (tid == 0) tn0 = tn[0];
        if (tid < 27) tn1 = tn[(1 + 2 * tid) * st];
        if (tid < 28) tn2 = tn[(2 + 2 * tid) * st];
    }
    for (;;) {
        const int itn = it + (int)gridDim.x;
        int4 itemn = make_int4(0, 0, 0, 0);
        if (itn < nitems) itemn = a.items[itn];
        const int tile = item.x, part = item.y, nparts = item.z;
        int org[kMaxDim] = {0, 0, 0}, Bt[kMaxDim] = {1, 1, 1}, Kd[kMaxDim] = {1, 1, 1}, E[kMaxDim] = {1, 1, 1};
        {
            int r = tile;
            for (int d = D - 1; d >= 0; --d) {
                const int nbd = a.nb[d];
                const int bc = r % nbd;
                r /= nbd;
                Kd[d] = a.K[d];
                org[d] = bc * a.B[d];
                Bt[d] = min(a.B[d], Kd[d] - org[d]);
                E[d] = Bt[d] + J - 1;
            }
        }
        const int NB = D == 2 ? E[0] : E[0] * E[1];   // buckets
        const int P = a.P;
        const int c0 = blockIdx.y * CPT;
        const int ncc = min(CPT, a.C - c0);
        const int tcells = Bt[0] * Bt[1] * Bt[2];
        const int Bl = Bt[D - 1];
        const int R = tcells / Bl;                    // tile rows
        // shared: tile [tcells][CPT], y [P][YP], weights [P][WP], last start e_l [P], bucket [P],
        // sorted hits [P], bucket offsets [NB + 1], cursors [NB]; odd row pitches YP, WP keep the
        // one-candidate-per-thread staging stores on distinct banks
        constexpr int YP = CPT + 1, WP = D * J + ((D * J + 1) & 1);
        float2* s_acc = (float2*)smem4;
        float2* s_y = s_acc + (size_t)tcells * CPT;
        float* s_w = (float*)(s_y + (size_t)P * YP);
        int* s_el = (int*)(s_w + P * WP);
        int* s_bk = s_el + P;
        int* s_list = s_bk + P;
        int* s_off = s_list + P;
        int* s_cur = s_off + NB + 1;

        if (tid == 0) { s_nn = tn0; s_nh = 0; }
        if (tid < 27) s_start[tid] = tn1;      // entries past the count are never used
        if (tid < 28) s_pref[tid] = tn2;
        for (int i = tid; i < tcells * CPT; i += nt) s_acc[i] = make_float2(0.f, 0.f);
        for (int i = tid; i < NB; i += nt) s_cur[i] = 0;
        __syncthreads();

        // ------------------------------------------------ stage and count the hits
        const int nn = s_nn;
        const int lo = part * P, hi = min(s_pref[nn], lo + P);
        for (int t = tid; t < P; t += nt) {
            const int cand = lo + t;
            if (cand >= hi) break;
            int q = 0;
            while (q + 1 < nn && s_pref[q + 1] <= cand) ++q;
            const int64_t pidx = s_start[q] + (cand - s_pref[q]);
            const int4 ix = a.pts.idx[pidx];
            // weights and (sorted) coil values are loaded with the record, before the window test, so
            // that staging takes one memory round trip; a miss wastes these reads
            float wv[D * J];
            const float* pw = a.pts.w + pidx * a.pts.ws;
#pragma unroll
            for (int q = 0; q < D * J; ++q) wv[q] = __ldg(pw + q);
            float2 yl[CPT];   // clamped coil, zero past the chunk
            if (a.y_sorted) {
#pragma unroll
                for (int c = 0; c < CPT; ++c) yl[c] = __ldg(a.y + (int64_t)(c0 + min(c, ncc - 1)) * a.M + pidx);
            }
            bool hit = true;
            int e[kMaxDim] = {0, 0, 0};
#pragma unroll
            for (int d = 0; d < D; ++d) {
                int sd = (d == 0 ? ix.x : (d == 1 ? ix.y : ix.z)) - org[d];
                if (sd < 0) sd += Kd[d];
                if (sd > Kd[d] - J) sd -= Kd[d];           // starts up to J-1 cells before the tile
                hit = hit && sd >= -(J - 1) && sd < Bt[d];
                e[d] = sd + J - 1;
            }
            if (!hit) continue;
            if (!a.y_sorted) {
#pragma unroll
                for (int c = 0; c < CPT; ++c) yl[c] = __ldg(a.y + (int64_t)(c0 + min(c, ncc - 1)) * a.M + ix.w);
            }
            const int slot = atomicAdd(&s_nh, 1);
            const int bk = D == 2 ? e[0] : e[0] * E[1] + e[1];
            s_el[slot] = e[D - 1] - (J - 1);               // window start along the last axis, tile-relative
            s_bk[slot] = bk;
            float* w = s_w + slot * WP;
#pragma unroll
            for (int q = 0; q < D * J; ++q) w[q] = wv[q];
            float2* yv = s_y + (size_t)slot * YP;
#pragma unroll
            for (int c = 0; c < CPT; ++c) yv[c] = c < ncc ? yl[c] : make_float2(0.f, 0.f);
            atomicAdd(&s_cur[bk], 1);
        }
        if (itn < nitems) {   // the next item's bin list, consumed at its start
            const int* tn = a.tile_nbr + itemn.x;
            const int64_t st = a.nbins;
            if (tid == 0) tn0 = tn[0];
            if (tid < 27) tn1 = tn[(1 + 2 * tid) * st];
            if (tid < 28) tn2 = tn[(2 + 2 * tid) * st];
        }
        __syncthreads();
        // exclusive scan of the bucket counts (one warp)
        if (warp == 0) {
            int carry = 0;
            for (int b0 = 0; b0 < NB; b0 += 32) {
                const int b = b0 + lane;
                const int v = b < NB ? s_cur[b] : 0;
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += u;
                }
                if (b < NB) {
                    s_off[b] = carry + incl - v;
                    s_cur[b] = carry + incl - v;
                }
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) s_off[NB] = carry;
        }
        __syncthreads();
        const int nh = s_nh;
        for (int h = tid; h < nh; h += nt) s_list[atomicAdd(&s_cur[s_bk[h]], 1)] = h;
        __syncthreads();

        // ------------------------------------------------------------- accumulate
        constexpr int JPL = 32 / CPT;                 // last-axis taps per lane pass
        constexpr int NJX = (J + JPL - 1) / JPL;      // passes
        const int c = lane & (CPT - 1), jg = lane / CPT;
        const int nseg = R >= NW ? 1 : (NW + R - 1) / R;   // row segments when rows are fewer than warps
        const int segw = (Bl + nseg - 1) / nseg;
        if constexpr (D == 2) {
            // The points covering tile row r are those of buckets r .. r + J - 1: one contiguous
            // range of the sorted hit list, with outer tap J - 1 - (bucket - r).  The loop is
            // software-pipelined: the next point's metadata is read (from arrays this phase never
            // writes) before the current point's cells are updated.
            for (int u = warp; u < R * nseg; u += NW) {
                const int r = u / nseg, sg = u - r * nseg;
                const int x_lo = sg * segw, x_hi = min(Bl, x_lo + segw);
                const int hb = s_off[r], he = s_off[r + J];
                if (hb >= he) continue;
                float2* arow = s_acc + (size_t)r * Bl * CPT + c;
                int hx = s_list[hb];
                float won = s_w[hx * WP + J - 1 - (s_bk[hx] - r)];
                float2 yn = s_y[(size_t)hx * YP + c];
                int sln = s_el[hx];
                float wxn[NJX];
#pragma unroll
                for (int k = 0; k < NJX; ++k) wxn[k] = s_w[hx * WP + J + min(jg + k * JPL, J - 1)];
                for (int hh = hb; hh < he; ++hh) {
                    const float wo = won;
                    const float2 yv = yn;
                    const int sl = sln;
                    float wx[NJX];
#pragma unroll
                    for (int k = 0; k < NJX; ++k) wx[k] = wxn[k];
                    hx = s_list[min(hh + 1, he - 1)];
                    won = s_w[hx * WP + J - 1 - (s_bk[hx] - r)];
                    yn = s_y[(size_t)hx * YP + c];
                    sln = s_el[hx];
#pragma unroll
                    for (int k = 0; k < NJX; ++k) wxn[k] = s_w[hx * WP + J + min(jg + k * JPL, J - 1)];
#pragma unroll
                    for (int k = 0; k < NJX; ++k) {
                        const int jx = jg + k * JPL;
                        const int col = sl + jx;
                        if (jx < J && col >= x_lo && col < x_hi) {
                            const float wt = wo * wx[k];
                            float2* t = arow + col * CPT;
                            float2 v = *t;
                            v.x = fmaf(wt, yv.x, v.x);
                            v.y = fmaf(wt, yv.y, v.y);
                            *t = v;
                        }
                    }
                    __syncwarp();   // the next point's cells may be another lane's
                }
            }
        } else {
            for (int u = warp; u < R * nseg; u += NW) {
                const int r = u / nseg, sg = u - r * nseg;
                const int x_lo = sg * segw, x_hi = min(Bl, x_lo + segw);
                int l0 = r, l1 = 0;
                if (D == 3) {
                    l0 = r / Bt[1];
                    l1 = r - l0 * Bt[1];
                }
                float2* arow = s_acc + (size_t)r * Bl * CPT + c;
#pragma unroll 1
                for (int a0 = 0; a0 < J; ++a0) {
#pragma unroll 1
                    for (int a1 = 0; a1 < (D > 2 ? J : 1); ++a1) {
                        const int b = D == 2 ? l0 + a0 : (l0 + a0) * E[1] + (l1 + a1);
                        const int h1 = s_off[b + 1];
                        for (int hh = s_off[b]; hh < h1; ++hh) {
                            const int h = s_list[hh];
                            const float* w = s_w + h * WP;
                            float wo = w[J - 1 - a0];
                            if (D > 2) wo *= w[J + J - 1 - a1];
                            const float2 yv = s_y[(size_t)h * YP + c];
                            const int sl = s_el[h];
#pragma unroll
                            for (int k = 0; k < NJX; ++k) {
                                const int jx = jg + k * JPL;
                                const int col = sl + jx;
                                if (jx < J && col >= x_lo && col < x_hi) {
                                    const float wt = wo * w[(D - 1) * J + jx];
                                    float2* t = arow + col * CPT;
                                    float2 v = *t;
                                    v.x = fmaf(wt, yv.x, v.x);
                                    v.y = fmaf(wt, yv.y, v.y);
                                    *t = v;
                                }
                            }
                            __syncwarp();   // the next point's cells may be another lane's
                        }
                    }
                }
            }
        }
        __syncthreads();   // every warp's rows are complete

        // write the tile coil-fastest: a tile row is Bt_last cells, contiguous in the grid
        const int K1 = D > 1 ? Kd[1] : 1, K2 = D > 2 ? Kd[2] : 1;
        if (D == 2 && nparts == 1 && ncc == CPT && a.C == CPT) {
            // all coils in this block: each tile row is one contiguous run of Bl * CPT complex
            const int per_row4 = Bl * CPT / 2;
            for (int row = warp; row < R; row += NW) {
                const float4* src = (const float4*)(s_acc + (size_t)row * Bl * CPT);
                float4* dst = (float4*)(a.grid + ((int64_t)(org[0] + row) * K1 + org[1]) * CPT);
                for (int i = lane; i < per_row4; i += 32) dst[i] = src[i];
            }
        } else {
            const int rowlen = Bl * ncc;
            const uint32_t mg = ncc > 1 ? (uint32_t)((((uint64_t)1 << 32) + ncc - 1) / ncc) : 0u;
            for (int f = tid; f < R * rowlen; f += nt) {
                const int row = f / rowlen, i = f - row * rowlen;
                const int cr = (int)div_magic((uint32_t)i, (uint32_t)ncc, mg);
                const int cc = i - cr * ncc;
                int r0 = row, r1 = 0;
                if (D == 3) { r1 = row % Bt[1]; r0 = row / Bt[1]; }
                const int64_t gcell = D == 2 ? (int64_t)(org[0] + r0) * K1 + org[1] + cr
                                             : ((int64_t)(org[0] + r0) * K1 + (org[1] + r1)) * K2 + org[2] + cr;
                const float2 v = s_acc[(size_t)(row * Bl + cr) * CPT + cc];
                float2* dst = a.grid + gcell * a.C + c0 + cc;
                if (nparts == 1) *dst = v;
                else if (v.x != 0.f || v.y != 0.f) atomicAdd(dst, v);
            }
        }
        if (itn >= nitems) break;
        it = itn;
        item = itemn;
        __syncthreads();   // the shared tile and lists are reused by the next item
    }
}

// Streaming multiprocessors of the current device (queried once per device).
static int device_sms() {
    static std::atomic<int> n[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    int v = n[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        n[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

template <int D, int J>
static cudaError_t spread_rows_cpt(const SpreadArgs& a, cudaStream_t s, int threads) {
    const int cpt = a.CC <= 4 ? 4 : (a.CC <= 8 ? 8 : 16);
    int NB = 1, tcells = 1;   // buckets, tile cells
    for (int d = 0; d < D - 1; ++d) NB *= a.B[d] + J - 1;
    for (int d = 0; d < D; ++d) tcells *= a.B[d];
    const int WP = D * J + ((D * J + 1) & 1);
    const size_t smem = (size_t)tcells * cpt * sizeof(float2) + (size_t)a.P * (cpt + 1) * sizeof(float2) +
                        (size_t)a.P * WP * sizeof(float) + 3 * (size_t)a.P * sizeof(int) +
                        (size_t)(2 * NB + 1) * sizeof(int);
    // persistent: two blocks per SM (the shared tile and lists take ~84 KB) walk the items
    dim3 grid((unsigned)std::min<int64_t>(a.max_items, 2 * (int64_t)device_sms()), (unsigned)((a.C + cpt - 1) / cpt));
    if (cpt == 4) {
        ensure_smem<k_spread_rows<D, J, 4>>(smem);
        (void)launch_pdl(k_spread_rows<D, J, 4>, grid, threads, smem, s, a);
    } else if (cpt == 8) {
        ensure_smem<k_spread_rows<D, J, 8>>(smem);
        (void)launch_pdl(k_spread_rows<D, J, 8>, grid, threads, smem, s, a);
    } else {
        ensure_smem<k_spread_rows<D, J, 16>>(smem);
        (void)launch_pdl(k_spread_rows<D, J, 16>, grid, threads, smem, s, a);
    }
    return cudaGetLastError();
}

template <int D>
static cudaError_t spread_rows_d(const SpreadArgs& a, cudaStream_t s, int threads) {
    switch (a.J) {
        case 4: return spread_rows_cpt<D, 4>(a, s, threads);
        case 5: return spread_rows_cpt<D, 5>(a, s, threads);
        case 6: return spread_rows_cpt<D, 6>(a, s, threads);
        case 7: return spread_rows_cpt<D, 7>(a, s, threads);
        default: return spread_rows_cpt<D, 8>(a, s, threads);
    }
}

// 2-D: row-owner tiles (lanes over taps and coils, measured 1.3x faster than
// cell owners on radial 640x640 / 16 coils, where the cell owners diverge);
// 3-D: cell owners (8 coils and 8-cell rows leave the row owners' lanes idle,
// while each cell sums about J^3 x density hits in registers: 1.8x faster on
// 3-D radial 256x256x192 / 8 coils).
cudaError_t launch_spread_cells(const SpreadArgs& a, cudaStream_t s) {
    if (a.max_items == 0) return cudaSuccess;
    if (a.D == 3) return launch_spread_cells_3d(a, s);
    // one staging thread per candidate slot, whole warps, at most 512
    int threads = std::min(512, ((a.P + 31) / 32) * 32);
    return spread_rows_d<2>(a, s, threads);
}

// Clears the cells (all coils) of the tiles that are split over several work items.
__global__ void k_permute_y(const int4* __restrict__ idx, const float2* __restrict__ y, float2* __restrict__ ys,
                            int64_t M, int C) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int64_t o = idx[i].w;
    int c = 0;
    for (; c + 4 <= C; c += 4) {   // four independent loads in flight
        float2 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = __ldg(y + (int64_t)(c + q) * M + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) ys[(int64_t)(c + q) * M + i] = v[q];
    }
    for (; c < C; ++c) ys[(int64_t)c * M + i] = __ldg(y + (int64_t)c * M + o);
}

cudaError_t launch_permute_y(const int4* idx, const float2* y, float2* ys, int64_t M, int C, cudaStream_t s) {
    if (M == 0) return cudaSuccess;
    (void)launch_pdl(k_permute_y, (unsigned)((M + 255) / 256), 256, 0, s, idx, y, ys, M, C);
    return cudaGetLastError();
}

// The sort lists these tiles; blocks walk the list, warps take tile rows (all axes but the
// last), and each row's cells times coils are one contiguous run of the grid.
__global__ void k_zero_heavy_tiles(SpreadArgs a) {
    pdl_wait();
    const int nh = a.heavy[0];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = blockIdx.x; i < nh; i += gridDim.x) {
        int r = a.heavy[1 + i], org[kMaxDim] = {0, 0, 0}, Bt[kMaxDim] = {1, 1, 1}, Kd[kMaxDim] = {1, 1, 1};
        for (int d = a.D - 1; d >= 0; --d) {
            const int bc = r % a.nb[d];
            r /= a.nb[d];
            Kd[d] = a.K[d];
            org[d] = bc * a.B[d];
            Bt[d] = min(a.B[d], Kd[d] - org[d]);
        }
        const int Dl = a.D - 1;
        const int rows = a.D == 1 ? 1 : (a.D == 2 ? Bt[0] : Bt[0] * Bt[1]);
        const int run = Bt[Dl] * a.C;
        for (int row = warp; row < rows; row += nw) {
            int64_t cell0;
            if (a.D == 1) cell0 = org[0];
            else if (a.D == 2) cell0 = (int64_t)(org[0] + row) * Kd[1] + org[1];
            else cell0 = ((int64_t)(org[0] + row / Bt[1]) * Kd[1] + (org[1] + row % Bt[1])) * Kd[2] + org[2];
            float2* dst = a.grid + cell0 * a.C;
            for (int f = lane; f < run; f += 32) dst[f] = make_float2(0.f, 0.f);
        }
    }
}

template <int D, int J>
static cudaError_t spread_j(const SpreadArgs& a, cudaStream_t s, size_t smem, dim3 grid) {
    ensure_smem<k_spread<D, J>>(smem);
    (void)launch_pdl(k_spread<D, J>, grid, 256, smem, s, a);
    return cudaGetLastError();
}

template <int D>
static cudaError_t spread_d(const SpreadArgs& a, cudaStream_t s, size_t smem, dim3 grid) {
    switch (a.J) {
        case 4: return spread_j<D, 4>(a, s, smem, grid);
        case 5: return spread_j<D, 5>(a, s, smem, grid);
        case 6: return spread_j<D, 6>(a, s, smem, grid);
        case 7: return spread_j<D, 7>(a, s, smem, grid);
        default: return spread_j<D, 8>(a, s, smem, grid);
    }
}

int spread_min_slots(int D, int J) {
    switch (D * 16 + J) {
#define NJ_NS(DD, JJ) case DD * 16 + JJ: return SpreadShape<DD, JJ>::NS_MIN;
        NJ_NS(1, 4) NJ_NS(1, 5) NJ_NS(1, 6) NJ_NS(1, 7) NJ_NS(1, 8)
        NJ_NS(2, 4) NJ_NS(2, 5) NJ_NS(2, 6) NJ_NS(2, 7) NJ_NS(2, 8)
        NJ_NS(3, 4) NJ_NS(3, 5) NJ_NS(3, 6) NJ_NS(3, 7) NJ_NS(3, 8)
#undef NJ_NS
        default: return 32;
    }
}

cudaError_t launch_spread(const SpreadArgs& a, int /*cpl*/, cudaStream_t s, size_t smem) {
    dim3 grid((unsigned)a.max_items, (unsigned)((a.C + a.CC - 1) / a.CC));
    if (a.max_items == 0) return cudaSuccess;
    if (a.D == 1) return spread_d<1>(a, s, smem, grid);
    if (a.D == 2) return spread_d<2>(a, s, smem, grid);
    return spread_d<3>(a, s, smem, grid);
}

cudaError_t launch_zero_heavy_tiles(const SpreadArgs& a, cudaStream_t s) {
    (void)launch_pdl(k_zero_heavy_tiles, std::min(a.nbins, 152 * 4), 256, 0, s, a);
    return cudaGetLastError();
}

}  // namespace nj

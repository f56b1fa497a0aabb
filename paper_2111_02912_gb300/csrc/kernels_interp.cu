// Interpolation (gather) and its adjoint (spread) on the oversampled grid.
//
// Gather, step (3) of the Appendix: y_i = sum over the J^D window taps of
// prod_d psi(u_d) G[k mod K].  A group of G lanes (a power of two) handles one
// sample; lane l owns coils l, l+G, ...  The J*D kernel weights of the sample
// are evaluated once by the group (one psi per lane) and reused for every
// channel of every coil: the unweighted grid and the D coordinate-weighted
// grids x . r^[d] of Eq. (e,Ax).  Epilogues:
//   FWD  y_c = g_c0
//   JVP  dy_c = -i sum_d domega^[d] g_cd  (and y_c when the plain channel is present)
//   VJP  grad^[d] = sum_c Re{conj(v_c) (-i) g_cd} = sum_c Im{conj(v_c) g_cd}   (Eq. (e,jac,Ax,v))
// so the D interpolated channels per coil never leave registers.
//
// Spread, the transpose of the gather (Sec. II-D): points are bin-sorted by
// window start; a sub-problem is up to P points of one bin.  A block spreads
// its points into a shared-memory tile covering the bin plus the J-1 halo
// (shared atomics; the lanes of a group touch different coils, so a group
// never conflicts with itself), then adds the non-zero tile cells to the
// global grid with float2 vector atomics.
#include "internal.h"

namespace nj {

__device__ __forceinline__ int wrap1(int k, int K) { return k >= K ? k - K : k; }

// Weights of one sample into w[d * kJMax + j] (shared, per group).
__device__ __forceinline__ void group_weights(float* w, const float* coef, float two_over_j, int D, int J, float4 fr,
                                              int lane_g, int G) {
    for (int q = lane_g; q < D * J; q += G) {
        const int d = q / J, j = q - d * J;
        const float u0 = d == 0 ? fr.x : (d == 1 ? fr.y : fr.z);
        w[d * kJMax + j] = kb_psi(coef, two_over_j, u0 - (float)j);
    }
}

template <int D, int ND, int CPL, int MODE>
__global__ void __launch_bounds__(256) k_gather(GatherArgs a) {
    __shared__ float coef[kKbTerms];
    extern __shared__ float wsm[];   // [groups][D][kJMax]
    const int tid = threadIdx.x;
    if (tid < kKbTerms) coef[tid] = a.kb.a[tid];
    __syncthreads();

    const int G = a.G;
    const int lane_g = tid & (G - 1);
    const int grp = tid >> a.lgG;
    const int gpb = blockDim.x >> a.lgG;
    const int64_t pt = (int64_t)blockIdx.x * gpb + grp;
    const bool valid = pt < a.pts.m;
    float* w = wsm + grp * (D * kJMax);
    int4 ix = make_int4(0, 0, 0, 0);
    float4 fr = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        ix = a.pts.idx[pt];
        fr = a.pts.frac[pt];
        group_weights(w, coef, a.kb.two_over_j, D, a.J, fr, lane_g, G);
    }
    __syncwarp();
    if (!valid) return;

    const int J = a.J, C = a.C;
    const int64_t ch = (int64_t)ND * C;
    float2 acc[ND][CPL];
#pragma unroll
    for (int q = 0; q < ND; ++q)
#pragma unroll
        for (int k = 0; k < CPL; ++k) acc[q][k] = make_float2(0.f, 0.f);

    // innermost dimension: columns and weights in registers
    const int Kl = D == 1 ? a.K[0] : (D == 2 ? a.K[1] : a.K[2]);
    const int kl0 = D == 1 ? ix.x : (D == 2 ? ix.y : ix.z);
    const float* wl = w + (D - 1) * kJMax;
    int col[kJMax];
    float wcol[kJMax];
#pragma unroll
    for (int j = 0; j < kJMax; ++j) {
        col[j] = wrap1(kl0 + (j < J ? j : 0), Kl);
        wcol[j] = j < J ? wl[j] : 0.f;
    }

    auto tap_row = [&](int64_t rowbase, float wrow) {
#pragma unroll
        for (int j = 0; j < kJMax; ++j) {
            if (j < J) {
                const float wt = wrow * wcol[j];
                const float2* gp = a.grid + (rowbase + col[j]) * ch + lane_g;
#pragma unroll
                for (int q = 0; q < ND; ++q)
#pragma unroll
                    for (int k = 0; k < CPL; ++k) {
                        if (lane_g + k * G < C) {
                            const float2 g = __ldg(gp + q * C + k * G);
                            acc[q][k].x = fmaf(wt, g.x, acc[q][k].x);
                            acc[q][k].y = fmaf(wt, g.y, acc[q][k].y);
                        }
                    }
            }
        }
    };

    if (D == 1) {
        tap_row(0, 1.f);
    } else if (D == 2) {
        const int K0 = a.K[0], K1 = a.K[1];
        for (int j0 = 0; j0 < J; ++j0) tap_row((int64_t)wrap1(ix.x + j0, K0) * K1, w[j0]);
    } else {
        const int K0 = a.K[0], K1 = a.K[1], K2 = a.K[2];
        for (int j0 = 0; j0 < J; ++j0) {
            const int64_t r0 = (int64_t)wrap1(ix.x + j0, K0) * K1;
            const float w0 = w[j0];
            for (int j1 = 0; j1 < J; ++j1)
                tap_row((r0 + wrap1(ix.y + j1, K1)) * K2, w0 * w[kJMax + j1]);
        }
    }

    const int64_t orig = ix.w;
    const int64_t M = a.M;
    if (MODE == GM_FWD) {
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int c = lane_g + k * G;
            if (c < C) a.y[(int64_t)c * M + orig] = acc[0][k];
        }
    } else if (MODE == GM_JVP) {
        const int hp = a.has_plain;
        float dom[D];
#pragma unroll
        for (int d = 0; d < D; ++d) dom[d] = a.domega[(int64_t)d * M + orig];
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int c = lane_g + k * G;
            if (c >= C) continue;
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float2 g = acc[(ND > D ? 1 : 0) + d][k];
                s.x = fmaf(dom[d], g.y, s.x);    // -i * g = (g.y, -g.x)
                s.y = fmaf(-dom[d], g.x, s.y);
            }
            a.dy[(int64_t)c * M + orig] = s;
            if (ND > D && hp) a.y[(int64_t)c * M + orig] = acc[0][k];
        }
    } else {   // GM_VJP
        float gsum[D];
#pragma unroll
        for (int d = 0; d < D; ++d) gsum[d] = 0.f;
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            const int c = lane_g + k * G;
            if (c >= C) continue;
            const float2 v = __ldg(a.v + (int64_t)c * M + orig);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float2 g = acc[d][k];
                gsum[d] += v.x * g.y - v.y * g.x;   // Im{conj(v) g}
            }
        }
        const unsigned mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) & ~(G - 1)));
#pragma unroll
        for (int d = 0; d < D; ++d)
            for (int off = G >> 1; off > 0; off >>= 1) gsum[d] += __shfl_xor_sync(mask, gsum[d], off, G);
        if (lane_g == 0) {
#pragma unroll
            for (int d = 0; d < D; ++d) a.grad[(int64_t)d * M + orig] = gsum[d];
        }
    }
}

template <int D, int ND, int MODE>
static cudaError_t gather_cpl(const GatherArgs& a, int cpl, cudaStream_t s) {
    const int threads = 256;
    const int gpb = threads / a.G;
    const unsigned blocks = (unsigned)((a.pts.m + gpb - 1) / gpb);
    const size_t smem = (size_t)gpb * D * kJMax * sizeof(float);
    if (blocks == 0) return cudaSuccess;
    switch (cpl) {
        case 1: k_gather<D, ND, 1, MODE><<<blocks, threads, smem, s>>>(a); break;
        case 2: k_gather<D, ND, 2, MODE><<<blocks, threads, smem, s>>>(a); break;
        default: k_gather<D, ND, 4, MODE><<<blocks, threads, smem, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <int D>
static cudaError_t gather_d(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s) {
    if (mode == GM_FWD) return gather_cpl<D, 1, GM_FWD>(a, cpl, s);
    if (mode == GM_VJP) return gather_cpl<D, D, GM_VJP>(a, cpl, s);
    if (a.nd == D) return gather_cpl<D, D, GM_JVP>(a, cpl, s);
    return gather_cpl<D, D + 1, GM_JVP>(a, cpl, s);
}

cudaError_t launch_gather(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s) {
    switch (a.D) {
        case 1: return gather_d<1>(mode, a, cpl, s);
        case 2: return gather_d<2>(mode, a, cpl, s);
        default: return gather_d<3>(mode, a, cpl, s);
    }
}

// ------------------------------------------------------------------ spread
template <int D, int CPL>
__global__ void __launch_bounds__(256) k_spread(SpreadArgs a) {
    extern __shared__ float4 smem4[];
    __shared__ float coef[kKbTerms];
    const int sp = blockIdx.x;
    if (sp >= a.nsubp[0]) return;             // block-uniform
    const int tid = threadIdx.x, nt = blockDim.x;
    const int G = a.G, lane_g = tid & (G - 1), grp = tid >> a.lgG, gpb = nt >> a.lgG;
    const int c0 = blockIdx.y * a.CC;
    const int ncc = min(a.CC, a.C - c0);
    const int CC = a.CC;
    const int T0 = a.T[0], T1 = D > 1 ? a.T[1] : 1, T2 = D > 2 ? a.T[2] : 1;
    const int tcells = T0 * T1 * T2;
    float2* tile = (float2*)smem4;                         // [tcells][CC]
    float* wsm = (float*)(tile + (size_t)tcells * CC);      // [gpb][D][kJMax]
    float* w = wsm + grp * (D * kJMax);

    if (tid < kKbTerms) coef[tid] = a.kb.a[tid];
    for (int i = tid; i < tcells * CC; i += nt) tile[i] = make_float2(0.f, 0.f);
    const int4 sub = a.subp[sp];
    int bz = sub.x, bc[3] = {0, 0, 0};
    for (int d = D - 1; d >= 0; --d) {
        const int nbd = d == 0 ? a.nb[0] : (d == 1 ? a.nb[1] : a.nb[2]);
        bc[d] = bz % nbd;
        bz /= nbd;
    }
    const int org0 = bc[0] * a.B[0], org1 = D > 1 ? bc[1] * a.B[1] : 0, org2 = D > 2 ? bc[2] * a.B[2] : 0;
    __syncthreads();

    const int J = a.J, C = a.C;
    for (int base = 0; base < sub.z; base += gpb) {
        const int q = base + grp;
        const bool valid = q < sub.z;
        int4 ix = make_int4(0, 0, 0, 0);
        float4 fr = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
            ix = a.pts.idx[sub.y + q];
            fr = a.pts.frac[sub.y + q];
            group_weights(w, coef, a.kb.two_over_j, D, J, fr, lane_g, G);
        }
        __syncwarp();
        if (valid) {
            float2 yv[CPL];
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const int cl = lane_g + k * G;
                yv[k] = cl < ncc ? __ldg(a.y + (int64_t)(c0 + cl) * a.M + ix.w) : make_float2(0.f, 0.f);
            }
            const int l0 = ix.x - org0, l1 = D > 1 ? ix.y - org1 : 0, l2 = D > 2 ? ix.z - org2 : 0;
            for (int j0 = 0; j0 < J; ++j0) {
                const float w0 = w[j0];
                for (int j1 = 0; j1 < (D > 1 ? J : 1); ++j1) {
                    const float w01 = D > 1 ? w0 * w[kJMax + j1] : w0;
                    for (int j2 = 0; j2 < (D > 2 ? J : 1); ++j2) {
                        const float wt = D > 2 ? w01 * w[2 * kJMax + j2] : w01;
                        const int cell = ((l0 + j0) * T1 + (D > 1 ? l1 + j1 : 0)) * T2 + (D > 2 ? l2 + j2 : 0);
                        float2* tp = tile + (size_t)cell * CC + lane_g;
#pragma unroll
                        for (int k = 0; k < CPL; ++k) {
                            if (lane_g + k * G < ncc) {
                                atomicAdd(&tp[k * G].x, wt * yv[k].x);
                                atomicAdd(&tp[k * G].y, wt * yv[k].y);
                            }
                        }
                    }
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();

    // flush: tile cell (l0, l1, l2) -> grid cell ((org + l) mod K)
    const int K0 = a.K[0], K1 = D > 1 ? a.K[1] : 1, K2 = D > 2 ? a.K[2] : 1;
    const int n = tcells * ncc;
    for (int f = tid; f < n; f += nt) {
        const int cl = f % ncc, cell = f / ncc;
        const float2 v = tile[(size_t)cell * CC + cl];
        if (v.x == 0.f && v.y == 0.f) continue;
        const int l2 = cell % T2, r = cell / T2;
        const int l1 = r % T1, l0 = r / T1;
        const int g0 = (org0 + l0) % K0, g1 = (org1 + l1) % K1, g2 = (org2 + l2) % K2;
        const int64_t gcell = ((int64_t)g0 * K1 + g1) * K2 + g2;
        atomicAdd((float2*)(a.grid + gcell * C + c0 + cl), v);
    }
}

cudaError_t launch_spread(const SpreadArgs& a, int cpl, cudaStream_t s, size_t smem) {
    dim3 grid((unsigned)a.max_subp, (unsigned)((a.C + a.CC - 1) / a.CC));
    if (a.max_subp == 0) return cudaSuccess;
#define NJ_SPREAD(DD, CP)                                                                               \
    do {                                                                                                \
        cudaFuncSetAttribute(k_spread<DD, CP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        k_spread<DD, CP><<<grid, 256, smem, s>>>(a);                                                    \
    } while (0)
    if (a.D == 1) { if (cpl == 1) NJ_SPREAD(1, 1); else if (cpl == 2) NJ_SPREAD(1, 2); else NJ_SPREAD(1, 4); }
    else if (a.D == 2) { if (cpl == 1) NJ_SPREAD(2, 1); else if (cpl == 2) NJ_SPREAD(2, 2); else NJ_SPREAD(2, 4); }
    else { if (cpl == 1) NJ_SPREAD(3, 1); else if (cpl == 2) NJ_SPREAD(3, 2); else NJ_SPREAD(3, 4); }
#undef NJ_SPREAD
    return cudaGetLastError();
}

}  // namespace nj

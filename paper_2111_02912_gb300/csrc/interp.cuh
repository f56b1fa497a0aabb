// Interpolation (gather) kernel template, instantiated per dimension in
// kernels_gather_d{1,2,3}.cu.
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
#pragma once
#include "internal.h"

namespace nj {

// Weights of one sample into w[d * J + j] (shared, per group), copied from the
// sort's per-point weights (at d * wd + j): lane q of the group loads q, q + G, ...
template <int D, int J>
__device__ __forceinline__ void group_weights(float* w, const float* pw, int wd, int lane_g, int G) {
    for (int q = lane_g; q < D * J; q += G) {
        const int d = q / J;
        w[q] = __ldg(pw + d * wd + (q - d * J));
    }
}

// 32-byte read-only load (four complex coil values), one instruction.
__device__ __forceinline__ void ldg_v8(const float2* p, float4& lo, float4& hi) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(lo.x), "=f"(lo.y), "=f"(lo.z), "=f"(lo.w), "=f"(hi.x), "=f"(hi.y), "=f"(hi.z), "=f"(hi.w)
        : "l"(p));
}

// W coils per lane slot: lane l owns coils W (l + k G) .. W (l + k G) + W - 1, read as one load of
// 8 W bytes (W = 2: a 16-byte load, C even; W = 4: a 32-byte load, C a multiple of 4; W = 1: one
// coil).
template <int D, int J, int ND, int CPL, int MODE, int W>
__device__ __forceinline__ void gather_body(const GatherArgs& a) {
    extern __shared__ float wsm[];   // [groups][D * J]
    const int tid = threadIdx.x;

    const int G = a.G;
    const int lane_g = tid & (G - 1);
    const int grp = tid >> a.lgG;
    const int gpb = blockDim.x >> a.lgG;
    const int64_t pt = (int64_t)blockIdx.x * gpb + grp;
    const bool valid = pt < a.pts.m;
    float* w = wsm + grp * (D * J);
    int4 ix = make_int4(0, 0, 0, 0);
    if (valid) {
        ix = a.pts.idx[pt];
        group_weights<D, J>(w, a.pts.w + pt * a.pts.ws, a.pts.wd, lane_g, G);
    }
    __syncwarp();
    if (!valid) return;

    const int C = a.C;
    const int chs = ND * C;   // channel stride of one grid cell
    bool ok[CPL];
    int lofs[CPL];   // coil offset of slot k; slots past the last coil read coil 0 (never stored)
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        ok[k] = W * (lane_g + k * G) < C;
        lofs[k] = ok[k] ? W * (lane_g + k * G) : 0;
    }
    float2 acc[ND][CPL][W];
#pragma unroll
    for (int q = 0; q < ND; ++q)
#pragma unroll
        for (int k = 0; k < CPL; ++k)
#pragma unroll
            for (int i = 0; i < W; ++i) acc[q][k][i] = make_float2(0.f, 0.f);

    // innermost axis: column offsets and weights in registers
    const int Kl = a.K[D - 1];
    const int kl0 = D == 1 ? ix.x : (D == 2 ? ix.y : ix.z);
    int coff[J];
    float wl[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        int k = kl0 + j;
        if (k >= Kl) k -= Kl;
        coff[j] = k * chs;
        wl[j] = w[(D - 1) * J + j];
    }
    const float2* g0 = a.grid;

    auto row = [&](const float2* rp, float wr) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const float wt = wr * wl[j];
            const float2* gp = rp + coff[j];
#pragma unroll
            for (int q = 0; q < ND; ++q)
#pragma unroll
                for (int k = 0; k < CPL; ++k) {   // unconditional loads: all taps in flight together
                        if constexpr (W == 4) {
                            float4 g, h;
                            ldg_v8(gp + q * C + lofs[k], g, h);
                            acc[q][k][0].x = fmaf(wt, g.x, acc[q][k][0].x);
                            acc[q][k][0].y = fmaf(wt, g.y, acc[q][k][0].y);
                            acc[q][k][1].x = fmaf(wt, g.z, acc[q][k][1].x);
                            acc[q][k][1].y = fmaf(wt, g.w, acc[q][k][1].y);
                            acc[q][k][2].x = fmaf(wt, h.x, acc[q][k][2].x);
                            acc[q][k][2].y = fmaf(wt, h.y, acc[q][k][2].y);
                            acc[q][k][W - 1].x = fmaf(wt, h.z, acc[q][k][W - 1].x);
                            acc[q][k][W - 1].y = fmaf(wt, h.w, acc[q][k][W - 1].y);
                        } else if constexpr (W == 2) {
                            const float4 g = __ldg((const float4*)(gp + q * C + lofs[k]));
                            acc[q][k][0].x = fmaf(wt, g.x, acc[q][k][0].x);
                            acc[q][k][0].y = fmaf(wt, g.y, acc[q][k][0].y);
                            acc[q][k][W - 1].x = fmaf(wt, g.z, acc[q][k][W - 1].x);
                            acc[q][k][W - 1].y = fmaf(wt, g.w, acc[q][k][W - 1].y);
                        } else {
                            const float2 g = __ldg(gp + q * C + lofs[k]);
                            acc[q][k][0].x = fmaf(wt, g.x, acc[q][k][0].x);
                            acc[q][k][0].y = fmaf(wt, g.y, acc[q][k][0].y);
                        }
                    }
        }
    };

    if (D == 1) {
        row(g0, 1.f);
    } else if (D == 2) {
        const int K0 = a.K[0];
        const int64_t rstride = (int64_t)a.K[1] * chs;
#pragma unroll
        for (int j0 = 0; j0 < J; ++j0) {
            int k0 = ix.x + j0;
            if (k0 >= K0) k0 -= K0;
            row(g0 + k0 * rstride, w[j0]);
        }
    } else {
        const int K0 = a.K[0], K1 = a.K[1];
        const int64_t pstride = (int64_t)a.K[1] * a.K[2] * chs, rstride = (int64_t)a.K[2] * chs;
#pragma unroll 1
        for (int j0 = 0; j0 < J; ++j0) {
            int k0 = ix.x + j0;
            if (k0 >= K0) k0 -= K0;
            const float2* pp = g0 + k0 * pstride;
            const float w0 = w[j0];
#pragma unroll
            for (int j1 = 0; j1 < J; ++j1) {
                int k1 = ix.y + j1;
                if (k1 >= K1) k1 -= K1;
                row(pp + k1 * rstride, w0 * w[J + j1]);
            }
        }
    }

    const int64_t orig = ix.w;
    const int64_t M = a.M;
    if (MODE == GM_FWD) {
#pragma unroll
        for (int k = 0; k < CPL; ++k)
#pragma unroll
            for (int i = 0; i < W; ++i)
                if (ok[k]) a.y[(int64_t)(W * (lane_g + k * G) + i) * M + orig] = acc[0][k][i];
    } else if (MODE == GM_JVP) {
        float dom[D];
#pragma unroll
        for (int d = 0; d < D; ++d) dom[d] = a.domega[(int64_t)d * M + orig];
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            if (!ok[k]) continue;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int64_t c = W * (lane_g + k * G) + i;
                float2 s = make_float2(0.f, 0.f);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const float2 g = acc[(ND > D ? 1 : 0) + d][k][i];
                    s.x = fmaf(dom[d], g.y, s.x);    // -i * g = (g.y, -g.x)
                    s.y = fmaf(-dom[d], g.x, s.y);
                }
                a.dy[c * M + orig] = s;
                if (ND > D) a.y[c * M + orig] = acc[0][k][i];
            }
        }
    } else {   // GM_VJP
        float gsum[D];
#pragma unroll
        for (int d = 0; d < D; ++d) gsum[d] = 0.f;
#pragma unroll
        for (int k = 0; k < CPL; ++k) {
            if (!ok[k]) continue;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int64_t cv = W * (lane_g + k * G) + i;
                const float2 v = __ldg(a.v + cv * M + orig);
                if (a.v_sorted) {   // for the adjoint spread of the same v
                    if (a.v_sorted_cpt) {
                        const int64_t cg = cv / a.v_sorted_cpt;
                        a.v_sorted[(cg * M + pt) * a.v_sorted_cpt + (cv - cg * a.v_sorted_cpt)] = v;
                    } else {
                        a.v_sorted[cv * M + pt] = v;
                    }
                }
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const float2 g = acc[d][k][i];
                    gsum[d] += v.x * g.y - v.y * g.x;   // Im{conj(v) g}
                }
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

template <int D, int J, int ND, int CPL, int MODE, int W>
__global__ void __launch_bounds__(256) k_gather(GatherArgs a) {
    pdl_wait();
    gather_body<D, J, ND, CPL, MODE, W>(a);
}

// The gathers wait on their tap loads.  The 2-D VJP with coil pairs is held to 64 registers (no
// spill for any J) so that four blocks share an SM: measured 40.3 -> 39.1 us on the 640^2, 16-coil
// case.  The forward at 40 or 48 registers spills and gains nothing; the other VJP kinds spill at 64.
template <int D, int J, int ND, int CPL, int MODE, int W>
__global__ void __launch_bounds__(256, 4) k_gather_occ4(GatherArgs a) {
    pdl_wait();
    gather_body<D, J, ND, CPL, MODE, W>(a);
}

template <int D, int J, int ND, int MODE>
static cudaError_t gather_cpl(const GatherArgs& a, int cpl, cudaStream_t s) {
    const int threads = 256;
    const int gpb = threads / a.G;
    const unsigned blocks = (unsigned)((a.pts.m + gpb - 1) / gpb);
    const size_t smem = (size_t)gpb * D * J * sizeof(float);
    if (blocks == 0) return cudaSuccess;
    if (cpl == kGatherQuads) {   // coil quads
        (void)launch_pdl(k_gather<D, J, ND, 1, MODE, 4>, blocks, threads, smem, s, a);
    } else if (cpl == 0) {   // coil pairs
        if constexpr (D == 2 && MODE == GM_VJP) (void)launch_pdl(k_gather_occ4<D, J, ND, 1, MODE, 2>, blocks, threads, smem, s, a);
        else (void)launch_pdl(k_gather<D, J, ND, 1, MODE, 2>, blocks, threads, smem, s, a);
    }
    else if (cpl == 1) (void)launch_pdl(k_gather<D, J, ND, 1, MODE, 1>, blocks, threads, smem, s, a);
    else (void)launch_pdl(k_gather<D, J, ND, 4, MODE, 1>, blocks, threads, smem, s, a);   // C up to 4 G = 128
    return cudaGetLastError();
}

template <int D, int J>
static cudaError_t gather_mode(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s) {
    if (mode == GM_FWD) return gather_cpl<D, J, 1, GM_FWD>(a, cpl, s);
    if (mode == GM_VJP) return gather_cpl<D, J, D, GM_VJP>(a, cpl, s);
    if (a.nd == D) return gather_cpl<D, J, D, GM_JVP>(a, cpl, s);
    return gather_cpl<D, J, D + 1, GM_JVP>(a, cpl, s);
}

template <int D>
cudaError_t gather_dim(GatherMode mode, const GatherArgs& a, int cpl, cudaStream_t s) {
    switch (a.J) {
        case 4: return gather_mode<D, 4>(mode, a, cpl, s);
        case 5: return gather_mode<D, 5>(mode, a, cpl, s);
        case 6: return gather_mode<D, 6>(mode, a, cpl, s);
        case 7: return gather_mode<D, 7>(mode, a, cpl, s);
        default: return gather_mode<D, 8>(mode, a, cpl, s);
    }
}

}  // namespace nj

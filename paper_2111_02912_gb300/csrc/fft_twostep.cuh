// Register-resident line FFT for L = L1 * L2 (both at most 32): the four-step
// split of one transform, with a single shared-memory transpose.
//
// Step (2) of the Appendix's NUFFT along one axis of a channel-interleaved
// grid, like k_line_fft (same LinePass arguments and pass kinds), but every
// butterfly runs in registers.  With n = L2 n1 + n2 and k = k1 + L1 k2:
//
//   X[k1 + L1 k2] = sum_n2 W_L2^(n2 k2) [ W_L^(n2 k1) sum_n1 x[L2 n1 + n2] W_L1^(n1 k1) ]
//
// Phase 1: thread (line, n2) holds the L1 elements x[L2 n1 + n2], takes the
// L1-point DFT, multiplies by W_L^(n2 k1) (table, FP64-computed) and writes
// row k1 of the tile line in shared memory.  Phase 2: thread (line, k1) reads
// the L2 values of row k1, takes the L2-point DFT and writes X[k1 + L1 k2].
// Consecutive threads work on consecutive lines (the lines of a tile are
// adjacent in memory), so global loads and stores are coalesced along the
// channel axis.  Shared layout: row k1 of a line at k1 (L2 + 1) (position
// p = n1 L2 + n2 at p + p / L2), lines LP apart with LP = 16 / H mod 16 for
// H lines per half-warp (odd for H = 16): a half-warp's 64-bit accesses then
// fall on distinct banks in both phases.
//
// Pass kinds: FWD_FIRST stages its input from the image (scaling s_n of the
// Appendix, coil map of Sec. II-G, coordinate weight r^[d] of Eq. (e,Ax), zero
// padding) with loads coalesced along the image row; FWD_MID reads only the
// n_in nonzero positions of its input lines; INV_MID keeps the n_out cropped
// positions; INV_LAST crops, stages the line in shared memory, then applies
// the scaling and conj(s_c) and sums the tile's coils with loads and stores
// coalesced along the image row (with pair_add, the two coil chunks of a row
// each add their sum into the image that INV_MID cleared: x = 0 + a + b has the
// same bits in either order, so the result does not depend on which comes first).
#pragma once
#include "fft_dft.cuh"
#include "internal.h"

namespace nj {

// Row factors of an image line: scaling of the non-last dims and its
// coordinates r^[d] = n_d - N_d/2 for d < D-1.
__device__ __forceinline__ void image_row_factors(const ImageSide& im, int64_t b, float& scale, float& r0, float& r1) {
    scale = 1.f;
    r0 = r1 = 0.f;
    if (im.D == 2) {
        const int n0 = (int)b;
        scale = im.deap[0][n0];
        r0 = (float)(n0 - im.N[0] / 2);
    } else if (im.D == 3) {
        const int n0 = (int)(b / im.N[1]), n1 = (int)(b - (int64_t)n0 * im.N[1]);
        scale = im.deap[0][n0] * im.deap[1][n1];
        r0 = (float)(n0 - im.N[0] / 2);
        r1 = (float)(n1 - im.N[1] / 2);
    }
}

// Registers: with L2 = 32 (256-thread blocks of 8 lines) 80 per thread, so that three blocks share
// an SM (24 warps; the passes are issue- and latency-bound): the register DFTs fit with at most a
// few bytes of spill (measured on the 640-point passes: FWD_MID 37.6 -> 31.5 us, INV_MID 26.4 ->
// 22.4 us against 128 registers at two blocks per SM).  Other sizes keep 128: on the 400-point
// passes (320-thread blocks) 80 registers cost FWD_FIRST 24.5 -> 28.3 us and FWD_MID 17.3 -> 19.0
// us.  The coil-summing INV_LAST takes 8 coils per block as well when its two chunks add into the
// image (9..16 coils: 640 blocks in 1.4 waves against 320 one-per-SM blocks of 16 coils in 2.1);
// with more coils it runs 512-thread blocks of 16 at one block per SM.
// Half-length pruning fixed at compile time (HALF: n_in = L / 2 on the forward side, n_out = L / 2 on
// the inverse side, i.e. sigma = 2).  Then the kept positions p < L/4 or p >= 3L/4 are whole phase-1
// registers n1 (p = L2 n1 + n2, L1 % 4 == 0) on the forward side and whole phase-2 outputs k2
// (k = k1 + L1 k2, L2 % 4 == 0) on the inverse side: the zero inputs are never loaded and the
// dropped outputs never computed.
template <int L1, int L2, PassKind KIND>
__host__ __device__ constexpr bool fft2_half_applies() {
    return (KIND == PASS_FWD_FIRST || KIND == PASS_FWD_MID) ? L1 % 4 == 0 : L2 % 4 == 0;
}

template <int L1, int L2, PassKind KIND, bool HALF>
__global__ void __maxnreg__(L2 != 32 ? 128 : 80) k_line_fft2(LinePass a) {
    pdl_wait();
    if (KIND == PASS_INV_MID && a.clear) {   // the image the next pass's two coil chunks add into
        const int64_t nthr = (int64_t)gridDim.x * gridDim.y * blockDim.x;
        for (int64_t i = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x; i < a.nclear;
             i += nthr)
            a.clear[i] = make_float2(0.f, 0.f);
    }
    constexpr int DIR = (KIND == PASS_FWD_FIRST || KIND == PASS_FWD_MID) ? -1 : 1;
    constexpr int L = L1 * L2;
    constexpr bool FH = HALF && DIR < 0 && fft2_half_applies<L1, L2, KIND>();   // forward: n1 kept iff
    constexpr bool IH = HALF && DIR > 0 && fft2_half_applies<L1, L2, KIND>();   // inverse: k2 kept iff
    constexpr int Q = L / 4;
    constexpr int RP = L2 + 1;   // row pitch inside a line
    const int LP = a.TLP;        // line pitch (>= L1 RP, >= n_out)
    extern __shared__ float2 buf[];   // [TL][LP]
    const int lgTS = a.lgTS, lgTL = a.lgTL;
    const int TS = 1 << lgTS, TL = 1 << lgTL, TB = TL >> lgTS;
    const int tid = threadIdx.x;
    const int line = tid & (TL - 1), col = tid >> lgTL;
    const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
    uint32_t tile_b, tile_s;
    line_tile(a.ntiles_s, tile_b, tile_s);
    const int64_t b0 = (int64_t)tile_b * TB, s0 = (int64_t)tile_s * TS;
    const int64_t S = a.S;
    const int Si = (int)a.S;   // fits in 32 bits (checked when the plan is made)
    const int64_t b = b0 + (line >> lgTS), sl = s0 + (line & (TS - 1));
    const bool valid = b < a.B && sl < S;
    float2* row = buf + line * LP;

    const int Dm1 = a.im.D - 1;
    const int nlast = a.im.N[Dm1];
    const float* deap_last = a.im.deap[Dm1];

    // ---------------------------------------------------------------- input
    if (KIND == PASS_FWD_FIRST) {
        // Lines are (image row, channel); channel = dblk * C + coil, dblk 0 the
        // plain image when has_plain, then the r^[d]-weighted ones.
        const int h = a.n_in >> 1;
        for (int ln = warp; ln < TL; ln += nwarps) {
            const int64_t bb = b0 + (ln >> lgTS), ss = s0 + (ln & (TS - 1));
            const bool ok = bb < a.B && ss < S;
            const float2* xrow = a.im.x;
            const float2* mrow = nullptr;
            float rs = 0.f, wr = 0.f;
            int kind = -1;
            if (ok) {
                const int dblk = (int)ss / a.im.C, c = (int)ss - dblk * a.im.C;
                kind = a.im.has_plain ? dblk - 1 : dblk;
                float r0, r1;
                image_row_factors(a.im, bb, rs, r0, r1);
                if (kind >= 0 && kind < Dm1) wr = kind == 0 ? r0 : r1;
                if (a.im.smaps) {
                    xrow = a.im.x + bb * nlast;
                    mrow = a.im.smaps + (int64_t)c * a.im.nimg + bb * nlast;
                } else {
                    xrow = a.im.x + (int64_t)c * a.im.nimg + bb * nlast;
                }
            }
            float2* dst = buf + ln * LP;
            if (!FH)   // zero padding (with FH the padded registers are never read)
                for (int p = h + lane; p < L - h; p += 32) dst[p + p / L2] = make_float2(0.f, 0.f);
            // image element e sits at position (e - n_in/2) mod L.  A row of up to 384
            // elements is loaded in one batch of 12 per lane; indices are clamped so the
            // loads are unconditional and independent (all in flight before the first use).
            const int n = a.n_in;
            if (!ok) {
                for (int e = lane; e < n; e += 32) {
                    const int p = e < h ? e - h + L : e - h;
                    dst[p + p / L2] = make_float2(0.f, 0.f);
                }
                continue;
            }
            const float wgt = kind == Dm1 ? 0.f : (kind >= 0 ? wr : 1.f);   // row factor; last-axis weight below
            for (int e0 = 0; e0 < n; e0 += 32 * 12) {
                float2 xv[12], mv[12];
                float dv[12];
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    const int e = min(e0 + q * 32 + lane, n - 1);
                    xv[q] = __ldg(xrow + e);
                    dv[q] = __ldg(deap_last + e);
                }
                if (mrow) {
#pragma unroll
                    for (int q = 0; q < 12; ++q) mv[q] = __ldg(mrow + min(e0 + q * 32 + lane, n - 1));
#pragma unroll
                    for (int q = 0; q < 12; ++q) xv[q] = cmul(xv[q], mv[q]);
                }
#pragma unroll
                for (int q = 0; q < 12; ++q) {
                    const int e = e0 + q * 32 + lane;
                    if (e < n) {
                        float sc = rs * dv[q];
                        sc *= kind == Dm1 ? (float)(e - nlast / 2) : wgt;
                        const int p = e < h ? e - h + L : e - h;
                        dst[p + p / L2] = cscale(xv[q], sc);
                    }
                }
            }
        }
        __syncthreads();
    }

    // -------------------------------------------------------------- phase 1
    if (col < L2) {
        const int n2 = col;
        float2 v[L1];
        if (KIND == PASS_FWD_FIRST) {
            sfor<0, L1>([&](auto n1_) {
                constexpr int n1 = decltype(n1_)::value;
                if constexpr (FH && n1 >= L1 / 4 && n1 < 3 * L1 / 4) v[n1] = make_float2(0.f, 0.f);
                else v[n1] = row[n1 * RP + n2];
            });
        } else if constexpr (FH && KIND == PASS_FWD_MID) {
            // kept rows: element e = p + L/4 for p < L/4, p - 3L/4 for p >= 3L/4 (n_in = L/2)
            const float2* base = a.in + (valid ? b * a.n_in * S + sl : 0) + (int64_t)n2 * Si;
            sfor<0, L1>([&](auto n1_) {
                constexpr int n1 = decltype(n1_)::value;
                if constexpr (n1 >= L1 / 4 && n1 < 3 * L1 / 4) {
                    v[n1] = make_float2(0.f, 0.f);
                } else {
                    constexpr int e0 = n1 < L1 / 4 ? n1 * L2 + Q : n1 * L2 - 3 * Q;   // e - n2
                    const float2 t = __ldg(base + (int64_t)e0 * Si);   // in bounds for every line
                    v[n1] = valid ? t : make_float2(0.f, 0.f);
                }
            });
        } else {
            const float2* in_line = a.in + (valid ? b * a.n_in * S + sl : 0);
            if (DIR < 0) {   // pruned input: position p holds element (p + n_in/2) mod L when kept
                const int h = a.n_in >> 1;
                sfor<0, L1>([&](auto n1_) {
                    constexpr int n1 = decltype(n1_)::value;
                    const int p = n1 * L2 + n2;
                    const bool keep = valid && (p < h || p >= L - h);
                    const int e = p < h ? p + h : p - (L - h);
                    v[n1] = keep ? __ldg(in_line + (int64_t)e * Si) : make_float2(0.f, 0.f);
                });
            } else {
                sfor<0, L1>([&](auto n1_) {
                    constexpr int n1 = decltype(n1_)::value;
                    const int p = n1 * L2 + n2;
                    const float2 t = __ldg(in_line + (int64_t)(valid ? p : 0) * Si);   // unconditional load
                    v[n1] = valid ? t : make_float2(0.f, 0.f);
                });
            }
        }
        dft<L1, DIR>(v);
        if (n2 > 0) {
            const float2* tw = a.ax.tw2 + n2 * L1;   // row n2: exp(-2 pi i n2 k1 / L) at k1
            sfor<1, L1>([&](auto k1_) {
                constexpr int k1 = decltype(k1_)::value;
                float2 w = __ldg(tw + k1);
                if (DIR > 0) w.y = -w.y;
                v[k1] = cmul(v[k1], w);
            });
        }
        sfor<0, L1>([&](auto k1_) {
            constexpr int k1 = decltype(k1_)::value;
            row[k1 * RP + n2] = v[k1];
        });
    }
    __syncthreads();

    // -------------------------------------------------------------- phase 2
    const int k1 = col;
    float2 w[L2];
    if (k1 < L1) {
        sfor<0, L2>([&](auto n2_) {
            constexpr int n2 = decltype(n2_)::value;
            w[n2] = row[k1 * RP + n2];
        });
        dft<L2, DIR>(w);   // w[k2] = X[k1 + L1 k2]
    }

    if (KIND == PASS_FWD_FIRST || KIND == PASS_FWD_MID) {
        if (k1 < L1 && valid) {
            float2* out_line = a.out + b * (int64_t)L * S + sl + (int64_t)k1 * Si;
            sfor<0, L2>([&](auto k2_) {
                constexpr int k2 = decltype(k2_)::value;
                out_line[(int64_t)(L1 * k2) * Si] = w[k2];
            });
        }
    } else if (KIND == PASS_INV_MID) {
        if (k1 < L1 && valid) {
            const int h = a.n_out >> 1;
            float2* out_line = a.out + b * a.n_out * S + sl;
            sfor<0, L2>([&](auto k2_) {
                constexpr int k2 = decltype(k2_)::value;
                if constexpr (IH) {   // kept: k2 < L2/4 (e = k + L/4) or k2 >= 3 L2/4 (e = k - 3L/4)
                    if constexpr (k2 < L2 / 4 || k2 >= 3 * L2 / 4) {
                        constexpr int c = k2 < L2 / 4 ? L1 * k2 + Q : L1 * k2 - 3 * Q;
                        out_line[(int64_t)(k1 + c) * Si] = w[k2];
                    }
                } else {
                    const int k = k1 + L1 * k2;
                    const int e = k < h ? k + h : k - (L - h);
                    if (k < h || k >= L - h) out_line[(int64_t)e * Si] = w[k2];
                }
            });
        }
    } else {   // PASS_INV_LAST: crop into shared memory, then the image side
        const int h = a.n_out >> 1;
        __syncthreads();   // every thread has read its phase-2 row
        if (k1 < L1) {
            sfor<0, L2>([&](auto k2_) {
                constexpr int k2 = decltype(k2_)::value;
                if constexpr (IH) {
                    if constexpr (k2 < L2 / 4 || k2 >= 3 * L2 / 4) {
                        constexpr int c = k2 < L2 / 4 ? L1 * k2 + Q : L1 * k2 - 3 * Q;
                        row[k1 + c] = w[k2];
                    }
                } else {
                    const int k = k1 + L1 * k2;
                    const int e = k < h ? k + h : k - (L - h);
                    if (k < h || k >= L - h) row[e] = w[k2];
                }
            });
        }
        __syncthreads();
        const int n = a.n_out, nt = blockDim.x;
        if (a.coil_sum) {
            // x_b[e] = s_b s_e sum_c conj(s_c[b, e]) X_c[e] over the tile's coils, in coil order
            float2* xo = a.im.xout + tile_s * a.im.xout_stride;
            for (int lb = 0; lb < TB; ++lb) {
                const int64_t bb = b0 + lb;
                if (bb >= a.B) break;
                float rs, r0, r1;
                image_row_factors(a.im, bb, rs, r0, r1);
                const float2* maps = a.im.smaps + s0 * a.im.nimg + bb * nlast;
                const int ncoil = (int)(S - s0 < TS ? S - s0 : TS);
                for (int e = tid; e < n; e += nt) {
                    float2 sum = make_float2(0.f, 0.f);
                    for (int l0 = 0; l0 < ncoil; l0 += 8) {   // map loads batched eight deep
                        float2 m[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            m[q] = l0 + q < ncoil ? __ldg(maps + (int64_t)(l0 + q) * a.im.nimg + e) : make_float2(0.f, 0.f);
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            if (l0 + q < ncoil) sum = cadd(sum, cmulc(buf[(lb * TS + l0 + q) * LP + e], m[q]));
                    }
                    const float2 xv = cscale(sum, rs * __ldg(deap_last + e));
                    if (a.pair_add) atomicAdd(xo + bb * nlast + e, xv);   // 2 adds onto 0: order-free
                    else xo[bb * nlast + e] = xv;
                }
            }
        } else {
            for (int ln = 0; ln < TL; ++ln) {
                const int64_t bb = b0 + (ln >> lgTS), c = s0 + (ln & (TS - 1));
                if (bb >= a.B || c >= S) continue;
                float rs, r0, r1;
                image_row_factors(a.im, bb, rs, r0, r1);
                for (int e = tid; e < n; e += nt)
                    a.im.xout[c * a.im.nimg + bb * nlast + e] = cscale(buf[ln * LP + e], rs * deap_last[e]);
            }
        }
    }
}

}  // namespace nj

namespace nj {

// Launches k_line_fft2<L1, L2, KIND> when (L1, L2) has a compiled kernel.
template <PassKind KIND>
cudaError_t launch_fft2_kind(int L1, int L2, const LinePass& a, dim3 grid, int threads, size_t smem, cudaStream_t s) {
#define NJ_FFT2_CASE(A, B)                                                                   \
    if (L1 == A && L2 == B) {                                                                 \
        if constexpr (fft2_half_applies<A, B, KIND>()) {                                      \
            if (2 * ((KIND == PASS_FWD_FIRST || KIND == PASS_FWD_MID) ? a.n_in : a.n_out) == A * B) { \
                ensure_smem<k_line_fft2<A, B, KIND, true>>(smem);                             \
                (void)launch_pdl(k_line_fft2<A, B, KIND, true>, grid, threads, smem, s, a);   \
                return cudaGetLastError();                                                    \
            }                                                                                 \
        }                                                                                     \
        ensure_smem<k_line_fft2<A, B, KIND, false>>(smem);                                    \
        (void)launch_pdl(k_line_fft2<A, B, KIND, false>, grid, threads, smem, s, a);          \
        return cudaGetLastError();                                                            \
    }
    NJ_FFT2_SIZES(NJ_FFT2_CASE)
#undef NJ_FFT2_CASE
    return cudaErrorInvalidValue;
}

}  // namespace nj

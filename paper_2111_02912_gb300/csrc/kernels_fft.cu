// Shared-memory Stockham FFT passes over one axis of a channel-interleaved grid.
//
// Step (2) of the Appendix's NUFFT: a K-point FFT of the zero-padded, scaled
// signal, applied one axis at a time.  A pass transforms every line of a
// [B][L][S] array along its middle axis (S = stride of the faster axes,
// channels innermost).  A block holds a tile of TB x TS lines in shared memory
// as [L][TLP] (element-major, line-minor, TLP = TL + 1), so that consecutive
// threads of a butterfly work on consecutive lines (conflict-free) and the
// global loads and stores of a strided axis are coalesced along S.
//
// Stockham autosort, mixed radix (16, 8, 4, 2, 3, 5): stage with radix R and
// running length Ns reads a[j + r L/R], twiddles by W^(r (j mod Ns) L/(Ns R)),
// takes an R-point DFT and writes b[(j div Ns) Ns R + (j mod Ns) + r Ns].
// Stages alternate between two shared buffers (ping-pong), one butterfly per
// thread at a time, so register use is independent of the tile size.  On the
// grid side the first stage reads its R inputs straight from global memory and
// the last stage writes its R outputs straight back (the last stage's output
// positions are j + r L/R, the same pattern as the first stage's inputs), so a
// pass costs (stages - 1) shared-memory round trips.
//
// Forward passes read N of the L input positions (zero padding: element e of
// the image axis sits at position (e - N/2) mod L) and write all L; inverse
// passes read all L and keep the N cropped positions.  The first forward pass
// builds its input from the image (scaling s_n of the Appendix, coil map s_c
// of Sec. II-G and coordinate weight r^[d] of Eq. (e,Ax)); the last inverse
// pass applies the scaling, conj(s_c) and the coil sum.
#include <algorithm>

#include "fft_dft.cuh"
#include "internal.h"

namespace nj {

// Global side of a fused first / last stage, for the one tile line a thread
// works on (the block size is a multiple of the tile's line count, so butterfly
// u = tid + k * blockDim always falls on line tid mod TL).  Position p of the
// transform holds element e(p) of the line (zero padding / crop: e = (p + n/2)
// mod L when p is one of the n kept positions); elements are S apart.
struct LineIO {
    const float2* in_line;   // element 0 of the thread's input line
    float2* out_line;        // element 0 of the thread's output line
    int64_t S;
    int L, n_in, n_out;
    bool valid, pruned_in, cropped_out;

    __device__ __forceinline__ float2 load(int p) const {
        int e = p;
        if (pruned_in) {
            const int h = n_in >> 1;
            e = p < h ? p + h : (p >= L - h ? p - (L - h) : -1);
        }
        if (e < 0 || !valid) return make_float2(0.f, 0.f);
        return in_line[e * S];
    }
    __device__ __forceinline__ void store(int p, float2 v) const {
        int e = p;
        if (cropped_out) {
            const int h = n_out >> 1;
            e = p < h ? p + h : (p >= L - h ? p - (L - h) : -1);
        }
        if (e < 0 || !valid) return;
        out_line[e * S] = v;
    }
};

enum { ST_SMEM = 0, ST_GLOBAL = 1 };

// One Stockham stage.  SRC / DST: shared tile or, for the first / last stage of
// a pass, the global array itself (no shared round trip).
template <int R, int DIR, int SRC, int DST>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                          const float2* __restrict__ tw, int L, int TLP, int lgTL, const FftStage st,
                                          const LineIO& io) {
    const int LR = L / R;
    const int TL = 1 << lgTL;
    const int total = LR << lgTL;
    const int sstride = LR * TLP, dstride = st.Ns * TLP;
    for (int u = threadIdx.x; u < total; u += blockDim.x) {
        const int line = u & (TL - 1);
        const int j = u >> lgTL;
        const int jq = (int)div_magic((uint32_t)j, (uint32_t)st.Ns, st.magic);
        const int kk = j - jq * st.Ns;
        float2 v[R];
        if (SRC == ST_SMEM) {
            const float2* sp = src + j * TLP + line;
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = sp[r * sstride];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[r] = io.load(j + r * LR);
        }
        if (st.Ns > 1) {
            const int tstep = kk * st.tw_step;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = tw[r * tstep];
                if (DIR > 0) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        Dft<R, DIR>::run(v);
        const int d0 = jq * st.Ns * R + kk;
        if (DST == ST_SMEM) {
            float2* dp = dst + d0 * TLP + line;
#pragma unroll
            for (int r = 0; r < R; ++r) dp[r * dstride] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) io.store(d0 + r * st.Ns, v[r]);
        }
    }
    __syncthreads();
}

template <int R, int DIR>
__device__ __forceinline__ void fft_stage_any(bool gin, bool gout, const float2* src, float2* dst, const float2* tw,
                                              int L, int TLP, int lgTL, const FftStage st, const LineIO& io) {
    if (gin && gout) fft_stage<R, DIR, ST_GLOBAL, ST_GLOBAL>(src, dst, tw, L, TLP, lgTL, st, io);
    else if (gin) fft_stage<R, DIR, ST_GLOBAL, ST_SMEM>(src, dst, tw, L, TLP, lgTL, st, io);
    else if (gout) fft_stage<R, DIR, ST_SMEM, ST_GLOBAL>(src, dst, tw, L, TLP, lgTL, st, io);
    else fft_stage<R, DIR, ST_SMEM, ST_SMEM>(src, dst, tw, L, TLP, lgTL, st, io);
}

// Runs all stages.  gin: the first stage reads the global input; gout: the last
// stage writes the global output.  Returns the shared buffer holding the result
// when !gout.
template <int DIR>
__device__ float2* fft_all_stages(float2* buf0, float2* buf1, const float2* tw, const FftStage* sst, int nstages,
                                  int L, int TLP, int lgTL, bool gin, bool gout, const LineIO& io) {
    float2* src = buf0;
    float2* dst = buf1;
    for (int s = 0; s < nstages; ++s) {
        const FftStage st = sst[s];
        const bool fi = gin && s == 0, fo = gout && s == nstages - 1;
        switch (st.R) {
            case 16: fft_stage_any<16, DIR>(fi, fo, src, dst, tw, L, TLP, lgTL, st, io); break;
            case 8: fft_stage_any<8, DIR>(fi, fo, src, dst, tw, L, TLP, lgTL, st, io); break;
            case 4: fft_stage_any<4, DIR>(fi, fo, src, dst, tw, L, TLP, lgTL, st, io); break;
            case 2: fft_stage_any<2, DIR>(fi, fo, src, dst, tw, L, TLP, lgTL, st, io); break;
            case 3: fft_stage_any<3, DIR>(fi, fo, src, dst, tw, L, TLP, lgTL, st, io); break;
            default: fft_stage_any<5, DIR>(fi, fo, src, dst, tw, L, TLP, lgTL, st, io); break;
        }
        float2* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// Row factors of an image line: scaling of the non-last dims and its
// coordinates r^[d] = n_d - N_d/2 for d < D-1.
__device__ __forceinline__ void image_row(int D, int N0, int N1, const float* deap0, const float* deap1, int64_t b,
                                          float& scale, float& r0, float& r1) {
    scale = 1.f;
    r0 = r1 = 0.f;
    if (D == 2) {
        const int n0 = (int)b;
        scale = deap0[n0];
        r0 = (float)(n0 - N0 / 2);
    } else if (D == 3) {
        const int n0 = (int)(b / N1), n1 = (int)(b - (int64_t)n0 * N1);
        scale = deap0[n0] * deap1[n1];
        r0 = (float)(n0 - N0 / 2);
        r1 = (float)(n1 - N1 / 2);
    }
}

template <PassKind KIND>
__global__ void __launch_bounds__(256) k_line_fft(LinePass a) {
    pdl_wait();
    constexpr int DIR = (KIND == PASS_FWD_FIRST || KIND == PASS_FWD_MID) ? -1 : 1;
    extern __shared__ float2 smem[];
    const int L = a.ax.L;
    const int TS = a.TS, TB = a.TB, TL = TB * TS, TLP = a.TLP;
    float2* tw = smem;
    float2* buf = smem + L;
    float2* buf1 = buf + (size_t)L * TLP;
    float2* acc = buf1 + (size_t)L * TLP;                // coil-sum accumulator [TB][n_out]
    float* row_scale = (float*)(acc + (a.coil_sum ? TB * a.n_out : 0));
    float* row_r = row_scale + TB;                        // [TB][2]
    __shared__ FftStage sst[kMaxStages];
    const int tid = threadIdx.x, nt = blockDim.x;
    uint32_t tile_b, tile_s;
    line_tile(a.ntiles_s, tile_b, tile_s);
    const int64_t by = tile_s;
    const int64_t b0 = (int64_t)tile_b * TB;

    for (int i = tid; i < L; i += nt) tw[i] = a.ax.tw[i];
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < kMaxStages; ++i) sst[i] = a.ax.st[i];
    }
    if (KIND == PASS_FWD_FIRST || KIND == PASS_INV_LAST) {
        for (int lb = tid; lb < TB; lb += nt) {
            float sc = 0.f, r0 = 0.f, r1 = 0.f;
            if (b0 + lb < a.B) image_row(a.im.D, a.im.N[0], a.im.N[1], a.im.deap[0], a.im.deap[1], b0 + lb, sc, r0, r1);
            row_scale[lb] = sc;
            row_r[2 * lb] = r0;
            row_r[2 * lb + 1] = r1;
        }
    }
    if (KIND == PASS_INV_LAST && a.coil_sum)
        for (int i = tid; i < TB * a.n_out; i += nt) acc[i] = make_float2(0.f, 0.f);
    __syncthreads();

    const int Dm1 = a.im.D - 1;
    const int nlast = Dm1 == 2 ? a.im.N[2] : (Dm1 == 1 ? a.im.N[1] : a.im.N[0]);
    const float* deap_last = Dm1 == 2 ? a.im.deap[2] : (Dm1 == 1 ? a.im.deap[1] : a.im.deap[0]);
    const int nstages = a.ax.nstages;
    const int half_in = a.n_in / 2;
    const int nchunks = a.nchunks;

    for (int chunk = 0; chunk < nchunks; ++chunk) {
        const int64_t s0 = (by * nchunks + chunk) * TS;
        LineIO io;
        {
            const int line = tid & (TL - 1);
            const int64_t b = b0 + (line >> a.lgTS), sl = s0 + (line & (TS - 1));
            io.valid = b < a.B && sl < a.S;
            io.in_line = a.in + (io.valid ? b * a.n_in * a.S + sl : 0);
            io.out_line = a.out + (io.valid ? b * a.n_out * a.S + sl : 0);
            io.S = a.S;
            io.L = L;
            io.n_in = a.n_in;
            io.n_out = a.n_out;
            io.pruned_in = DIR < 0;
            io.cropped_out = DIR > 0;
        }
        // ---------------- prologue: the first pass builds the tile from the image
        const int nfill = KIND == PASS_FWD_FIRST ? L * TL : 0;
        for (int f = tid; f < nfill; f += nt) {
            // positions fastest: image rows are contiguous
            const int line = (int)div_magic((uint32_t)f, (uint32_t)L, a.magic_L);
            const int p = f - line * L;
            const int lb = line >> a.lgTS, ls = line & (TS - 1);
            const int e = p < half_in ? p + half_in : (p >= L - half_in ? p - (L - half_in) : -1);
            float2 val = make_float2(0.f, 0.f);
            const int64_t b = b0 + lb, s = s0 + ls;
            if (e >= 0 && b < a.B && s < a.S) {
                const int dblk = (int)(s / a.im.C), c = (int)(s - (int64_t)dblk * a.im.C);
                const int kind = a.im.has_plain ? dblk - 1 : dblk;   // -1: plain image
                const int64_t pix = b * nlast + e;
                float2 xv = a.im.smaps ? cmul(a.im.x[pix], a.im.smaps[(int64_t)c * a.im.nimg + pix])
                                       : a.im.x[(int64_t)c * a.im.nimg + pix];
                float sc = row_scale[lb] * deap_last[e];
                if (kind == Dm1) sc *= (float)(e - nlast / 2);
                else if (kind >= 0) sc *= row_r[2 * lb + kind];
                val = cscale(xv, sc);
            }
            buf[p * TLP + lb * TS + ls] = val;
        }
        __syncthreads();

        const bool gin = KIND != PASS_FWD_FIRST, gout = KIND != PASS_INV_LAST;
        const float2* res = fft_all_stages<DIR>(buf, buf1, tw, sst, nstages, L, TLP, a.lgTL, gin, gout, io);

        // ---------------- epilogue
        const int half_out = a.n_out / 2;
        if (KIND == PASS_INV_LAST) {   // crop, scale, coil maps
            if (a.coil_sum) {
                const int nst = a.n_out * TB;
                for (int f = tid; f < nst; f += nt) {
                    const int lb = (int)div_magic((uint32_t)f, (uint32_t)a.n_out, a.magic_n);
                    const int e = f - lb * a.n_out;
                    const int p = e < half_out ? e + L - half_out : e - half_out;
                    const int64_t b = b0 + lb;
                    if (b >= a.B) continue;
                    const int64_t pix = b * nlast + e;
                    float2 sum = acc[lb * a.n_out + e];
                    for (int ls = 0; ls < TS; ++ls) {
                        const int64_t c = s0 + ls;
                        if (c >= a.S) break;
                        sum = cadd(sum, cmulc(res[p * TLP + lb * TS + ls], a.im.smaps[c * a.im.nimg + pix]));
                    }
                    acc[lb * a.n_out + e] = sum;
                }
            } else {
                const int nst = a.n_out * TL;
                for (int f = tid; f < nst; f += nt) {
                    const int line = (int)div_magic((uint32_t)f, (uint32_t)a.n_out, a.magic_n);
                    const int e = f - line * a.n_out;
                    const int lb = line >> a.lgTS, ls = line & (TS - 1);
                    const int p = e < half_out ? e + L - half_out : e - half_out;
                    const int64_t b = b0 + lb, c = s0 + ls;
                    if (b < a.B && c < a.S)
                        a.im.xout[c * a.im.nimg + b * nlast + e] =
                            cscale(res[p * TLP + lb * TS + ls], row_scale[lb] * deap_last[e]);
                }
            }
        }
        __syncthreads();
    }
    if (KIND == PASS_INV_LAST && a.coil_sum) {
        float2* xo = a.im.xout + by * a.im.xout_stride;
        for (int f = tid; f < TB * a.n_out; f += nt) {
            const int lb = f / a.n_out, e = f - lb * a.n_out;
            const int64_t b = b0 + lb;
            if (b < a.B) xo[b * nlast + e] = cscale(acc[f], row_scale[lb] * deap_last[e]);
        }
    }
}

__global__ void k_sum_chunks(const float2* __restrict__ part, int nparts, int64_t n, float2* __restrict__ x) {
    pdl_wait();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float2 acc = part[i];
        for (int k = 1; k < nparts; ++k) acc = cadd(acc, part[(int64_t)k * n + i]);
        x[i] = acc;
    }
}

cudaError_t launch_sum_chunks(const float2* part, int nparts, int64_t n, float2* x, cudaStream_t s) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    (void)launch_pdl(k_sum_chunks, blocks, 256, 0, s, part, nparts, n, x);
    return cudaGetLastError();
}

cudaError_t launch_line_pass(PassKind kind, const LinePass& a, dim3 grid, int threads, size_t smem,
                             cudaStream_t s) {
    switch (kind) {
        case PASS_FWD_FIRST:
            ensure_smem<k_line_fft<PASS_FWD_FIRST>>(smem);
            (void)launch_pdl(k_line_fft<PASS_FWD_FIRST>, grid, threads, smem, s, a);
            break;
        case PASS_FWD_MID:
            ensure_smem<k_line_fft<PASS_FWD_MID>>(smem);
            (void)launch_pdl(k_line_fft<PASS_FWD_MID>, grid, threads, smem, s, a);
            break;
        case PASS_INV_MID:
            ensure_smem<k_line_fft<PASS_INV_MID>>(smem);
            (void)launch_pdl(k_line_fft<PASS_INV_MID>, grid, threads, smem, s, a);
            break;
        case PASS_INV_LAST:
            ensure_smem<k_line_fft<PASS_INV_LAST>>(smem);
            (void)launch_pdl(k_line_fft<PASS_INV_LAST>, grid, threads, smem, s, a);
            break;
    }
    return cudaGetLastError();
}

}  // namespace nj

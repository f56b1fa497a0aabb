/*
 * nufftjac.h -- C ABI of the GB300 (sm_103a) NUFFT / NUFFT-Jacobian library.
 *
 * Operations (Wang & Fessler, "Efficient approximation of Jacobian matrices
 * involving a non-uniform fast Fourier transform"):
 *   forward  y = A(omega) x, A_ij = exp(-i omega_i . r_j)       Sec. II-B, Eq. (e,ndft)
 *            approximated by a NUFFT: scaling s_n, zero-padded K-point FFT,
 *            J-tap interpolation                                  Appendix (NUFFT entries)
 *   adjoint  x = A' y                                             Sec. II-D
 *   sensitivity maps E = (I kron A) S, S_c = diag(s_c)            Sec. II-G
 *   d(Ax)/d omega^[d] = -i diag{A (x . r^[d])}                    Sec. II-C, Eq. (e,Ax)
 *   VJP  dL/d omega = Re{(-i A(x . r^[d]))' . v}                  Sec. III, Eq. (e,jac,Ax,v)
 *   d(A'y)/d omega^[d] = i diag{r^[d]} A' diag{y}                 Sec. II-D, Eq. (e,A'y)
 *
 * Conventions shared by every entry point
 *   - Every array argument is DEVICE memory owned by the caller, contiguous,
 *     and must stay valid until the work queued on `stream` has finished.
 *     Complex arrays are interleaved float pairs (re, im), 8-byte aligned.
 *   - Images are C-ordered (N_1, ..., N_D), last axis fastest.  Voxel centre
 *     r_j^[d] = n_d - N_d/2 (integer voxel units; every N_d must be even).
 *   - omega is float32 [D][M] (row d holds omega^[d]) in radians per voxel;
 *     any value is accepted (A is 2*pi-periodic in omega because r is integer).
 *   - k-space arrays (y, v, dy) are [C][M] in the caller's point order.
 *   - smaps == NULL: x is [C][N] (one image per channel) and the adjoint
 *     returns [C][N].  smaps != NULL: smaps is [C][N], x is [N], and the
 *     adjoint returns sum_c conj(s_c) A' y_c, shape [N].
 *   - Gradients follow the real-valued convention: for a real loss L and
 *     k-space output y, v = dL/dRe(y) + i dL/dIm(y); grad_x is returned in the
 *     same convention and grad_omega = dL/d omega exactly (no factor 2).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All calls
 *     are asynchronous and stream-ordered; none synchronises the host except
 *     nufft_plan / nufft_set_points when the point capacity must grow.  A plan
 *     owns a second stream (highest priority) for its point sort: a call forks
 *     it from `stream` and joins it back before returning, so every call is
 *     self-contained and may be recorded into a CUDA graph.
 *   - Return NUFFT_OK (0) or a negative status.  Nothing is thrown across the
 *     ABI.  An asynchronous kernel fault is reported by a later call.
 *     nufft_last_error() gives a readable message for the calling thread.
 *   - A plan is not thread-safe; distinct plans are independent.
 */
#ifndef NUFFTJAC_H
#define NUFFTJAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nufft_plan_s* nufft_plan_t;

typedef struct {
    float re, im;
} nufft_cfloat;

enum {
    NUFFT_OK = 0,
    NUFFT_ERR_INVALID_ARG = -1, /* null pointer, bad size, C out of range */
    NUFFT_ERR_UNSUPPORTED = -2, /* D not in {1,2,3}, odd N_d, J out of [4,8], grid too large */
    NUFFT_ERR_OOM = -3,         /* device allocation failed */
    NUFFT_ERR_CUDA = -4,        /* a CUDA runtime call or kernel launch failed */
    NUFFT_ERR_TIMEOUT = -5      /* reserved, never returned: no kernel of this library waits on
                                   another kernel, a flag or another GPU */
};

/* Largest channel count of one call (coils, or images of a map-free call). */
#define NUFFT_MAX_COILS 128

/* Plan options.  Fields left 0 take the defaults noted. */
typedef struct {
    int dim;          /* D, 1..3 */
    int64_t n[3];     /* image size N_d (even), d < dim */
    double sigma;     /* oversampling factor, > 1 (0 -> 2.0); K_d = smallest even
                         2,3,5-smooth integer >= sigma N_d, K_d <= 4096 */
    int J;            /* interpolation width, 4..8 (0 -> 6) */
    double beta;      /* Kaiser-Bessel shape (<= 0 -> Beatty et al.:
                         pi sqrt((J/sigma)^2 (sigma-1/2)^2 - 0.8)) */
    int max_coils;    /* largest C any call on this plan will pass, 1..NUFFT_MAX_COILS (0 -> 1) */
    int bin_size[3];  /* spread tile edge per dim (0 -> automatic: 256, 16x16, 8x8x8) */
    int deterministic; /* 1: every output is bitwise reproducible from call to call (the strip
                          adjoint adds its terms in an order fixed by the sort; needs the strip
                          spread); 0: fastest order (the adjoint then agrees to rounding between
                          calls) */
    int spread_variant; /* adjoint spread kernel: NUFFT_SPREAD_AUTO (0), _STRIPS, _TILES, _GENERAL */
    int strip_part;   /* strip spread: hits one warp adds before a unit is split into parts
                         (a power of two, 8..4096; 0 -> 64) */
    int kernel_mode;  /* how the interpolation weights psi(u) are evaluated (once per omega, by the
                         bin sort): NUFFT_KERNEL_DIRECT (0), the Kaiser-Bessel function itself as
                         its I0 power series in FP32; NUFFT_KERNEL_TABLE, psi sampled at
                         table_density points per grid unit and read by linear interpolation (the
                         table interpolator of Sec. II-B / Sec. IV-A, for comparison; less accurate) */
    int table_density; /* NUFFT_KERNEL_TABLE: samples per grid unit, 16..65536 (0 -> 512) */
    int gather_variant; /* lanes of the forward gather: NUFFT_GATHER_AUTO (0), _PAIRS, _QUADS */
} nufft_opts;

enum { NUFFT_KERNEL_DIRECT = 0, NUFFT_KERNEL_TABLE = 1 };

/* Forward gather (interpolation, Appendix step 3) lane layouts (nufft_opts.gather_variant), all
 * computing the same sums: a lane owns two adjacent coils (PAIRS: one 16-byte load per tap) or
 * four (QUADS: one 32-byte load per tap, twice the points per warp; for C a multiple of 4 from 8
 * on, else pairs).  AUTO takes quads for the 2-D forward with C a multiple of 4 from 16 on, where
 * they measured faster, and pairs elsewhere.  The JVP and VJP gathers always use pairs. */
enum { NUFFT_GATHER_AUTO = 0, NUFFT_GATHER_PAIRS = 1, NUFFT_GATHER_QUADS = 2 };

/* Adjoint spread kernels (nufft_opts.spread_variant), all computing the transpose of the
 * interpolation (Sec. II-D); AUTO takes STRIPS where it applies, else TILES, else GENERAL.
 *   STRIPS  2-D and 3-D: a warp owns NSL grid rows x 16 cells of the last axis in registers
 *           (NSL = 64 / coils per warp: 4 for 16 coils, from max_coils; in 3-D a row is a (k0, k1)
 *           pair of an R0 x R1 block, R0 R1 = NSL); needs a grid of at least 16 + J - 1 cells
 *           along the last axis and R + J - 1 along each other axis (R = NSL in 2-D, R0 and R1
 *           in 3-D).
 *   TILES   2-D / 3-D: a block owns one bin tile in shared memory (row or cell owners).
 *   GENERAL any D: shared-memory atomics on bin tiles.
 * Asking for a variant that does not apply to the plan returns NUFFT_ERR_UNSUPPORTED. */
enum { NUFFT_SPREAD_AUTO = 0, NUFFT_SPREAD_STRIPS = 1, NUFFT_SPREAD_TILES = 2, NUFFT_SPREAD_GENERAL = 3 };

/* Fill *o with defaults for a D-dimensional image of size n[0..D-1]. */
void nufft_default_opts(nufft_opts* o, int dim, const int64_t* n);

/* Create a plan: tables, workspace for max_coils channels, and the bin sort of
 * the m points in omega (Appendix: offsets k_m and coefficients u_j(omega_m)
 * depend on omega only).  m may be 0.  *out receives the plan. */
int nufft_plan(nufft_plan_t* out, const nufft_opts* o, int64_t m, const float* omega, void* stream);

/* New sample locations (every trajectory update).  The Appendix's interpolation
 * offsets k_m and coefficients u_j(omega_m) depend on omega only, so this is where
 * they are fixed: the bin sort computes each point's window start and its D*J
 * kernel weights once, and every later gather and spread of these points reads
 * them.  m may differ from the plan's current m; growing past the capacity
 * reallocates (synchronising).  The call copies omega into the plan on `stream`
 * (the caller's buffer is free once that copy has run); the bin sort itself runs
 * in the next call that needs the points, on the plan's own stream, beside that
 * call's FFT passes. */
int nufft_set_points(nufft_plan_t p, int64_t m, const float* omega, void* stream);

/* Run the bin sort of the points last given to nufft_set_points now, on `stream`
 * (forked to the plan's own stream and joined back before the call returns), instead
 * of in the next call that needs them: for a caller that has omega on the device
 * before the other inputs of the next call (e.g. while they are still being copied
 * from the host) and orders that call after this stream.  Does nothing when the
 * points are sorted already.  Same Appendix passage as nufft_set_points. */
int nufft_sort_points(nufft_plan_t p, void* stream);

/* y[C][M] = E x: forward NUFFT of each coil image (Sec. II-B, II-G). */
int nufft_forward(nufft_plan_t p, int C, const nufft_cfloat* x, const nufft_cfloat* smaps,
                  nufft_cfloat* y, void* stream);

/* x = E' y: adjoint NUFFT (Sec. II-D), summed over coils when smaps != NULL. */
int nufft_adjoint(nufft_plan_t p, int C, const nufft_cfloat* y, const nufft_cfloat* smaps,
                  nufft_cfloat* x, void* stream);

/* Forward-mode product (Eq. (e,Ax)): dy_c = sum_d domega^[d] . (-i) A(s_c . x . r^[d]).
 * domega is float [D][M].  If y_or_null != NULL, y = E x comes out of the same
 * interpolation launch (1+D channels per coil share the kernel weights). */
int nufft_jvp_omega(nufft_plan_t p, int C, const nufft_cfloat* x, const nufft_cfloat* smaps,
                    const float* domega, nufft_cfloat* dy, nufft_cfloat* y_or_null, void* stream);

/* Reverse-mode products for incoming gradient v [C][M] (Eq. (e,jac,Ax,v)):
 *   grad_omega[d][i] = sum_c Re{ conj(v_ci) (-i) [A(s_c . x . r^[d])]_i }   (float [D][M])
 *   grad_x = E' v                                                          (as nufft_adjoint)
 * Either output may be NULL to skip it.  The adjoint operator's omega-VJP
 * (Eq. (e,A'y)) is this call with (x, v) <- (incoming image gradient, y).
 * With both outputs on a 2-D strip plan (and at most 16 coils when smaps != NULL),
 * grad_x is computed on a second stream of the plan beside grad_omega, forked from
 * and joined back into `stream` inside the call; the call stays stream-ordered. */
int nufft_vjp_omega_x(nufft_plan_t p, int C, const nufft_cfloat* x, const nufft_cfloat* smaps,
                      const nufft_cfloat* v, float* grad_omega, nufft_cfloat* grad_x, void* stream);

/* Device bytes a plan with these options, m points and calls of up to C coils would allocate
 * (C <= 0: o->max_coils).  Returns 0 for options nufft_plan would reject. */
size_t nufft_workspace_bytes(const nufft_opts* o, int64_t m, int C);

/* Plan facts for callers and benchmarks. */
typedef struct {
    int dim;
    int64_t n[3], k[3];      /* image and oversampled grid sizes */
    int J;
    double sigma, beta;
    int64_t m;               /* current number of points */
    int bin_size[3], nbins;  /* spread tiles */
    int max_coils;
    size_t workspace_bytes;  /* device bytes held by the plan */
} nufft_plan_info;
int nufft_get_info(nufft_plan_t p, nufft_plan_info* info);

/* Free the plan and its device memory (synchronises the plan's last stream). */
void nufft_destroy(nufft_plan_t p);

const char* nufft_status_string(int status);
const char* nufft_last_error(void);

/* ---- allocation-free forward (the paper has no counterpart) --------------
 * For callers that cannot allocate device memory: code whose device memory is
 * owned by another allocator (a framework's caching allocator, a service with
 * a fixed memory budget) or that must not allocate while it runs.  Same result
 * as nufft_plan + nufft_forward on the same arguments, but without a plan: all
 * scratch (scaling and twiddle tables, the bin sort, the FFT workspace) lives
 * in one file-scope device array of NUFFT_NOALLOC_SCRATCH_BYTES that every GPU
 * loading this library holds until the process exits.  The call allocates
 * nothing (no cudaMalloc / cudaFree, no allocating library routine).
 *   - o, m, omega, C, x, smaps, y as for nufft_plan / nufft_forward.
 *   - A problem whose scratch would exceed the array returns
 *     NUFFT_ERR_UNSUPPORTED with the byte counts in nufft_last_error().
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and keeps it for the life of the process; make
 *     that first call before any stream capture, and do not use the call on a
 *     device after cudaDeviceReset (the kept address would be stale).
 *   - Every call uses the same array and leaves its contents behind; calls
 *     whose work overlaps on the GPU (other streams, other host threads)
 *     race on it and must be serialised by the caller.  The call itself
 *     zeroes what must start at zero (the sort counters).
 *   - The scaling and twiddle tables are computed on the device into the
 *     array; nothing is copied from host memory and the host does not wait
 *     for the stream (the call is asynchronous like the others). */
#define NUFFT_NOALLOC_SCRATCH_BYTES (32u << 20)
int nufft_forward_noalloc(const nufft_opts* o, int64_t m, const float* omega, int C, const nufft_cfloat* x,
                          const nufft_cfloat* smaps, nufft_cfloat* y, void* stream);

/* ---- measurement hooks -------------------------------------------------
 * Kernel launches made by this library in this process (all plans). */
int64_t nufft_launch_count(void);

/* When enabled, every kernel the plan launches is bracketed by CUDA events on
 * the launching stream.  nufft_profile_read synchronises those events and
 * returns, per kernel kind, the launch count and summed milliseconds, then
 * clears them.  names[i] points to static strings. */
int nufft_profile_enable(nufft_plan_t p, int enable);
int nufft_profile_read(nufft_plan_t p, int max_kinds, const char** names, int* launches,
                       double* total_ms, int* n_kinds);

#ifdef __cplusplus
}
#endif
#endif /* NUFFTJAC_H */

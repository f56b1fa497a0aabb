// C ABI of libnufftjac: plans, tables, workspace and the orchestration of the
// kernels for forward / adjoint / JVP / VJP (declarations in nufftjac.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/nufftjac.h"
#include "internal.h"

using namespace nj;

namespace {

thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};

int fail(int status, const std::string& msg) {
    g_last_error = msg;
    return status;
}

#define NJ_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(NUFFT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    } while (0)

enum ProfKind {
    PK_ZERO, PK_BIN_COUNT, PK_BIN_SCAN, PK_TILE_SCAN, PK_BIN_SCATTER, PK_BIN_ITEMS, PK_FFT_FWD_FIRST, PK_FFT_FWD_MID,
    PK_FFT_INV_MID, PK_FFT_INV_LAST, PK_GATHER_FWD, PK_GATHER_JVP, PK_GATHER_VJP, PK_ZERO_HEAVY, PK_SPREAD, PK_SUM_CHUNKS, PK_PERMUTE_Y,
    PK_STRIP_PLAN_A, PK_STRIP_PLAN_B, PK_STRIP_FILL, PK_DET_PLACE, PK_DET_RANK, PK_STRIP_ORDER, PK_COUNT
};
const char* kProfNames[PK_COUNT] = {"zero", "bin_count", "bin_scan", "tile_scan", "bin_scatter", "bin_items", "fft_fwd_first",
                                    "fft_fwd_mid", "fft_inv_mid", "fft_inv_last", "gather_fwd", "gather_jvp",
                                    "gather_vjp", "zero_heavy", "spread", "sum_chunks", "permute_y",
                                    "strip_plan_a", "strip_plan_b", "strip_fill", "det_place", "det_rank",
                                    "strip_order"};

int64_t grid_size(int64_t n, double sigma) {
    int64_t k = (int64_t)std::ceil(sigma * (double)n - 1e-9);
    for (;; ++k) {
        if (k % 2) continue;
        int64_t q = k;
        for (int p : {2, 3, 5})
            while (q % p == 0) q /= p;
        if (q == 1) return k;
    }
}

int pow2_ceil(int64_t v) {
    int p = 1;
    while (p < v) p *= 2;
    return p;
}
int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}
uint32_t magic_of(uint32_t d) { return d <= 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + d - 1) / d); }

}  // namespace

struct nufft_plan_s {
    int D = 0;
    int64_t N[3] = {1, 1, 1}, K[3] = {1, 1, 1};
    int J = 6;
    double sigma = 2.0, beta = 0.0;
    int maxC = 1;
    int64_t M = 0, M_cap = 0;
    int64_t Nimg = 1, Ktot = 1;
    KbPoly kb{};
    float* d_deap[3] = {nullptr, nullptr, nullptr};
    float2* d_tw[3] = {nullptr, nullptr, nullptr};
    FftAxis axis[3]{};
    // bins
    int B[3] = {1, 1, 1}, nb[3] = {1, 1, 1}, nbins = 1, cpb = 1, P = 1024, CCmax = 1;
    bool cell_spread = false;   // spread by the row-owner tile kernel (else the general kernel)
    // strip spread (2-D and 3-D): strip units of NSL rows x kStripW columns of the last axis
    bool strip = false;
    bool deterministic = false;    // stable bin order and hit lists ordered by sorted point
    int kernel_mode = NUFFT_KERNEL_DIRECT, tab_L = 0, tab_n = 0;   // table mode: L samples per unit
    int gather_variant = NUFFT_GATHER_AUTO;
    float* d_kbtab = nullptr;      // [tab_n + 2] psi(l / tab_L), zero from tab_n on
    int2* d_hits_tmp = nullptr;    // [hit_cap] the fill's list before ordering (deterministic only)
    int NSL = 2, SR0 = 2, SR1 = 1, nunits = 0, strip_P = 64, strip_slots = 0, ncg_max = 1;
    float2* d_ys = nullptr;        // [ncg_max][M_cap][64 / NSL] coil values in sorted point order
    float2* d_partial = nullptr;   // [strip_slots][ncg_max][kStripW][32] coil pairs (float4)
    int* d_counters = nullptr;     // [strip_slots][ncg_max], zero between calls
    int* d_hcount = nullptr;       // [nunits] hits per strip unit
    int* d_hcur = nullptr;         // [nunits] fill cursors
    int* d_plan_sums = nullptr;    // per-block totals of the strip plan
    int* d_hoff = nullptr;         // [nunits + 1]
    int2* d_hits = nullptr;        // [hit_cap] strip hit lists
    int64_t hit_cap = 0;
    int4* d_splits = nullptr;      // [strip_slots]
    int* d_kcount = nullptr;
    bool kcount_clear = false;   // the bin histogram is known to be zero (the bin scan clears it)
    int* d_offsets = nullptr;
    int* d_item_off = nullptr;
    int* d_tile_parts = nullptr;
    int* d_heavy = nullptr;
    int* d_tile_nbr = nullptr;
    int* d_nitems = nullptr;
    int4* d_items = nullptr;
    int* d_local = nullptr;   // [M_cap] rank within the bin, then (after the scatter) sorted position
    int* d_keyid = nullptr;
    int4* d_pidx = nullptr;
    float4* d_pfrac = nullptr;
    float* d_om = nullptr;   // [D][M_cap] copy of omega taken by set_points
    // The sort runs at the first call after set_points that needs the points, on a stream of the
    // plan, beside that call's FFT passes (which do not need them); the call joins it before its
    // first kernel that reads the sorted points.  Fork and join stay inside one call.
    cudaStream_t aux = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr, join2_ev = nullptr;
    // A VJP with both outputs on 2-D strips runs its adjoint (grad_x) on aux2 beside the
    // omega-gradient gather, forked and joined inside the call.
    cudaStream_t aux2 = nullptr;
    cudaEvent_t fork2_ev = nullptr, done2_ev = nullptr;
    bool sort_pending = false;   // eager: omega copied by set_points, not yet sorted
    bool join_pending = false;   // sort launched on aux, not yet joined into a stream
    bool join2_pending = false;  // strip plan and fill launched on aux after the join event, not yet joined
    bool cap_pending = false;    // the same for a set_points recorded into capture cap_id
    unsigned long long cap_id = 0;
    float* d_pw = nullptr;   // [M_cap][ws] kernel weights of the sorted points
    int ws = 4;              // D*J rounded up to a multiple of 4 (8 D for the strips)
    int wd = 6;              // weights per dimension in a row (J; 8 for the strips)
    float c_hi[3] = {0, 0, 0}, c_lo[3] = {0, 0, 0};
    // workspace
    float2* d_G = nullptr;
    float2* d_T = nullptr;
    size_t G_elems = 0, T_elems = 0;
    size_t bytes = 0;
    cudaStream_t last_stream = nullptr;
    // profiling
    bool prof = false;
    struct Ev {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Ev> events;
    std::vector<cudaEvent_t> pool;
};

namespace {

cudaEvent_t get_event(nufft_plan_s* p) {
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Wraps one kernel launch: counts it and, when profiling, brackets it with events.
template <typename F>
int launch(nufft_plan_s* p, int kind, cudaStream_t s, F&& f) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (p->prof) {
        a = get_event(p);
        b = get_event(p);
        cudaEventRecord(a, s);
    }
    cudaError_t e = f();
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (p->prof) {
        cudaEventRecord(b, s);
        p->events.push_back({kind, a, b});
    }
    if (e != cudaSuccess) return fail(NUFFT_ERR_CUDA, std::string("kernel ") + kProfNames[kind] + ": " + cudaGetErrorString(e));
    return NUFFT_OK;
}

void build_fft_axis(int L, FftAxis& ax) {
    std::vector<int> rad;
    int q = L;
    while (q % 16 == 0) { rad.push_back(16); q /= 16; }
    while (q % 8 == 0) { rad.push_back(8); q /= 8; }
    while (q % 4 == 0) { rad.push_back(4); q /= 4; }
    while (q % 2 == 0) { rad.push_back(2); q /= 2; }
    while (q % 3 == 0) { rad.push_back(3); q /= 3; }
    while (q % 5 == 0) { rad.push_back(5); q /= 5; }
    ax.L = L;
    ax.nstages = (int)rad.size();
    int Ns = 1;
    for (size_t i = 0; i < rad.size(); ++i) {
        ax.st[i].R = rad[i];
        ax.st[i].Ns = Ns;
        ax.st[i].tw_step = L / (Ns * rad[i]);
        ax.st[i].magic = magic_of((uint32_t)Ns);
        Ns *= rad[i];
    }
}

// psi(u) = I0(beta sqrt(1 - (2u/J)^2)) for |u| < J/2, else 0, by the power series of I0 in FP64
// (terms past 1e-17 of the sum dropped).
double kb_psi_fp64(double u, int J, double beta) {
    const double s = 2.0 * u / J, z = 1.0 - s * s;
    if (z <= 0.0) return 0.0;
    const double q = beta * beta / 4.0 * z;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 200 && term > 1e-17 * sum; ++k) {
        term *= q / ((double)k * k);
        sum += term;
    }
    return sum;
}

// Kaiser-Bessel Fourier transform int psi(u) exp(-2 pi i f u) du in closed form.
double kb_ft(double f, int J, double beta) {
    const double a = beta * beta - (M_PI * J * f) * (M_PI * J * f);
    if (a > 0) { const double s = std::sqrt(a); return J * std::sinh(s) / s; }
    if (a < 0) { const double s = std::sqrt(-a); return J * std::sin(s) / s; }
    return J;
}

void free_plan(nufft_plan_s* p) {
    for (int d = 0; d < 3; ++d) { cudaFree(p->d_deap[d]); cudaFree(p->d_tw[d]); }
    cudaFree(p->d_kbtab);
    cudaFree(p->d_kcount); cudaFree(p->d_offsets); cudaFree(p->d_item_off); cudaFree(p->d_tile_parts); cudaFree(p->d_heavy); cudaFree(p->d_tile_nbr);
    cudaFree(p->d_nitems); cudaFree(p->d_items); cudaFree(p->d_local); cudaFree(p->d_keyid); cudaFree(p->d_pidx); cudaFree(p->d_pfrac);
    cudaFree(p->d_pw); cudaFree(p->d_om);
    cudaFree(p->d_G); cudaFree(p->d_T);
    cudaFree(p->d_partial); cudaFree(p->d_counters); cudaFree(p->d_ys); cudaFree(p->d_hcount); cudaFree(p->d_hoff);
    cudaFree(p->d_hits); cudaFree(p->d_splits); cudaFree(p->d_hcur); cudaFree(p->d_plan_sums);
    cudaFree(p->d_hits_tmp);
    if (p->aux) cudaStreamDestroy(p->aux);
    if (p->fork_ev) cudaEventDestroy(p->fork_ev);
    if (p->join_ev) cudaEventDestroy(p->join_ev);
    if (p->join2_ev) cudaEventDestroy(p->join2_ev);
    if (p->aux2) cudaStreamDestroy(p->aux2);
    if (p->fork2_ev) cudaEventDestroy(p->fork2_ev);
    if (p->done2_ev) cudaEventDestroy(p->done2_ev);
    for (auto& e : p->events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (auto e : p->pool) cudaEventDestroy(e);
    delete p;
}

int validate_opts(const nufft_opts* o, nufft_plan_s& p) {
    if (!o) return fail(NUFFT_ERR_INVALID_ARG, "opts is NULL");
    if (o->dim < 1 || o->dim > 3) return fail(NUFFT_ERR_UNSUPPORTED, "dim must be 1, 2 or 3");
    p.D = o->dim;
    p.sigma = o->sigma > 0 ? o->sigma : 2.0;
    if (p.sigma <= 1.0 || p.sigma > 4.0) return fail(NUFFT_ERR_UNSUPPORTED, "sigma must lie in (1, 4]");
    p.J = o->J ? o->J : 6;
    if (p.J < kJMin || p.J > kJMax) return fail(NUFFT_ERR_UNSUPPORTED, "J must lie in [4, 8]");
    p.maxC = o->max_coils ? o->max_coils : 1;
    if (p.maxC < 1 || p.maxC > NUFFT_MAX_COILS) return fail(NUFFT_ERR_UNSUPPORTED, "max_coils must lie in [1, 128]");
    p.Nimg = 1;
    p.Ktot = 1;
    for (int d = 0; d < p.D; ++d) {
        const int64_t n = o->n[d];
        if (n < 2 || n % 2) return fail(NUFFT_ERR_UNSUPPORTED, "every N_d must be even and >= 2");
        p.N[d] = n;
        p.K[d] = grid_size(n, p.sigma);
        if (p.K[d] > 4096) return fail(NUFFT_ERR_UNSUPPORTED, "oversampled grid edge exceeds 4096");
        if (p.K[d] < p.J) return fail(NUFFT_ERR_UNSUPPORTED, "oversampled grid edge smaller than J");
        p.Nimg *= n;
        p.Ktot *= p.K[d];
    }
    // the line passes index within a line in 32 bits: the channel stride of the first axis,
    // (1 + D) max_coils prod_{d > 0} K_d complex elements, must fit
    if ((int64_t)(1 + p.D) * p.maxC * (p.Ktot / p.K[0]) > (int64_t)INT32_MAX)
        return fail(NUFFT_ERR_UNSUPPORTED, "oversampled grid too large for max_coils");
    p.beta = o->beta > 0 ? o->beta
                         : M_PI * std::sqrt(std::pow(p.J / p.sigma, 2) * std::pow(p.sigma - 0.5, 2) - 0.8);
    // bins = spread tiles of B_d cells per axis; coils per spread block from the tile size
    const int defB[3][3] = {{256, 1, 1}, {16, 16, 1}, {8, 8, 8}};
    size_t tcells = 1;
    for (int d = 0; d < p.D; ++d) {
        int b = o->bin_size[d] > 0 ? o->bin_size[d] : defB[p.D - 1][d];
        b = (int)std::min<int64_t>(b, p.K[d]);
        if (b < p.J) b = (int)std::min<int64_t>(p.J, p.K[d]);   // a window must not pass a whole tile
        p.B[d] = b;
        p.nb[d] = (int)((p.K[d] + b - 1) / b);
        tcells *= b;
    }
    p.nbins = 1;
    for (int d = 0; d < p.D; ++d) p.nbins *= p.nb[d];
    if (p.nbins > (1 << 24)) return fail(NUFFT_ERR_UNSUPPORTED, "too many bins; enlarge bin_size");
    p.cpb = (int)tcells;
    if ((int64_t)p.nbins * p.cpb >= ((int64_t)1 << 31)) return fail(NUFFT_ERR_UNSUPPORTED, "grid too large for the point sort");
    const size_t tile_budget = 32 * 1024;
    if (tcells * sizeof(float2) > tile_budget)
        return fail(NUFFT_ERR_UNSUPPORTED, "spread tile does not fit in shared memory; reduce bin_size");
    p.CCmax = (int)std::max<size_t>(1, std::min<size_t>(32, tile_budget / (tcells * sizeof(float2))));
    // spread path: row-owner tiles when no window can cover a tile twice, else the general kernel
    p.cell_spread = p.D >= 2 && tcells <= 512;
    for (int d = 0; d < p.D; ++d) p.cell_spread = p.cell_spread && p.B[d] + p.J - 1 <= p.K[d];
    p.P = p.cell_spread ? (int)tcells : (p.D == 3 ? 1024 : 512);
    // strips (2-D and 3-D): lanes are NSL row slots x 32 / NSL coil pairs, chosen from max_coils;
    // a window must not reach a unit twice along any axis
    {
        // coils per warp (a coil pair per lane): 16, 8, 4 or 2; NSL = 64 / coils per warp
        const int cpw = p.maxC >= 9 ? 16 : (p.maxC >= 5 ? 8 : (p.maxC >= 3 ? 4 : 2));
        p.NSL = 64 / cpw;
        p.ncg_max = (p.maxC + cpw - 1) / cpw;
        p.SR1 = p.D == 3 ? strip_rows1(p.NSL) : 1;
        p.SR0 = p.NSL / p.SR1;
        // a window must not reach a unit twice: 16 + J - 1 columns along the last axis, R + J - 1
        // rows along each row axis (R = NSL in 2-D, R0 and R1 in 3-D)
        const int64_t KL = p.K[p.D - 1];
        p.strip = p.D >= 2 && KL >= kStripW + p.J - 1 && p.K[0] >= p.SR0 + p.J - 1 &&
                  (p.D == 2 || p.K[1] >= p.SR1 + p.J - 1);
        if (o->spread_variant == NUFFT_SPREAD_TILES || o->spread_variant == NUFFT_SPREAD_GENERAL) p.strip = false;
        if (o->spread_variant == NUFFT_SPREAD_GENERAL) p.cell_spread = false;
        if (o->spread_variant == NUFFT_SPREAD_STRIPS && !p.strip)
            return fail(NUFFT_ERR_UNSUPPORTED, "strip spread needs D >= 2 and a grid of at least 16 + J - 1 cells "
                                               "along the last axis and R + J - 1 along the others (R: unit rows)");
        if (o->spread_variant == NUFFT_SPREAD_TILES && !p.cell_spread)
            return fail(NUFFT_ERR_UNSUPPORTED, "tile spread needs D >= 2, at most 512 cells per bin and bins of at "
                                               "most K - J + 1 cells");
        if (o->spread_variant < 0 || o->spread_variant > NUFFT_SPREAD_GENERAL)
            return fail(NUFFT_ERR_INVALID_ARG, "unknown spread_variant");
        if (o->strip_part) {
            if (o->strip_part < 8 || o->strip_part > 4096 || (o->strip_part & (o->strip_part - 1)))
                return fail(NUFFT_ERR_INVALID_ARG, "strip_part must be a power of two in [8, 4096]");
            p.strip_P = o->strip_part;
        }
        p.deterministic = o->deterministic != 0;
        if (p.deterministic && !p.strip)
            return fail(NUFFT_ERR_UNSUPPORTED, "deterministic results need the strip spread");
        if (p.strip) {
            int64_t nu = ((p.K[0] + p.SR0 - 1) / p.SR0) * ((KL + kStripW - 1) / kStripW);
            if (p.D == 3) nu *= (p.K[1] + p.SR1 - 1) / p.SR1;
            if (nu >= ((int64_t)1 << 30)) return fail(NUFFT_ERR_UNSUPPORTED, "too many strip units");
            p.nunits = (int)nu;
            // partial-sum slots for split units (8 KB each): ~nunits / 4, at most 16 MB (the plan
            // lengthens the parts of split units when they would need more)
            p.strip_slots = std::max(64, std::min(2048 / p.ncg_max, p.nunits / 4));
        }
    }
    // KB power-series coefficients a_k = (beta^2/4)^k / (k!)^2
    double ak = 1.0, sum = 0.0;
    const double q = p.beta * p.beta / 4.0;
    for (int k = 0; k < kKbTerms; ++k) {
        if (k > 0) ak *= q / ((double)k * k);
        p.kb.a[k] = (float)ak;
        sum += ak;
    }
    if (ak > 1e-9 * sum) return fail(NUFFT_ERR_UNSUPPORTED, "beta too large for the kernel power series");
    p.kb.two_over_j = (float)(2.0 / p.J);
    p.gather_variant = o->gather_variant;
    if (p.gather_variant < NUFFT_GATHER_AUTO || p.gather_variant > NUFFT_GATHER_QUADS)
        return fail(NUFFT_ERR_INVALID_ARG, "unknown gather_variant");
    p.kernel_mode = o->kernel_mode;
    if (p.kernel_mode != NUFFT_KERNEL_DIRECT && p.kernel_mode != NUFFT_KERNEL_TABLE)
        return fail(NUFFT_ERR_INVALID_ARG, "kernel_mode must be NUFFT_KERNEL_DIRECT or NUFFT_KERNEL_TABLE");
    if (p.kernel_mode == NUFFT_KERNEL_TABLE) {
        p.tab_L = o->table_density ? o->table_density : 512;
        if (p.tab_L < 16 || p.tab_L > 65536) return fail(NUFFT_ERR_INVALID_ARG, "table_density must lie in [16, 65536]");
        p.tab_n = p.tab_L * p.J / 2;
    }
    p.wd = p.strip ? 8 : p.J;   // the strip spread reads the column weights as two 16-byte loads
    p.ws = p.strip ? 8 * p.D : (p.D * p.J + 3) & ~3;
    for (int d = 0; d < p.D; ++d) {
        const double c = (double)p.K[d] / (2.0 * M_PI);
        p.c_hi[d] = (float)c;
        p.c_lo[d] = (float)(c - (double)p.c_hi[d]);
    }
    return NUFFT_OK;
}

// Workspace element counts for max channels chmax = maxC (1 + D).
void workspace_elems(const nufft_plan_s& p, size_t& G, size_t& T) {
    const int64_t chmax = (int64_t)p.maxC * (1 + p.D);
    G = (size_t)(p.Ktot * chmax);
    T = 0;
    // forward intermediates: after the pass over dim d, [N_0..N_{d-1}][K_d..K_{D-1}]
    for (int d = p.D - 1; d >= 0; --d) {
        int64_t n = 1;
        for (int e = 0; e < d; ++e) n *= p.N[e];
        for (int e = d; e < p.D; ++e) n *= p.K[e];
        if ((d % 2) == 1) T = std::max<size_t>(T, (size_t)(n * chmax));
        else G = std::max<size_t>(G, (size_t)(n * chmax));
    }
    // inverse intermediates: after the pass over dim d < D-1, [N_0..N_d][K_{d+1}..]
    for (int d = 0; d < p.D - 1; ++d) {
        int64_t n = 1;
        for (int e = 0; e <= d; ++e) n *= p.N[e];
        for (int e = d + 1; e < p.D; ++e) n *= p.K[e];
        if ((d % 2) == 0) T = std::max<size_t>(T, (size_t)(n * p.maxC));
        else G = std::max<size_t>(G, (size_t)(n * p.maxC));
    }
    // the coil-summing last inverse pass keeps up to C partial images in the buffer it does not read
    T = std::max<size_t>(T, (size_t)(p.maxC * p.Nimg));
    G = std::max<size_t>(G, (size_t)(p.maxC * p.Nimg));
}

// Upper bound of the spread work items: one per tile plus one per P candidates;
// every point is a candidate of at most 3^D tiles.
size_t max_items(const nufft_plan_s& p, int64_t cap) {
    int nbr = 1;
    for (int d = 0; d < p.D; ++d) nbr *= std::min(3, p.nb[d]);
    size_t n = (size_t)p.nbins + (size_t)((nbr * cap + p.P - 1) / p.P) + 1;
    // strips: one item per unit, plus the extra parts of split units (at most the partial slots)
    if (p.strip) n = std::max(n, (size_t)p.nunits + (size_t)p.strip_slots + 1);
    return n;
}

// Sort histogram entries: one per bin.
int64_t sort_keys(const nufft_plan_s& p) { return (int64_t)p.nbins; }

size_t strip_bytes(const nufft_plan_s& p) {
    if (!p.strip) return 0;
    return (size_t)p.strip_slots * (p.ncg_max * (kStripW * 32 * sizeof(float4) + sizeof(int)) + sizeof(int4)) +
           (size_t)(3 * p.nunits + 3) * sizeof(int);
}

// Strip units a point's window can reach: its J rows span at most ceil((J - 1) / NSL) + 1 row
// groups, one more where they wrap past the shorter last group, and its J columns at most three
// column tiles (two, and a narrow last one).
int64_t strip_hits_per_point(const nufft_plan_s& p) {
    const int64_t rows0 = (p.J - 2) / p.SR0 + 3;
    return p.D == 3 ? 3 * rows0 * ((p.J - 2) / p.SR1 + 3) : 3 * rows0;
}

size_t point_bytes(const nufft_plan_s& p, int64_t cap) {
    size_t b = (size_t)cap * (2 * sizeof(int) + sizeof(int4) + sizeof(float4) + (p.ws + p.D) * sizeof(float)) +
               max_items(p, cap) * sizeof(int4);
    if (p.strip)
        b += (size_t)cap * ((size_t)p.ncg_max * (64 / p.NSL) * sizeof(float2) +
                            (p.deterministic ? 2 : 1) * strip_hits_per_point(p) * sizeof(int2));
    return b;
}

int alloc_points(nufft_plan_s* p, int64_t cap) {
    cudaFree(p->d_items); cudaFree(p->d_local); cudaFree(p->d_keyid); cudaFree(p->d_pidx); cudaFree(p->d_pfrac);
    cudaFree(p->d_pw); cudaFree(p->d_om); cudaFree(p->d_ys); cudaFree(p->d_hits); cudaFree(p->d_hits_tmp);
    p->d_items = nullptr; p->d_local = p->d_keyid = nullptr; p->d_pidx = nullptr; p->d_pfrac = nullptr;
    p->d_pw = nullptr;
    p->d_om = nullptr;
    p->d_ys = nullptr;
    p->d_hits = nullptr;
    p->d_hits_tmp = nullptr;
    const size_t c = (size_t)std::max<int64_t>(cap, 1);
    if (p->strip) {
        p->hit_cap = (int64_t)c * strip_hits_per_point(*p);
        if (cudaMalloc(&p->d_ys, c * (size_t)p->ncg_max * (64 / p->NSL) * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&p->d_hits, (size_t)p->hit_cap * sizeof(int2)) != cudaSuccess ||
            (p->deterministic && cudaMalloc(&p->d_hits_tmp, (size_t)p->hit_cap * sizeof(int2)) != cudaSuccess)) {
            cudaGetLastError();
            return fail(NUFFT_ERR_OOM, "device allocation of the strip hit lists failed");
        }
    }
    if (cudaMalloc(&p->d_items, max_items(*p, cap) * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(&p->d_local, c * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&p->d_keyid, c * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&p->d_pidx, c * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(&p->d_pfrac, c * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&p->d_pw, c * p->ws * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&p->d_om, c * p->D * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(NUFFT_ERR_OOM, "device allocation of point arrays failed");
    }
    p->M_cap = cap;
    return NUFFT_OK;
}

StripTables strip_tables(const nufft_plan_s& p) {
    StripTables t{};
    t.hcount = p.d_hcount;
    t.hcur = p.d_hcur;
    t.partial_sums = p.d_plan_sums;
    t.hoff = p.d_hoff;
    t.hits = p.d_hits;
    t.fill_to = p.deterministic ? p.d_hits_tmp : p.d_hits;
    t.hit_cap = p.hit_cap;
    t.items = p.d_items;
    t.splits = p.d_splits;
    t.nitems = p.d_nitems;
    t.P = p.strip_P;
    t.slots = p.strip_slots;
    return t;
}

StripGeom strip_geom(const nufft_plan_s& p) {
    StripGeom g{};
    g.D = p.D;
    g.K0 = (int)p.K[0];
    g.K1 = p.D >= 2 ? (int)p.K[1] : 1;
    g.KL = (int)p.K[p.D - 1];
    g.R0 = p.SR0;
    g.R1 = p.SR1;
    g.ng1 = p.D == 3 ? (int)((p.K[1] + p.SR1 - 1) / p.SR1) : 1;
    g.nbl = (int)((g.KL + kStripW - 1) / kStripW);
    g.J = p.J;
    g.NSL = p.NSL;
    return g;
}

SortArgs sort_args(nufft_plan_s* p, const float* omega) {
    SortArgs a{};
    a.omega = omega;
    a.m = p->M;
    a.D = p->D;
    a.J = p->J;
    for (int d = 0; d < 3; ++d) {
        a.K[d] = (int)p->K[d];
        a.B[d] = p->B[d];
        a.nb[d] = p->nb[d];
        a.c_hi[d] = p->c_hi[d];
        a.c_lo[d] = p->c_lo[d];
    }
    a.nbins = p->nbins;
    a.P = p->P;
    a.kcount = p->d_kcount;
    a.local = p->d_local;
    a.keyid = p->d_keyid;
    a.offsets = p->d_offsets;
    a.item_off = p->d_item_off;
    a.tile_parts = p->d_tile_parts;
    a.heavy = p->d_heavy;
    a.tile_nbr = p->d_tile_nbr;
    a.items = p->d_items;
    a.nitems = p->d_nitems;
    a.pidx = p->d_pidx;
    a.pfrac = p->d_pfrac;
    a.pw = p->d_pw;
    a.ws = p->ws;
    a.wd = p->wd;
    a.kb = p->kb;
    a.kbtab = p->d_kbtab;
    a.tab_L = (float)p->tab_L;
    a.tab_n = p->tab_n;
    a.strip = p->strip ? 1 : 0;
    a.nunits = p->nunits;
    a.sg = strip_geom(*p);
    a.st = strip_tables(*p);
    return a;
}

int sort_rest(nufft_plan_s* p, cudaStream_t s);

// True, with the capture sequence id, when s is recording into a CUDA graph.
bool capture_id(cudaStream_t s, unsigned long long& id) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamGetCaptureInfo(s, &cs, &id) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusActive;
}

int do_set_points(nufft_plan_s* p, int64_t m, const float* omega, cudaStream_t s) {
    if (m < 0 || m > (int64_t)INT32_MAX) return fail(NUFFT_ERR_INVALID_ARG, "m out of range");
    if (m > 0 && !omega) return fail(NUFFT_ERR_INVALID_ARG, "omega is NULL");
    if (m > p->M_cap) {
        NJ_CUDA(cudaStreamSynchronize(s));
        if (p->aux) NJ_CUDA(cudaStreamSynchronize(p->aux));
        int st = alloc_points(p, m);
        if (st) return st;
        p->bytes = 0;
    }
    p->M = m;
    p->last_stream = s;
    // the plan keeps its own copy of omega (the caller's buffer is free once the copy has run);
    // the sort itself runs in the next call that needs the points (sort_rest)
    if (m > 0) NJ_CUDA(cudaMemcpyAsync(p->d_om, omega, sizeof(float) * p->D * m, cudaMemcpyDeviceToDevice, s));
    unsigned long long id = 0;
    if (capture_id(s, id)) {
        p->cap_id = id;
        p->cap_pending = true;
    } else {
        p->sort_pending = true;
    }
    if (!p->aux) return sort_rest(p, s);   // plans without a stream of their own sort in line
    return NUFFT_OK;
}

// The sort of the plan's copy of omega: histogram, scan, tile lists and items, scatter of the point
// records and weights; on the plan's stream, forked from s and joined by sort_join, when the plan
// has one.  An eager call sorts what the last eager set_points left; a call recorded into a graph
// sorts when that graph, or the eager state, has points not yet sorted, and then clears the
// histogram itself, so that every replay sorts completely.
int sort_rest(nufft_plan_s* p, cudaStream_t s) {
    unsigned long long id = 0;
    const bool capturing = capture_id(s, id);
    bool run;
    if (capturing) {
        run = (p->cap_pending && p->cap_id == id) || p->sort_pending;
        if (p->cap_id == id) p->cap_pending = false;
    } else {
        run = p->sort_pending;
        p->sort_pending = false;
    }
    if (!run) return NUFFT_OK;
    SortArgs a = sort_args(p, p->d_om);
    cudaStream_t ss = s;
    if (p->aux) {
        NJ_CUDA(cudaEventRecord(p->fork_ev, s));
        NJ_CUDA(cudaStreamWaitEvent(p->aux, p->fork_ev, 0));
        ss = p->aux;
    }
    int st;
    // every scan leaves the histogram zero for the next sort; a fresh one, or one in a graph, is cleared
    if ((capturing || !p->kcount_clear) &&
        (st = launch(p, PK_ZERO, ss, [&] { return launch_zero(p->d_kcount, sizeof(int) * sort_keys(*p), ss); })))
        return st;
    if ((st = launch(p, PK_BIN_COUNT, ss, [&] { return launch_key_count(a, ss); }))) return st;
    if (p->strip && (capturing || !p->kcount_clear) &&
        (st = launch(p, PK_ZERO, ss, [&] { return launch_zero(p->d_hcount, sizeof(int) * p->nunits, ss); })))
        return st;
    if (p->strip) {   // bin offsets only: the strip spread needs no tile lists
        if ((st = launch(p, PK_BIN_SCAN, ss, [&] { return launch_bin_scan(a, ss); }))) return st;
    } else if (p->nbins <= kFusedTablesMaxBins) {
        if ((st = launch(p, PK_BIN_SCAN, ss, [&] { return launch_sort_tables(a, ss); }))) return st;
    } else {
        if ((st = launch(p, PK_BIN_SCAN, ss, [&] { return launch_bin_scan(a, ss); }))) return st;
        if ((st = launch(p, PK_TILE_SCAN, ss, [&] { return launch_tile_lists(a, ss); }))) return st;
        if ((st = launch(p, PK_BIN_ITEMS, ss, [&] { return launch_item_scan(a, ss); }))) return st;
    }
    if (!capturing) p->kcount_clear = true;
    if (p->deterministic) {   // bins ordered by original index (the point records' buffer is scratch here)
        if ((st = launch(p, PK_DET_PLACE, ss, [&] { return launch_det_ranks(a, 0, (int*)p->d_pfrac, ss); })) ||
            (st = launch(p, PK_DET_RANK, ss, [&] { return launch_det_ranks(a, 1, (int*)p->d_pfrac, ss); })))
            return st;
    }
    if ((st = launch(p, PK_BIN_SCATTER, ss, [&] { return launch_bin_scatter(a, ss); }))) return st;
    if (p->aux) {
        NJ_CUDA(cudaEventRecord(p->join_ev, p->aux));
        p->join_pending = true;
    }
    // The strip tables (hit offsets, work items, hit lists) are needed by the adjoint spread only:
    // they run behind the join event, beside the kernels that read the sorted points, and are
    // joined before the spread or at the end of the call (strip_join).
    if (p->strip) {
        if ((st = launch(p, PK_STRIP_PLAN_A, ss, [&] { return launch_strip_plan(a, 0, ss); }))) return st;
        if ((st = launch(p, PK_STRIP_PLAN_B, ss, [&] { return launch_strip_plan(a, 1, ss); }))) return st;
        if ((st = launch(p, PK_STRIP_FILL, ss, [&] { return launch_strip_fill(a, ss); }))) return st;
        if (p->deterministic &&
            (st = launch(p, PK_STRIP_ORDER, ss, [&] { return launch_strip_order(a, p->d_hits_tmp, ss); })))
            return st;
        if (p->aux) {
            NJ_CUDA(cudaEventRecord(p->join2_ev, p->aux));
            p->join2_pending = true;
        }
    }
    return NUFFT_OK;
}

int sort_join(nufft_plan_s* p, cudaStream_t s);

// Makes s wait for the strip tables (before the strip spread, and at the end of every call that
// started a sort, so that each call stays self-contained).
int strip_join(nufft_plan_s* p, cudaStream_t s) {
    if (!p->join2_pending) return NUFFT_OK;
    p->join2_pending = false;
    NJ_CUDA(cudaStreamWaitEvent(s, p->join2_ev, 0));
    return NUFFT_OK;
}

// End of an entry point: every piece of the plan's second stream is joined into s.
int finish_call(nufft_plan_s* p, cudaStream_t s, int st) {
    if (st) return st;
    if ((st = sort_join(p, s))) return st;
    return strip_join(p, s);
}

// Makes s wait for the sort before a kernel that reads the sorted points.
int sort_join(nufft_plan_s* p, cudaStream_t s) {
    if (!p->join_pending) return NUFFT_OK;
    p->join_pending = false;
    NJ_CUDA(cudaStreamWaitEvent(s, p->join_ev, 0));
    return NUFFT_OK;
}

// Two-phase line pass of kind `kind` (kernels instantiated one kind per translation unit).
cudaError_t launch_line_pass2(PassKind kind, int L1, int L2, const LinePass& a, dim3 grid, int threads,
                                     size_t smem, cudaStream_t s) {
    switch (kind) {
        case PASS_FWD_FIRST: return launch_fft2_kind<PASS_FWD_FIRST>(L1, L2, a, grid, threads, smem, s);
        case PASS_FWD_MID: return launch_fft2_kind<PASS_FWD_MID>(L1, L2, a, grid, threads, smem, s);
        case PASS_INV_MID: return launch_fft2_kind<PASS_INV_MID>(L1, L2, a, grid, threads, smem, s);
        default: return launch_fft2_kind<PASS_INV_LAST>(L1, L2, a, grid, threads, smem, s);
    }
}

// Tile shape of a line pass: TL lines (TB rows x TS channels) of length L.
// L1 > 0: the register-resident two-phase kernel for L = L1 L2; else the
// shared-memory Stockham kernel.
struct Tile {
    int TB, TS, TL, threads;
    size_t smem;
    int L1, L2, LP;   // two-phase kernel: factors and shared line pitch
};

Tile pick_tile(int L, int64_t B, int64_t S, bool coil_sum, int n_out, bool pair = false) {
    Tile t{};
    if (fft2_factor(L, t.L1, t.L2)) {
        // 8 adjacent lines (64-byte segments along the channel axis), two or three blocks per SM:
        // measured faster than 4 or 16 lines on the 640-point passes.  The coil-summing last
        // inverse pass takes 8 coils per block when its two coil chunks add into a cleared image
        // (pair), else up to 16, so 16 coils need no partial-sum pass.
        int TL = (coil_sum && S > 8 && !pair) ? 16 : 8;
        t.TS = std::min<int>(TL, pow2_ceil(S));
        t.TB = std::min<int>(TL / t.TS, pow2_ceil(B));
        t.TL = t.TB * t.TS;
        while ((t.TL * t.L2) % 32 != 0) {   // whole warps; extra lines are masked
            t.TB *= 2;
            t.TL *= 2;
        }
        t.threads = t.TL * t.L2;
        // line pitch: >= L1 (L2 + 1), congruent to 16 / H mod 16 for H lines per half-warp
        const int H = std::min(t.TL, 16), want = H == 16 ? 1 : 16 / H;
        t.LP = t.L1 * (t.L2 + 1);
        while (t.LP % 16 != want) ++t.LP;
        t.smem = (size_t)t.TL * t.LP * sizeof(float2);
        return t;
    }
    t.L1 = t.L2 = 0;
    const size_t budget = 58 * 1024;   // three to four blocks per SM
    int TL = 32;
    while (TL > 1 && (size_t)(2 * (size_t)L * (TL + 1) + L) * sizeof(float2) > budget) TL /= 2;
    t.TS = std::min<int>(TL, pow2_ceil(S));
    t.TB = std::min<int>(TL / t.TS, pow2_ceil(B));
    t.TL = t.TB * t.TS;
    int work = (L / 4) * t.TL;   // butterflies of a radix-4 stage
    t.threads = std::min(256, std::max(64, ((work + 31) / 32) * 32));
    t.smem = (size_t)(L + 2 * (size_t)L * (t.TL + 1)) * sizeof(float2) + (size_t)t.TB * 3 * sizeof(float);
    if (coil_sum) t.smem += (size_t)t.TB * n_out * sizeof(float2);
    return t;
}

ImageSide image_side(nufft_plan_s* p, int C, const float2* x, const float2* smaps, float2* xout, int has_plain) {
    ImageSide im{};
    im.x = x;
    im.smaps = smaps;
    im.xout = xout;
    im.C = C;
    im.has_plain = has_plain;
    im.D = p->D;
    for (int d = 0; d < 3; ++d) {
        im.N[d] = (int)p->N[d];
        im.deap[d] = p->d_deap[d] ? p->d_deap[d] : p->d_deap[0];
    }
    im.nimg = p->Nimg;
    return im;
}

// Forward grids: channel (dblk, c) = dblk * C + c, dblk 0 = plain image when
// has_plain, then r^[d]-weighted images.  Result in p->d_G, layout [K...][nd*C].
int forward_grids(nufft_plan_s* p, int C, int nd, int has_plain, const float2* x, const float2* smaps, cudaStream_t s) {
    const int D = p->D;
    const int64_t ch = (int64_t)nd * C;
    ImageSide im = image_side(p, C, x, smaps, nullptr, has_plain);
    const float2* in = nullptr;
    for (int k = 0; k < D; ++k) {
        const int d = D - 1 - k;
        const int L = (int)p->K[d];
        int64_t B = 1, S = ch;
        for (int e = 0; e < d; ++e) B *= p->N[e];
        for (int e = d + 1; e < D; ++e) S *= p->K[e];
        float2* out = (d % 2 == 0) ? p->d_G : p->d_T;
        Tile t = pick_tile(L, B, S, false, L);
        LinePass a{};
        a.ax = p->axis[d];
        a.n_in = (int)p->N[d];
        a.n_out = L;
        a.B = B;
        a.S = S;
        a.TB = t.TB;
        a.TS = t.TS;
        a.lgTS = ilog2(t.TS);
        a.lgTL = ilog2(t.TL);
        a.TLP = t.L1 ? t.LP : t.TL + 1;
        a.nchunks = 1;
        a.coil_sum = 0;
        a.in = in;
        a.out = out;
        a.im = im;
        a.magic_L = magic_of((uint32_t)L);
        a.magic_n = magic_of((uint32_t)a.n_out);
        a.ntiles_s = (S + t.TS - 1) / t.TS;
        const dim3 grid = line_grid((B + t.TB - 1) / t.TB, a.ntiles_s);
        const PassKind kind = (k == 0) ? PASS_FWD_FIRST : PASS_FWD_MID;
        int st = launch(p, k == 0 ? PK_FFT_FWD_FIRST : PK_FFT_FWD_MID, s, [&] {
            return t.L1 ? launch_line_pass2(kind, t.L1, t.L2, a, grid, t.threads, t.smem, s)
                        : launch_line_pass(kind, a, grid, t.threads, t.smem, s);
        });
        if (st) return st;
        in = out;
    }
    return NUFFT_OK;
}

int inverse_passes(nufft_plan_s* p, int C, const float2* smaps, float2* xout, cudaStream_t s,
                   float2* gbuf = nullptr, float2* tbuf = nullptr);

// Adjoint of the interpolation + FFT + scaling for C coil channels of y.
// ysorted: y already copied into T in sorted point order (by the VJP gather), else null.
int adjoint_impl(nufft_plan_s* p, int C, const float2* y, const float2* smaps, float2* xout, cudaStream_t s,
                 const float2* ysorted = nullptr, float2* gbuf = nullptr, float2* tbuf = nullptr) {
    const int D = p->D;
    int st;
    if (!gbuf) gbuf = p->d_G;
    if (!tbuf) tbuf = p->d_T;
    if (p->strip) {
        // strips: every grid cell written once by its unit; y in sorted point-major order
        StripArgs ta{};
        ta.pts = PointsView{p->d_pidx, p->d_pfrac, p->M, p->d_pw, p->ws, p->wd};
        ta.g = strip_geom(*p);
        ta.t = strip_tables(*p);
        ta.max_items = p->nunits + p->strip_slots;
        ta.C = C;
        const int cpt = 64 / p->NSL;   // coils per warp
        ta.ncg = (C + cpt - 1) / cpt;
        ta.grid = gbuf;
        ta.partial = p->d_partial;
        ta.counters = p->d_counters;
        if (ysorted) {
            ta.y = ysorted;
        } else {
            if ((st = launch(p, PK_PERMUTE_Y, s,
                             [&] { return launch_permute_y_strips(p->d_local, y, p->d_ys, p->M, C, cpt, s); })))
                return st;
            ta.y = p->d_ys;
        }
        if ((st = strip_join(p, s))) return st;
        if ((st = launch(p, PK_SPREAD, s, [&] { return launch_spread_strips(ta, s); }))) return st;
        return inverse_passes(p, C, smaps, xout, s, gbuf, tbuf);
    }
    // spread: output-driven tiles; only tiles split over several work items are cleared first
    SpreadArgs sa{};
    sa.pts = PointsView{p->d_pidx, p->d_pfrac, p->M, p->d_pw, p->ws, p->wd};
    sa.D = D;
    sa.J = p->J;
    for (int d = 0; d < 3; ++d) {
        sa.K[d] = (int)p->K[d];
        sa.B[d] = p->B[d];
        sa.nb[d] = p->nb[d];
    }
    sa.nbins = p->nbins;
    sa.offsets = p->d_offsets;
    sa.tile_nbr = p->d_tile_nbr;
    sa.items = p->d_items;
    sa.nitems = p->d_nitems;
    sa.tile_parts = p->d_tile_parts;
    sa.heavy = p->d_heavy;
    sa.max_items = (int)max_items(*p, p->M);
    sa.P = p->P;
    sa.y = y;
    sa.M = p->M;
    sa.C = C;
    sa.CC = std::min(C, p->CCmax);
    // row slots per warp: at least the kernel's minimum, at least 2 (<= 16 coils staged per pass)
    sa.G = std::max(std::max(spread_min_slots(D, p->J), 2), 32 / std::min(32, pow2_ceil(sa.CC)));
    sa.lgG = ilog2(sa.G);
    const int cpl = 1;
    sa.kb = p->kb;
    sa.grid = p->d_G;
    const size_t ssm = (size_t)p->cpb * sa.CC * sizeof(float2);
    if ((st = launch(p, PK_ZERO_HEAVY, s, [&] { return launch_zero_heavy_tiles(sa, s); }))) return st;
    if (p->cell_spread) {
        sa.CC = C <= 4 ? 4 : (C <= 8 ? 8 : 16);
        // y in sorted point order (in T, free until the inverse FFT passes): the tile kernels then
        // read it coalesced and without waiting for the point record
        if (ysorted) {
            sa.y = ysorted;
            sa.y_sorted = 1;
        } else if ((size_t)C * (size_t)p->M <= p->T_elems && p->M > 0) {
            if ((st = launch(p, PK_PERMUTE_Y, s,
                             [&] { return launch_permute_y(p->d_pidx, y, p->d_T, p->M, C, s); })))
                return st;
            sa.y = p->d_T;
            sa.y_sorted = 1;
        }
        if ((st = launch(p, PK_SPREAD, s, [&] { return launch_spread_cells(sa, s); }))) return st;
    } else {
        if ((st = launch(p, PK_SPREAD, s, [&] { return launch_spread(sa, cpl, s, ssm); }))) return st;
    }
    return inverse_passes(p, C, smaps, xout, s);
}

// Inverse FFT passes over the spread grid in gbuf (p->d_G), dim 0 first, intermediates alternating
// with tbuf (p->d_T); the last one crops, scales and applies the conjugate maps (summing the coils)
// or writes one image per coil.
int inverse_passes(nufft_plan_s* p, int C, const float2* smaps, float2* xout, cudaStream_t s, float2* gbuf,
                   float2* tbuf) {
    const int D = p->D;
    int st;
    if (!gbuf) gbuf = p->d_G;
    if (!tbuf) tbuf = p->d_T;
    const float2* in = gbuf;
    ImageSide im = image_side(p, C, nullptr, smaps, xout, 0);
    // 9..16 coils summed by two-phase passes: the last pass runs two 8-coil chunks that both add
    // into the image, which the pass before it clears
    bool pair = false;
    if (smaps && D >= 2 && C > 8 && C <= 16) {
        int l1, l2;
        pair = fft2_factor((int)p->K[D - 1], l1, l2) && fft2_factor((int)p->K[D - 2], l1, l2);
    }
    for (int d = 0; d < D; ++d) {
        const int L = (int)p->K[d];
        int64_t B = 1, S = C;
        for (int e = 0; e < d; ++e) B *= p->N[e];
        for (int e = d + 1; e < D; ++e) S *= p->K[e];
        const bool last = d == D - 1;
        const bool coil_sum = last && smaps != nullptr;
        float2* out = last ? nullptr : ((d % 2 == 0) ? tbuf : gbuf);
        Tile t = pick_tile(L, B, S, coil_sum, (int)p->N[d], pair);
        LinePass a{};
        a.ax = p->axis[d];
        a.n_in = L;
        a.n_out = (int)p->N[d];
        a.B = B;
        a.S = S;
        a.TB = t.TB;
        a.TS = t.TS;
        a.lgTS = ilog2(t.TS);
        a.lgTL = ilog2(t.TL);
        a.TLP = t.L1 ? t.LP : t.TL + 1;
        a.coil_sum = coil_sum ? 1 : 0;
        a.nchunks = 1;   // one channel chunk per block
        const int chunks = (int)((S + t.TS - 1) / t.TS);
        a.in = in;
        a.out = out;
        a.im = im;
        float2* part = nullptr;
        if (pair && d == D - 2) {
            a.clear = xout;
            a.nclear = p->Nimg;
        }
        if (pair && last) {
            a.pair_add = 1;
            a.im.xout_stride = 0;
        } else if (coil_sum && chunks > 1) {   // partial coil sums per chunk, added in order afterwards
            part = (in == gbuf) ? tbuf : gbuf;
            a.im.xout = part;
            a.im.xout_stride = p->Nimg;
        }
        a.magic_L = magic_of((uint32_t)L);
        a.magic_n = magic_of((uint32_t)a.n_out);
        a.ntiles_s = chunks;
        const dim3 grid = line_grid((B + t.TB - 1) / t.TB, chunks);
        const PassKind kind = last ? PASS_INV_LAST : PASS_INV_MID;
        st = launch(p, last ? PK_FFT_INV_LAST : PK_FFT_INV_MID, s, [&] {
            return t.L1 ? launch_line_pass2(kind, t.L1, t.L2, a, grid, t.threads, t.smem, s)
                        : launch_line_pass(kind, a, grid, t.threads, t.smem, s);
        });
        if (st) return st;
        if (part) {
            st = launch(p, PK_SUM_CHUNKS, s, [&] { return launch_sum_chunks(part, chunks, p->Nimg, xout, s); });
            if (st) return st;
        }
        in = out;
    }
    return NUFFT_OK;
}

// The forward gather on coil quads: a lane owns four adjacent coils (32-byte loads, twice the
// points per warp).  AUTO takes them for the 2-D forward with C a multiple of 4 from 16 on (640^2 /
// 16 coils: 23.0 -> 22.0 us); the VJP kinds (40.1 -> 46.5 us: half the resident warps) and the 3-D
// gathers (1.35 -> 1.64 ms on 8 coils) lose with them.  QUADS takes them wherever C is a multiple
// of 4 from 8 on; PAIRS never.
void forward_quads(const nufft_plan_s* p, GatherArgs& g) {
    const bool quads = p->gather_variant == NUFFT_GATHER_QUADS
                           ? (g.C % 4 == 0 && g.C >= 8)
                           : (p->gather_variant == NUFFT_GATHER_AUTO && g.D == 2 && g.C % 4 == 0 && g.C >= 16);
    if (quads && g.C <= 128) {
        g.W = 4;
        g.G = pow2_ceil(g.C / 4);
        g.lgG = ilog2(g.G);
    }
}

GatherArgs gather_args(nufft_plan_s* p, int C, int nd, int has_plain) {
    GatherArgs g{};
    g.pts = PointsView{p->d_pidx, p->d_pfrac, p->M, p->d_pw, p->ws, p->wd};
    g.D = p->D;
    g.J = p->J;
    for (int d = 0; d < 3; ++d) g.K[d] = (int)p->K[d];
    g.grid = p->d_G;
    g.C = C;
    g.nd = nd;
    g.has_plain = has_plain;
    // even C up to 64: a lane owns two adjacent coils (16-byte loads), else one
    g.W = (C % 2 == 0 && C <= 64) ? 2 : 1;
    g.G = g.W == 2 ? pow2_ceil(C / 2) : std::min(32, pow2_ceil(C));
    g.lgG = ilog2(g.G);
    g.kb = p->kb;
    g.M = p->M;
    return g;
}

int gather_cpl(const GatherArgs& g) {
    if (g.W == 4) return kGatherQuads;
    if (g.W == 2) return 0;
    return (g.C + g.G - 1) / g.G;
}

int check_call(nufft_plan_s* p, int C) {
    if (!p) return fail(NUFFT_ERR_INVALID_ARG, "plan is NULL");
    if (C < 1 || C > p->maxC) return fail(NUFFT_ERR_INVALID_ARG, "C must lie in [1, max_coils]");
    return NUFFT_OK;
}

}  // namespace

// =========================================================================== C ABI
extern "C" {

void nufft_default_opts(nufft_opts* o, int dim, const int64_t* n) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->dim = dim;
    for (int d = 0; d < dim && d < 3 && n; ++d) o->n[d] = n[d];
    o->sigma = 2.0;
    o->J = 6;
    o->beta = 0.0;
    o->max_coils = 1;
}

size_t nufft_workspace_bytes(const nufft_opts* o, int64_t m, int C) {
    if (!o) return 0;
    nufft_opts oc = *o;
    if (C > 0) oc.max_coils = C;
    nufft_plan_s p;
    if (validate_opts(&oc, p) != NUFFT_OK) return 0;
    size_t G, T;
    workspace_elems(p, G, T);
    size_t b = (G + T) * sizeof(float2) + point_bytes(p, std::max<int64_t>(m, 1));
    b += (size_t)((4 + kNbrStride) * p.nbins + 2 * sort_keys(p) + 8) * sizeof(int) + strip_bytes(p);
    for (int d = 0; d < p.D; ++d) b += (size_t)p.N[d] * sizeof(float) + 2 * (size_t)p.K[d] * sizeof(float2);
    if (p.kernel_mode == NUFFT_KERNEL_TABLE) b += (size_t)(p.tab_n + 2) * sizeof(float);
    return b;
}

int nufft_plan(nufft_plan_t* out, const nufft_opts* o, int64_t m, const float* omega, void* stream) {
    if (!out) return fail(NUFFT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    nufft_plan_s* p = new (std::nothrow) nufft_plan_s();
    if (!p) return fail(NUFFT_ERR_OOM, "host allocation failed");
    int st = validate_opts(o, *p);
    if (st) { delete p; return st; }
    auto oom = [&](const char* what) {
        cudaGetLastError();
        free_plan(p);
        return fail(NUFFT_ERR_OOM, std::string("device allocation failed: ") + what);
    };
    // tables: scaling factors s_d[n] = 1 / psi_hat((n - N/2) / K) and twiddles
    for (int d = 0; d < p->D; ++d) {
        std::vector<float> dp(p->N[d]);
        for (int64_t n = 0; n < p->N[d]; ++n)
            dp[n] = (float)(1.0 / kb_ft((double)(n - p->N[d] / 2) / (double)p->K[d], p->J, p->beta));
        if (cudaMalloc(&p->d_deap[d], dp.size() * sizeof(float)) != cudaSuccess) return oom("scaling table");
        cudaMemcpy(p->d_deap[d], dp.data(), dp.size() * sizeof(float), cudaMemcpyHostToDevice);
        const int L = (int)p->K[d];
        int L1 = 0, L2 = 0;
        const bool two = fft2_factor(L, L1, L2);
        std::vector<float2> tw(2 * (size_t)L);
        auto unit = [&](int t) {
            const double ang = -2.0 * M_PI * (double)t / (double)L;
            return make_float2((float)std::cos(ang), (float)std::sin(ang));
        };
        for (int t = 0; t < L; ++t) tw[t] = unit(t);
        if (two)   // [n2][k1]: a thread's L1 - 1 twiddles sit at fixed offsets from its row
            for (int n2 = 0; n2 < L2; ++n2)
                for (int k1 = 0; k1 < L1; ++k1) tw[L + (size_t)n2 * L1 + k1] = unit(n2 * k1);
        if (cudaMalloc(&p->d_tw[d], tw.size() * sizeof(float2)) != cudaSuccess) return oom("twiddles");
        cudaMemcpy(p->d_tw[d], tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
        build_fft_axis(L, p->axis[d]);
        p->axis[d].tw = p->d_tw[d];
        p->axis[d].tw2 = p->d_tw[d] + L;
    }
    if (p->kernel_mode == NUFFT_KERNEL_TABLE) {
        // psi(l / L) for l = 0 .. n + 1 from the FP64 power series, zero from l = n = L J / 2 on
        std::vector<float> tab(p->tab_n + 2, 0.f);
        for (int l = 0; l < p->tab_n; ++l) tab[l] = (float)kb_psi_fp64((double)l / p->tab_L, p->J, p->beta);
        if (cudaMalloc(&p->d_kbtab, tab.size() * sizeof(float)) != cudaSuccess) return oom("kernel table");
        cudaMemcpy(p->d_kbtab, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (cudaMalloc(&p->d_kcount, sizeof(int) * sort_keys(*p)) != cudaSuccess ||
        cudaMalloc(&p->d_offsets, sizeof(int) * (sort_keys(*p) + 1)) != cudaSuccess ||
        cudaMalloc(&p->d_item_off, sizeof(int) * (p->nbins + 1)) != cudaSuccess ||
        cudaMalloc(&p->d_tile_parts, sizeof(int) * p->nbins) != cudaSuccess ||
        cudaMalloc(&p->d_heavy, sizeof(int) * (p->nbins + 1)) != cudaSuccess ||
        cudaMalloc(&p->d_tile_nbr, sizeof(int) * kNbrStride * p->nbins) != cudaSuccess ||
        cudaMalloc(&p->d_nitems, 2 * sizeof(int)) != cudaSuccess)
        return oom("bins");
    cudaMemset(p->d_nitems, 0, 2 * sizeof(int));
    if (p->strip) {
        const size_t nslot = (size_t)p->strip_slots * p->ncg_max;
        if (cudaMalloc(&p->d_partial, nslot * kStripW * 32 * sizeof(float4)) != cudaSuccess ||
            cudaMalloc(&p->d_counters, nslot * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&p->d_hcount, (size_t)p->nunits * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&p->d_hcur, (size_t)p->nunits * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&p->d_plan_sums, (size_t)strip_plan_blocks(p->nunits) * strip_plan_vals() * sizeof(int)) !=
                cudaSuccess ||
            cudaMalloc(&p->d_hoff, (size_t)(p->nunits + 1) * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&p->d_splits, (size_t)p->strip_slots * sizeof(int4)) != cudaSuccess)
            return oom("strip partial sums");
        cudaMemset(p->d_counters, 0, nslot * sizeof(int));
        cudaMemset(p->d_hcount, 0, (size_t)p->nunits * sizeof(int));
    }
    workspace_elems(*p, p->G_elems, p->T_elems);
    if (cudaMalloc(&p->d_G, p->G_elems * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&p->d_T, p->T_elems * sizeof(float2)) != cudaSuccess)
        return oom("workspace");
    // the sort is short and on the path to the first gather: its blocks go before queued FFT blocks
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
        cudaGetLastError();
        prio_hi = 0;
    }
    if (cudaStreamCreateWithPriority(&p->aux, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->join_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->join2_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->aux2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->fork2_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->done2_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return fail(NUFFT_ERR_CUDA, "stream or event creation failed");
    }
    if ((st = alloc_points(p, std::max<int64_t>(m, 1)))) { free_plan(p); return st; }
    if ((st = do_set_points(p, m, omega, (cudaStream_t)stream))) { free_plan(p); return st; }
    *out = p;
    return NUFFT_OK;
}

int nufft_set_points(nufft_plan_t p, int64_t m, const float* omega, void* stream) {
    if (!p) return fail(NUFFT_ERR_INVALID_ARG, "plan is NULL");
    return do_set_points(p, m, omega, (cudaStream_t)stream);
}

int nufft_sort_points(nufft_plan_t p, void* stream) {
    if (!p) return fail(NUFFT_ERR_INVALID_ARG, "plan is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    return finish_call(p, s, sort_rest(p, s));
}

int nufft_forward(nufft_plan_t p, int C, const nufft_cfloat* x, const nufft_cfloat* smaps, nufft_cfloat* y,
                  void* stream) {
    int st;
    if ((st = check_call(p, C))) return st;
    if (!x || (!y && p->M > 0)) return fail(NUFFT_ERR_INVALID_ARG, "x or y is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    if ((st = sort_rest(p, s))) return st;
    if (p->M == 0) return finish_call(p, s, NUFFT_OK);
    if ((st = forward_grids(p, C, 1, 1, (const float2*)x, (const float2*)smaps, s))) return st;
    if ((st = sort_join(p, s))) return st;
    GatherArgs g = gather_args(p, C, 1, 1);
    forward_quads(p, g);
    g.y = (float2*)y;
    const int cpl = gather_cpl(g);
    return finish_call(p, s, launch(p, PK_GATHER_FWD, s, [&] { return launch_gather(GM_FWD, g, cpl, s); }));
}

int nufft_adjoint(nufft_plan_t p, int C, const nufft_cfloat* y, const nufft_cfloat* smaps, nufft_cfloat* x,
                  void* stream) {
    int st;
    if ((st = check_call(p, C))) return st;
    if (!x || (!y && p->M > 0)) return fail(NUFFT_ERR_INVALID_ARG, "x or y is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    if ((st = sort_rest(p, s)) || (st = sort_join(p, s))) return st;
    return finish_call(p, s, adjoint_impl(p, C, (const float2*)y, (const float2*)smaps, (float2*)x, s));
}

int nufft_jvp_omega(nufft_plan_t p, int C, const nufft_cfloat* x, const nufft_cfloat* smaps, const float* domega,
                    nufft_cfloat* dy, nufft_cfloat* y_or_null, void* stream) {
    int st;
    if ((st = check_call(p, C))) return st;
    if (!x || (p->M > 0 && (!domega || !dy))) return fail(NUFFT_ERR_INVALID_ARG, "x, domega or dy is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    if ((st = sort_rest(p, s))) return st;
    if (p->M == 0) return finish_call(p, s, NUFFT_OK);
    const int hp = y_or_null ? 1 : 0;
    const int nd = p->D + hp;
    if ((st = forward_grids(p, C, nd, hp, (const float2*)x, (const float2*)smaps, s))) return st;
    if ((st = sort_join(p, s))) return st;
    GatherArgs g = gather_args(p, C, nd, hp);
    g.y = (float2*)y_or_null;
    g.dy = (float2*)dy;
    g.domega = domega;
    const int cpl = gather_cpl(g);
    return finish_call(p, s, launch(p, PK_GATHER_JVP, s, [&] { return launch_gather(GM_JVP, g, cpl, s); }));
}

// The two-stream VJP applies to 2-D strip plans with their own streams, with points, and with a
// last inverse pass that needs no partial coil sums (16 coils or fewer with maps: one block sums
// them all, or two 8-coil blocks add into the cleared image), whose buffer would be the one the
// omega chain uses.
bool dual_vjp(const nufft_plan_s* p, int C, bool maps) {
    return p->aux2 && p->strip && p->D == 2 && p->M > 0 && (!maps || C <= 16);
}

int nufft_vjp_omega_x(nufft_plan_t p, int C, const nufft_cfloat* x, const nufft_cfloat* smaps, const nufft_cfloat* v,
                      float* grad_omega, nufft_cfloat* grad_x, void* stream) {
    int st;
    if ((st = check_call(p, C))) return st;
    if ((p->M > 0 && !v) || (grad_omega && !x)) return fail(NUFFT_ERR_INVALID_ARG, "x or v is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    // With both outputs the gather also writes v in sorted point order into T (free once the
    // last forward pass has read it) for the adjoint's spread, which then needs no reorder pass.
    const float2* vsorted = nullptr;
    if ((st = sort_rest(p, s))) return st;
    if (grad_omega && grad_x && dual_vjp(p, C, smaps != nullptr)) {
        // grad_x on aux2 beside the omega-gradient chain on s: the adjoint's grid and intermediate
        // take the channel block that the D-channel forward grids leave free (the workspace holds
        // 1 + D channel blocks), so the two chains share no buffer
        const int64_t N0K1 = p->N[0] * p->K[1];
        float2* gbuf = p->d_G + (size_t)p->Ktot * C * p->D;
        float2* tbuf = p->d_T + (size_t)N0K1 * C * p->D;
        NJ_CUDA(cudaEventRecord(p->fork2_ev, s));
        NJ_CUDA(cudaStreamWaitEvent(p->aux2, p->fork2_ev, 0));
        // the sorted points and the strip tables, when they come from a sort of this call
        if (p->join2_pending) NJ_CUDA(cudaStreamWaitEvent(p->aux2, p->join2_ev, 0));
        else if (p->join_pending) NJ_CUDA(cudaStreamWaitEvent(p->aux2, p->join_ev, 0));
        if ((st = adjoint_impl(p, C, (const float2*)v, (const float2*)smaps, (float2*)grad_x, p->aux2, nullptr,
                               gbuf, tbuf)))
            return st;
        NJ_CUDA(cudaEventRecord(p->done2_ev, p->aux2));
        if ((st = forward_grids(p, C, p->D, 0, (const float2*)x, (const float2*)smaps, s))) return st;
        if ((st = sort_join(p, s))) return st;
        GatherArgs g = gather_args(p, C, p->D, 0);
        g.v = (const float2*)v;
        g.grad = grad_omega;
        const int cpl = gather_cpl(g);
        if ((st = launch(p, PK_GATHER_VJP, s, [&] { return launch_gather(GM_VJP, g, cpl, s); }))) return st;
        NJ_CUDA(cudaStreamWaitEvent(s, p->done2_ev, 0));
        return finish_call(p, s, NUFFT_OK);
    }
    if (grad_omega && p->M > 0) {
        if ((st = forward_grids(p, C, p->D, 0, (const float2*)x, (const float2*)smaps, s))) return st;
        if ((st = sort_join(p, s))) return st;
        GatherArgs g = gather_args(p, C, p->D, 0);
        g.v = (const float2*)v;
        g.grad = grad_omega;
        if (grad_x && p->strip) {
            g.v_sorted = p->d_ys;
            g.v_sorted_cpt = 64 / p->NSL;
            vsorted = p->d_ys;
        } else if (grad_x && p->cell_spread && (size_t)C * (size_t)p->M <= p->T_elems) {
            g.v_sorted = p->d_T;
            vsorted = p->d_T;
        }
        const int cpl = gather_cpl(g);
        if ((st = launch(p, PK_GATHER_VJP, s, [&] { return launch_gather(GM_VJP, g, cpl, s); }))) return st;
    }
    if ((st = sort_join(p, s))) return st;
    if (grad_x) st = adjoint_impl(p, C, (const float2*)v, (const float2*)smaps, (float2*)grad_x, s, vsorted);
    return finish_call(p, s, st);
}

int nufft_get_info(nufft_plan_t p, nufft_plan_info* info) {
    if (!p || !info) return fail(NUFFT_ERR_INVALID_ARG, "plan or info is NULL");
    std::memset(info, 0, sizeof(*info));
    info->dim = p->D;
    for (int d = 0; d < 3; ++d) {
        info->n[d] = d < p->D ? p->N[d] : 1;
        info->k[d] = d < p->D ? p->K[d] : 1;
        info->bin_size[d] = d < p->D ? p->B[d] : 1;
    }
    info->J = p->J;
    info->sigma = p->sigma;
    info->beta = p->beta;
    info->m = p->M;
    info->nbins = p->nbins;
    info->max_coils = p->maxC;
    info->workspace_bytes = (p->G_elems + p->T_elems) * sizeof(float2) + point_bytes(*p, p->M_cap) + strip_bytes(*p);
    return NUFFT_OK;
}

void nufft_destroy(nufft_plan_t p) {
    if (!p) return;
    if (p->last_stream) cudaStreamSynchronize(p->last_stream);
    else cudaDeviceSynchronize();
    if (p->aux) cudaStreamSynchronize(p->aux);
    free_plan(p);
}

const char* nufft_status_string(int status) {
    switch (status) {
        case NUFFT_OK: return "ok";
        case NUFFT_ERR_INVALID_ARG: return "invalid argument";
        case NUFFT_ERR_UNSUPPORTED: return "unsupported configuration";
        case NUFFT_ERR_OOM: return "out of device memory";
        case NUFFT_ERR_CUDA: return "CUDA error";
        case NUFFT_ERR_TIMEOUT: return "device wait timed out";
        default: return "unknown status";
    }
}

const char* nufft_last_error(void) { return g_last_error.c_str(); }

int64_t nufft_launch_count(void) { return g_launches.load(); }

int nufft_profile_enable(nufft_plan_t p, int enable) {
    if (!p) return fail(NUFFT_ERR_INVALID_ARG, "plan is NULL");
    p->prof = enable != 0;
    return NUFFT_OK;
}

int nufft_profile_read(nufft_plan_t p, int max_kinds, const char** names, int* launches, double* total_ms,
                       int* n_kinds) {
    if (!p) return fail(NUFFT_ERR_INVALID_ARG, "plan is NULL");
    int cnt[PK_COUNT] = {0};
    double ms[PK_COUNT] = {0};
    for (auto& e : p->events) {
        cudaError_t r = cudaEventSynchronize(e.b);
        if (r != cudaSuccess) return fail(NUFFT_ERR_CUDA, std::string("event sync: ") + cudaGetErrorString(r));
        float t = 0.f;
        cudaEventElapsedTime(&t, e.a, e.b);
        cnt[e.kind] += 1;
        ms[e.kind] += t;
        p->pool.push_back(e.a);
        p->pool.push_back(e.b);
    }
    p->events.clear();
    int k = 0;
    for (int i = 0; i < PK_COUNT; ++i) {
        if (!cnt[i]) continue;
        if (k < max_kinds) {
            if (names) names[k] = kProfNames[i];
            if (launches) launches[k] = cnt[i];
            if (total_ms) total_ms[k] = ms[i];
        }
        ++k;
    }
    if (n_kinds) *n_kinds = k;
    return NUFFT_OK;
}

}  // extern "C"

// ============================================================ allocation-free forward
// nufft_forward_noalloc: the forward NUFFT without a plan and without any
// device allocation.  For callers that cannot call cudaMalloc: code that runs
// under a device-memory budget owned by another allocator (a framework's
// caching allocator, a real-time or embedded service with a fixed footprint),
// or that must not allocate while it runs.  All scratch (tables, bin sort,
// FFT workspace) is carved from one file-scope device array of
// NUFFT_NOALLOC_SCRATCH_BYTES; every GPU that loads this library holds it
// until the process exits.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[NUFFT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once
// per device, with that device current).
int noalloc_scratch(void** out) {
    int dev = 0;
    NJ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(NUFFT_ERR_UNSUPPORTED, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(NUFFT_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return NUFFT_OK;
}

// Scaling factors s[n] = 1 / psi_hat((n - N/2) / K) (the Kaiser-Bessel transform in closed form, FP64)
// and twiddles exp(-2 pi i t / L) of one axis, written into the scratch array on the device, so that
// the call copies nothing from host memory.
__global__ void k_noalloc_tables(float* deap, int64_t N, int64_t K, int J, double beta, float2* tw, int L, int L1) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const double f = (double)(i - N / 2) / (double)K;
        const double x = M_PI * J * f;
        const double q = beta * beta - x * x;
        double ft = J;
        if (q > 0) ft = J * sinh(sqrt(q)) / sqrt(q);
        else if (q < 0) ft = J * sin(sqrt(-q)) / sqrt(-q);
        deap[i] = (float)(1.0 / ft);
    }
    if (i < L) {
        double sn, cs;
        sincospi(-2.0 * (double)i / (double)L, &sn, &cs);
        tw[i] = make_float2((float)cs, (float)sn);
        if (L1 > 0) {   // the two-phase table [n2][k1] = exp(-2 pi i n2 k1 / L), behind the linear one
            const int n2 = (int)i / L1, k1 = (int)i - n2 * L1;
            sincospi(-2.0 * (double)(n2 * k1) / (double)L, &sn, &cs);
            tw[L + i] = make_float2((float)cs, (float)sn);
        }
    }
}

struct Carve {
    size_t off = 0;
    template <typename T>
    size_t take(size_t n) {
        const size_t at = off;
        off = (off + n * sizeof(T) + 255) / 256 * 256;
        return at;
    }
};

}  // namespace

extern "C" int nufft_forward_noalloc(const nufft_opts* o, int64_t m, const float* omega, int C,
                                     const nufft_cfloat* x, const nufft_cfloat* smaps, nufft_cfloat* y,
                                     void* stream) {
    nufft_plan_s p;   // host-side description only; every device pointer below is scratch
    int st = validate_opts(o, p);
    if (st) return st;
    p.strip = false;   // forward only: the bin sort without the adjoint's strip tables
    if (p.kernel_mode != NUFFT_KERNEL_DIRECT)
        return fail(NUFFT_ERR_UNSUPPORTED, "nufft_forward_noalloc evaluates the kernel directly only");
    p.wd = p.J;
    p.ws = (p.D * p.J + 3) & ~3;
    if (C < 1 || C > NUFFT_MAX_COILS) return fail(NUFFT_ERR_INVALID_ARG, "C must lie in [1, 128]");
    if (m < 0 || m > (int64_t)INT32_MAX) return fail(NUFFT_ERR_INVALID_ARG, "m out of range");
    if (m > 0 && (!omega || !x || !y)) return fail(NUFFT_ERR_INVALID_ARG, "omega, x or y is NULL");
    p.maxC = C;
    // forward workspace for C channels: the pass over dim d leaves [N_0..N_{d-1}][K_d..][C]
    size_t G = (size_t)p.Ktot * C, T = 1;
    for (int d = p.D - 1; d >= 0; --d) {
        int64_t n = C;
        for (int e = 0; e < d; ++e) n *= p.N[e];
        for (int e = d; e < p.D; ++e) n *= p.K[e];
        if (d % 2) T = std::max<size_t>(T, (size_t)n);
        else G = std::max<size_t>(G, (size_t)n);
    }
    const int64_t mc = std::max<int64_t>(m, 1);
    Carve cv;
    size_t o_deap[3], o_tw[3];
    for (int d = 0; d < p.D; ++d) {
        o_deap[d] = cv.take<float>(p.N[d]);
        o_tw[d] = cv.take<float2>(2 * p.K[d]);
    }
    const size_t o_kcount = cv.take<int>(p.nbins),
                 o_offsets = cv.take<int>(p.nbins + 1),
                 o_item_off = cv.take<int>(p.nbins + 1), o_tile_parts = cv.take<int>(p.nbins),
                 o_heavy = cv.take<int>(p.nbins + 1),
                 o_tile_nbr = cv.take<int>((size_t)kNbrStride * p.nbins),
                 o_nitems = cv.take<int>(1), o_items = cv.take<int4>(max_items(p, mc)), o_local = cv.take<int>(mc),
                 o_keyid = cv.take<int>(mc), o_pidx = cv.take<int4>(mc), o_pfrac = cv.take<float4>(mc),
                 o_pw = cv.take<float>((size_t)mc * p.ws),
                 o_om = cv.take<float>((size_t)mc * p.D),
                 o_G = cv.take<float2>(G), o_T = cv.take<float2>(T);
    if (cv.off > (size_t)NUFFT_NOALLOC_SCRATCH_BYTES)
        return fail(NUFFT_ERR_UNSUPPORTED, "problem needs " + std::to_string(cv.off) +
                                               " bytes of scratch; nufft_forward_noalloc is limited to " +
                                               std::to_string((size_t)NUFFT_NOALLOC_SCRATCH_BYTES));
    void* base = nullptr;
    if ((st = noalloc_scratch(&base))) return st;
    unsigned char* b = (unsigned char*)base;
    cudaStream_t s = (cudaStream_t)stream;
    // tables, computed in FP64 on the device into the scratch array (nothing is copied from the host)
    for (int d = 0; d < p.D; ++d) {
        const int L = (int)p.K[d];
        p.d_deap[d] = (float*)(b + o_deap[d]);
        p.d_tw[d] = (float2*)(b + o_tw[d]);
        int L1 = 0, L2 = 0;
        if (!fft2_factor(L, L1, L2)) L1 = 0;
        const int64_t n = std::max<int64_t>(p.N[d], L);
        NJ_CUDA(launch_pdl(k_noalloc_tables, (unsigned)((n + 255) / 256), 256, 0, s, p.d_deap[d], p.N[d], p.K[d], p.J,
                           p.beta, p.d_tw[d], L, L1));
        build_fft_axis(L, p.axis[d]);
        p.axis[d].tw = p.d_tw[d];
        p.axis[d].tw2 = p.d_tw[d] + L;
    }
    p.d_kcount = (int*)(b + o_kcount);
    p.d_offsets = (int*)(b + o_offsets);
    p.d_item_off = (int*)(b + o_item_off);
    p.d_tile_parts = (int*)(b + o_tile_parts);
    p.d_heavy = (int*)(b + o_heavy);
    p.d_tile_nbr = (int*)(b + o_tile_nbr);
    p.d_nitems = (int*)(b + o_nitems);
    p.d_items = (int4*)(b + o_items);
    p.d_local = (int*)(b + o_local);
    p.d_keyid = (int*)(b + o_keyid);
    p.d_pidx = (int4*)(b + o_pidx);
    p.d_pfrac = (float4*)(b + o_pfrac);
    p.d_pw = (float*)(b + o_pw);
    p.d_om = (float*)(b + o_om);
    p.d_G = (float2*)(b + o_G);
    p.d_T = (float2*)(b + o_T);
    p.G_elems = G;
    p.T_elems = T;
    p.M_cap = mc;   // capacity is the scratch slice: the sort never reallocates
    // the bin sort zeroes its own counters; every workspace element is written before it is read
    if ((st = do_set_points(&p, m, omega, s))) return st;
    if (m == 0) return NUFFT_OK;
    if ((st = forward_grids(&p, C, 1, 1, (const float2*)x, (const float2*)smaps, s))) return st;
    GatherArgs g = gather_args(&p, C, 1, 1);
    forward_quads(&p, g);
    g.y = (float2*)y;
    const int cpl = gather_cpl(g);
    return launch(&p, PK_GATHER_FWD, s, [&] { return launch_gather(GM_FWD, g, cpl, s); });
}

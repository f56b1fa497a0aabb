// In-register DFTs of the line-FFT kernels.
//
// Dft<R, DIR>: hand-written R-point butterflies (R = 2, 3, 4, 5, 8, 16) with
// exp(DIR 2 pi i n k / R).  dft<N, DIR>: any 2,3,5-smooth N as a compile-time
// Cooley-Tukey split N = R M (decimation in time): M-point DFTs of the R
// decimated subsequences, twiddles W_N^(r k2) folded to immediates, then
// R-point butterflies; X[k2 + M k1] = sum_r W_R^(r k1) W_N^(r k2) Y_r[k2].
#pragma once
#include <type_traits>

#include "common.cuh"

namespace nj {

template <int DIR>
__device__ __forceinline__ float2 mul_si(float2 z) {   // (DIR * i) * z
    return DIR < 0 ? make_float2(z.y, -z.x) : make_float2(-z.y, z.x);
}

// In-register R-point DFT with exp(DIR * 2 pi i n k / R).
template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(float2* a) {
        const float2 t = a[1];
        a[1] = csub(a[0], t);
        a[0] = cadd(a[0], t);
    }
};

template <int DIR>
struct Dft<4, DIR> {
    __device__ __forceinline__ static void run(float2* a) {
        const float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        const float2 t2 = cadd(a[1], a[3]), t3 = mul_si<DIR>(csub(a[1], a[3]));
        a[0] = cadd(t0, t2);
        a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3);
        a[3] = csub(t1, t3);
    }
};

template <int DIR>
struct Dft<8, DIR> {
    __device__ __forceinline__ static void run(float2* a) {
        float2 e[4] = {a[0], a[2], a[4], a[6]};
        float2 o[4] = {a[1], a[3], a[5], a[7]};
        Dft<4, DIR>::run(e);
        Dft<4, DIR>::run(o);
        const float h = 0.70710678118654752f;
        // o[k] *= exp(DIR 2 pi i k / 8)
        o[1] = make_float2(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
        o[2] = mul_si<DIR>(o[2]);
        o[3] = make_float2(h * (-o[3].x - DIR * o[3].y), h * (-o[3].y + DIR * o[3].x));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            a[k] = cadd(e[k], o[k]);
            a[k + 4] = csub(e[k], o[k]);
        }
    }
};

template <int DIR>
struct Dft<3, DIR> {
    __device__ __forceinline__ static void run(float2* a) {
        const float s3 = 0.86602540378443865f;   // sin(2 pi / 3)
        const float2 t1 = cadd(a[1], a[2]);
        const float2 t2 = cscale(mul_si<DIR>(csub(a[1], a[2])), s3);
        const float2 m = make_float2(a[0].x - 0.5f * t1.x, a[0].y - 0.5f * t1.y);
        a[0] = cadd(a[0], t1);
        a[1] = cadd(m, t2);
        a[2] = csub(m, t2);
    }
};

template <int DIR>
struct Dft<5, DIR> {
    __device__ __forceinline__ static void run(float2* a) {
        const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;   // cos(2pi/5), cos(4pi/5)
        const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;    // sin(2pi/5), sin(4pi/5)
        const float2 b1 = cadd(a[1], a[4]), b2 = cadd(a[2], a[3]);
        const float2 d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
        const float2 m1 = make_float2(a[0].x + c1 * b1.x + c2 * b2.x, a[0].y + c1 * b1.y + c2 * b2.y);
        const float2 m2 = make_float2(a[0].x + c2 * b1.x + c1 * b2.x, a[0].y + c2 * b1.y + c1 * b2.y);
        const float2 n1 = mul_si<DIR>(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
        const float2 n2 = mul_si<DIR>(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
        a[0] = cadd(a[0], cadd(b1, b2));
        a[1] = cadd(m1, n1);
        a[4] = csub(m1, n1);
        a[2] = cadd(m2, n2);
        a[3] = csub(m2, n2);
    }
};

template <int DIR>
struct Dft<16, DIR> {
    // 16 = 4 x 4: DFT4 over n1 for each n2, twiddle W16^(n2 k1), DFT4 over n2 for each k1.
    __device__ __forceinline__ static void run(float2* a) {
        const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
        // W16^m = (cos 2pi m/16, DIR sin 2pi m/16) for m = 0..9
        const float wc[10] = {1.f, c1, h, s1, 0.f, -s1, -h, -c1, -1.f, -c1};
        const float ws[10] = {0.f, s1, h, c1, 1.f, c1, h, s1, 0.f, -s1};
        float2 b[4][4];
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) {
            float2 t[4] = {a[n2], a[4 + n2], a[8 + n2], a[12 + n2]};
            Dft<4, DIR>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < 4; ++k1) {
                const int m = n2 * k1;
                if (m == 0) b[n2][k1] = t[k1];
                else b[n2][k1] = cmul(t[k1], make_float2(wc[m], DIR * ws[m]));
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 t[4] = {b[0][k1], b[1][k1], b[2][k1], b[3][k1]};
            Dft<4, DIR>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = t[k2];
        }
    }
};

// Calls f(integral_constant<int, I>) for I = B .. E-1 (indices stay compile-time).
template <int B, int E, typename F>
__device__ __forceinline__ void sfor(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

// cos and sin of 2 pi e / n, evaluated by the compiler (argument reduced to
// (-pi, pi], then the Taylor series to order 39: error below 1e-16).
struct CosSin {
    double c, s;
};
__host__ __device__ constexpr CosSin cis_turns(int e, int n) {
    const double two_pi = 6.283185307179586476925286766559;
    int r = e % n;
    if (r < 0) r += n;
    double x = two_pi * r / n;
    if (2 * r > n) x -= two_pi;
    const double x2 = x * x;
    double tc = 1.0, ts = x, c = 1.0, s = x;
    for (int k = 1; k < 20; ++k) {
        tc *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
        ts *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
        c += tc;
        s += ts;
    }
    return CosSin{c, s};
}

// z * W_N^E, W_N = exp(DIR 2 pi i / N); quarter turns are exact swaps.
template <int N, int DIR, int E>
__device__ __forceinline__ float2 twiddle_const(float2 z) {
    constexpr int e = ((E % N) + N) % N;
    if constexpr (e == 0) {
        return z;
    } else if constexpr (4 * e == N) {
        return mul_si<DIR>(z);
    } else if constexpr (2 * e == N) {
        return make_float2(-z.x, -z.y);
    } else if constexpr (4 * e == 3 * N) {
        return mul_si<-DIR>(z);
    } else {
        constexpr CosSin w = cis_turns(e, N);
        constexpr float c = (float)w.c, s = (float)(DIR * w.s);
        return make_float2(fmaf(z.x, c, -z.y * s), fmaf(z.x, s, z.y * c));
    }
}

template <int N>
struct DftSplit {
    static constexpr bool base = N == 2 || N == 3 || N == 4 || N == 5 || N == 8 || N == 16;
    static constexpr int R = base ? N : (N % 4 == 0 ? 4 : (N % 2 == 0 ? 2 : (N % 3 == 0 ? 3 : 5)));
    static constexpr int M = N / R;
};

template <int N, int DIR>
__device__ __forceinline__ void dft(float2* a) {
    if constexpr (N == 1) {
        return;
    } else if constexpr (DftSplit<N>::base) {
        Dft<N, DIR>::run(a);
    } else {
        constexpr int R = DftSplit<N>::R, M = DftSplit<N>::M;
        static_assert(R * M == N && (M % 2 == 0 || M % 3 == 0 || M % 5 == 0 || M == 1), "N must be 2,3,5-smooth");
        float2 y[R][M];
        sfor<0, R>([&](auto r_) {
            constexpr int r = decltype(r_)::value;
            sfor<0, M>([&](auto m_) {
                constexpr int m = decltype(m_)::value;
                y[r][m] = a[R * m + r];
            });
            dft<M, DIR>(y[r]);
        });
        sfor<0, M>([&](auto k2_) {
            constexpr int k2 = decltype(k2_)::value;
            float2 t[R];
            sfor<0, R>([&](auto r_) {
                constexpr int r = decltype(r_)::value;
                t[r] = twiddle_const<N, DIR, r * k2>(y[r][k2]);
            });
            Dft<R, DIR>::run(t);
            sfor<0, R>([&](auto k1_) {
                constexpr int k1 = decltype(k1_)::value;
                a[k2 + M * k1] = t[k1];
            });
        });
    }
}

}  // namespace nj

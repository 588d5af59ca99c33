// Compile-time helpers for in-register DFTs: unrolled loops, twiddle constants
// and an in-register radix-2 decimation-in-frequency FFT.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace corr {

// ------------------------------------------------------------------ compile-time trig
// cos / sin of 2 pi j / L, evaluated at compile time from their Taylor series after
// reducing the angle to [-pi/4, pi/4] by quadrant (exact integer arithmetic).
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int n = 1; n < 14; ++n) {
        term *= -x2 / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}

constexpr double taylor_cos(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int n = 1; n < 14; ++n) {
        term *= -x2 / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}

// angle 2 pi j / L = 2 pi (4 j - q L) / (4 L) + q pi / 2 with q = round(4 j / L)
constexpr int quad_of(int j, int L) { return (8 * j + L) / (2 * L); }  // j in [0, L)

constexpr double cos2pi(int j, int L) {
    int jj = ((j % L) + L) % L;
    int q = quad_of(jj, L);
    double r = 2.0 * kPi * (double)(4 * jj - q * L) / (4.0 * L);
    switch (q & 3) {
        case 0: return taylor_cos(r);
        case 1: return -taylor_sin(r);
        case 2: return -taylor_cos(r);
        default: return taylor_sin(r);
    }
}

constexpr double sin2pi(int j, int L) {
    int jj = ((j % L) + L) % L;
    int q = quad_of(jj, L);
    double r = 2.0 * kPi * (double)(4 * jj - q * L) / (4.0 * L);
    switch (q & 3) {
        case 0: return taylor_sin(r);
        case 1: return taylor_cos(r);
        case 2: return -taylor_sin(r);
        default: return -taylor_cos(r);
    }
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

constexpr int bitrev(int x, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((x >> b) & 1) << (bits - 1 - b);
    return r;
}

// ------------------------------------------------------------------ unrolled loops
template <int B, int E, class F>
__device__ __forceinline__ void sfor(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

// ------------------------------------------------------------------ packed FP32 pairs
// Blackwell's add/sub/mul.f32x2 operate on both components of a float2 with one
// instruction (same per-lane FP32 throughput, half the issue slots).
__device__ __forceinline__ unsigned long long f2_pack(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)));
    return f2_unpack(r);
}

__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_pack(a)), "l"(f2_pack(b)), "l"(f2_pack(c)));
    return f2_unpack(r);
}

// v * W_L^J with W_L = exp(-j 2 pi / L); trivial factors cost no multiply.
template <int J, int L>
__device__ __forceinline__ float2 mul_w(float2 v) {
    constexpr int Jr = J % L;
    if constexpr (Jr == 0) {
        return v;
    } else if constexpr (4 * Jr == L) {
        return make_float2(v.y, -v.x);  // * (-j)
    } else if constexpr (2 * Jr == L) {
        return make_float2(-v.x, -v.y);  // * (-1)
    } else if constexpr (4 * Jr == 3 * L) {
        return make_float2(-v.y, v.x);  // * (+j)
    } else {
        constexpr float c = (float)cos2pi(Jr, L);
        constexpr float s = (float)sin2pi(Jr, L);
        // (x + j y)(c - j s) = (x c + y s) + j (y c - x s)
        return make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -(v.x * s)));
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -(a.y * b.y)), fmaf(a.x, b.y, a.y * b.x));
}

// In-register P-point DFT (Eq. 1 on P points) of v[0 .. P-1], radix-2 decimation in
// frequency (v may hold more than P values), from stage S0 on (S0 = 0: the whole
// transform; S0 = 1 when the caller has done the first stage). On return v[bitrev(k)]
// holds X[k].
template <int P, int L, int S0 = 0>
__device__ __forceinline__ void fft_dif(float2 (&v)[L]) {
    static_assert(P <= L, "DFT longer than the register array");
    constexpr int LG = ilog2(P);
    sfor<S0, LG>([&](auto S) {
        constexpr int half = P >> (decltype(S)::value + 1);
        constexpr int len = 2 * half;
        sfor<0, P / len>([&](auto Bk) {
            sfor<0, half>([&](auto J) {
                constexpr int a = decltype(Bk)::value * len + decltype(J)::value;
                constexpr int b = a + half;
                const float2 x = v[a], y = v[b];
                v[a] = f2_add(x, y);
                v[b] = mul_w<decltype(J)::value, len>(f2_sub(x, y));
            });
        });
    });
}

}  // namespace corr

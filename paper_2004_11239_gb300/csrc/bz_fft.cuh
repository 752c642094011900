// Register-resident mixed-radix (4, 2, 3) FFTs of compile-time length N in FP32.
//
// One thread transforms one length-N line held in registers: a decimation-in-frequency
// recursion N = R * (N / R) with radix-4, -2 or -3 butterflies; every index is a
// compile-time constant after unrolling, so the line stays in registers and the
// output digit reversal is register renaming.  Twiddles exp(+-2 pi i j / N) come from
// a __constant__ table built at compile time from a Taylor series of sin and cos
// (octant-reduced), so they are FFMA constant-bank operands.
//
// fft_inplace<N, SIGN>(x): x[k] <- sum_j x[j] exp(SIGN 2 pi i j k / N), unnormalised.
#pragma once

#include <cuda_runtime.h>

namespace bz {

struct TwCS { double c, s; };

constexpr double kPiD = 3.14159265358979323846264338327950288;

// Taylor series on [0, pi/4]: 14 terms are far below double rounding there.
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

// (cos, sin) of 2 pi j / N for N divisible by 8, reduced to an octant by integer math.
constexpr TwCS unit_root(int j, int N) {
    j = ((j % N) + N) % N;
    int e = 8 * j;
    int o = e / N;                      // octant
    int rem = e % N;                    // position inside the octant, in units of (pi/4)/N
    double t = (kPiD / 4.0) * rem / N;
    double tp = (kPiD / 4.0) * (N - rem) / N;   // pi/4 - t
    double c = taylor_cos(t), s = taylor_sin(t);
    double cp = taylor_cos(tp), sp = taylor_sin(tp);
    switch (o) {
        case 0: return {c, s};
        case 1: return {sp, cp};
        case 2: return {-s, c};
        case 3: return {-cp, sp};
        case 4: return {-c, -s};
        case 5: return {-sp, -cp};
        case 6: return {s, -c};
        default: return {cp, -sp};
    }
}

// Table layout: lengths 8, 16, 24, 32, 48, 64 back to back.
template <int N> __host__ __device__ constexpr int tw_off() {
    static_assert(N == 8 || N == 16 || N == 24 || N == 32 || N == 48 || N == 64 || N == 4 ||
                  N == 2 || N == 12 || N == 6 || N == 3 || N == 1, "unsupported FFT length");
    return N == 8 ? 0 : N == 16 ? 8 : N == 24 ? 24 : N == 32 ? 48 : N == 48 ? 80 :
           N == 64 ? 128 : N == 12 ? 192 : N == 6 ? 204 : N == 4 ? 210 : N == 3 ? 214 :
           N == 2 ? 217 : 219;
}
constexpr int kTwTotal = 220;

struct TwTable { float2 v[kTwTotal]; };

constexpr TwTable make_tw_table() {
    TwTable t{};
    const int lens[12] = {8, 16, 24, 32, 48, 64, 12, 6, 4, 3, 2, 1};
    const int offs[12] = {0, 8, 24, 48, 80, 128, 192, 204, 210, 214, 217, 219};
    for (int a = 0; a < 12; ++a) {
        int N = lens[a];
        for (int j = 0; j < N; ++j) {
            // lengths not divisible by 8: evaluate 2 pi j / N as 2 pi (j * 8L/N) / (8L), L = lcm
            TwCS cs = unit_root(j * (192 / N), 192);
            t.v[offs[a] + j].x = (float)cs.c;
            t.v[offs[a] + j].y = (float)cs.s;
        }
    }
    return t;
}

static __constant__ TwTable c_tw = make_tw_table();

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// multiply by SIGN * i
template <int SIGN> __device__ __forceinline__ float2 mul_i(float2 a) {
    return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int N, int SIGN> __device__ __forceinline__ void mul_tw(float2 &v, int j) {
    // j is a compile-time constant after unrolling; trivial roots skip the multiply
    if (j == 0) return;
    if (4 * j == N) { v = mul_i<SIGN>(v); return; }
    if (2 * j == N) { v = make_float2(-v.x, -v.y); return; }
    if (4 * j == 3 * N) { v = mul_i<-SIGN>(v); return; }
    float2 w = c_tw.v[tw_off<N>() + j];
    if (SIGN < 0) w.y = -w.y;
    v = cmul(v, w);
}

template <int SIGN> __device__ __forceinline__ void bfly2(float2 &a, float2 &b) {
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int SIGN> __device__ __forceinline__ void bfly4(float2 &a, float2 &b, float2 &c, float2 &d) {
    float2 s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = mul_i<SIGN>(csub(b, d));
    a = cadd(s0, s1);
    c = csub(s0, s1);
    b = cadd(d0, d1);
    d = csub(d0, d1);
}

template <int SIGN> __device__ __forceinline__ void bfly3(float2 &a, float2 &b, float2 &c) {
    const float h = 0.86602540378443864676f;   // sqrt(3)/2
    float2 t1 = cadd(b, c), t2 = csub(b, c);
    float2 m = make_float2(a.x - 0.5f * t1.x, a.y - 0.5f * t1.y);
    float2 r = mul_i<SIGN>(make_float2(h * t2.x, h * t2.y));
    a = cadd(a, t1);
    b = cadd(m, r);
    c = csub(m, r);
}

template <int N> __host__ __device__ constexpr int first_radix() {
    return (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 3);
}

// In-place DIF on x[0], x[S], ..., x[(N-1) S]; output in digit-reversed slots.
template <int N, int SIGN, int S> __device__ __forceinline__ void dif(float2 *x) {
    if constexpr (N > 1) {
        constexpr int R = first_radix<N>();
        constexpr int M = N / R;
        #pragma unroll
        for (int nm = 0; nm < M; ++nm) {
            if constexpr (R == 4) bfly4<SIGN>(x[S * nm], x[S * (nm + M)], x[S * (nm + 2 * M)], x[S * (nm + 3 * M)]);
            else if constexpr (R == 2) bfly2<SIGN>(x[S * nm], x[S * (nm + M)]);
            else bfly3<SIGN>(x[S * nm], x[S * (nm + M)], x[S * (nm + 2 * M)]);
            #pragma unroll
            for (int kr = 1; kr < R; ++kr) mul_tw<N, SIGN>(x[S * (nm + M * kr)], nm * kr);
        }
        #pragma unroll
        for (int kr = 0; kr < R; ++kr) dif<M, SIGN, S>(x + S * M * kr);
    }
}

// Slot holding frequency k after dif<N>: frequency k = R k_m + k_r sits at M k_r + slot_M(k_m).
template <int N> __host__ __device__ constexpr int slot_of(int k) {
    if constexpr (N == 1) {
        return 0;
    } else {
        constexpr int R = first_radix<N>();
        constexpr int M = N / R;
        return M * (k % R) + slot_of<M>(k / R);
    }
}

template <int N, int SIGN> __device__ __forceinline__ void fft_inplace(float2 (&x)[N]) {
    dif<N, SIGN, 1>(x);
    float2 y[N];
    #pragma unroll
    for (int k = 0; k < N; ++k) y[k] = x[slot_of<N>(k)];
    #pragma unroll
    for (int k = 0; k < N; ++k) x[k] = y[k];
}

}  // namespace bz

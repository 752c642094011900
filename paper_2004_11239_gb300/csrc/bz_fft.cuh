// Register-resident mixed-radix (4, 2, 3) FFTs of compile-time length N in FP32 (float2)
// or FP64 (double2).
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
struct TwTableD { double2 v[kTwTotal]; };

constexpr TwTableD make_tw_table_d() {
    TwTableD t{};
    const int lens[12] = {8, 16, 24, 32, 48, 64, 12, 6, 4, 3, 2, 1};
    const int offs[12] = {0, 8, 24, 48, 80, 128, 192, 204, 210, 214, 217, 219};
    for (int a = 0; a < 12; ++a) {
        int N = lens[a];
        for (int j = 0; j < N; ++j) {
            TwCS cs = unit_root(j * (192 / N), 192);
            t.v[offs[a] + j].x = cs.c;
            t.v[offs[a] + j].y = cs.s;
        }
    }
    return t;
}

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

// Double-float numbers: an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2
// (Dekker 1971; Knuth's TwoSum, FMA-based TwoProduct).  About 48 significant bits on the
// FP32 pipes.  _rn intrinsics keep the compiler from contracting the error-free steps.
struct ff { float hi, lo; };
struct cff { ff x, y; };

struct TwTableFF { cff v[kTwTotal]; };

constexpr TwTableFF make_tw_table_ff() {
    TwTableFF t{};
    const int lens[12] = {8, 16, 24, 32, 48, 64, 12, 6, 4, 3, 2, 1};
    const int offs[12] = {0, 8, 24, 48, 80, 128, 192, 204, 210, 214, 217, 219};
    for (int a = 0; a < 12; ++a) {
        int N = lens[a];
        for (int j = 0; j < N; ++j) {
            TwCS cs = unit_root(j * (192 / N), 192);
            float ch = (float)cs.c, sh = (float)cs.s;
            t.v[offs[a] + j].x.hi = ch;
            t.v[offs[a] + j].x.lo = (float)(cs.c - (double)ch);
            t.v[offs[a] + j].y.hi = sh;
            t.v[offs[a] + j].y.lo = (float)(cs.s - (double)sh);
        }
    }
    return t;
}

static __constant__ TwTable c_tw = make_tw_table();
static __constant__ TwTableD c_twd = make_tw_table_d();
static __constant__ TwTableFF c_twff = make_tw_table_ff();

__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {   // |a| >= |b|
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    ff t = ff_two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = ff_fast_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return ff_fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_from(double d) {
    float h = (float)d;
    return {h, (float)(d - (double)h)};
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ double2 cneg(double2 a) { return make_double2(-a.x, -a.y); }
__device__ __forceinline__ cff cadd(cff a, cff b) { return {ff_add(a.x, b.x), ff_add(a.y, b.y)}; }
__device__ __forceinline__ cff csub(cff a, cff b) { return {ff_add(a.x, ff_neg(b.x)), ff_add(a.y, ff_neg(b.y))}; }
__device__ __forceinline__ cff cmul(cff a, cff b) {
    return {ff_add(ff_mul(a.x, b.x), ff_neg(ff_mul(a.y, b.y))), ff_add(ff_mul(a.x, b.y), ff_mul(a.y, b.x))};
}
__device__ __forceinline__ cff cscale(cff a, ff s) { return {ff_mul(a.x, s), ff_mul(a.y, s)}; }
__device__ __forceinline__ cff cneg(cff a) { return {ff_neg(a.x), ff_neg(a.y)}; }
__device__ __forceinline__ ff neg_of(ff a) { return ff_neg(a); }
__device__ __forceinline__ float neg_of(float a) { return -a; }
__device__ __forceinline__ double neg_of(double a) { return -a; }
// multiply by SIGN * i
template <int SIGN, class T> __device__ __forceinline__ T mul_i(T a) {
    T r;
    if (SIGN > 0) { r.x = neg_of(a.y); r.y = a.x; }
    else { r.x = a.y; r.y = neg_of(a.x); }
    return r;
}

__device__ __forceinline__ float2 tw_entry(const float2 *, int i) { return c_tw.v[i]; }
__device__ __forceinline__ double2 tw_entry(const double2 *, int i) { return c_twd.v[i]; }
__device__ __forceinline__ cff tw_entry(const cff *, int i) { return c_twff.v[i]; }

// real constants in the element precision
__device__ __forceinline__ float real_const(const float2 *, double c) { return (float)c; }
__device__ __forceinline__ double real_const(const double2 *, double c) { return c; }
__device__ __forceinline__ ff real_const(const cff *, double c) { return ff_from(c); }

template <int N, int SIGN, class T> __device__ __forceinline__ void mul_tw(T &v, int j) {
    // j is a compile-time constant after unrolling; trivial roots skip the multiply
    if (j == 0) return;
    if (4 * j == N) { v = mul_i<SIGN>(v); return; }
    if (2 * j == N) { v = cneg(v); return; }
    if (4 * j == 3 * N) { v = mul_i<-SIGN>(v); return; }
    T w = tw_entry((const T *)nullptr, tw_off<N>() + j);
    if (SIGN < 0) w.y = neg_of(w.y);
    v = cmul(v, w);
}

template <int SIGN, class T> __device__ __forceinline__ void bfly2(T &a, T &b) {
    T t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int SIGN, class T> __device__ __forceinline__ void bfly4(T &a, T &b, T &c, T &d) {
    T s0 = cadd(a, c), d0 = csub(a, c), s1 = cadd(b, d), d1 = mul_i<SIGN>(csub(b, d));
    a = cadd(s0, s1);
    c = csub(s0, s1);
    b = cadd(d0, d1);
    d = csub(d0, d1);
}

template <int SIGN, class T> __device__ __forceinline__ void bfly3(T &a, T &b, T &c) {
    // sqrt(3)/2 and 1/2 in the element precision
    const auto h = real_const((const T *)nullptr, 0.86602540378443864676372317075294);
    const auto half = real_const((const T *)nullptr, 0.5);
    T t1 = cadd(b, c), t2 = csub(b, c);
    T m = csub(a, cscale(t1, half));
    T r = mul_i<SIGN>(cscale(t2, h));
    a = cadd(a, t1);
    b = cadd(m, r);
    c = csub(m, r);
}

template <int N> __host__ __device__ constexpr int first_radix() {
    return (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 3);
}

// In-place DIF on x[0], x[S], ..., x[(N-1) S]; output in digit-reversed slots.
template <int N, int SIGN, int S, class T> __device__ __forceinline__ void dif(T *x) {
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

template <int N, int SIGN, class T> __device__ __forceinline__ void fft_inplace(T (&x)[N]) {
    dif<N, SIGN, 1>(x);
    T y[N];
    #pragma unroll
    for (int k = 0; k < N; ++k) y[k] = x[slot_of<N>(k)];
    #pragma unroll
    for (int k = 0; k < N; ++k) x[k] = y[k];
}

}  // namespace bz

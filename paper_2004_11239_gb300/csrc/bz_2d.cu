// The 2D operator (Sec. 4 with d = 2; Sec. 4.1 (i)) on an N x N grid, N <= 64.
//
// A whole term's field fits one CTA: N threads, the field in shared memory [N][N+1], FP32
// register FFTs.  Per term (twiddles beta_p per axis, alpha_p = c_p F / N^2):
//   columns (thread = k2):  x = beta_p fhat over k1, IFFT over k1 -> S            (sync)
//   rows    (thread = j1):  IFFT over k2, times h, FFT over j2 -> S              (sync)
//   columns (thread = k2):  FFT over j1, acc += alpha_p x  (acc[., k2] is the thread's own)
// A column pass writes and reads only its own column of S, so the next term's first pass
// needs no barrier.  Work items are (term block) per CTA, persistent over a grid of resident
// CTAs; each item's FP32 sum goes to its partial, summed over blocks in a fixed order by
// k_reduce_parts.  h = IFFT(fhat) is formed beforehand in FP64 (k_h64_2d, or the four-step
// k_h64_2d_64 at N = 64) and stored FP32.
#include "bz_fft.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

template <int N> struct D2 {
    static constexpr int LD = N + 1;
    static constexpr size_t SMEM = 2 * (size_t)N * LD * sizeof(float2);   // S and acc
    static constexpr size_t SMEM64 = (size_t)N * LD * sizeof(double2);    // the h pass
};

__device__ __forceinline__ double2 load_c2(const void *f, int dtype, size_t i) {
    if (dtype == BZ_C128) return ((const double2 *)f)[i];
    const float2 v = ((const float2 *)f)[i];
    return make_double2(v.x, v.y);
}

// h = IFFT(fhat) in FP64 for N <= 32: one CTA, thread c transforms column c, then row c.
template <int N>
__global__ void __launch_bounds__(N) k_h64_2d(const void *__restrict__ f, int dtype, float2 *__restrict__ h) {
    extern __shared__ double2 sd[];
    constexpr int LD = D2<N>::LD;
    const int c = threadIdx.x;
    double2 x[N];
    #pragma unroll
    for (int i = 0; i < N; ++i) x[i] = load_c2(f, dtype, (size_t)i * N + c);
    fft_inplace<N, +1>(x);
    #pragma unroll
    for (int i = 0; i < N; ++i) sd[i * LD + c] = x[i];
    __syncthreads();
    #pragma unroll
    for (int j = 0; j < N; ++j) x[j] = sd[c * LD + j];
    fft_inplace<N, +1>(x);
    #pragma unroll
    for (int j = 0; j < N; ++j) h[(size_t)c * N + j] = make_float2((float)x[j].x, (float)x[j].y);
}

// N = 64: an FP64 line transform of length 64 = 8 x 8 by the 8 threads of one CTA (four-step
// Cooley-Tukey): thread t holds x[t + 8 m], transforms over m, multiplies by exp(+2 pi i t k2 / 64)
// and, after a transpose through shared memory, thread k2 transforms over t, ending with
// X[k2 + 8 k1].  FP64 rate per SM is low on this GPU, so each line gets its own CTA (64 per
// pass).  AXIS 0: column c of f -> scr (FP64); AXIS 1: row r of scr -> h (FP32).
template <int AXIS>
__global__ void __launch_bounds__(8) k_h64_2d_64(const void *__restrict__ f, int dtype, double2 *__restrict__ scr,
                                                float2 *__restrict__ h) {
    constexpr int N = 64;
    __shared__ double2 tr[8][9];
    const int line = blockIdx.x, t = threadIdx.x;
    double2 y[8];
    #pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int n = t + 8 * m;
        y[m] = AXIS == 0 ? load_c2(f, dtype, (size_t)n * N + line) : scr[(size_t)line * N + n];
    }
    fft_inplace<8, +1>(y);                                   // over m -> k2
    #pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) {
        mul_tw<64, +1>(y[k2], t * k2);                       // exp(+2 pi i t k2 / 64)
        tr[k2][t] = y[k2];
    }
    __syncthreads();
    #pragma unroll
    for (int u = 0; u < 8; ++u) y[u] = tr[t][u];              // thread k2 = t gathers over t' = u
    fft_inplace<8, +1>(y);                                   // over t' -> k1; index k = t + 8 k1
    #pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
        const int k = t + 8 * k1;
        if (AXIS == 0) scr[(size_t)k * N + line] = y[k1];
        else h[(size_t)line * N + k] = make_float2((float)y[k1].x, (float)y[k1].y);
    }
}

template <int N>
__global__ void __launch_bounds__(N)
k_collide_2d(const float2 *__restrict__ fin, const float2 *__restrict__ h, const float2 *__restrict__ tw,
             const float2 *__restrict__ alpha, float2 *__restrict__ part, int p0, int p1, int TB, int nblk) {
    extern __shared__ float2 s2[];
    constexpr int LD = D2<N>::LD, N2 = N * N;
    float2 *S = s2, *acc = s2 + (size_t)N * LD;
    const int c = threadIdx.x;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int t0 = p0 + blk * TB, t1 = min(p1, t0 + TB);
        #pragma unroll 8
        for (int i = 0; i < N; ++i) acc[i * LD + c] = make_float2(0.f, 0.f);
        for (int p = t0; p < t1; ++p) {
            const float2 *twp = tw + (size_t)p * 3 * N;       // [axis][m]; the third axis is unused in 2D
            const float2 t2 = __ldg(twp + N + c);
            float2 x[N];
            #pragma unroll
            for (int i = 0; i < N; ++i) x[i] = cmul(fin[i * N + c], cmul(__ldg(twp + i), t2));
            fft_inplace<N, +1>(x);                           // k1 -> j1
            #pragma unroll
            for (int i = 0; i < N; ++i) S[i * LD + c] = x[i];
            __syncthreads();
            #pragma unroll
            for (int j = 0; j < N; ++j) x[j] = S[c * LD + j];
            fft_inplace<N, +1>(x);                           // k2 -> j2 (row j1 = c)
            #pragma unroll
            for (int j = 0; j < N; ++j) x[j] = cmul(x[j], __ldg(h + (size_t)c * N + j));
            fft_inplace<N, -1>(x);                           // j2 -> k2
            #pragma unroll
            for (int j = 0; j < N; ++j) S[c * LD + j] = x[j];
            __syncthreads();
            #pragma unroll
            for (int i = 0; i < N; ++i) x[i] = S[i * LD + c];
            fft_inplace<N, -1>(x);                           // j1 -> k1 (column k2 = c)
            const float2 *al = alpha + (size_t)p * N2 + c;
            #pragma unroll
            for (int i = 0; i < N; ++i) {
                const float2 a = al[i * N];
                float2 s = acc[i * LD + c];
                s.x = fmaf(x[i].x, a.x, fmaf(-x[i].y, a.y, s.x));
                s.y = fmaf(x[i].x, a.y, fmaf(x[i].y, a.x, s.y));
                acc[i * LD + c] = s;
            }
        }
        float2 *out = part + (size_t)blk * N2 + c;
        #pragma unroll 8
        for (int i = 0; i < N; ++i) out[i * N] = acc[i * LD + c];
    }
}

template <int N> cudaError_t setup_n(Plan &pl) {
    cudaError_t e = cudaFuncSetAttribute(k_collide_2d<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D2<N>::SMEM);
    if constexpr (N < 64) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_h64_2d<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)D2<N>::SMEM64);
    }
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_collide_2d<N>, N, D2<N>::SMEM);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    pl.fused_G = per_sm * sms;
    pl.fused_C = 1;
    return pl.fused_G > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <int N> bz_status run_n(Plan &pl, int p0, int p1, cudaStream_t st, int *launches) {
    const int n2 = N * N;
    const int nt = p1 - p0;
    const int TB = nt > 0 ? (nt + pl.fused_G - 1) / pl.fused_G : 1;
    const int nblk = nt > 0 ? (nt + TB - 1) / TB : 0;
    const void *src = pl.src ? pl.src : (const void *)pl.fin;
    const int sdt = pl.src ? pl.src_dtype : BZ_C64;
    tm_begin(pl, st);
    if constexpr (N == 64) {
        k_h64_2d_64<0><<<N, 8, 0, st>>>(src, sdt, pl.scr64, nullptr);
        k_h64_2d_64<1><<<N, 8, 0, st>>>(nullptr, BZ_C128, pl.scr64, pl.h);
    } else {
        k_h64_2d<N><<<1, N, D2<N>::SMEM64, st>>>(src, sdt, pl.h);
    }
    tm_end(pl, st, TK_OTHER);
    tm_begin(pl, st);
    if (nblk > 0)
        k_collide_2d<N><<<nblk < pl.fused_G ? nblk : pl.fused_G, N, D2<N>::SMEM, st>>>(
            pl.fin, pl.h, pl.tw, pl.alpha, pl.part, p0, p1, TB, nblk);
    tm_end(pl, st, TK_FUSED);
    tm_begin(pl, st);
    reduce_parts(pl.part, nblk, n2, pl.acc, st);
    tm_end(pl, st, TK_REDUCE);
    BZ_CUDA_TRY(cudaGetLastError());
    if (launches) *launches += (nblk > 0 ? 3 : 2) + (N == 64 ? 1 : 0);
    return BZ_OK;
}

}  // namespace

cudaError_t setup_2d(Plan &pl) {
    switch (pl.N) {
        case 8: return setup_n<8>(pl);
        case 16: return setup_n<16>(pl);
        case 32: return setup_n<32>(pl);
        case 64: return setup_n<64>(pl);
    }
    return cudaErrorInvalidValue;
}

bz_status collide_2d(Plan &pl, int p0, int p1, cudaStream_t st, int *launches) {
    switch (pl.N) {
        case 8: return run_n<8>(pl, p0, p1, st, launches);
        case 16: return run_n<16>(pl, p0, p1, st, launches);
        case 32: return run_n<32>(pl, p0, p1, st, launches);
        case 64: return run_n<64>(pl, p0, p1, st, launches);
    }
    return BZ_ERR_UNSUPPORTED;
}

}  // namespace bz

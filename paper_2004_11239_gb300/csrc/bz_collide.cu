// The per-term pipeline of eq. realQ (Sec. 4) in FP32 with FP64 accumulation over terms.
//
// For each chunk of T terms, four kernels run over a scratch buffer S[T][N^3] sized to
// stay in L2 (where the plan has more streams, chunk i runs on stream i % lanes over that
// stream's scratch and accumulator, overlapping the others; the sums are added at the end):
//   plane_inv  (planes k1):  S = IFFT_{axes 3,2}( beta_p(m) fhat_m )       twiddle + 2 axes
//   pencil     (lines k1):   S = FFT_1( h . IFFT_1(S) )                     product in registers
// (at N = 64 the plane and pencil passes are the radix-8 x 8 kernels of bz_chunk64.cu)
//   plane_fwd  (planes k1):  S = alpha_p . FFT_{axes 3,2}(S)                 weight in the epilogue
//   reduce     (modes k):    acc += sum_t S[t]  (compensated FP32 over every term, FP64 at the end)
// h = IFFT(fhat) is formed once per call by plane_inv without twiddles plus an
// inverse-only pencil pass.  Inverse transforms are unnormalised; alpha carries N^-3.
#include <algorithm>
#include <cstdio>

#include "bz_fft.cuh"
#include "bz_internal.h"

namespace bz {

template <int N> struct Cfg {
    // planes per CTA; N = 64 takes two so that three CTAs (12 warps) share an SM
    static constexpr int PPC = N <= 8 ? 8 : (N <= 16 ? 16 : (N <= 32 ? 8 : (N <= 48 ? 4 : 2)));
    static constexpr int LD = N + 1;                                              // padded row
    static constexpr int THREADS = PPC * N;
    static constexpr size_t SMEM = ((size_t)PPC * N * LD + 6 * N) * sizeof(float2);   // planes + a pair's twiddles
    // resident CTAs per SM the register budget is held to (shared memory allows as many)
    static constexpr int MINB = N == 64 ? 3 : (N == 48 ? 2 : 1);
};

// ---------------------------------------------------------------------------------------
// plane_inv: one CTA holds PPC planes k1 of one term; N threads per plane.
// ---------------------------------------------------------------------------------------
// PAIR (BZ_DATA_REAL): unit t is the term pair (2u, 2u + 1), u = p0 + t, and the twiddle is
// beta_2u + i beta_2u+1 (both terms' [3][N] vectors, contiguous).
template <int N, bool PAIR = false>
__global__ void __launch_bounds__(Cfg<N>::THREADS, Cfg<N>::MINB)
k_plane_inv(const float2 *__restrict__ fin, const float2 *__restrict__ tw, float2 *__restrict__ S,
            int p0, int use_tw) {
    constexpr int PPC = Cfg<N>::PPC, LD = Cfg<N>::LD, NT = (PAIR ? 6 : 3) * N;
    extern __shared__ float2 sm[];
    float2 *stw = sm + PPC * N * LD;                  // the term's twiddle vectors
    const int lane = threadIdx.x % N, pid = threadIdx.x / N;
    const int k1 = blockIdx.x * PPC + pid;
    const int t = blockIdx.y;
    float2 *s = sm + pid * N * LD;
    const float2 *f = fin + (size_t)k1 * N * N;
    const float2 *twp = tw + (size_t)(p0 + t) * NT;
    float2 x[N];
    #pragma unroll
    for (int i = 0; i < N; ++i) x[i] = f[i * N + lane];   // every load of the plane in flight at once
    if (use_tw) {
        for (int i = threadIdx.x; i < NT; i += Cfg<N>::THREADS) stw[i] = twp[i];
        __syncthreads();
        const float2 t13 = cmul(stw[k1], stw[2 * N + lane]);
        if constexpr (PAIR) {
            const float2 t13b = cmul(stw[3 * N + k1], stw[5 * N + lane]);
            #pragma unroll
            for (int i = 0; i < N; ++i) {
                const float2 u = cmul(t13, stw[N + i]), w = cmul(t13b, stw[4 * N + i]);
                x[i] = cmul(x[i], make_float2(u.x - w.y, u.y + w.x));
            }
        } else {
            #pragma unroll
            for (int i = 0; i < N; ++i) x[i] = cmul(x[i], cmul(t13, stw[N + i]));
        }
    }
    #pragma unroll
    for (int i = 0; i < N; ++i) s[i * LD + lane] = x[i];
    __syncthreads();
    #pragma unroll
    for (int j = 0; j < N; ++j) x[j] = s[lane * LD + j];
    fft_inplace<N, +1>(x);                       // axis 3: k3 -> j3
    #pragma unroll
    for (int j = 0; j < N; ++j) s[lane * LD + j] = x[j];
    __syncthreads();
    #pragma unroll
    for (int i = 0; i < N; ++i) x[i] = s[i * LD + lane];
    fft_inplace<N, +1>(x);                       // axis 2: k2 -> j2
    float2 *out = S + (size_t)t * N * N * N + (size_t)k1 * N * N;
    #pragma unroll
    for (int i = 0; i < N; ++i) out[i * N + lane] = x[i];
}

// ---------------------------------------------------------------------------------------
// pencil: one thread per (j2, j3) line along axis 1 of one term.
//   MODE 0: out = IFFT_1(S)                         (forms h)
//   MODE 1: S = FFT_1( h . IFFT_1(S) )              (in place)
//   MODE 2: as MODE 1 with the real part of h (BZ_DATA_REAL: h is real)
// ---------------------------------------------------------------------------------------
template <int N, int MODE>
__global__ void __launch_bounds__(128, 3)
k_pencil(float2 *__restrict__ S, const float2 *__restrict__ h, float2 *__restrict__ out) {
    constexpr int N2 = N * N;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N2) return;
    float2 *base = S + (size_t)blockIdx.y * N * N2 + g;
    float2 x[N];
    #pragma unroll
    for (int k = 0; k < N; ++k) x[k] = base[k * N2];
    fft_inplace<N, +1>(x);                       // axis 1: k1 -> j1
    if constexpr (MODE == 0) {
        #pragma unroll
        for (int j = 0; j < N; ++j) out[j * N2 + g] = x[j];
    } else {
        #pragma unroll
        for (int j = 0; j < N; ++j) {
            if constexpr (MODE == 2) {
                const float hv = h[j * N2 + g].x;
                x[j].x *= hv;
                x[j].y *= hv;
            } else {
                x[j] = cmul(x[j], h[j * N2 + g]);
            }
        }
        fft_inplace<N, -1>(x);                   // axis 1: j1 -> k1
        #pragma unroll
        for (int k = 0; k < N; ++k) base[k * N2] = x[k];
    }
}

// ---------------------------------------------------------------------------------------
// plane_fwd: forward transform along axes 2 and 3, times alpha_p, in place.
// ---------------------------------------------------------------------------------------
// PAIR (BZ_DATA_REAL): alpha is the pair table A, and the chunk's Nyquist sums X = C Z go to
// Ss[t][3][N][N] (family layout; every entry written, zero where C is zero).  gsc (or null):
// a batch slot's radial scale r_i^(gamma_slot - gamma_plan) per radial node i of the M-point
// sphere rule (a pair shares its node), applied to the transformed field.
template <int N, bool PAIR = false>
__global__ void __launch_bounds__(Cfg<N>::THREADS, Cfg<N>::MINB)
k_plane_fwd(float2 *__restrict__ S, const float2 *__restrict__ alpha, int p0, const float2 *__restrict__ cpair = nullptr,
            float2 *__restrict__ Ss = nullptr, const float *__restrict__ gsc = nullptr, int M = 1) {
    constexpr int PPC = Cfg<N>::PPC, LD = Cfg<N>::LD;
    extern __shared__ float2 sm[];
    const int lane = threadIdx.x % N, pid = threadIdx.x / N;
    const int k1 = blockIdx.x * PPC + pid;
    const int t = blockIdx.y;
    float2 *s = sm + pid * N * LD;
    float2 *pl = S + (size_t)t * N * N * N + (size_t)k1 * N * N;
    const float2 *al = alpha + (size_t)(p0 + t) * N * N * N + (size_t)k1 * N * N;
    float2 x[N];
    #pragma unroll
    for (int i = 0; i < N; ++i) x[i] = pl[i * N + lane];     // column j3 = lane, over j2
    fft_inplace<N, -1>(x);                                    // axis 2: j2 -> k2
    #pragma unroll
    for (int i = 0; i < N; ++i) s[i * LD + lane] = x[i];
    __syncthreads();
    #pragma unroll
    for (int j = 0; j < N; ++j) x[j] = s[lane * LD + j];     // row k2 = lane, over j3
    fft_inplace<N, -1>(x);                                    // axis 3: j3 -> k3
    #pragma unroll
    for (int j = 0; j < N; ++j) s[lane * LD + j] = x[j];
    __syncthreads();
    #pragma unroll
    for (int i = 0; i < N; ++i) x[i] = al[i * N + lane];    // every weight load in flight at once
    const float sc = gsc ? gsc[(PAIR ? 2 * (p0 + t) : p0 + t) / M] : 1.f;
    #pragma unroll
    for (int i = 0; i < N; ++i) pl[i * N + lane] = cscale(cmul(s[i * LD + lane], x[i]), sc);
    if constexpr (PAIR) {
        const float2 *cq = cpair + (size_t)(p0 + t) * 3 * N * N;
        float2 *xs = Ss + (size_t)t * 3 * N * N;
        // family k2 = -N/2 at [k1][k3 = lane]; family k3 = -N/2 at [k1][k2 = lane]
        xs[N * N + k1 * N + lane] = cscale(cmul(s[(N / 2) * LD + lane], cq[N * N + k1 * N + lane]), sc);
        xs[2 * N * N + k1 * N + lane] = cscale(cmul(s[lane * LD + N / 2], cq[2 * N * N + k1 * N + lane]), sc);
        if (k1 == N / 2) {                                    // the plane k1 = -N/2: [k2][k3]
            #pragma unroll 4
            for (int i = 0; i < N; ++i) xs[i * N + lane] = cscale(cmul(s[i * LD + lane], cq[i * N + lane]), sc);
        }
    }
}

// ---------------------------------------------------------------------------------------
// reduce: acc[k] += sum_t S[t][k], one Kahan-compensated FP32 sum over every term of the
// collide in term order (per lane), carried from chunk to chunk in the accumulator's memory
// and turned into FP64 after the last chunk.  Each thread takes two adjacent modes (16-byte
// loads) and issues the loads of up to kRedBatch terms before it adds them, so the chunk's
// loads are in flight together.  A second array (S2, n2 modes, acc2) may follow the first in
// the same launch: thread pairs past n3 / 2 take it.
// ---------------------------------------------------------------------------------------
constexpr int kRedBatch = 8;

struct Kahan4 {
    float s[4], c[4];
    __device__ __forceinline__ Kahan4(float4 s0, float4 c0)
        : s{s0.x, s0.y, s0.z, s0.w}, c{c0.x, c0.y, c0.z, c0.w} {}
    __device__ __forceinline__ void add(float4 v) {
        const float x[4] = {v.x, v.y, v.z, v.w};
        #pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float y = x[i] - c[i], t = s[i] + y;
            c[i] = (t - s[i]) - y;
            s[i] = t;
        }
    }
};

// acc += sum over the chunk's T terms, compensated in FP32 across every chunk of the collide:
// while the chunks run, the 32 bytes of acc[2 k2], acc[2 k2 + 1] (FP64 modes 2 k2, 2 k2 + 1)
// hold the running sums s and compensations c of the pair's four components as two float4
// (zero bytes are the empty sum), and k_kahan_fold turns them into FP64 once at the end.  The
// per-chunk pass thus runs no FP64 arithmetic, whose rate on this part is a small fraction of
// FP32's.  S2 / n2 / acc2 (or null): a second field summed the same way (the Nyquist sums).
__global__ void __launch_bounds__(256, 4)        // <= 64 registers: a launch at N = 64 fits one wave
k_reduce(const float2 *__restrict__ S, int T, int n3, double2 *__restrict__ acc,
         const float2 *__restrict__ S2 = nullptr, int n2 = 0, double2 *__restrict__ acc2 = nullptr) {
    int k2 = blockIdx.x * blockDim.x + threadIdx.x;          // mode pair index
    const float4 *src = (const float4 *)S;
    int n = n3;
    float4 *dst = (float4 *)acc;
    if (k2 >= n3 / 2) {
        k2 -= n3 / 2;
        if (!S2 || k2 >= n2 / 2) return;
        src = (const float4 *)S2;
        n = n2;
        dst = (float4 *)acc2;
    }
    const size_t stride = (size_t)n / 2;                     // float4 per term
    Kahan4 sum(dst[2 * k2], dst[2 * k2 + 1]);
    for (int t0 = 0; t0 < T; t0 += kRedBatch) {
        float4 v[kRedBatch];
        #pragma unroll
        for (int i = 0; i < kRedBatch; ++i)
            if (t0 + i < T) v[i] = src[(size_t)(t0 + i) * stride + k2];
        #pragma unroll
        for (int i = 0; i < kRedBatch; ++i)
            if (t0 + i < T) sum.add(v[i]);
    }
    dst[2 * k2] = make_float4(sum.s[0], sum.s[1], sum.s[2], sum.s[3]);
    dst[2 * k2 + 1] = make_float4(sum.c[0], sum.c[1], sum.c[2], sum.c[3]);
}

// In place, after the last chunk: the compensated state of k_reduce to FP64, s - c per component.
__global__ void k_kahan_fold(double2 *__restrict__ acc, int n, double2 *__restrict__ acc2 = nullptr, int n2 = 0) {
    int k2 = blockIdx.x * blockDim.x + threadIdx.x;
    double2 *a = acc;
    if (k2 >= n / 2) {
        k2 -= n / 2;
        if (!acc2 || k2 >= n2 / 2) return;
        a = acc2;
    }
    const float4 s = ((const float4 *)a)[2 * k2], c = ((const float4 *)a)[2 * k2 + 1];
    a[2 * k2] = make_double2((double)s.x - (double)c.x, (double)s.y - (double)c.y);
    a[2 * k2 + 1] = make_double2((double)s.z - (double)c.z, (double)s.w - (double)c.w);
}

__global__ void k_c128_to_c64(const double2 *__restrict__ in, float2 *__restrict__ out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

__global__ void k_acc_to_c64(const double2 *__restrict__ in, float2 *__restrict__ out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// a[i] += b[i]: the second stream's accumulator into the first.
__global__ void k_acc_add(double2 *__restrict__ a, const double2 *__restrict__ b, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        double2 v = a[i];
        const double2 w = b[i];
        v.x += w.x;
        v.y += w.y;
        a[i] = v;
    }
}

// The plan's result to the caller's array in its dtype, raising the non-finite flag.
__global__ void k_acc_out(const double2 *__restrict__ in, void *__restrict__ out, int dtype, int n, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double2 v = in[i];
    if (dtype == BZ_C128) {
        ((double2 *)out)[i] = v;
        note_finite(v, flag);
    } else {
        const float2 w = make_float2((float)v.x, (float)v.y);
        ((float2 *)out)[i] = w;
        note_finite(w, flag);
    }
}

// Padded plans (BZ_CONV_PADDED): the caller's Nin-grid lives inside the N = 2 Nin grid at the
// same signed modes.  Embed: one thread per N-grid mode, zero outside the caller's range.
__global__ void k_embed(const void *__restrict__ f, int dtype, int Nin, int N, float2 *__restrict__ out,
                        double2 *__restrict__ out64) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * N * N) return;
    const int h = Nin / 2;
    int s[3] = {i / (N * N), (i / N) % N, i % N};
    bool in = true;
    size_t src = 0;
    #pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int k = s[d] < N / 2 ? s[d] : s[d] - N;
        in = in && k >= -h && k < h;
        src = src * Nin + (size_t)((k + Nin) % Nin);
    }
    double2 v = make_double2(0.0, 0.0);
    if (in) {
        if (dtype == BZ_C128) v = ((const double2 *)f)[src];
        else { const float2 w = ((const float2 *)f)[src]; v = make_double2(w.x, w.y); }
    }
    out[i] = make_float2((float)v.x, (float)v.y);
    if (out64) out64[i] = v;
}

// Extract: one thread per caller mode, from the FP64 accumulator of the N grid.
__global__ void k_extract(const double2 *__restrict__ acc, int Nin, int N, void *__restrict__ Q, int dtype,
                          int *flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nin * Nin * Nin) return;
    int s[3] = {i / (Nin * Nin), (i / Nin) % Nin, i % Nin};
    size_t src = 0;
    #pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int k = s[d] < Nin / 2 ? s[d] : s[d] - Nin;
        src = src * N + (size_t)((k + N) % N);
    }
    const double2 v = acc[src];
    if (dtype == BZ_C128) {
        ((double2 *)Q)[i] = v;
        note_finite(v, flag);
    } else {
        const float2 w = make_float2((float)v.x, (float)v.y);
        ((float2 *)Q)[i] = w;
        note_finite(w, flag);
    }
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
int supported_N(int N) {
    return N == 8 || N == 16 || N == 24 || N == 32 || N == 48 || N == 64;
}

template <int N> static cudaError_t set_attrs() {
    if constexpr (N == 64) {
        const cudaError_t e = chunk64_set_attributes();
        if (e != cudaSuccess) return e;
    }
    const void *ks[4] = {(const void *)k_plane_inv<N, false>, (const void *)k_plane_inv<N, true>,
                         (const void *)k_plane_fwd<N, false>, (const void *)k_plane_fwd<N, true>};
    for (const void *k : ks) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<N>::SMEM);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Terms per chunk: two waves of plane CTAs (resident CTAs / CTAs per term, twice), so that
// the second wave's loads overlap the first wave's arithmetic, capped by a scratch of 64 MB
// that stays in L2 (measured at N = 64, P = 1024, real data: 2.56 ms per collide with one
// wave of 14 pairs, 2.18 ms with two).
template <int N> static int chunk_for() {
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plane_inv<N, false>, Cfg<N>::THREADS, Cfg<N>::SMEM) !=
        cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int wave = 2 * per_sm * sms / (N / Cfg<N>::PPC);
    const int l2 = (int)(((size_t)64 << 20) / ((size_t)N * N * N * sizeof(float2)));
    const int c = wave < l2 ? wave : l2;
    return c > 0 ? c : 1;
}

int chunk_terms_for(int N) {
    switch (N) {
        case 8: return chunk_for<8>();
        case 16: return chunk_for<16>();
        case 24: return chunk_for<24>();
        case 32: return chunk_for<32>();
        case 48: return chunk_for<48>();
        case 64: return chunk_for<64>();
    }
    return 1;
}

cudaError_t collide_set_attributes(int N) {
    switch (N) {
        case 8: return set_attrs<8>();
        case 16: return set_attrs<16>();
        case 24: return set_attrs<24>();
        case 32: return set_attrs<32>();
        case 48: return set_attrs<48>();
        case 64: return set_attrs<64>();
    }
    return cudaErrorInvalidValue;
}

// Plane passes of a chunk: at N = 64 the radix-8 one-plane-per-CTA kernels, else the generic ones.
template <int N, bool PAIR>
static void plane_inv(const float2 *fin, const float2 *tw, float2 *S, int p0, int T, int use_tw, cudaStream_t st) {
    constexpr int PPC = Cfg<N>::PPC;
    if constexpr (N == 64) plane_inv64(fin, tw, S, p0, T, use_tw, PAIR, st);
    else k_plane_inv<N, PAIR><<<dim3(N / PPC, T), Cfg<N>::THREADS, Cfg<N>::SMEM, st>>>(fin, tw, S, p0, use_tw);
}

template <int N, bool PAIR>
static void plane_fwd(float2 *S, const float2 *alpha, int p0, int T, const float2 *cpair, float2 *Ss, const float *gsc,
                      int M, cudaStream_t st) {
    constexpr int PPC = Cfg<N>::PPC;
    if constexpr (N == 64) plane_fwd64(S, alpha, p0, T, cpair, Ss, gsc, M, PAIR, st);
    else k_plane_fwd<N, PAIR><<<dim3(N / PPC, T), Cfg<N>::THREADS, Cfg<N>::SMEM, st>>>(S, alpha, p0, cpair, Ss, gsc, M);
}

template <int N, int MODE>
static void pencil(float2 *S, const float2 *h, float2 *out, int T, cudaStream_t st) {
    if constexpr (N == 64) pencil64(S, h, out, T, MODE, st);
    else k_pencil<N, MODE><<<dim3((N * N + 127) / 128, T), 128, 0, st>>>(S, h, out);
}

// BZ_DATA_REAL: the Hermitian part of the input (sym_input) feeds h and the pair passes; the
// chunks run over term pairs [p0 / 2, p1 / 2) with the pair table A, the Nyquist sums X are
// reduced beside V, and Q is symmetrised after the last chunk.
template <int N>
static bz_status run_chunks_real(Plan &pl, int p0, int p1, cudaStream_t st, int *launches) {
    const int n3 = N * N * N, ns = 3 * N * N;
    if ((p0 | p1) & 1) return BZ_ERR_ARG;
    const int u0 = p0 / 2, u1 = p1 / 2;
    const int chunk = pl.chunk;
    tm_begin(pl, st);
    bz_status s = sym_input(pl, pl.src ? pl.src : (const void *)pl.fin, pl.src ? pl.src_dtype : BZ_C64, st);
    if (s != BZ_OK) return s;
    plane_inv<N, false>(pl.fsym, pl.tw, pl.S, 0, 1, 0, st);
    // h is real: at N = 64 it is stored as N^3 packed floats (half the bytes the pair pencils read)
    if constexpr (N == 64) pencil64(pl.S, nullptr, pl.h, 1, 3, st);
    else pencil<N, 0>(pl.S, nullptr, pl.h, 1, st);
    BZ_CUDA_TRY(cudaMemsetAsync(pl.acc, 0, (size_t)n3 * sizeof(double2), st));
    BZ_CUDA_TRY(cudaMemsetAsync(pl.acc_s, 0, (size_t)ns * sizeof(double2), st));
    tm_end(pl, st, TK_OTHER);
    int nl = 3;
    // lanes: as many streams as chunks, up to 1 + pl.xn
    const int nchunks = (u1 - u0 + chunk - 1) / chunk;
    const int lanes = 1 + (pl.xn < nchunks - 1 ? pl.xn : (nchunks > 1 ? nchunks - 1 : 0));
    if (lanes > 1) {
        BZ_CUDA_TRY(cudaEventRecord(pl.ev_fork, st));
        for (int e = 0; e + 1 < lanes; ++e) {
            BZ_CUDA_TRY(cudaStreamWaitEvent(pl.xst[e], pl.ev_fork, 0));
            BZ_CUDA_TRY(cudaMemsetAsync(pl.xacc[e], 0, (size_t)n3 * sizeof(double2), pl.xst[e]));
            BZ_CUDA_TRY(cudaMemsetAsync(pl.xacc_s[e], 0, (size_t)ns * sizeof(double2), pl.xst[e]));
        }
    }
    for (int c0 = u0, i = 0; c0 < u1; c0 += chunk, ++i) {
        const int T = (u1 - c0) < chunk ? (u1 - c0) : chunk;
        const int ln = i % lanes;
        cudaStream_t cs = ln ? pl.xst[ln - 1] : st;
        float2 *S = ln ? pl.xS[ln - 1] : pl.S, *Ss = ln ? pl.xS_s[ln - 1] : pl.S_s;
        double2 *acc = ln ? pl.xacc[ln - 1] : pl.acc, *acc_s = ln ? pl.xacc_s[ln - 1] : pl.acc_s;
        tm_begin(pl, cs);
        plane_inv<N, true>(pl.fsym, pl.tw, S, c0, T, 1, cs);
        tm_end(pl, cs, TK_PLANE_INV);
        tm_begin(pl, cs);
        pencil<N, 2>(S, pl.h, nullptr, T, cs);
        tm_end(pl, cs, TK_PENCIL);
        tm_begin(pl, cs);
        plane_fwd<N, true>(S, pl.apair, c0, T, pl.cpair, Ss, pl.gsc_cur, pl.M, cs);
        tm_end(pl, cs, TK_PLANE_FWD);
        tm_begin(pl, cs);
        k_reduce<<<(n3 / 2 + ns / 2 + 255) / 256, 256, 0, cs>>>(S, T, n3, acc, Ss, ns, acc_s);
        tm_end(pl, cs, TK_REDUCE);
        nl += 4;
    }
    for (int ln = 0; ln < lanes; ++ln) {
        cudaStream_t cs = ln ? pl.xst[ln - 1] : st;
        k_kahan_fold<<<(n3 / 2 + ns / 2 + 255) / 256, 256, 0, cs>>>(ln ? pl.xacc[ln - 1] : pl.acc, n3,
                                                                   ln ? pl.xacc_s[ln - 1] : pl.acc_s, ns);
        ++nl;
    }
    for (int e = 0; e + 1 < lanes; ++e) {
        // the other lanes' sums join the first's in a fixed order
        BZ_CUDA_TRY(cudaEventRecord(pl.xev_join[e], pl.xst[e]));
        BZ_CUDA_TRY(cudaStreamWaitEvent(st, pl.xev_join[e], 0));
        k_acc_add<<<(n3 + 255) / 256, 256, 0, st>>>(pl.acc, pl.xacc[e], n3);
        k_acc_add<<<(ns + 255) / 256, 256, 0, st>>>(pl.acc_s, pl.xacc_s[e], ns);
        nl += 2;
    }
    tm_begin(pl, st);
    s = sym_output(pl, st);
    if (s != BZ_OK) return s;
    tm_end(pl, st, TK_OTHER);
    ++nl;
    BZ_CUDA_TRY(cudaGetLastError());
    if (launches) *launches += nl;
    return BZ_OK;
}

template <int N>
static bz_status run_chunks(Plan &pl, int p0, int p1, cudaStream_t st, int *launches) {
    const int n3 = N * N * N;
    if (pl.real) return run_chunks_real<N>(pl, p0, p1, st, launches);
    // h = IFFT(fhat): planes without twiddles into S[0], then an inverse-only pencil pass
    tm_begin(pl, st);
    plane_inv<N, false>(pl.fin, pl.tw, pl.S, 0, 1, 0, st);
    pencil<N, 0>(pl.S, nullptr, pl.h, 1, st);
    BZ_CUDA_TRY(cudaMemsetAsync(pl.acc, 0, (size_t)n3 * sizeof(double2), st));
    tm_end(pl, st, TK_OTHER);
    int nl = 2;
    const int nchunks = (p1 - p0 + pl.chunk - 1) / pl.chunk;
    const int lanes = 1 + (pl.xn < nchunks - 1 ? pl.xn : (nchunks > 1 ? nchunks - 1 : 0));
    if (lanes > 1) {
        BZ_CUDA_TRY(cudaEventRecord(pl.ev_fork, st));
        for (int e = 0; e + 1 < lanes; ++e) {
            BZ_CUDA_TRY(cudaStreamWaitEvent(pl.xst[e], pl.ev_fork, 0));
            BZ_CUDA_TRY(cudaMemsetAsync(pl.xacc[e], 0, (size_t)n3 * sizeof(double2), pl.xst[e]));
        }
    }
    for (int c0 = p0, i = 0; c0 < p1; c0 += pl.chunk, ++i) {
        const int T = (p1 - c0) < pl.chunk ? (p1 - c0) : pl.chunk;
        const int ln = i % lanes;
        cudaStream_t cs = ln ? pl.xst[ln - 1] : st;
        float2 *S = ln ? pl.xS[ln - 1] : pl.S;
        double2 *acc = ln ? pl.xacc[ln - 1] : pl.acc;
        tm_begin(pl, cs);
        plane_inv<N, false>(pl.fin, pl.tw, S, c0, T, 1, cs);
        tm_end(pl, cs, TK_PLANE_INV);
        tm_begin(pl, cs);
        pencil<N, 1>(S, pl.h, nullptr, T, cs);
        tm_end(pl, cs, TK_PENCIL);
        tm_begin(pl, cs);
        plane_fwd<N, false>(S, pl.alpha, c0, T, nullptr, nullptr, pl.gsc_cur, pl.M, cs);
        tm_end(pl, cs, TK_PLANE_FWD);
        tm_begin(pl, cs);
        k_reduce<<<(n3 / 2 + 255) / 256, 256, 0, cs>>>(S, T, n3, acc);
        tm_end(pl, cs, TK_REDUCE);
        nl += 4;
    }
    for (int ln = 0; ln < lanes; ++ln) {
        k_kahan_fold<<<(n3 / 2 + 255) / 256, 256, 0, ln ? pl.xst[ln - 1] : st>>>(ln ? pl.xacc[ln - 1] : pl.acc, n3);
        ++nl;
    }
    for (int e = 0; e + 1 < lanes; ++e) {
        BZ_CUDA_TRY(cudaEventRecord(pl.xev_join[e], pl.xst[e]));
        BZ_CUDA_TRY(cudaStreamWaitEvent(st, pl.xev_join[e], 0));
        k_acc_add<<<(n3 + 255) / 256, 256, 0, st>>>(pl.acc, pl.xacc[e], n3);
        ++nl;
    }
    BZ_CUDA_TRY(cudaGetLastError());
    if (launches) *launches += nl;
    return BZ_OK;
}

template <int N> static void h_fp32_n(Plan &pl, const float2 *fin, cudaStream_t st) {
    plane_inv<N, false>(fin, pl.tw, pl.S, 0, 1, 0, st);
    k_pencil<N, 0><<<dim3((N * N + 127) / 128, 1), 128, 0, st>>>(pl.S, nullptr, pl.h);
}

bz_status h_fp32(Plan &pl, const float2 *fin, cudaStream_t st) {
    switch (pl.N) {
        case 8: h_fp32_n<8>(pl, fin, st); break;
        case 16: h_fp32_n<16>(pl, fin, st); break;
        case 32: h_fp32_n<32>(pl, fin, st); break;
        default: return BZ_ERR_UNSUPPORTED;
    }
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

bz_status load_input(Plan &pl, const void *fhat, int dtype, cudaStream_t st, int *launches) {
    const int n3 = (int)modes(pl);
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    if (pl.Nin) {
        // padded: embed into the 2N grid, in FP32 and (where the FP64 h pass reads it) FP64
        k_embed<<<(n3 + 255) / 256, 256, 0, st>>>(fhat, dtype, pl.Nin, pl.N, pl.fin, pl.fin64);
        BZ_CUDA_TRY(cudaGetLastError());
        pl.src = pl.fin64;
        pl.src_dtype = BZ_C128;
        if (launches) *launches += 1;
        return BZ_OK;
    }
    pl.src = fhat;                 // the fused path forms h from the caller's array in FP64
    pl.src_dtype = dtype;
    if (dtype == BZ_C64) {
        BZ_CUDA_TRY(cudaMemcpyAsync(pl.fin, fhat, (size_t)n3 * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    } else if (dtype == BZ_C128) {
        k_c128_to_c64<<<(n3 + 255) / 256, 256, 0, st>>>((const double2 *)fhat, pl.fin, n3);
        BZ_CUDA_TRY(cudaGetLastError());
        if (launches) *launches += 1;
    } else {
        return BZ_ERR_ARG;
    }
    return BZ_OK;
}

// Q over terms [p0, p1) of the FP32 input already in pl.fin; result in pl.acc (FP64).
bz_status collide_core(Plan &pl, int p0, int p1, cudaStream_t st, int *launches) {
    if (pl.dim == 2) return collide_2d(pl, p0, p1, st, launches);
    if (pl.use_fused) return collide_fused(pl, p0, p1, st, launches);
    switch (pl.N) {
        case 8: return run_chunks<8>(pl, p0, p1, st, launches);
        case 16: return run_chunks<16>(pl, p0, p1, st, launches);
        case 24: return run_chunks<24>(pl, p0, p1, st, launches);
        case 32: return run_chunks<32>(pl, p0, p1, st, launches);
        case 48: return run_chunks<48>(pl, p0, p1, st, launches);
        case 64: return run_chunks<64>(pl, p0, p1, st, launches);
    }
    return BZ_ERR_ARG;
}

bz_status collide_range(Plan &pl, int p0, int p1, const void *fhat, int in_dtype, cudaStream_t st,
                        int *launches) {
    bz_status s = load_input(pl, fhat, in_dtype, st, launches);
    if (s != BZ_OK) return s;
    return collide_core(pl, p0, p1, st, launches);
}

bz_status write_output(Plan &pl, void *Qhat, int dtype, cudaStream_t st, int *launches) {
    const int n3 = (int)modes(pl);
    if (pl.Nin) {
        if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
        const int m3 = pl.Nin * pl.Nin * pl.Nin;
        k_extract<<<(m3 + 255) / 256, 256, 0, st>>>(pl.acc, pl.Nin, pl.N, Qhat, dtype, nonfinite_flag(pl));
        BZ_CUDA_TRY(cudaGetLastError());
        if (launches) *launches += 1;
        return BZ_OK;
    }
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    k_acc_out<<<(n3 + 255) / 256, 256, 0, st>>>(pl.acc, Qhat, dtype, n3, nonfinite_flag(pl));
    BZ_CUDA_TRY(cudaGetLastError());
    if (launches) *launches += 1;
    return BZ_OK;
}

}  // namespace bz

// =======================================================================================
// Allocation-free collide.
//
// Some callers cannot let this library allocate device memory during a call: an
// application whose device memory is fully reserved up front by its own pool
// allocator, a latency-critical time loop that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree, or a host process that forbids a library
// from growing its footprint after start-up.  bz_collide_noalloc serves them: its
// scratch (FP32 input copy, h, the FP64 accumulator and the term chunk) lives in one
// file-scope device array of kNoallocBytes, which every GPU that loads libbz holds
// until the process exits.  The caller passes the plan (built beforehand) and the
// input and output arrays; nothing is allocated or freed during the call.  h is formed as
// bz_collide forms it on the same plan (FP64 on the fused pipeline unless the plan asks for
// FP32 h, FP32 on the chunked one), so both compute the same operator.
// =======================================================================================
namespace bz {
namespace {

constexpr size_t kNoallocBytes = (size_t)8 << 20;   // 8 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Device address of the scratch array on the current device.  In host code the symbol is
// only a stand-in, so the address is looked up with the device current, on every call: the
// lookup allocates nothing, and a fresh address after cudaDeviceReset is picked up.  The first
// lookup on a device may load the module there.
bz_status noalloc_scratch(unsigned char **out) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return BZ_ERR_CUDA;
    *out = (unsigned char *)p;
    return BZ_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Scratch layout (256-byte blocks): fin (8 N^3 bytes), h (8 N^3), acc (16 N^3), the FP64 h
// pass's scratch where the plan forms h in FP64 (16 N^3), then T terms of 8 N^3.
template <int N>
bz_status run_noalloc(const Plan &pl, const void *fhat, void *Qhat, int dtype, unsigned char *base,
                      bool h64, int T, cudaStream_t st) {
    constexpr int PPC = Cfg<N>::PPC;
    const int n3 = N * N * N;
    const size_t field = (size_t)n3 * sizeof(float2);
    float2 *fin = (float2 *)base;
    float2 *h = (float2 *)(base + align256(field));
    double2 *acc = (double2 *)(base + 2 * align256(field));
    double2 *scr64 = (double2 *)(base + 2 * align256(field) + align256(2 * field));
    float2 *S = (float2 *)(base + 2 * align256(field) + (h64 ? 2 : 1) * align256(2 * field));
    if (dtype == BZ_C64) {
        BZ_CUDA_TRY(cudaMemcpyAsync(fin, fhat, field, cudaMemcpyDeviceToDevice, st));
    } else {
        k_c128_to_c64<<<(n3 + 255) / 256, 256, 0, st>>>((const double2 *)fhat, fin, n3);
    }
    if (h64) {
        // as bz_collide on this plan: h from the caller's coefficients in FP64, stored FP32
        const bz_status s = h64_launch(N, fhat, dtype, nullptr, nullptr, 1, scr64, h, st);
        if (s != BZ_OK) return s;
    } else {
        k_plane_inv<N><<<dim3(N / PPC, 1), Cfg<N>::THREADS, Cfg<N>::SMEM, st>>>(fin, pl.tw, S, 0, 0);
        k_pencil<N, 0><<<dim3((N * N + 127) / 128, 1), 128, 0, st>>>(S, nullptr, h);
    }
    BZ_CUDA_TRY(cudaMemsetAsync(acc, 0, (size_t)n3 * sizeof(double2), st));   // left over from the last call
    for (int c0 = 0; c0 < pl.P; c0 += T) {
        const int Tc = (pl.P - c0) < T ? (pl.P - c0) : T;
        k_plane_inv<N><<<dim3(N / PPC, Tc), Cfg<N>::THREADS, Cfg<N>::SMEM, st>>>(fin, pl.tw, S, c0, 1);
        k_pencil<N, 1><<<dim3((N * N + 127) / 128, Tc), 128, 0, st>>>(S, h, nullptr);
        k_plane_fwd<N><<<dim3(N / PPC, Tc), Cfg<N>::THREADS, Cfg<N>::SMEM, st>>>(S, pl.alpha, c0);
        k_reduce<<<(n3 / 2 + 255) / 256, 256, 0, st>>>(S, Tc, n3, acc);
    }
    k_kahan_fold<<<(n3 / 2 + 255) / 256, 256, 0, st>>>(acc, n3);
    if (dtype == BZ_C128) {
        BZ_CUDA_TRY(cudaMemcpyAsync(Qhat, acc, (size_t)n3 * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    } else {
        k_acc_to_c64<<<(n3 + 255) / 256, 256, 0, st>>>(acc, (float2 *)Qhat, n3);
    }
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

}  // namespace

const Plan *plan_internal(const bz_plan *plan);

}  // namespace bz

extern "C" bz_status bz_collide_noalloc(const bz_plan *plan, const void *fhat, void *Qhat, int dtype,
                                        void *stream) {
    using namespace bz;
    if (!plan || !fhat || !Qhat || fhat == Qhat) return BZ_ERR_ARG;
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    const Plan &pl = *plan_internal(plan);
    if (pl.Nin || pl.dim == 2 || pl.real) return BZ_ERR_UNSUPPORTED;   // padded, 2D and real-data plans: bz_collide
    if (pl.precision != BZ_PREC_FP32) return BZ_ERR_UNSUPPORTED;        // split-BF16 plans: bz_collide
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return BZ_ERR_CUDA;
    if (dev != pl.device) return BZ_ERR_ARG;
    // h as bz_collide forms it on this plan: FP64 on the fused pipeline with FP64 h, else FP32
    const bool h64 = pl.use_fused && pl.h_fp64;
    const size_t n3 = (size_t)pl.N * pl.N * pl.N;
    const size_t field = n3 * sizeof(float2);
    const size_t fixed = 2 * align256(field) + (h64 ? 2 : 1) * align256(2 * field);   // fin, h, acc (, scr64)
    if (fixed + field > kNoallocBytes) return BZ_ERR_ARG;               // not even one term fits
    const int T = (int)std::min<size_t>((kNoallocBytes - fixed) / field, (size_t)pl.P);
    unsigned char *base = nullptr;
    bz_status s = noalloc_scratch(&base);
    if (s != BZ_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    switch (pl.N) {
        case 8: return run_noalloc<8>(pl, fhat, Qhat, dtype, base, h64, T, st);
        case 16: return run_noalloc<16>(pl, fhat, Qhat, dtype, base, h64, T, st);
        case 24: return run_noalloc<24>(pl, fhat, Qhat, dtype, base, h64, T, st);
        case 32: return run_noalloc<32>(pl, fhat, Qhat, dtype, base, h64, T, st);
        case 48: return run_noalloc<48>(pl, fhat, Qhat, dtype, base, h64, T, st);
        case 64: return run_noalloc<64>(pl, fhat, Qhat, dtype, base, h64, T, st);
    }
    return BZ_ERR_ARG;
}

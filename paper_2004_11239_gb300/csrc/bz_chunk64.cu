// The plane and pencil passes of the chunked pipeline (Sec. 4, eq. realQ) at N = 64: one plane
// per CTA, or 32 lines along axis 1 per CTA.
//
// A 64-point transform is split as 64 = 8 x 8 (n = 8 n1 + n2, k = k1 + 8 k2):
//     X[k1 + 8 k2] = sum_n2 W8^(n2 k2) [ W64^(n2 k1) sum_n1 x[8 n1 + n2] W8^(n1 k1) ],
// so each of 8 threads takes one n2 (stage 1: an 8-point DFT over n1, then the twiddle
// W64^(n2 k1)), the 8 x 8 block is transposed through shared memory, and each thread takes one
// k1 (stage 2: an 8-point DFT over n2).  A thread holds 8 values instead of a whole line, so a
// 512-thread CTA transforms a 64 x 64 plane with about 64 registers per thread (the generic
// kernels hold a line of 64 per thread: 168 registers, 12 warps per SM).
//   rows (contiguous axis): the 8 threads of a row sit in one warp, the transpose needs only
//     __syncwarp; its shared-memory slots are XOR-swizzled (8 k1 + (n2 ^ k1)) so that neither
//     the stage-1 stores nor the stage-2 loads conflict;
//   columns: a warp holds 32 consecutive columns of one n2, every access is a contiguous row
//     segment; the transpose needs __syncthreads.
// k_plane_inv64: twiddle (beta_p, or the pair's beta_p + i beta_p') on load from global, inverse
//   transform along k3 (rows) then k2 (columns), result to S[t][k1][j2][j3].
// k_plane_fwd64: forward transform along j2 (columns, loaded from S) then j3 (rows), times the
//   weight alpha_p (or the pair table A), whose 8 values per thread are loaded at the start so
//   the HBM stream overlaps the transforms (a batch slot's radial scale, if given, multiplies
//   the transformed field); result to S; the pair form also writes the Nyquist
//   sums X = C Z of the plane (family layout [3][N][N], every entry of this k1 written).
#include "bz_fft.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

constexpr int N64 = 64;
constexpr int RP = 72;                 // row pitch (float2): rows r, r + 1 fall on opposite bank halves
constexpr int T64 = 512;               // threads per CTA
constexpr size_t kTileBytes = (size_t)N64 * RP * sizeof(float2);
constexpr size_t kInvSmem = kTileBytes + (6 * N64 + N64) * sizeof(float2);   // tile, twiddles, W64
constexpr size_t kFwdSmem = kTileBytes + N64 * sizeof(float2);

// W64^(SIGN j) from the table w[j] = exp(+2 pi i j / 64)
template <int SIGN> __device__ __forceinline__ float2 w64(const float2 *w, int j) {
    float2 v = w[j & 63];
    if (SIGN < 0) v.y = -v.y;
    return v;
}

__device__ __forceinline__ void load_w64(float2 *w) {
    if (threadIdx.x < N64) w[threadIdx.x] = c_tw.v[tw_off<64>() + threadIdx.x];
}

// Stage 1 of a 64-point transform on the thread's 8 values x[n1] = x(8 n1 + n2): the 8-point
// DFT over n1 and the twiddle W64^(SIGN n2 k1); x[k1] holds Y[n2][k1] after it.
template <int SIGN> __device__ __forceinline__ void stage1(float2 (&x)[8], int n2, const float2 *w) {
    fft_inplace<8, SIGN>(x);
    #pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) x[k1] = cmul(x[k1], w64<SIGN>(w, n2 * k1));
}

// stage1 where n2 = q is the same across the warp: the twiddles come from the constant table
// as broadcasts instead of from shared memory.
template <int SIGN> __device__ __forceinline__ void stage1u(float2 (&x)[8], int q) {
    fft_inplace<8, SIGN>(x);
    #pragma unroll
    for (int k1 = 1; k1 < 8; ++k1) {
        float2 w = c_tw.v[tw_off<64>() + ((q * k1) & 63)];
        if (SIGN < 0) w.y = -w.y;
        x[k1] = cmul(x[k1], w);
    }
}

// Row pass of the plane held in `tile` (natural order) or, for the first pass of plane_inv, in
// registers: thread (r, n2) = (tid / 8, tid % 8) holds x[n1] = row r element 8 n1 + n2 on entry
// and y[k2] = row r element kk + 8 k2 of the transform (kk = n2) on exit.  The row's slots of
// the tile are overwritten (swizzled scratch).
template <int SIGN> __device__ __forceinline__ void row_pass(float2 (&x)[8], float2 *tile, int r, int n2,
                                                             const float2 *w) {
    stage1<SIGN>(x, n2, w);
    float2 *row = tile + r * RP;
    __syncwarp();                                         // the row's natural-order loads are done
    #pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) row[8 * k1 + (n2 ^ k1)] = x[k1];
    __syncwarp();
    #pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = row[8 * n2 + (m ^ n2)];   // Y[m][kk], kk = n2
    fft_inplace<8, SIGN>(x);                              // x[k2] = X[kk + 8 k2]
}

template <bool PAIR>
__global__ void __launch_bounds__(T64, 2)
k_plane_inv64(const float2 *__restrict__ fin, const float2 *__restrict__ tw, float2 *__restrict__ S, int p0,
              int use_tw) {
    extern __shared__ float2 sm[];
    float2 *tile = sm;
    float2 *stw = sm + N64 * RP;
    float2 *w = stw + 6 * N64;
    const int tid = threadIdx.x, k1p = blockIdx.x, t = blockIdx.y;
    const int r = tid >> 3, n2 = tid & 7;
    // the plane's row r, elements 8 n1 + n2, straight from global (L2)
    const float2 *f = fin + ((size_t)k1p * N64 + r) * N64 + n2;
    float2 x[8];
    #pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) x[n1] = f[8 * n1];
    load_w64(w);
    if (use_tw) {
        constexpr int NT = (PAIR ? 6 : 3) * N64;
        const float2 *twp = tw + (size_t)(p0 + t) * NT;
        for (int i = tid; i < NT; i += T64) stw[i] = twp[i];
    }
    __syncthreads();
    if (use_tw) {
        // beta(k1, k2, k3) = b1(k1) b2(k2) b3(k3) per term; the pair form takes b + i b'
        const float2 a = cmul(stw[k1p], stw[N64 + r]);
        if constexpr (PAIR) {
            const float2 b = cmul(stw[3 * N64 + k1p], stw[4 * N64 + r]);
            #pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) {
                const int k3 = 8 * n1 + n2;
                const float2 u = cmul(a, stw[2 * N64 + k3]), v = cmul(b, stw[5 * N64 + k3]);
                x[n1] = cmul(x[n1], make_float2(u.x - v.y, u.y + v.x));
            }
        } else {
            #pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) x[n1] = cmul(x[n1], cmul(a, stw[2 * N64 + 8 * n1 + n2]));
        }
    }
    row_pass<+1>(x, tile, r, n2, w);                      // axis 3: k3 -> j3
    __syncwarp();                                         // the row's swizzled loads are done
    #pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) tile[r * RP + n2 + 8 * k2] = x[k2];
    __syncthreads();
    // axis 2: k2 -> j2, column c, thread (c, m2) = (tid % 64, tid / 64)
    const int c = tid & 63, m2 = tid >> 6;
    #pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) x[n1] = tile[(8 * n1 + m2) * RP + c];
    stage1u<+1>(x, m2);
    #pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) tile[(8 * k1 + m2) * RP + c] = x[k1];   // the rows it read: no hazard
    __syncthreads();
    #pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = tile[(8 * m2 + m) * RP + c];
    fft_inplace<8, +1>(x);                                // x[k2] = column c at j2 = m2 + 8 k2
    float2 *out = S + (size_t)t * N64 * N64 * N64 + (size_t)k1p * N64 * N64 + c;
    #pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) out[(m2 + 8 * k2) * N64] = x[k2];
}

template <bool PAIR>
__global__ void __launch_bounds__(T64, 2)
k_plane_fwd64(float2 *__restrict__ S, const float2 *__restrict__ alpha, int p0, const float2 *__restrict__ cpair,
              float2 *__restrict__ Ss, const float *__restrict__ gsc, int M) {
    extern __shared__ float2 sm[];
    float2 *tile = sm;
    float2 *w = sm + N64 * RP;
    const int tid = threadIdx.x, k1p = blockIdx.x, t = blockIdx.y;
    const int r = tid >> 3, n2 = tid & 7;                 // row-pass roles
    const int c = tid & 63, m2 = tid >> 6;                // column-pass roles
    float2 *pl = S + (size_t)t * N64 * N64 * N64 + (size_t)k1p * N64 * N64;
    // the weights of this thread's 8 outputs (row r, k3 = n2 + 8 k2): from HBM, in flight
    // during both transforms
    const float2 *al = alpha + ((size_t)(p0 + t) * N64 * N64 * N64 + (size_t)k1p * N64 * N64 + (size_t)r * N64 + n2);
    float2 a[8];
    #pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) a[k2] = al[8 * k2];
    float2 x[8];
    #pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) x[n1] = pl[(8 * n1 + m2) * N64 + c];
    load_w64(w);
    __syncthreads();
    // axis 2: j2 -> k2 on column c
    stage1u<-1>(x, m2);
    #pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) tile[(8 * k1 + m2) * RP + c] = x[k1];
    __syncthreads();
    #pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = tile[(8 * m2 + m) * RP + c];
    fft_inplace<8, -1>(x);                                // x[k2] = column c at k2 = m2 + 8 k2
    __syncthreads();                                      // every stage-2 load is done
    #pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) tile[(m2 + 8 * k2) * RP + c] = x[k2];
    __syncthreads();
    // axis 3: j3 -> k3 on row r (= k2)
    #pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) x[n1] = tile[r * RP + 8 * n1 + n2];
    row_pass<-1>(x, tile, r, n2, w);                      // x[k2] = Z(k2 = r, k3 = n2 + 8 k2)
    if (gsc) {                                            // a batch slot's radial scale (a pair shares its node)
        const float sc = gsc[(PAIR ? 2 * (p0 + t) : p0 + t) / M];
        #pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) x[k2] = cscale(x[k2], sc);
    }
    float2 *o = pl + (size_t)r * N64 + n2;
    #pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) o[8 * k2] = cmul(x[k2], a[k2]);
    if constexpr (PAIR) {
        const float2 *cq = cpair + (size_t)(p0 + t) * 3 * N64 * N64;
        float2 *xs = Ss + (size_t)t * 3 * N64 * N64;
        if (r == N64 / 2) {                               // family k2 = -N/2: [k1][k3]
            #pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) {
                const int k3 = n2 + 8 * k2;
                xs[N64 * N64 + k1p * N64 + k3] = cmul(x[k2], cq[N64 * N64 + k1p * N64 + k3]);
            }
        }
        if (n2 == 0)                                      // family k3 = -N/2 (k3 = 32: k2 = 4): [k1][k2]
            xs[2 * N64 * N64 + k1p * N64 + r] = cmul(x[4], cq[2 * N64 * N64 + k1p * N64 + r]);
        if (k1p == N64 / 2) {                             // the plane k1 = -N/2: [k2][k3]
            #pragma unroll
            for (int k2 = 0; k2 < 8; ++k2) {
                const int k3 = n2 + 8 * k2;
                xs[r * N64 + k3] = cmul(x[k2], cq[r * N64 + k3]);
            }
        }
    }
}

// The pencil pass at N = 64: 32 lines (j2, j3), (j2, j3 + 1), ... of one term per 256-thread
// CTA, each 64-point transform along axis 1 split 8 x 8 as in the plane passes: warp q holds
// the elements 8 n1 + q of its lane's line, and the 8 x 8 transposes go through shared memory
// (every warp access is 32 consecutive slots: no bank conflict).  The inverse transform leaves
// warp q with j1 = q + 8 k2, which is the order the forward transform's first stage takes
// (n2 = q, n1 = k2), so the product with h needs no transpose in between.
//   MODE 0: out = IFFT_1(S)               (forms h)
//   MODE 1: S = FFT_1(h . IFFT_1(S))      (in place)
//   MODE 2: as MODE 1 with h real, read as N^3 packed floats (BZ_DATA_REAL)
//   MODE 3: out = Re IFFT_1(S) as N^3 packed floats (forms the real h of MODE 2)
constexpr int PL = 32;                 // lines per CTA, one per lane
constexpr int TP = 256;                // threads per CTA: warp q = n2 in stage 1, k1 in stage 2

// x[k1] = Y[q][k1] on entry; x[k2] = X[q + 8 k2] on exit (tile free again once every thread
// has passed the caller's next barrier)
template <int SIGN> __device__ __forceinline__ void pencil_stage2(float2 (&x)[8], float2 *tile, int q, int lane) {
    #pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) tile[(8 * k1 + q) * PL + lane] = x[k1];
    __syncthreads();
    #pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = tile[(8 * q + m) * PL + lane];
    fft_inplace<8, SIGN>(x);
}

template <int MODE>
__global__ void __launch_bounds__(TP, 4)
k_pencil64(float2 *__restrict__ S, const float2 *__restrict__ h, float2 *__restrict__ out) {
    constexpr int N2 = N64 * N64;
    __shared__ float2 tile[N64 * PL];
    const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
    const int g = blockIdx.x * PL + lane;                 // line (j2, j3) = g
    float2 *base = S + (size_t)blockIdx.y * N64 * N2 + g;
    float2 x[8];
    #pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) x[n1] = base[(size_t)(8 * n1 + q) * N2];
    stage1u<+1>(x, q);                                    // axis 1: k1 -> j1
    pencil_stage2<+1>(x, tile, q, lane);                  // x[k2] = line at j1 = q + 8 k2
    if constexpr (MODE == 0) {
        #pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) out[(size_t)(q + 8 * k2) * N2 + g] = x[k2];
    } else if constexpr (MODE == 3) {
        #pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) ((float *)out)[(size_t)(q + 8 * k2) * N2 + g] = x[k2].x;
    } else {
        #pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) {
            const size_t j = (size_t)(q + 8 * k2) * N2 + g;
            if constexpr (MODE == 2) {
                const float hv = ((const float *)h)[j];
                x[k2].x *= hv;
                x[k2].y *= hv;
            } else {
                x[k2] = cmul(x[k2], h[j]);
            }
        }
        stage1u<-1>(x, q);                                // axis 1: j1 -> k1 (n1 = k2, n2 = q)
        __syncthreads();                                  // every read of the first transpose is done
        pencil_stage2<-1>(x, tile, q, lane);              // x[k2] = k1 = q + 8 k2
        #pragma unroll
        for (int k2 = 0; k2 < 8; ++k2) base[(size_t)(q + 8 * k2) * N2] = x[k2];
    }
}

}  // namespace

cudaError_t chunk64_set_attributes() {
    const void *inv[2] = {(const void *)k_plane_inv64<false>, (const void *)k_plane_inv64<true>};
    const void *fwd[2] = {(const void *)k_plane_fwd64<false>, (const void *)k_plane_fwd64<true>};
    for (const void *k : inv) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kInvSmem);
        if (e != cudaSuccess) return e;
    }
    for (const void *k : fwd) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void plane_inv64(const float2 *fin, const float2 *tw, float2 *S, int p0, int T, int use_tw, bool pair,
                 cudaStream_t st) {
    if (pair) k_plane_inv64<true><<<dim3(N64, T), T64, kInvSmem, st>>>(fin, tw, S, p0, use_tw);
    else k_plane_inv64<false><<<dim3(N64, T), T64, kInvSmem, st>>>(fin, tw, S, p0, use_tw);
}

void plane_fwd64(float2 *S, const float2 *alpha, int p0, int T, const float2 *cpair, float2 *Ss, const float *gsc,
                 int M, bool pair, cudaStream_t st) {
    if (pair) k_plane_fwd64<true><<<dim3(N64, T), T64, kFwdSmem, st>>>(S, alpha, p0, cpair, Ss, gsc, M);
    else k_plane_fwd64<false><<<dim3(N64, T), T64, kFwdSmem, st>>>(S, alpha, p0, nullptr, nullptr, gsc, M);
}

void pencil64(float2 *S, const float2 *h, float2 *out, int T, int mode, cudaStream_t st) {
    const dim3 grid(N64 * N64 / PL, T);
    if (mode == 0) k_pencil64<0><<<grid, TP, 0, st>>>(S, nullptr, out);
    else if (mode == 1) k_pencil64<1><<<grid, TP, 0, st>>>(S, h, nullptr);
    else if (mode == 2) k_pencil64<2><<<grid, TP, 0, st>>>(S, h, nullptr);
    else k_pencil64<3><<<grid, TP, 0, st>>>(S, nullptr, out);
}

}  // namespace bz

// Free streaming df/dt + v_1 df/dx = 0 of nx cells of Fourier coefficients (bz_transport_x).
//
// With f(x_c, v) = sum_k fhat_c(k) exp(i pi k.v / L) the exact solution f(x - v_1 t, v) at the
// velocity nodes needs the values along v_1 only: for each (k2, k3), the nx x N array
// fhat_c(k1, k2, k3) is transformed over the cells (x-DFT), over k1 to the node values
// f(v_1j) = sum_k1 (-1)^k1 fhat(k1) exp(2 pi i k1 j / N) (the factor (-1)^k1 = exp(-i pi k1)
// from the grid origin -L), multiplied by exp(-2 pi i kappa v_1j t / Lx), and transformed back.
// One CTA per (k2, k3); FP64 register FFTs; the array sits in shared memory between the passes.
#include <cmath>

#include "bz_fft.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

__device__ __forceinline__ double2 load_cd(const void *f, int dtype, size_t i) {
    if (dtype == BZ_C128) return ((const double2 *)f)[i];
    const float2 v = ((const float2 *)f)[i];
    return make_double2(v.x, v.y);
}
__device__ __forceinline__ void store_cd(void *f, int dtype, size_t i, double2 v) {
    if (dtype == BZ_C128) ((double2 *)f)[i] = v;
    else ((float2 *)f)[i] = make_float2((float)v.x, (float)v.y);
}

template <int N, int NX>
__global__ void __launch_bounds__(N > NX ? N : NX) k_transport(void *f, int dtype, double L, double Lx, double t) {
    __shared__ double2 s[NX][N + 1];
    const size_t n3 = (size_t)N * N * N;
    const size_t line = blockIdx.x;                          // k2 N + k3
    const int tid = threadIdx.x;
    if (tid < N) {                                           // column k1 = tid over the cells
        double2 x[NX];
        #pragma unroll
        for (int c = 0; c < NX; ++c) x[c] = load_cd(f, dtype, c * n3 + (size_t)tid * N * N + line);
        fft_inplace<NX, -1>(x);                              // cells -> x-modes kappa
        #pragma unroll
        for (int c = 0; c < NX; ++c) s[c][tid] = x[c];
    }
    __syncthreads();
    if (tid < NX) {                                          // x-mode row c over k1
        double2 y[N];
        #pragma unroll
        for (int i = 0; i < N; ++i) {
            const double2 v = s[tid][i];
            y[i] = (i & 1) ? make_double2(-v.x, -v.y) : v;
        }
        fft_inplace<N, +1>(y);                               // k1 -> node values f(v_1j)
        const double kappa = tid < NX / 2 ? tid : tid - NX;
        const double a = -2.0 * kappa * t / Lx;              // phase exp(i pi a v_1j)
        #pragma unroll
        for (int j = 0; j < N; ++j) {
            double sn, cs;
            sincospi(a * (-L + 2.0 * L * j / N), &sn, &cs);
            y[j] = make_double2(y[j].x * cs - y[j].y * sn, y[j].x * sn + y[j].y * cs);
        }
        fft_inplace<N, -1>(y);                               // node values -> k1
        const double inv = 1.0 / ((double)N * NX);           // both inverse normalisations
        #pragma unroll
        for (int i = 0; i < N; ++i) {
            const double sg = (i & 1) ? -inv : inv;
            s[tid][i] = make_double2(y[i].x * sg, y[i].y * sg);
        }
    }
    __syncthreads();
    if (tid < N) {
        double2 x[NX];
        #pragma unroll
        for (int c = 0; c < NX; ++c) x[c] = s[c][tid];
        fft_inplace<NX, +1>(x);                              // x-modes -> cells
        #pragma unroll
        for (int c = 0; c < NX; ++c) store_cd(f, dtype, c * n3 + (size_t)tid * N * N + line, x[c]);
    }
}

template <int N, int NX> bz_status run(void *f, int dtype, double L, double Lx, double t, cudaStream_t st) {
    k_transport<N, NX><<<N * N, N > NX ? N : NX, 0, st>>>(f, dtype, L, Lx, t);
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

template <int N> bz_status run_nx(int nx, void *f, int dtype, double L, double Lx, double t, cudaStream_t st) {
    switch (nx) {
        case 8: return run<N, 8>(f, dtype, L, Lx, t, st);
        case 16: return run<N, 16>(f, dtype, L, Lx, t, st);
        case 24: return run<N, 24>(f, dtype, L, Lx, t, st);
        case 32: return run<N, 32>(f, dtype, L, Lx, t, st);
    }
    return BZ_ERR_UNSUPPORTED;
}

}  // namespace

bz_status transport_x(int N, double L, int nx, double Lx, void *f, int dtype, double t, cudaStream_t st) {
    switch (N) {
        case 8: return run_nx<8>(nx, f, dtype, L, Lx, t, st);
        case 16: return run_nx<16>(nx, f, dtype, L, Lx, t, st);
        case 24: return run_nx<24>(nx, f, dtype, L, Lx, t, st);
        case 32: return run_nx<32>(nx, f, dtype, L, Lx, t, st);
    }
    return BZ_ERR_UNSUPPORTED;
}

}  // namespace bz

extern "C" bz_status bz_transport_x(int N, double L, int nx, double Lx, void *fcells, int dtype, double t,
                                    void *stream) {
    if (!fcells || !(L > 0) || !(Lx > 0) || !std::isfinite(t)) return BZ_ERR_ARG;
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    return bz::transport_x(N, L, nx, Lx, fcells, dtype, t, (cudaStream_t)stream);
}

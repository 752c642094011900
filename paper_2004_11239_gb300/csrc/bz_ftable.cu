// FP64 weight table F(k, r_i, qhat_j) on the GPU (Sec. 2.1 eq. FF, Sec. 4.1 split, 3D).
//
// With a = pi r / (2L), kappa = k.qhat, kperp = |k - kappa qhat|, x = a kappa, y = a kperp
// and g(t) = sin(t) b(cos t), the phi integral of eq. FF3D1 is exact (2 pi J0), so
//   F = 2 pi [ i x A1 - x^2 A2 / 2 - y^2 A3 / 4 ]                          (part I, [0, eps])
//     + 2 pi sum_n W_n [ (exp(i x c_n) - 1) J0(y s_n) + (J0(y s_n) - 1) ]   (part II, [eps, pi])
// with c_n = 1 - cos t_n, s_n = sin t_n, W_n = w_n g(t_n) from the host rule of the
// radial node.  The table stores alpha_p(k) = c_p F / N^3 in FP32 (the N^-3 of the
// forward transform folded in).  J0 is CUDA's double-precision j0; J0 - 1 uses its
// power series for small arguments to avoid cancellation.
#include <cmath>
#include <vector>

#include "bz_internal.h"

namespace bz {

namespace {

__device__ __forceinline__ double j0m1(double z) {
    if (fabs(z) < 0.25) {
        // J0(z) - 1 = sum_{m >= 1} (-(z/2)^2)^m / (m!)^2, Horner form to m = 8
        double u = -0.25 * z * z;
        double s = 1.0;
        #pragma unroll
        for (int m = 8; m >= 2; --m) s = 1.0 + s * u / ((double)m * (double)m);
        return u * s;
    }
    return j0(z) - 1.0;
}

// F for one (x, y) pair over one radial node's rule (nodes staged in shared memory).
__device__ __forceinline__ double2 f_value(double x, double y, const double *A, int n,
                                           const double *omc, const double *sn, const double *W) {
    double sr = -0.5 * x * x * A[1] - 0.25 * y * y * A[2];
    double si = x * A[0];
    for (int q = 0; q < n; ++q) {
        double jm1 = j0m1(y * sn[q]);
        double J = 1.0 + jm1;
        double sh, ch;
        sincos(0.5 * x * omc[q], &sh, &ch);
        // exp(i x c) - 1 = -2 sin^2(x c / 2) + i 2 sin(x c / 2) cos(x c / 2)
        sr += W[q] * (-2.0 * sh * sh * J + jm1);
        si += W[q] * (2.0 * sh * ch * J);
    }
    return make_double2(2.0 * M_PI * sr, 2.0 * M_PI * si);
}

struct TableArgs {
    int N, M, P, p0;
    int nin;                 // > 0: alpha is zero outside the signed range [-nin/2, nin/2) per axis
    double L, inv_n3;
    double A0, A1, A2;
    const double *term;      // [P][5]: r, q0, q1, q2, c
    const double *rule;      // concatenated omc | sn | W per radial node
    const int *rule_off;     // [N_rho + 1]
    float2 *alpha;           // [P][N^3]
};

// grid: x over N^3 / blockDim, y over terms p0 + blockIdx.y
__global__ void ftable_kernel(TableArgs a) {
    extern __shared__ double sm[];
    const int p = a.p0 + blockIdx.y;
    const int i = p / a.M;
    const int off = a.rule_off[i];
    const int n = a.rule_off[i + 1] - off;
    double *omc = sm, *sn = sm + n, *W = sm + 2 * n;
    const double *src = a.rule + 3 * (size_t)off;
    for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) sm[t] = src[t];
    __syncthreads();
    const int n3 = a.N * a.N * a.N;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n3) return;
    const int N = a.N;
    int i1 = idx / (N * N), i2 = (idx / N) % N, i3 = idx % N;
    int k1 = i1 < N / 2 ? i1 : i1 - N;
    int k2 = i2 < N / 2 ? i2 : i2 - N;
    int k3 = i3 < N / 2 ? i3 : i3 - N;
    // F(-k) = conj F(k) (eq. FF): the entry of the smaller index of each pair (k, -k) is computed
    // and written to both; modes with a Nyquist component (-N/2) have no partner.
    const bool nyq = k1 == -N / 2 || k2 == -N / 2 || k3 == -N / 2;
    int midx = -1;
    if (!nyq) {
        midx = (((-k1 + N) % N) * N + ((-k2 + N) % N)) * N + ((-k3 + N) % N);
        if (midx < idx) return;                           // written by the partner's thread
    }
    // padded plans: only the modes of the caller's grid carry a weight (both members of the pair
    // are tested: -k leaves the range when a component of k is -nin/2)
    const int h = a.nin / 2;
    const bool in_k = a.nin == 0 || (k1 >= -h && k1 < h && k2 >= -h && k2 < h && k3 >= -h && k3 < h);
    const bool in_m = midx >= 0 && (a.nin == 0 || (-k1 >= -h && -k1 < h && -k2 >= -h && -k2 < h && -k3 >= -h && -k3 < h));
    if (!in_k && !in_m) {
        a.alpha[(size_t)p * n3 + idx] = make_float2(0.f, 0.f);
        if (midx > idx) a.alpha[(size_t)p * n3 + midx] = make_float2(0.f, 0.f);
        return;
    }
    const double *tp = a.term + 5 * (size_t)p;
    double r = tp[0];
    double kap = k1 * tp[1] + k2 * tp[2] + k3 * tp[3];
    double kk = (double)k1 * k1 + (double)k2 * k2 + (double)k3 * k3;
    double kp2 = kk - kap * kap;
    double kp = kp2 > 0.0 ? sqrt(kp2) : 0.0;
    double aa = M_PI * r / (2.0 * a.L);
    double A[3] = {a.A0, a.A1, a.A2};
    double2 F = f_value(aa * kap, aa * kp, A, n, omc, sn, W);
    double sc = tp[4] * a.inv_n3;
    a.alpha[(size_t)p * n3 + idx] = in_k ? make_float2((float)(sc * F.x), (float)(sc * F.y)) : make_float2(0.f, 0.f);
    if (midx > idx)
        a.alpha[(size_t)p * n3 + midx] = in_m ? make_float2((float)(sc * F.x), (float)(-sc * F.y)) : make_float2(0.f, 0.f);
}

// 2D (Sec. 4.1 (i)): with x = a k.qhat, y = a k.qperp the odd terms cancel between parts I and
// III and part II folds onto [eps, pi], so
//   F = 2 [ i x A1 - x^2 A2 / 2 - y^2 A3 / 2 ] + 2 sum_n W_n [ (exp(i x c_n) - 1) cos(y s_n) + (cos(y s_n) - 1) ]
// with W_n = w_n b(t_n) (the circle's measure carries no sin t).
__device__ __forceinline__ double2 f_value_2d(double x, double y, const double *A, int n,
                                              const double *omc, const double *sn, const double *W) {
    double sr = -0.5 * x * x * A[1] - 0.5 * y * y * A[2];
    double si = x * A[0];
    for (int q = 0; q < n; ++q) {
        double sy, cy, sh, ch;
        sincos(0.5 * y * sn[q], &sy, &cy);
        const double cs = 1.0 - 2.0 * sy * sy;             // cos(y s), its deficit -2 sin^2(y s / 2)
        sincos(0.5 * x * omc[q], &sh, &ch);
        sr += W[q] * (-2.0 * sh * sh * cs - 2.0 * sy * sy);
        si += W[q] * (2.0 * sh * ch * cs);
    }
    return make_double2(2.0 * sr, 2.0 * si);
}

// 2D table: one thread per (mode of the N x N grid, term); alpha = c_p F / N^2.
__global__ void ftable2d_kernel(TableArgs a) {
    extern __shared__ double sm[];
    const int p = a.p0 + blockIdx.y;
    const int i = p / a.M;
    const int off = a.rule_off[i];
    const int n = a.rule_off[i + 1] - off;
    double *omc = sm, *sn = sm + n, *W = sm + 2 * n;
    const double *src = a.rule + 3 * (size_t)off;
    for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) sm[t] = src[t];
    __syncthreads();
    const int N = a.N, n2 = N * N;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n2) return;
    const int i1 = idx / N, i2 = idx % N;
    const int k1 = i1 < N / 2 ? i1 : i1 - N;
    const int k2 = i2 < N / 2 ? i2 : i2 - N;
    const double *tp = a.term + 5 * (size_t)p;
    const double aa = M_PI * tp[0] / (2.0 * a.L);
    const double A[3] = {a.A0, a.A1, a.A2};
    const double2 F = f_value_2d(aa * (k1 * tp[1] + k2 * tp[2]), aa * (-k1 * tp[2] + k2 * tp[1]), A, n, omc, sn, W);
    const double sc = tp[4] * a.inv_n3;
    a.alpha[(size_t)p * n2 + idx] = make_float2((float)(sc * F.x), (float)(sc * F.y));
}

struct EntryArgs {
    int N, M, P, count, dim;
    double L;
    double A0, A1, A2;
    const double *term;
    const double *rule;
    const int *rule_off;
    const int *k_idx;
    const int *tsel;
    double *out;
};

// One thread per requested entry; rule read from global memory.
__global__ void fentries_kernel(EntryArgs a) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.count) return;
    const int N = a.N;
    int p = a.tsel[e];
    int i1 = a.k_idx[3 * e], i2 = a.k_idx[3 * e + 1], i3 = a.dim == 2 ? 0 : a.k_idx[3 * e + 2];
    if (p < 0 || p >= a.P || i1 < 0 || i1 >= N || i2 < 0 || i2 >= N || i3 < 0 || i3 >= N) {
        a.out[2 * e] = nan("");          // out-of-range request: no table access
        a.out[2 * e + 1] = nan("");
        return;
    }
    int i = p / a.M;
    int off = a.rule_off[i];
    int n = a.rule_off[i + 1] - off;
    const double *src = a.rule + 3 * (size_t)off;
    int k1 = i1 < N / 2 ? i1 : i1 - N;
    int k2 = i2 < N / 2 ? i2 : i2 - N;
    int k3 = i3 < N / 2 ? i3 : i3 - N;
    const double *tp = a.term + 5 * (size_t)p;
    double aa = M_PI * tp[0] / (2.0 * a.L);
    double A[3] = {a.A0, a.A1, a.A2};
    double2 F;
    if (a.dim == 2) {
        F = f_value_2d(aa * (k1 * tp[1] + k2 * tp[2]), aa * (-k1 * tp[2] + k2 * tp[1]), A, n, src, src + n, src + 2 * n);
    } else {
        double kap = k1 * tp[1] + k2 * tp[2] + k3 * tp[3];
        double kk = (double)k1 * k1 + (double)k2 * k2 + (double)k3 * k3;
        double kp2 = kk - kap * kap;
        double kp = kp2 > 0.0 ? sqrt(kp2) : 0.0;
        F = f_value(aa * kap, aa * kp, A, n, src, src + n, src + 2 * n);
    }
    a.out[2 * e] = F.x;
    a.out[2 * e + 1] = F.y;
}

}  // namespace

// Uploads terms and theta rules; fills pl.alpha with c_p F / N^3 (FP32).
bz_status ftable_build(Plan &pl) {
    const int P = pl.P, N = pl.N;
    std::vector<double> term(5 * (size_t)P);
    for (int p = 0; p < P; ++p) {
        term[5 * p] = pl.terms.r[p];
        for (int d = 0; d < 3; ++d) term[5 * p + 1 + d] = pl.terms.q[3 * p + d];
        term[5 * p + 4] = pl.terms.c[p];
    }
    std::vector<double> rule;
    std::vector<int> off(pl.N_rho + 1, 0);
    pl.rule_max = 0;
    for (int i = 0; i < pl.N_rho; ++i) {
        const ThetaRule &R = pl.rules[i];
        int n = (int)R.W.size();
        off[i + 1] = off[i] + n;
        pl.rule_max = n > pl.rule_max ? n : pl.rule_max;
        rule.insert(rule.end(), R.omc.begin(), R.omc.end());
        rule.insert(rule.end(), R.sn.begin(), R.sn.end());
        rule.insert(rule.end(), R.W.begin(), R.W.end());
    }
    BZ_CUDA_TRY(cudaMalloc(&pl.term_dev, term.size() * sizeof(double)));
    BZ_CUDA_TRY(cudaMalloc(&pl.rule_buf, rule.size() * sizeof(double)));
    BZ_CUDA_TRY(cudaMalloc(&pl.rule_off, off.size() * sizeof(int)));
    BZ_CUDA_TRY(cudaMemcpy(pl.term_dev, term.data(), term.size() * sizeof(double), cudaMemcpyHostToDevice));
    BZ_CUDA_TRY(cudaMemcpy(pl.rule_buf, rule.data(), rule.size() * sizeof(double), cudaMemcpyHostToDevice));
    BZ_CUDA_TRY(cudaMemcpy(pl.rule_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));

    const size_t smem = 3 * (size_t)pl.rule_max * sizeof(double);
    if (smem > 200 * 1024) return BZ_ERR_UNSUPPORTED;
    if (smem > 48 * 1024) {
        BZ_CUDA_TRY(cudaFuncSetAttribute(ftable_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        BZ_CUDA_TRY(cudaFuncSetAttribute(ftable2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    TableArgs a;
    a.N = N; a.M = pl.M; a.P = P; a.L = pl.L; a.nin = pl.Nin;
    a.inv_n3 = 1.0 / (double)modes(pl);      // the forward transform's N^-d
    a.A0 = pl.A[0]; a.A1 = pl.A[1]; a.A2 = pl.A[2];
    a.term = pl.term_dev; a.rule = pl.rule_buf; a.rule_off = pl.rule_off; a.alpha = pl.alpha;
    const int n3 = (int)modes(pl), bs = 128;
    const int ychunk = 32768;   // gridDim.y limit
    for (int p0 = 0; p0 < P; p0 += ychunk) {
        a.p0 = p0;
        dim3 grid((n3 + bs - 1) / bs, (P - p0) < ychunk ? (P - p0) : ychunk);
        if (pl.dim == 2) ftable2d_kernel<<<grid, bs, smem>>>(a);
        else ftable_kernel<<<grid, bs, smem>>>(a);
        BZ_CUDA_TRY(cudaGetLastError());
    }
    BZ_CUDA_TRY(cudaDeviceSynchronize());
    return BZ_OK;
}

bz_status ftable_entries(Plan &pl, int count, const int *k_idx, const int *term, double *out) {
    if (count <= 0) return count == 0 ? BZ_OK : BZ_ERR_ARG;
    EntryArgs a;
    a.N = pl.Nin ? pl.Nin : pl.N;      // indices address the caller's grid
    a.M = pl.M; a.P = pl.P; a.count = count; a.L = pl.L; a.dim = pl.dim;
    a.A0 = pl.A[0]; a.A1 = pl.A[1]; a.A2 = pl.A[2];
    a.term = pl.term_dev; a.rule = pl.rule_buf; a.rule_off = pl.rule_off;
    a.k_idx = k_idx; a.tsel = term; a.out = out;
    fentries_kernel<<<(count + 127) / 128, 128>>>(a);
    BZ_CUDA_TRY(cudaGetLastError());
    BZ_CUDA_TRY(cudaDeviceSynchronize());
    return BZ_OK;
}

}  // namespace bz

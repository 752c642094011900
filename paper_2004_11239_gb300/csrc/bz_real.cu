// Real-data form of the operator (BZ_DATA_REAL): f real, so fhat is Hermitian.
//
// Input: fs = Hermitian part of fhat, (fhat_k + conj fhat_{-k}) / 2, with every mode that has
// an index -N/2 (set S, the Nyquist planes) zero.  Then x_p = beta_p fs is Hermitian for every
// term (beta_p(-k) = conj beta_p(k) off S), so g_p = IFFT(x_p) and h = IFFT(fs) are real and
// U_p = FFT(h g_p) / N^3 is Hermitian (modulo N, S included).  For a term pair (p, p') with
// Z = FFT(h (g_p + i g_p')):
//     U_p = (Z + Z*) / 2,  U_p' = (Z - Z*) / (2 i),  Z*(k) = conj Z(-k),
//     alpha_p U_p + alpha_p' U_p' = A Z + B Z*,  A = (alpha_p - i alpha_p') / 2,
//                                                B = (alpha_p + i alpha_p') / 2.
// Off S, F(-k) = conj F(k) gives B = conj A(-k), so the pair adds W(k) + conj W(-k), W = A Z:
// the fused kernel accumulates V = sum of W over the pairs and Q(k) = V(k) + conj V(-k) is
// formed once per collide, in the reduction over the kernel's items (k_reduce_sym).  On S (where -k stays in S but alpha_p(-k) is not conj alpha_p(k))
// the kernel also accumulates X = sum of C Z with C(k) = conj B(-k), and Q(k) = V(k) +
// conj X(-k).  Q is eq. realQ applied to fs, every mode kept.
#include "bz_internal.h"
#include "bz_real.cuh"

namespace bz {

namespace {

// fs (FP32 and FP64) from the caller's array (c64 or c128).
__global__ void k_sym_in(const void *__restrict__ f, int dtype, int N, float2 *__restrict__ fs,
                         double2 *__restrict__ fs64) {
    const int n3 = N * N * N;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n3) return;
    const int i1 = k / (N * N), i2 = (k / N) % N, i3 = k % N;
    double2 v = make_double2(0.0, 0.0);
    if (!nyquist(i1, i2, i3, N)) {
        const size_t m = mirror(i1, i2, i3, N);
        double2 a, b;
        if (dtype == BZ_C128) {
            a = ((const double2 *)f)[k];
            b = ((const double2 *)f)[m];
        } else {
            const float2 fa = ((const float2 *)f)[k], fb = ((const float2 *)f)[m];
            a = make_double2(fa.x, fa.y);
            b = make_double2(fb.x, fb.y);
        }
        v = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    }
    fs[k] = make_float2((float)v.x, (float)v.y);
    fs64[k] = v;
}

// Kahan-compensated FP32 sum.
struct Kahan {
    float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
    __device__ __forceinline__ void add(float vr, float vi) {
        const float yr = vr - cr, yi = vi - ci;
        const float tr = sr + yr, ti = si + yi;
        cr = (tr - sr) - yr;
        ci = (ti - si) - yi;
        sr = tr;
        si = ti;
    }
};

// acc(k) = V(k) + conj V(-k) off S and V(k) + conj X(-k) on S, with V and X the sums over the
// G items of part and part_s.  Block: 32 modes k x 8 slices; slice s sums items s, s + 8, ...
// of the two entries mode k needs (V(k) and V(-k), or V(k) and X(-k)), then the eight slices are
// added in order (compensated, as k_reduce_parts).  Off S the lane of the smaller index of each
// pair {k, -k} writes both entries; k = 0 is its own mirror.
__global__ void __launch_bounds__(256) k_reduce_sym(const float2 *__restrict__ part, const float2 *__restrict__ part_s,
                                                   int G, int N, double2 *__restrict__ acc) {
    __shared__ float4 red[2][8][32];
    const int n3 = N * N * N;
    const int kk = threadIdx.x % 32, sl = threadIdx.x / 32;
    const int k = blockIdx.x * 32 + kk;
    // role of mode k: 0 none, 1 off S (pair k < -k, or k = 0), 2 on S
    int role = 0;
    const float2 *pb = part;
    size_t sb = n3, j = 0;
    if (k < n3) {
        const int i1 = k / (N * N), i2 = (k / N) % N, i3 = k % N;
        const int m1 = (N - i1) % N, m2 = (N - i2) % N, m3 = (N - i3) % N;
        if (nyquist(i1, i2, i3, N)) {
            role = 2;
            pb = part_s;
            sb = (size_t)3 * N * N;
            j = family_index(m1, m2, m3, N);
        } else {
            j = ((size_t)m1 * N + m2) * N + m3;
            role = (size_t)k <= j ? 1 : 0;
        }
    }
    Kahan a, b;
    if (role) {
        #pragma unroll 4
        for (int g = sl; g < G; g += 8) {
            const float2 va = __ldcs(part + (size_t)g * n3 + k), vb = __ldcs(pb + (size_t)g * sb + j);
            a.add(va.x, va.y);
            b.add(vb.x, vb.y);
        }
    }
    red[0][sl][kk] = make_float4(a.sr, a.si, a.cr, a.ci);
    red[1][sl][kk] = make_float4(b.sr, b.si, b.cr, b.ci);
    __syncthreads();
    if (sl != 0 || !role) return;
    Kahan ta, tb;
    #pragma unroll
    for (int u = 0; u < 8; ++u) {
        const float4 qa = red[0][u][kk], qb = red[1][u][kk];
        ta.add(qa.x, qa.y);
        ta.add(-qa.z, -qa.w);
        tb.add(qb.x, qb.y);
        tb.add(-qb.z, -qb.w);
    }
    const double2 va = make_double2((double)ta.sr - (double)ta.cr, (double)ta.si - (double)ta.ci);
    const double2 vb = make_double2((double)tb.sr - (double)tb.cr, (double)tb.si - (double)tb.ci);
    if (role == 2 || (size_t)k != j) {
        acc[k] = make_double2(va.x + vb.x, va.y - vb.y);
        if (role == 1) acc[j] = make_double2(vb.x + va.x, vb.y - va.y);
    } else {
        acc[k] = make_double2(2.0 * va.x, 0.0);                       // k = 0
    }
}

// In place: acc(k) <- V(k) + conj V(-k) off S, V(k) + conj X(-k) on S (xs: the FP64 sums X in
// the family layout).  Off S the thread of the smaller index of each pair {k, -k} writes both
// entries; k = 0 is its own mirror.
__global__ void k_sym_out(double2 *__restrict__ acc, const double2 *__restrict__ xs, int N) {
    const int n3 = N * N * N;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n3) return;
    const int i1 = k / (N * N), i2 = (k / N) % N, i3 = k % N;
    const int m1 = (N - i1) % N, m2 = (N - i2) % N, m3 = (N - i3) % N;
    const double2 a = acc[k];
    if (nyquist(i1, i2, i3, N)) {
        const double2 x = xs[family_index(m1, m2, m3, N)];
        acc[k] = make_double2(a.x + x.x, a.y - x.y);
        return;
    }
    const size_t m = ((size_t)m1 * N + m2) * N + m3;
    if ((size_t)k > m) return;
    if ((size_t)k == m) {
        acc[k] = make_double2(2.0 * a.x, 0.0);
        return;
    }
    const double2 b = acc[m];
    acc[k] = make_double2(a.x + b.x, a.y - b.y);
    acc[m] = make_double2(b.x + a.x, b.y - a.y);
}

// A_q(k) = (alpha_2q(k) - i alpha_2q+1(k)) / 2 for every k.
__global__ void k_pair_table(const float2 *__restrict__ alpha, int N, int pairs, float2 *__restrict__ ap) {
    const size_t n3 = (size_t)N * N * N;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n3 * pairs) return;
    const size_t q = t / n3, k = t % n3;
    const float2 a = alpha[(2 * q) * n3 + k], b = alpha[(2 * q + 1) * n3 + k];
    ap[t] = make_float2(0.5f * (a.x + b.y), 0.5f * (a.y - b.x));
}

// C_q on the Nyquist planes in the family layout: C(k) = conj B(-k) = (conj alpha_2q(-k) -
// i conj alpha_2q+1(-k)) / 2 where k belongs to the family, 0 at the family's other entries.
__global__ void k_pair_table_s(const float2 *__restrict__ alpha, int N, int pairs, float2 *__restrict__ cp) {
    const size_t n3 = (size_t)N * N * N, ns = (size_t)3 * N * N;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ns * pairs) return;
    const size_t q = t / ns;
    const int e = (int)(t % ns), fam = e / (N * N), u = (e / N) % N, w = e % N, h = N / 2;
    int i1, i2, i3;
    bool mine;
    if (fam == 0) { i1 = h; i2 = u; i3 = w; mine = true; }
    else if (fam == 1) { i1 = u; i2 = h; i3 = w; mine = u != h && w != h; }
    else { i1 = u; i2 = w; i3 = h; mine = u != h; }
    if (!mine) {
        cp[t] = make_float2(0.f, 0.f);
        return;
    }
    const size_t m = mirror(i1, i2, i3, N);
    const float2 a = alpha[(2 * q) * n3 + m], b = alpha[(2 * q + 1) * n3 + m];
    cp[t] = make_float2(0.5f * (a.x - b.y), -0.5f * (a.y + b.x));
}

}  // namespace

bz_status build_pair_table(Plan &pl) {
    const int pairs = pl.P / 2;
    const size_t n = modes(pl) * pairs, ns = (size_t)3 * pl.N * pl.N * pairs;
    k_pair_table<<<(unsigned)((n + 255) / 256), 256>>>(pl.alpha, pl.N, pairs, pl.apair);
    k_pair_table_s<<<(unsigned)((ns + 255) / 256), 256>>>(pl.alpha, pl.N, pairs, pl.cpair);
    BZ_CUDA_TRY(cudaGetLastError());
    BZ_CUDA_TRY(cudaDeviceSynchronize());
    return BZ_OK;
}

bz_status sym_input(Plan &pl, const void *f, int dtype, cudaStream_t st) {
    const int n3 = (int)modes(pl);
    k_sym_in<<<(n3 + 255) / 256, 256, 0, st>>>(f, dtype, pl.N, pl.fsym, pl.fsym64);
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

bz_status reduce_sym(Plan &pl, int nblk, cudaStream_t st) {
    const int n3 = (int)modes(pl);
    k_reduce_sym<<<(n3 + 31) / 32, 256, 0, st>>>(pl.part, pl.part_s, nblk, pl.N, pl.acc);
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

}  // namespace bz

namespace bz {

bz_status sym_output(Plan &pl, cudaStream_t st) {
    const int n3 = (int)modes(pl);
    k_sym_out<<<(n3 + 255) / 256, 256, 0, st>>>(pl.acc, pl.acc_s, pl.N);
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

}  // namespace bz

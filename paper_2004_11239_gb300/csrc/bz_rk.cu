// Classical RK4 for d fhat/dt = Q(fhat, fhat) (Sec. 5.2) and FP64 moments (Sec. 1, Sec. 4).
//
// RK4: the step state f0 and the running combination fsum = f0 + dt/6 (k1 + 2k2 + 2k3 + k4)
// are FP64; each stage's collide input is rounded to FP32 (pl.fin) and each stage
// derivative k_s arrives in the FP64 accumulator of the collide pipeline.
#include <cmath>

#include "bz_internal.h"

namespace bz {

namespace {

__global__ void k_rk_init(const void *fhat, int dtype, double2 *f0, float2 *fin, double2 *fin64, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v;
    if (dtype == BZ_C128) v = ((const double2 *)fhat)[i];
    else {
        float2 w = ((const float2 *)fhat)[i];
        v = make_double2(w.x, w.y);
    }
    f0[i] = v;
    fin[i] = make_float2((float)v.x, (float)v.y);
    if (fin64) fin64[i] = v;
}

// stage s in {1, 2, 3, 4}; k = acc (FP64 derivative of stage s)
__global__ void k_rk_stage(const double2 *__restrict__ k, double2 *__restrict__ f0,
                           double2 *__restrict__ fsum, float2 *__restrict__ fin, double2 *__restrict__ fin64,
                           int n, int stage, double dt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 kv = k[i], a = f0[i], y;
    if (stage == 1) {
        fsum[i] = make_double2(a.x + dt / 6.0 * kv.x, a.y + dt / 6.0 * kv.y);
        y = make_double2(a.x + 0.5 * dt * kv.x, a.y + 0.5 * dt * kv.y);
    } else if (stage == 2 || stage == 3) {
        double2 s = fsum[i];
        fsum[i] = make_double2(s.x + dt / 3.0 * kv.x, s.y + dt / 3.0 * kv.y);
        double c = stage == 2 ? 0.5 * dt : dt;
        y = make_double2(a.x + c * kv.x, a.y + c * kv.y);
    } else {
        double2 s = fsum[i];
        y = make_double2(s.x + dt / 6.0 * kv.x, s.y + dt / 6.0 * kv.y);
        f0[i] = y;
    }
    fin[i] = make_float2((float)y.x, (float)y.y);
    if (fin64) fin64[i] = y;
}

__global__ void k_rk_out(const double2 *f0, void *fhat, int dtype, int n, int *flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (dtype == BZ_C128) {
        ((double2 *)fhat)[i] = f0[i];
        note_finite(f0[i], flag);
    } else {
        const float2 w = make_float2((float)f0[i].x, (float)f0[i].y);
        ((float2 *)fhat)[i] = w;
        note_finite(w, flag);
    }
}

// Moments of f_N over [-L, L]^3.  Only the modes on the three axes contribute:
// int exp(i pi k v / L) dv = 2L delta_k0, int v exp(..) dv = (-1)^k 2 L^2 / (i pi k),
// int v^2 exp(..) dv = (-1)^k 4 L^3 / (pi k)^2 (k != 0) and 2 L^3 / 3 (k = 0).
// Thread q computes out[q] by a fixed-order loop.
__global__ void k_moments(const void *fhat, int dtype, int N, double L, double *out) {
    int q = threadIdx.x;
    if (q >= 5) return;
    auto get = [&](int i1, int i2, int i3) -> double2 {
        size_t idx = ((size_t)i1 * N + i2) * N + i3;
        if (dtype == BZ_C128) return ((const double2 *)fhat)[idx];
        float2 w = ((const float2 *)fhat)[idx];
        return make_double2(w.x, w.y);
    };
    const double L2 = 2.0 * L;
    if (q == 0) { out[0] = L2 * L2 * L2 * get(0, 0, 0).x; return; }
    double sum = 0.0;
    for (int d = 0; d < 3; ++d) {
        if (q >= 1 && q <= 3 && d != q - 1) continue;
        for (int i = 0; i < N; ++i) {
            int k = i < N / 2 ? i : i - N;
            double2 f = d == 0 ? get(i, 0, 0) : (d == 1 ? get(0, i, 0) : get(0, 0, i));
            double sg = (k & 1) ? -1.0 : 1.0;
            if (q <= 3) {
                if (k == 0) continue;
                // Re[f * (-i) sg 2 L^2 / (pi k)] = f.y * sg * 2 L^2 / (pi k)
                sum += f.y * sg * 2.0 * L * L / (M_PI * k);
            } else {
                double w = k == 0 ? 2.0 * L * L * L / 3.0 : sg * 4.0 * L * L * L / (M_PI * M_PI * k * k);
                sum += f.x * w;
            }
        }
    }
    out[q] = sum * L2 * L2;
}

}  // namespace

bz_status rk4_steps(Plan &pl, void *fhat, int dtype, double dt, int nsteps, cudaStream_t st,
                    int *launches) {
    const int n = (int)modes(pl);
    const int bs = 256, gs = (n + bs - 1) / bs;
    double2 *f0 = pl.rk, *fsum = pl.rk + n;
    k_rk_init<<<gs, bs, 0, st>>>(fhat, dtype, f0, pl.fin, pl.fin64, n);
    pl.src = pl.fin64;             // stage inputs for the FP64 h pass (fused plans)
    pl.src_dtype = BZ_C128;
    int nl = 1;
    for (int step = 0; step < nsteps; ++step) {
        for (int stage = 1; stage <= 4; ++stage) {
            bz_status s = collide_core(pl, 0, pl.P, st, &nl);
            if (s != BZ_OK) return s;
            k_rk_stage<<<gs, bs, 0, st>>>(pl.acc, f0, fsum, pl.fin, pl.fin64, n, stage, dt);
            ++nl;
        }
    }
    k_rk_out<<<gs, bs, 0, st>>>(f0, fhat, dtype, n, nonfinite_flag(pl));
    ++nl;
    BZ_CUDA_TRY(cudaGetLastError());
    if (launches) *launches += nl;
    return BZ_OK;
}

bz_status moments(Plan &pl, const void *fhat, int dtype, double out[5], cudaStream_t st) {
    k_moments<<<1, 32, 0, st>>>(fhat, dtype, pl.Nin ? pl.Nin : pl.N, pl.L, pl.mom);   // the caller's grid
    BZ_CUDA_TRY(cudaGetLastError());
    BZ_CUDA_TRY(cudaMemcpyAsync(out, pl.mom, 5 * sizeof(double), cudaMemcpyDeviceToHost, st));
    BZ_CUDA_TRY(cudaStreamSynchronize(st));
    for (int q = 0; q < 5; ++q)
        if (!std::isfinite(out[q])) return BZ_ERR_NONFINITE;
    return BZ_OK;
}

}  // namespace bz

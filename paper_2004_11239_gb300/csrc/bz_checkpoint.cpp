// Checkpoint and resume of an RK4 solve (Sec. 5.2 time stepping of d fhat/dt = Q(fhat, fhat)).
//
// The state of a solve between bz_step_rk calls is the coefficient array and t; with a
// complex128 array that state is exactly the FP64 RK state, so steps taken after a resume give
// the same bits as an uninterrupted run, provided the plan also makes the same choices (the
// term grouping of the collide decides the rounding of each sum).  The file therefore records
// the operator (every parameter of eq. approxG and the kernel) and the plan's pipeline choices
// (pipeline, CTAs per cluster, the pair kernel, terms per chunk), so that bz_checkpoint_plan_desc
// can rebuild an identical plan in a new process.  Layout (host byte order):
//   "BZCKPT1\0", int32 version = 1, int32 fields[16], double params[8], double t,
//   then N^d complex128 coefficients (d = 3, or 2 for a 2D plan).
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bz_internal.h"

struct bz_plan;

namespace bz {
const Plan *plan_internal(const bz_plan *plan);
}

namespace {

constexpr char kMagic[8] = {'B', 'Z', 'C', 'K', 'P', 'T', '1', '\0'};
enum { F_N, F_DIM, F_NRHO, F_M, F_KERNEL, F_PREC, F_DATA, F_CONV, F_HPREC, F_PIPE, F_CLUSTER, F_CTAS, F_CHUNK,
       F_COUNT = 16 };
enum { D_L, D_R, D_GAMMA, D_S, D_EPS, D_THETA0, D_COUNT = 8 };

struct Header {
    char magic[8];
    int32_t version;
    int32_t f[F_COUNT];
    double d[D_COUNT];
    double t;
};

void fill(const bz::Plan &pl, Header &h) {
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.f[F_N] = pl.Nin ? pl.Nin : pl.N;
    h.f[F_DIM] = pl.dim;
    h.f[F_NRHO] = pl.N_rho;
    h.f[F_M] = pl.M;
    h.f[F_KERNEL] = pl.kernel;
    h.f[F_PREC] = pl.precision;
    h.f[F_DATA] = pl.real ? BZ_DATA_REAL : BZ_DATA_COMPLEX;
    h.f[F_CONV] = pl.Nin ? BZ_CONV_PADDED : BZ_CONV_CIRCULAR;
    h.f[F_HPREC] = pl.h_fp64 ? BZ_H_FP64 : BZ_H_FP32;
    // 2D plans have one pipeline and split-BF16 plans one cluster size: left to the plan
    h.f[F_PIPE] = pl.dim == 2 ? BZ_PIPE_AUTO : (pl.use_fused ? BZ_PIPE_FUSED : BZ_PIPE_CHUNKED);
    h.f[F_CLUSTER] = pl.use_fused && pl.dim == 3 && pl.precision == BZ_PREC_FP32 ? pl.fused_C : 0;
    h.f[F_CTAS] = pl.pair3 ? 3 : 0;
    h.f[F_CHUNK] = pl.chunk;
    h.d[D_L] = pl.L;
    h.d[D_R] = pl.R;
    h.d[D_GAMMA] = pl.gamma;
    h.d[D_S] = pl.s;
    h.d[D_EPS] = pl.eps;
    h.d[D_THETA0] = pl.theta0;
}

bool read_header(FILE *fp, Header &h) {
    return std::fread(&h, sizeof(h), 1, fp) == 1 && std::memcmp(h.magic, kMagic, 8) == 0 && h.version == 1;
}

size_t field_modes(const Header &h) {
    const size_t N = (size_t)h.f[F_N];
    return h.f[F_DIM] == 2 ? N * N : N * N * N;
}

}  // namespace

extern "C" {

bz_status bz_checkpoint_write(const bz_plan *plan, const void *fhat, int dtype, double t, const char *path,
                              void *stream) {
    if (!plan || !fhat || !path) return BZ_ERR_ARG;
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    const bz::Plan &pl = *bz::plan_internal(plan);
    Header h;
    fill(pl, h);
    h.t = t;
    const size_t n = field_modes(h);
    std::vector<double2> host(n);
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == BZ_C128) {
        if (cudaMemcpyAsync(host.data(), fhat, n * sizeof(double2), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return BZ_ERR_CUDA;
    } else {
        std::vector<float2> f(n);
        if (cudaMemcpyAsync(f.data(), fhat, n * sizeof(float2), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return BZ_ERR_CUDA;
        for (size_t i = 0; i < n; ++i) host[i] = make_double2(f[i].x, f[i].y);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return BZ_ERR_CUDA;
    // written beside the target and renamed over it, so a reader never sees half a file
    const std::string tmp = std::string(path) + ".tmp";
    FILE *fp = std::fopen(tmp.c_str(), "wb");
    if (!fp) return BZ_ERR_ARG;
    const bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(host.data(), sizeof(double2), n, fp) == n;
    if (std::fclose(fp) != 0 || !ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return BZ_ERR_ARG;
    }
    return BZ_OK;
}

bz_status bz_checkpoint_plan_desc(const char *path, bz_plan_desc *desc, double *t) {
    if (!path || !desc) return BZ_ERR_ARG;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return BZ_ERR_ARG;
    Header h;
    const bool ok = read_header(fp, h);
    std::fclose(fp);
    if (!ok) return BZ_ERR_ARG;
    std::memset(desc, 0, sizeof(*desc));
    desc->N = h.f[F_N];
    desc->dim = h.f[F_DIM];
    desc->N_rho = h.f[F_NRHO];
    desc->M = h.f[F_M];
    desc->kernel = h.f[F_KERNEL];
    desc->precision = h.f[F_PREC];
    desc->data = h.f[F_DATA];
    desc->conv = h.f[F_CONV];
    desc->h_precision = h.f[F_HPREC];
    desc->pipeline = h.f[F_PIPE];
    desc->cluster = h.f[F_CLUSTER];
    desc->ctas_per_sm = h.f[F_CTAS] ? h.f[F_CTAS] : (h.f[F_DATA] == BZ_DATA_REAL && h.f[F_PIPE] == BZ_PIPE_FUSED ? 2 : 0);
    desc->chunk_terms = h.f[F_CHUNK];
    desc->L = h.d[D_L];
    desc->R = h.d[D_R];
    desc->gamma = h.d[D_GAMMA];
    desc->s = h.d[D_S];
    desc->eps = h.d[D_EPS];
    desc->theta0 = h.d[D_THETA0];
    if (t) *t = h.t;
    return BZ_OK;
}

bz_status bz_checkpoint_read(const bz_plan *plan, const char *path, void *fhat, int dtype, double *t, void *stream) {
    if (!plan || !path || !fhat) return BZ_ERR_ARG;
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    const bz::Plan &pl = *bz::plan_internal(plan);
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return BZ_ERR_ARG;
    Header h, mine;
    bool ok = read_header(fp, h);
    fill(pl, mine);
    // the same operator: every parameter of the terms and the kernel (the pipeline choices
    // may differ; they change only the rounding)
    ok = ok && std::memcmp(h.f, mine.f, sizeof(int32_t) * F_PIPE) == 0 &&
         std::memcmp(h.d, mine.d, sizeof(double) * D_COUNT) == 0;
    const size_t n = ok ? field_modes(h) : 0;
    std::vector<double2> host(n);
    ok = ok && std::fread(host.data(), sizeof(double2), n, fp) == n;
    std::fclose(fp);
    if (!ok) return BZ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == BZ_C128) {
        if (cudaMemcpyAsync(fhat, host.data(), n * sizeof(double2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return BZ_ERR_CUDA;
    } else {
        std::vector<float2> f(n);
        for (size_t i = 0; i < n; ++i) f[i] = make_float2((float)host[i].x, (float)host[i].y);
        if (cudaMemcpyAsync(fhat, f.data(), n * sizeof(float2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return BZ_ERR_CUDA;
    }
    if (t) *t = h.t;
    return BZ_OK;
}

}  // extern "C"

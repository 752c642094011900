// C ABI of libbz: plan lifetime, collide, RK4, moments and table accessors (include/bz.h).
#include <cmath>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "bz_internal.h"

struct bz_plan {
    bz::Plan p;
};

namespace bz {
const Plan *plan_internal(const bz_plan *plan) { return &plan->p; }
}  // namespace bz

namespace {

void free_timing(bz::Plan &p) {
    for (cudaEvent_t e : p.tm.ev) cudaEventDestroy(e);
    p.tm.ev.clear();
    p.tm.kind.clear();
    p.tm.used = 0;
    p.tm.on = false;
}

void free_plan(bz::Plan &p) {
    free_timing(p);
    cudaFree(p.alpha); cudaFree(p.tw); cudaFree(p.rule_buf); cudaFree(p.rule_off);
    cudaFree(p.term_dev); cudaFree(p.S); cudaFree(p.h); cudaFree(p.fin); cudaFree(p.acc);
    cudaFree(p.rk); cudaFree(p.mom); cudaFree(p.part); cudaFree(p.fin64); cudaFree(p.scr64);
    cudaFree(p.wimg); cudaFree(p.dev_err); cudaFree(p.apair); cudaFree(p.fsym); cudaFree(p.fsym64);
    cudaFree(p.cpair); cudaFree(p.part_s); cudaFree(p.S_s); cudaFree(p.acc_s);
    for (int e = 0; e < bz::kExtraStreams; ++e) {
        cudaFree(p.xS[e]); cudaFree(p.xS_s[e]); cudaFree(p.xacc[e]); cudaFree(p.xacc_s[e]);
        if (p.xev_join[e]) cudaEventDestroy(p.xev_join[e]);
        if (p.xst[e]) cudaStreamDestroy(p.xst[e]);
        p.xS[e] = nullptr; p.xS_s[e] = nullptr; p.xacc[e] = nullptr; p.xacc_s[e] = nullptr;
        p.xev_join[e] = nullptr; p.xst[e] = nullptr;
    }
    if (p.ev_fork) cudaEventDestroy(p.ev_fork);
    p.ev_fork = nullptr;
    p.xn = 0;
    p.wimg = nullptr; p.dev_err = nullptr; p.apair = nullptr; p.fsym = nullptr; p.fsym64 = nullptr;
    p.cpair = nullptr; p.part_s = nullptr; p.S_s = nullptr; p.acc_s = nullptr;
    p.part = nullptr; p.fin64 = nullptr; p.scr64 = nullptr; p.src = nullptr;
    p.alpha = nullptr; p.tw = nullptr; p.rule_buf = nullptr; p.rule_off = nullptr;
    p.term_dev = nullptr; p.S = nullptr; p.h = nullptr; p.fin = nullptr; p.acc = nullptr;
    p.rk = nullptr; p.mom = nullptr;
}

template <class T> bz_status dmalloc(T **ptr, size_t bytes) {
    if (cudaMalloc((void **)ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return BZ_ERR_OOM;
    }
    return BZ_OK;
}

// Twiddle vectors beta_p per axis: tw[p][d][i] = exp(-i pi r_p q_{p,d} m_i / L), m_i signed.
std::vector<float2> make_twiddles(const bz::Plan &pl) {
    const int N = pl.N;
    std::vector<float2> tw((size_t)pl.P * 3 * N);
    for (int p = 0; p < pl.P; ++p)
        for (int d = 0; d < 3; ++d)
            for (int i = 0; i < N; ++i) {
                int m = i < N / 2 ? i : i - N;
                double ph = -M_PI * pl.terms.r[p] * pl.terms.q[3 * p + d] * m / pl.L;
                tw[((size_t)p * 3 + d) * N + i] = make_float2((float)std::cos(ph), (float)std::sin(ph));
            }
    return tw;
}

// Times one full collide of a zero field for each compiled cluster size (or only `forced`)
// and keeps the fastest; allocates the partial-sum buffer for it.
bz_status select_fused(bz::Plan &pl, int forced, int ctas) {
    int cs[4];
    const bool mixed = pl.precision == BZ_PREC_BF16X3;
    int nc = mixed ? 1 : bz::fused_candidates(pl.N, cs);
    if (mixed) cs[0] = 8;
    // the real-data form at N = 32 also times the three-CTA pair kernel, k_pair3 (C = 8)
    const int pair3_c = (pl.real && pl.N == 32 && ctas != 2) ? nc : -1;
    if (pair3_c >= 0) cs[nc++] = 8;
    const size_t field = (size_t)pl.N * pl.N * pl.N * sizeof(float2);
    const size_t fields = (size_t)3 * pl.N * pl.N * sizeof(float2);   // BZ_DATA_REAL: Nyquist-plane sums
    int bestC = 0, bestG = 0, bestP3 = 0;
    float best = 1e30f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BZ_ERR_CUDA;
    if (cudaMemset(pl.fin, 0, field) != cudaSuccess) return BZ_ERR_CUDA;
    for (int c = 0; c < nc; ++c) {
        if (forced > 0 && cs[c] != forced) continue;
        if (ctas == 3 && c != pair3_c) continue;
        int G = 0;
        const cudaError_t se = mixed ? bz::mixed_setup(pl.N, &G)
                               : c == pair3_c ? bz::pair3_setup(&G) : bz::fused_setup(pl.N, cs[c], &G, pl.real != 0);
        if (se != cudaSuccess || G <= 0) { cudaGetLastError(); continue; }
        float2 *part = nullptr, *parts = nullptr;
        if (cudaMalloc(&part, (size_t)G * field) != cudaSuccess) { cudaGetLastError(); continue; }
        if (pl.real && cudaMalloc(&parts, (size_t)G * fields) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(part);
            continue;
        }
        std::swap(part, pl.part);
        std::swap(parts, pl.part_s);
        pl.use_fused = 1; pl.fused_C = cs[c]; pl.fused_G = G; pl.pair3 = c == pair3_c;
        float ms = 1e30f;
        if (bz::collide_fused(pl, 0, pl.P, nullptr, nullptr) == BZ_OK) {      // warm-up
            cudaEventRecord(e0);
            bz::collide_fused(pl, 0, pl.P, nullptr, nullptr);
            cudaEventRecord(e1);
            if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        }
        cudaGetLastError();
        std::swap(part, pl.part);
        std::swap(parts, pl.part_s);
        cudaFree(part);
        cudaFree(parts);
        if (ms < best) { best = ms; bestC = cs[c]; bestG = G; bestP3 = pl.pair3; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    pl.use_fused = 0;
    if (bestC == 0) return BZ_ERR_UNSUPPORTED;
    if (dmalloc(&pl.part, (size_t)bestG * field) != BZ_OK) return BZ_ERR_OOM;
    if (pl.real && dmalloc(&pl.part_s, (size_t)bestG * fields) != BZ_OK) return BZ_ERR_OOM;
    pl.use_fused = 1; pl.fused_C = bestC; pl.fused_G = bestG; pl.pair3 = bestP3;
    pl.fused_ms = best;
    pl.ws_bytes += (size_t)bestG * (field + (pl.real ? fields : 0));
    return BZ_OK;
}

bz_status create(bz_plan **out, const bz_plan_desc *d) {
    if (!out || !d) return BZ_ERR_ARG;
    *out = nullptr;
    if (!bz::supported_N(d->N) || d->N_rho < 1 || d->M < 1 || !(d->L > 0) || !(d->R > 0))
        return BZ_ERR_ARG;
    const int dim = d->dim == 0 ? 3 : d->dim;
    if (dim != 2 && dim != 3) return BZ_ERR_ARG;
    if (dim == 2) {
        if (d->N != 8 && d->N != 16 && d->N != 32 && d->N != 64) return BZ_ERR_ARG;
        if (d->kernel < BZ_KERNEL_B1 || d->kernel > BZ_KERNEL_B4) return BZ_ERR_ARG;
        if (d->precision != BZ_PREC_FP32 || d->conv != BZ_CONV_CIRCULAR || d->pipeline == BZ_PIPE_CHUNKED)
            return BZ_ERR_UNSUPPORTED;
    }
    if (d->precision != BZ_PREC_FP32 && d->precision != BZ_PREC_BF16X3) return BZ_ERR_ARG;
    if (d->conv != BZ_CONV_CIRCULAR && d->conv != BZ_CONV_PADDED) return BZ_ERR_ARG;
    const bool padded = d->conv == BZ_CONV_PADDED;
    if (padded && (d->N > 32 || d->precision != BZ_PREC_FP32)) return BZ_ERR_UNSUPPORTED;
    if (d->precision == BZ_PREC_BF16X3 && (d->N != 32 || d->pipeline == BZ_PIPE_CHUNKED))
        return BZ_ERR_UNSUPPORTED;
    if (d->pipeline < BZ_PIPE_AUTO || d->pipeline > BZ_PIPE_CHUNKED) return BZ_ERR_ARG;
    if (d->data != BZ_DATA_COMPLEX && d->data != BZ_DATA_REAL) return BZ_ERR_ARG;
    const bool real = d->data == BZ_DATA_REAL;
    // the real-data form: fused for N dividing 32, the chunked pipeline otherwise (or on request)
    if (real && (dim != 3 || d->precision != BZ_PREC_FP32 || padded || d->M % 2 != 0 ||
                 (d->pipeline == BZ_PIPE_FUSED && 32 % d->N != 0)))
        return BZ_ERR_UNSUPPORTED;
    if (d->ctas_per_sm == 3 && !(real && d->N == 32)) return BZ_ERR_UNSUPPORTED;
    if (d->ctas_per_sm > 0 && d->ctas_per_sm != 2 && d->ctas_per_sm != 3) return BZ_ERR_UNSUPPORTED;
    if (dim == 3 && !((d->kernel >= BZ_KERNEL_FAMILY && d->kernel <= BZ_KERNEL_B8) || d->kernel == BZ_KERNEL_DEBYE))
        return BZ_ERR_ARG;
    bz_plan *h = new (std::nothrow) bz_plan();
    if (!h) return BZ_ERR_OOM;
    bz::Plan &pl = h->p;
    pl.dim = dim;
    pl.N = padded ? 2 * d->N : d->N; pl.Nin = padded ? d->N : 0; pl.L = d->L; pl.R = d->R; pl.gamma = d->gamma; pl.s = d->s;
    pl.N_rho = d->N_rho; pl.M = d->M; pl.kernel = d->kernel; pl.precision = d->precision;
    pl.real = real ? 1 : 0;
    pl.eps = d->eps > 0 ? d->eps : M_PI / 1000.0;
    if (!(d->theta0 == 0.0 || (d->theta0 >= pl.eps && d->theta0 < M_PI))) { delete h; return BZ_ERR_ARG; }
    pl.theta0 = d->theta0;
    if (d->h_precision < BZ_H_AUTO || d->h_precision > BZ_H_FP32) { delete h; return BZ_ERR_ARG; }
    pl.h_fp64 = d->h_precision != BZ_H_FP32 || d->precision == BZ_PREC_BF16X3;   // BF16X3 reads h formed in FP64
    cudaGetDevice(&pl.device);
    bz_status s = bz::build_terms(pl, d->sphere_xyz, d->sphere_w);
    if (s == BZ_OK) s = bz::build_kernel_constants(pl);
    if (s != BZ_OK) { delete h; return s; }
    bz::build_theta_rules(pl);

    const int N = pl.N;
    const size_t n3 = bz::modes(pl);          // N^3, or N^2 for a 2D plan
    const size_t field = n3 * sizeof(float2);
    int chunk = d->chunk_terms;
    if (dim == 2) chunk = 1;                  // no chunked pipeline in 2D
    // the chunked pipeline (N > 32, or asked for) runs its chunks on two streams
    const bool two_streams = dim == 3 && (N > 32 || d->pipeline == BZ_PIPE_CHUNKED);
    if (chunk <= 0) {
        // two waves of plane CTAs, within an L2-sized scratch; one wave per stream on two streams
        if (bz::collide_set_attributes(N) != cudaSuccess) { delete h; return BZ_ERR_CUDA; }
        chunk = bz::chunk_terms_for(N);
        if (two_streams && chunk > 1) chunk = (chunk + bz::kExtraStreams) / (1 + bz::kExtraStreams);
    }
    if (chunk > pl.P) chunk = pl.P;
    if (chunk > 65535) chunk = 65535;
    pl.chunk = chunk;

    if ((s = dmalloc(&pl.alpha, (size_t)pl.P * field)) != BZ_OK ||
        (s = dmalloc(&pl.tw, (size_t)pl.P * 3 * N * sizeof(float2))) != BZ_OK ||
        (s = dmalloc(&pl.S, (size_t)chunk * field)) != BZ_OK ||
        (s = dmalloc(&pl.h, field)) != BZ_OK ||
        (s = dmalloc(&pl.fin, field)) != BZ_OK ||
        (s = dmalloc(&pl.acc, n3 * sizeof(double2))) != BZ_OK ||
        (s = dmalloc(&pl.rk, 2 * n3 * sizeof(double2))) != BZ_OK ||
        (s = dmalloc(&pl.mom, 8 * sizeof(double))) != BZ_OK ||
        (s = dmalloc(&pl.dev_err, 2 * sizeof(int))) != BZ_OK) {
        free_plan(pl);
        delete h;
        return s;
    }
    pl.ws_bytes = (size_t)chunk * field + 2 * field + 3 * n3 * sizeof(double2);
    std::vector<float2> tw = make_twiddles(pl);
    if (cudaMemcpy(pl.tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(pl.dev_err, 0, 2 * sizeof(int)) != cudaSuccess ||
        (pl.precision == BZ_PREC_BF16X3 && bz::mixed_upload(&pl.wimg) != BZ_OK) ||
        (dim == 3 && bz::collide_set_attributes(N) != cudaSuccess)) {
        free_plan(pl);
        delete h;
        return BZ_ERR_CUDA;
    }
    s = bz::ftable_build(pl);
    if (s == BZ_OK && pl.real) {
        // term pairs (2q, 2q + 1) share a radial node (M even) and one pair of transforms
        const size_t ns = (size_t)3 * N * N;
        if ((s = dmalloc(&pl.apair, (size_t)(pl.P / 2) * field)) == BZ_OK &&
            (s = dmalloc(&pl.cpair, (size_t)(pl.P / 2) * ns * sizeof(float2))) == BZ_OK &&
            (s = dmalloc(&pl.S_s, (size_t)pl.chunk * ns * sizeof(float2))) == BZ_OK &&
            (s = dmalloc(&pl.acc_s, ns * sizeof(double2))) == BZ_OK &&
            (s = dmalloc(&pl.fsym, field)) == BZ_OK && (s = dmalloc(&pl.fsym64, n3 * sizeof(double2))) == BZ_OK)
            s = bz::build_pair_table(pl);
        pl.ws_bytes += field + n3 * sizeof(double2) + (size_t)pl.chunk * ns * sizeof(float2) + ns * sizeof(double2);
    }
    if (s != BZ_OK) {
        free_plan(pl);
        delete h;
        return s;
    }
    if (dim == 2) {
        // one CTA per term block over a persistent grid; FP64 stage inputs for the h pass
        if (bz::setup_2d(pl) != cudaSuccess ||
            (s = dmalloc(&pl.part, (size_t)pl.fused_G * field)) != BZ_OK ||
            (s = dmalloc(&pl.fin64, n3 * sizeof(double2))) != BZ_OK ||
            (s = dmalloc(&pl.scr64, n3 * sizeof(double2))) != BZ_OK) {
            cudaGetLastError();
            free_plan(pl);
            delete h;
            return s != BZ_OK ? s : BZ_ERR_CUDA;
        }
        pl.ws_bytes += (size_t)pl.fused_G * field + 2 * n3 * sizeof(double2);
        *out = h;
        return BZ_OK;
    }
    // pipeline: the fused cluster kernel where it applies (cluster size timed on this
    // device, fastest kept), else the chunked kernels
    if (d->pipeline != BZ_PIPE_CHUNKED && N <= 32) {
        if (dmalloc(&pl.fin64, n3 * sizeof(double2)) == BZ_OK && dmalloc(&pl.scr64, n3 * sizeof(double2)) == BZ_OK) {
            pl.ws_bytes += 2 * n3 * sizeof(double2);
            if (select_fused(pl, d->cluster, d->ctas_per_sm) != BZ_OK) cudaGetLastError();
        }
    }
    if ((d->pipeline == BZ_PIPE_FUSED || pl.precision == BZ_PREC_BF16X3) && !pl.use_fused) {
        free_plan(pl);
        delete h;
        return BZ_ERR_UNSUPPORTED;
    }
    if (two_streams && !pl.use_fused) {
        // the other lanes' scratch and accumulators; without them the chunks stay on one stream
        const size_t ns = (size_t)3 * N * N;
        bool ok = cudaEventCreateWithFlags(&pl.ev_fork, cudaEventDisableTiming) == cudaSuccess;
        for (int e = 0; ok && e < bz::kExtraStreams; ++e) {
            ok = dmalloc(&pl.xS[e], (size_t)pl.chunk * field) == BZ_OK &&
                 dmalloc(&pl.xacc[e], n3 * sizeof(double2)) == BZ_OK;
            if (ok && pl.real)
                ok = dmalloc(&pl.xS_s[e], (size_t)pl.chunk * ns * sizeof(float2)) == BZ_OK &&
                     dmalloc(&pl.xacc_s[e], ns * sizeof(double2)) == BZ_OK;
            ok = ok && cudaStreamCreateWithFlags(&pl.xst[e], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&pl.xev_join[e], cudaEventDisableTiming) == cudaSuccess;
            if (ok) {
                pl.xn = e + 1;
                pl.ws_bytes += (size_t)pl.chunk * field + n3 * sizeof(double2) +
                               (pl.real ? (size_t)pl.chunk * ns * sizeof(float2) + ns * sizeof(double2) : 0);
            }
        }
        if (!ok) cudaGetLastError();   // the lanes that were set up stay in use
    }
    *out = h;
    return BZ_OK;
}

}  // namespace

extern "C" {

bz_status bz_plan_create(bz_plan **out, int N, double L, double R, double gamma, double s,
                         int N_rho, int M) {
    bz_plan_desc d;
    std::memset(&d, 0, sizeof(d));
    d.N = N; d.L = L; d.R = R; d.gamma = gamma; d.s = s; d.N_rho = N_rho; d.M = M;
    d.kernel = BZ_KERNEL_FAMILY; d.precision = BZ_PREC_FP32; d.eps = 0.0;
    return create(out, &d);
}

bz_status bz_plan_create_ex(bz_plan **out, const bz_plan_desc *desc) { return create(out, desc); }

void bz_plan_destroy(bz_plan *plan) {
    if (!plan) return;
    free_plan(plan->p);
    delete plan;
}

bz_status bz_plan_info(const bz_plan *plan, int *P, size_t *alpha_bytes, size_t *workspace_bytes) {
    if (!plan) return BZ_ERR_ARG;
    const bz::Plan &p = plan->p;
    size_t n3 = bz::modes(p);
    if (P) *P = p.P;
    if (alpha_bytes)
        *alpha_bytes = ((size_t)p.P * n3 + (p.real ? (size_t)(p.P / 2) * (n3 + 3 * (size_t)p.N * p.N) : 0)) *
                       sizeof(float2);
    if (workspace_bytes) *workspace_bytes = p.ws_bytes;
    return BZ_OK;
}

const char *bz_plan_kernel(const bz_plan *plan) {
    if (!plan) return nullptr;
    const bz::Plan &p = plan->p;
    if (p.dim == 2) return "k_collide_2d";
    if (!p.use_fused) return "chunked";
    if (p.precision == BZ_PREC_BF16X3) return "k_mixed";
    return p.pair3 ? "k_pair3" : "k_fused";
}

bz_status bz_plan_pipeline(const bz_plan *plan, int *pipeline, int *cluster, int *clusters, float *tuned_ms) {
    if (!plan) return BZ_ERR_ARG;
    const bz::Plan &p = plan->p;
    const bool fused = p.use_fused || p.dim == 2;       // the 2D kernel keeps a term's field on chip
    if (pipeline) *pipeline = fused ? BZ_PIPE_FUSED : BZ_PIPE_CHUNKED;
    if (cluster) *cluster = fused ? p.fused_C : 0;
    if (clusters) *clusters = fused ? p.fused_G : 0;
    if (tuned_ms) *tuned_ms = p.use_fused ? p.fused_ms : 0.f;
    return BZ_OK;
}

bz_status bz_plan_terms(const bz_plan *plan, double *r, double *w_r, double *qhat, double *w_q,
                        double *c) {
    if (!plan) return BZ_ERR_ARG;
    const bz::HostTerms &T = plan->p.terms;
    const int P = plan->p.P;
    for (int p = 0; p < P; ++p) {
        if (r) r[p] = T.r[p];
        if (w_r) w_r[p] = T.wr[p];
        if (w_q) w_q[p] = T.wq[p];
        if (c) c[p] = T.c[p];
        if (qhat) for (int d = 0; d < 3; ++d) qhat[3 * p + d] = T.q[3 * p + d];
    }
    return BZ_OK;
}

bz_status bz_collide_terms(bz_plan *plan, int p0, int p1, const void *fhat, void *Qhat, int dtype,
                           void *stream) {
    if (!plan || !fhat || !Qhat || fhat == Qhat) return BZ_ERR_ARG;
    bz::Plan &pl = plan->p;
    if (p0 < 0 || p1 < p0 || p1 > pl.P) return BZ_ERR_ARG;
    if (pl.real && ((p0 | p1) & 1)) return BZ_ERR_ARG;          // whole term pairs
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int nl = 0;
    bz_status s = bz::collide_range(pl, p0, p1, fhat, dtype, st, &nl);
    if (s == BZ_OK) s = bz::write_output(pl, Qhat, dtype, st, &nl);
    pl.last_launches = nl;
    return s;
}

bz_status bz_collide(bz_plan *plan, const void *fhat, void *Qhat, int dtype, void *stream) {
    if (!plan) return BZ_ERR_ARG;
    return bz_collide_terms(plan, 0, plan->p.P, fhat, Qhat, dtype, stream);
}

bz_status bz_step_rk(bz_plan *plan, void *fhat, int dtype, double *t, double dt, int nsteps,
                     void *workspace, void *stream) {
    (void)workspace;
    if (!plan || !fhat || nsteps < 0 || !std::isfinite(dt)) return BZ_ERR_ARG;
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    if (plan->p.Nin) return BZ_ERR_UNSUPPORTED;               // padded plans: bz_collide
    int nl = 0;
    bz_status s = bz::rk4_steps(plan->p, fhat, dtype, dt, nsteps, (cudaStream_t)stream, &nl);
    plan->p.last_launches = nl;
    if (s == BZ_OK && t) *t += dt * nsteps;
    return s;
}

bz_status bz_moments(bz_plan *plan, const void *fhat, int dtype, double out[5], void *stream) {
    if (!plan || !fhat || !out) return BZ_ERR_ARG;
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    if (plan->p.dim == 2) return BZ_ERR_UNSUPPORTED;
    return bz::moments(plan->p, fhat, dtype, out, (cudaStream_t)stream);
}

bz_status bz_ftable_entries(bz_plan *plan, int count, const int *k_idx, const int *term,
                            double *out) {
    if (!plan || count < 0 || (count > 0 && (!k_idx || !term || !out))) return BZ_ERR_ARG;
    return bz::ftable_entries(plan->p, count, k_idx, term, out);
}

bz_status bz_plan_alpha(const bz_plan *plan, int p0, int p1, void *dst, void *stream) {
    if (!plan || !dst) return BZ_ERR_ARG;
    const bz::Plan &pl = plan->p;
    if (p0 < 0 || p1 < p0 || p1 > pl.P) return BZ_ERR_ARG;
    if (pl.Nin) return BZ_ERR_UNSUPPORTED;                    // the padded table lives on the 2N grid
    size_t n3 = bz::modes(pl);
    if (cudaMemcpyAsync(dst, pl.alpha + (size_t)p0 * n3, (size_t)(p1 - p0) * n3 * sizeof(float2),
                        cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess)
        return BZ_ERR_CUDA;
    return BZ_OK;
}

int bz_plan_last_launches(const bz_plan *plan) { return plan ? plan->p.last_launches : 0; }

bz_status bz_plan_device_errors(bz_plan *plan, int *count) {
    if (!plan || !count) return BZ_ERR_ARG;
    int v = 0;
    if (cudaMemcpy(&v, plan->p.dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BZ_ERR_CUDA;
    *count = v != 0;
    return BZ_OK;
}

bz_status bz_plan_wait_selftest(bz_plan *plan, long long cycles, void *stream) {
    if (!plan || cycles < 1 || cycles > (1LL << 31)) return BZ_ERR_ARG;
    return bz::wait_selftest(plan->p, cycles, (cudaStream_t)stream);
}

bz_status bz_plan_check_finite(bz_plan *plan, int *nonfinite) {
    if (!plan) return BZ_ERR_ARG;
    int v = 0;
    if (cudaMemcpy(&v, plan->p.dev_err + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return BZ_ERR_CUDA;
    if (v && cudaMemset(plan->p.dev_err + 1, 0, sizeof(int)) != cudaSuccess) return BZ_ERR_CUDA;
    if (nonfinite) *nonfinite = v != 0;
    return v ? BZ_ERR_NONFINITE : BZ_OK;
}

bz_status bz_partition_terms(int P, int data, int world, int rank, int *p0, int *p1) {
    if (!p0 || !p1 || P < 0 || world < 1 || rank < 0 || rank >= world) return BZ_ERR_ARG;
    if (data != BZ_DATA_COMPLEX && data != BZ_DATA_REAL) return BZ_ERR_ARG;
    // contiguous near-equal ranges in rank order; BZ_DATA_REAL splits the P / 2 term pairs so
    // that both terms of a pair (2q, 2q + 1) stay on one rank
    const long u = data == BZ_DATA_REAL ? P / 2 : P;
    if (data == BZ_DATA_REAL && (P & 1)) return BZ_ERR_ARG;
    const long a = u * rank / world, b = u * (rank + 1) / world;
    const int scale = data == BZ_DATA_REAL ? 2 : 1;
    *p0 = (int)(a * scale);
    *p1 = (int)(b * scale);
    return BZ_OK;
}

bz_status bz_quadrature(int N_rho, double R, int M, double gamma, double *r, double *w_r, double *qhat,
                        double *w_q, double *c) {
    if (N_rho < 1 || M < 1 || !(R > 0) || !std::isfinite(gamma)) return BZ_ERR_ARG;
    bz::Plan pl;
    pl.N_rho = N_rho; pl.R = R; pl.M = M; pl.gamma = gamma;
    bz_status s = bz::build_terms(pl, nullptr, nullptr);
    if (s != BZ_OK) return s;
    const bz::HostTerms &T = pl.terms;
    for (int p = 0; p < pl.P; ++p) {
        if (r) r[p] = T.r[p];
        if (w_r) w_r[p] = T.wr[p];
        if (w_q) w_q[p] = T.wq[p];
        if (c) c[p] = T.c[p];
        if (qhat) for (int d = 0; d < 3; ++d) qhat[3 * p + d] = T.q[3 * p + d];
    }
    return BZ_OK;
}

bz_status bz_kernel_constants(int kernel, double s, double eps, double *c, double A[3]) {
    bz::Plan pl;
    pl.kernel = kernel; pl.s = s; pl.eps = eps > 0 ? eps : M_PI / 1000.0;
    bz_status st = bz::build_kernel_constants(pl);
    if (st != BZ_OK) return st;
    if (c) *c = pl.kc;
    if (A) for (int i = 0; i < 3; ++i) A[i] = pl.A[i];
    return BZ_OK;
}

bz_status bz_plan_set_timing(bz_plan *plan, int max_launches) {
    if (!plan || max_launches < 0) return BZ_ERR_ARG;
    bz::Plan &pl = plan->p;
    free_timing(pl);
    for (int k = 0; k < bz::TK_COUNT; ++k) { pl.tm.ms[k] = 0.0; pl.tm.n[k] = 0; }
    if (max_launches == 0) return BZ_OK;
    pl.tm.ev.resize(2 * (size_t)max_launches);
    for (size_t i = 0; i < pl.tm.ev.size(); ++i) {
        if (cudaEventCreate(&pl.tm.ev[i]) != cudaSuccess) {
            pl.tm.ev.resize(i);
            free_timing(pl);
            return BZ_ERR_CUDA;
        }
    }
    pl.tm.kind.assign(max_launches, 0);
    pl.tm.on = true;
    return BZ_OK;
}

bz_status bz_plan_timing(bz_plan *plan, int kind, long *launches, double *ms) {
    if (!plan || kind < 0 || kind >= bz::TK_COUNT) return BZ_ERR_ARG;
    bz::Plan &pl = plan->p;
    if (pl.tm.used > 0) {
        if (cudaEventSynchronize(pl.tm.ev[2 * pl.tm.used - 1]) != cudaSuccess) return BZ_ERR_CUDA;
        for (size_t i = 0; i < pl.tm.used; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, pl.tm.ev[2 * i], pl.tm.ev[2 * i + 1]) != cudaSuccess)
                return BZ_ERR_CUDA;
            pl.tm.ms[pl.tm.kind[i]] += t;
            pl.tm.n[pl.tm.kind[i]] += 1;
        }
        pl.tm.used = 0;
    }
    if (launches) *launches = pl.tm.n[kind];
    if (ms) *ms = pl.tm.ms[kind];
    return BZ_OK;
}

const char *bz_status_str(bz_status s) {
    switch (s) {
        case BZ_OK: return "ok";
        case BZ_ERR_ARG: return "invalid argument";
        case BZ_ERR_OOM: return "out of memory";
        case BZ_ERR_CUDA: return "CUDA error";
        case BZ_ERR_TIMEOUT: return "timeout";
        case BZ_ERR_NONFINITE: return "non-finite value";
        case BZ_ERR_BUSY: return "busy";
        case BZ_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

}  // extern "C"

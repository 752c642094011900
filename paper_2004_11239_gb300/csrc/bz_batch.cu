// Batched collides and RK4 over many independent instances of one plan geometry.
//
// Instances stand in for the spatial cells of an inhomogeneous solver: same N, L, R,
// kernel, N_rho, M (one F table), a gamma of their own.  gamma enters only through
// c_p = w_i w_j r_i^(gamma + 2), so instance b scales the plan's alpha_p by
// r_i^(gamma_b - gamma_plan), a per-radial-node factor applied in the accumulation.
//
// State lives in slots [0, capacity); each call names the active slots, so instances can
// join and leave between steps (continuous batching).  The fused item kernel processes
// (instance, block of TB terms) items; an instance's result is the fixed-order FP64 sum of
// its block partials, independent of the other instances in the call.  One RK4 step
// (4 x [fused items, stage update]) is captured once per dt into a CUDA graph and replayed;
// the active count and slot list are read from device memory at run time.
#include <cmath>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <vector>

#include "bz_internal.h"
#include "bz_real.cuh"

struct bz_plan;

namespace bz {
const Plan *plan_internal(const bz_plan *plan);
}

struct bz_batch {
    bz::Plan *pl = nullptr;
    int capacity = 0, TB = 0, nblk = 0;
    std::vector<double> gamma;
    float *gsc = nullptr;           // [capacity][N_rho]
    float2 *fin = nullptr;          // [capacity][N^3]
    float2 *part = nullptr;         // [capacity][nblk][N^3]
    double2 *f0 = nullptr, *fsum = nullptr;   // [capacity][N^3]
    double2 *fin64 = nullptr, *scr64 = nullptr;   // [capacity][N^3] FP64 stage input and h scratch
    float2 *h = nullptr;            // [capacity][N^3] h per instance
    int units = 0;                  // work units of the plan: terms, or term pairs (BZ_DATA_REAL)
    float2 *fsym = nullptr;         // BZ_DATA_REAL: [capacity][N^3] Hermitian, Nyquist-free inputs
    float2 *part_s = nullptr;       // BZ_DATA_REAL: [capacity][nblk][3][N][N] Nyquist sums
    int *slots_dev = nullptr;       // [capacity]
    int *count_dev = nullptr;       // [1]
    int *host_stage = nullptr;      // pinned [capacity + 1]
    cudaStream_t cap_stream = nullptr;
    std::map<double, cudaGraphExec_t> graphs;
    int last_launches = 0;
    bool chunked = false;           // the plan runs the chunked pipeline: slots step one by one
    // chunked plans: one captured RK4 step per (slot, dt, dtype, array) -- the slot's input,
    // four stages and its output as one graph launch
    std::map<std::tuple<int, double, int, const void *>, cudaGraphExec_t> slot_graphs;
    int slot_graph_launches = 0;    // kernel launches inside one such graph
};

namespace bz {
namespace {

__global__ void k_batch_load(const void *fhat, int dtype, const int *slots, const int *count_dev, int n3,
                             float2 *fin) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(e / n3), k = (int)(e % n3);
    if (b >= *count_dev) return;
    const size_t idx = (size_t)slots[b] * n3 + k;
    if (dtype == BZ_C128) {
        double2 v = ((const double2 *)fhat)[idx];
        fin[idx] = make_float2((float)v.x, (float)v.y);
    } else {
        fin[idx] = ((const float2 *)fhat)[idx];
    }
}

// Sum of an instance's block partials in block order, Kahan-compensated on the FP32 pipes
// (the FP64 units of this GPU are far slower); returned in FP64.
__device__ __forceinline__ double2 sum_blocks(const float2 *part, int slot, int nblk, int n3, size_t k) {
    float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
    const float2 *p = part + (size_t)slot * nblk * n3 + k;
    for (int blk = 0; blk < nblk; ++blk) {
        float2 v = p[(size_t)blk * n3];
        float yr = v.x - cr, yi = v.y - ci;
        float tr = sr + yr, ti = si + yi;
        cr = (tr - sr) - yr;
        ci = (ti - si) - yi;
        sr = tr;
        si = ti;
    }
    return make_double2((double)sr - (double)cr, (double)si - (double)ci);
}

__global__ void k_batch_out(const float2 *part, int nblk, const int *slots, const int *count_dev, int n3,
                            void *Qhat, int dtype, int *flag) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(e / n3), k = (int)(e % n3);
    if (b >= *count_dev) return;
    const int slot = slots[b];
    double2 q = sum_blocks(part, slot, nblk, n3, k);
    const size_t idx = (size_t)slot * n3 + k;
    if (dtype == BZ_C128) {
        ((double2 *)Qhat)[idx] = q;
        note_finite(q, flag);
    } else {
        const float2 w = make_float2((float)q.x, (float)q.y);
        ((float2 *)Qhat)[idx] = w;
        note_finite(w, flag);
    }
}

__global__ void k_batch_rk_init(const void *fhat, int dtype, const int *slots, const int *count_dev, int n3,
                                double2 *f0, float2 *fin, double2 *fin64) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(e / n3), k = (int)(e % n3);
    if (b >= *count_dev) return;
    const size_t idx = (size_t)slots[b] * n3 + k;
    double2 v;
    if (dtype == BZ_C128) v = ((const double2 *)fhat)[idx];
    else {
        float2 w = ((const float2 *)fhat)[idx];
        v = make_double2(w.x, w.y);
    }
    f0[idx] = v;
    fin[idx] = make_float2((float)v.x, (float)v.y);
    fin64[idx] = v;
}

// Stage s of RK4 (the same combination as the single-instance path), k_s from the partials.
__global__ void k_batch_rk_stage(const float2 *part, int nblk, const int *slots, const int *count_dev, int n3,
                                 double2 *f0, double2 *fsum, float2 *fin, double2 *fin64, int stage, double dt) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(e / n3), k = (int)(e % n3);
    if (b >= *count_dev) return;
    const int slot = slots[b];
    const size_t idx = (size_t)slot * n3 + k;
    const double2 kv = sum_blocks(part, slot, nblk, n3, k);
    const double2 a = f0[idx];
    double2 y;
    if (stage == 1) {
        fsum[idx] = make_double2(a.x + dt / 6.0 * kv.x, a.y + dt / 6.0 * kv.y);
        y = make_double2(a.x + 0.5 * dt * kv.x, a.y + 0.5 * dt * kv.y);
    } else if (stage == 2 || stage == 3) {
        double2 s = fsum[idx];
        fsum[idx] = make_double2(s.x + dt / 3.0 * kv.x, s.y + dt / 3.0 * kv.y);
        const double c = stage == 2 ? 0.5 * dt : dt;
        y = make_double2(a.x + c * kv.x, a.y + c * kv.y);
    } else {
        double2 s = fsum[idx];
        y = make_double2(s.x + dt / 6.0 * kv.x, s.y + dt / 6.0 * kv.y);
        f0[idx] = y;
    }
    fin[idx] = make_float2((float)y.x, (float)y.y);
    fin64[idx] = y;
}

// BZ_DATA_REAL: Q of mode k from the block sums V (part) and X (part_s): V(k) + conj V(-k) off
// the Nyquist planes, V(k) + conj X(-k) on them.  The thread of the smaller index of each
// mirror pair {k, -k} off the Nyquist planes produces both entries (mm = the mirror, or -1 when
// this thread has nothing to do); returns Q(k) and, for a pair, Q(-k) in qm.
__device__ __forceinline__ bool real_q(const float2 *part, const float2 *part_s, int slot, int nblk, int N, int k,
                                       double2 &qk, double2 &qm, long long &mm) {
    const int n3 = N * N * N;
    const int i1 = k / (N * N), i2 = (k / N) % N, i3 = k % N;
    const int m1 = (N - i1) % N, m2 = (N - i2) % N, m3 = (N - i3) % N;
    mm = -1;
    const double2 v = sum_blocks(part, slot, nblk, n3, (size_t)k);
    if (nyquist(i1, i2, i3, N)) {
        const double2 x = sum_blocks(part_s, slot, nblk, 3 * N * N, (size_t)family_index(m1, m2, m3, N));
        qk = make_double2(v.x + x.x, v.y - x.y);
        return true;
    }
    const size_t m = ((size_t)m1 * N + m2) * N + m3;
    if ((size_t)k > m) return false;
    if ((size_t)k == m) {
        qk = make_double2(2.0 * v.x, 0.0);
        return true;
    }
    const double2 w = sum_blocks(part, slot, nblk, n3, m);
    qk = make_double2(v.x + w.x, v.y - w.y);
    qm = make_double2(w.x + v.x, w.y - v.y);
    mm = (long long)m;
    return true;
}

__global__ void k_batch_out_real(const float2 *part, const float2 *part_s, int nblk, const int *slots,
                                 const int *count_dev, int N, void *Qhat, int dtype, int *flag) {
    const int n3 = N * N * N;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(e / n3), k = (int)(e % n3);
    if (b >= *count_dev) return;
    const int slot = slots[b];
    double2 qk, qm;
    long long mm;
    if (!real_q(part, part_s, slot, nblk, N, k, qk, qm, mm)) return;
    const size_t base = (size_t)slot * n3;
    auto put = [&](size_t i, double2 q) {
        if (dtype == BZ_C128) {
            ((double2 *)Qhat)[base + i] = q;
            note_finite(q, flag);
        } else {
            const float2 w = make_float2((float)q.x, (float)q.y);
            ((float2 *)Qhat)[base + i] = w;
            note_finite(w, flag);
        }
    };
    put((size_t)k, qk);
    if (mm >= 0) put((size_t)mm, qm);
}

// Stage s of RK4 on one mode (the same combination as k_batch_rk_stage).
__device__ __forceinline__ void rk_stage_mode(size_t idx, double2 kv, double2 *f0, double2 *fsum, float2 *fin,
                                              double2 *fin64, int stage, double dt) {
    const double2 a = f0[idx];
    double2 y;
    if (stage == 1) {
        fsum[idx] = make_double2(a.x + dt / 6.0 * kv.x, a.y + dt / 6.0 * kv.y);
        y = make_double2(a.x + 0.5 * dt * kv.x, a.y + 0.5 * dt * kv.y);
    } else if (stage == 2 || stage == 3) {
        const double2 s = fsum[idx];
        fsum[idx] = make_double2(s.x + dt / 3.0 * kv.x, s.y + dt / 3.0 * kv.y);
        const double c = stage == 2 ? 0.5 * dt : dt;
        y = make_double2(a.x + c * kv.x, a.y + c * kv.y);
    } else {
        const double2 s = fsum[idx];
        y = make_double2(s.x + dt / 6.0 * kv.x, s.y + dt / 6.0 * kv.y);
        f0[idx] = y;
    }
    fin[idx] = make_float2((float)y.x, (float)y.y);
    fin64[idx] = y;
}

__global__ void k_batch_rk_stage_real(const float2 *part, const float2 *part_s, int nblk, const int *slots,
                                      const int *count_dev, int N, double2 *f0, double2 *fsum, float2 *fin,
                                      double2 *fin64, int stage, double dt) {
    const int n3 = N * N * N;
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(e / n3), k = (int)(e % n3);
    if (b >= *count_dev) return;
    const int slot = slots[b];
    double2 qk, qm;
    long long mm;
    if (!real_q(part, part_s, slot, nblk, N, k, qk, qm, mm)) return;
    const size_t base = (size_t)slot * n3;
    rk_stage_mode(base + k, qk, f0, fsum, fin, fin64, stage, dt);
    if (mm >= 0) rk_stage_mode(base + (size_t)mm, qm, f0, fsum, fin, fin64, stage, dt);
}

__global__ void k_batch_rk_out(const double2 *f0, const int *slots, const int *count_dev, int n3, void *fhat,
                               int dtype, int *flag) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(e / n3), k = (int)(e % n3);
    if (b >= *count_dev) return;
    const size_t idx = (size_t)slots[b] * n3 + k;
    if (dtype == BZ_C128) {
        ((double2 *)fhat)[idx] = f0[idx];
        note_finite(f0[idx], flag);
    } else {
        const float2 w = make_float2((float)f0[idx].x, (float)f0[idx].y);
        ((float2 *)fhat)[idx] = w;
        note_finite(w, flag);
    }
}

ItemArgs item_args(const bz_batch &B) {
    const Plan &pl = *B.pl;
    ItemArgs a;
    a.fin = B.fin; a.tw = pl.tw; a.alpha = pl.alpha; a.gsc = B.gsc; a.part = B.part;
    a.hg = pl.h_fp64 ? B.h : nullptr;
    a.slots = B.slots_dev; a.count_dev = B.count_dev; a.count = 0;
    a.p0 = 0; a.p1 = B.units; a.TB = B.TB; a.nblk = B.nblk; a.M = pl.M; a.N_rho = pl.N_rho;
    if (pl.real) {                                   // units are term pairs
        a.real = 1; a.fin = B.fsym; a.alpha = pl.apair; a.cpair = pl.cpair; a.part_s = B.part_s;
    }
    return a;
}

unsigned grid_for(const bz_batch &B) {
    const size_t n = (size_t)B.capacity * B.pl->N * B.pl->N * B.pl->N;
    return (unsigned)((n + 255) / 256);
}

bz_status stage_slots(bz_batch &B, int count, const int *slots, cudaStream_t st) {
    if (count < 0 || count > B.capacity || (count > 0 && !slots)) return BZ_ERR_ARG;
    std::vector<char> seen(B.capacity, 0);
    for (int b = 0; b < count; ++b) {
        if (slots[b] < 0 || slots[b] >= B.capacity || seen[slots[b]]) return BZ_ERR_ARG;
        seen[slots[b]] = 1;
    }
    // the pinned staging buffer may still feed an earlier copy on this stream
    if (cudaStreamSynchronize(st) != cudaSuccess) return BZ_ERR_CUDA;
    B.host_stage[0] = count;
    for (int b = 0; b < count; ++b) B.host_stage[1 + b] = slots[b];
    BZ_CUDA_TRY(cudaMemcpyAsync(B.count_dev, B.host_stage, sizeof(int), cudaMemcpyHostToDevice, st));
    if (count > 0)
        BZ_CUDA_TRY(cudaMemcpyAsync(B.slots_dev, B.host_stage + 1, count * sizeof(int), cudaMemcpyHostToDevice, st));
    return BZ_OK;
}

void free_batch(bz_batch *B) {
    for (auto &g : B->graphs) cudaGraphExecDestroy(g.second);
    B->graphs.clear();
    for (auto &g : B->slot_graphs) cudaGraphExecDestroy(g.second);
    B->slot_graphs.clear();
    cudaFree(B->gsc); cudaFree(B->fin); cudaFree(B->part); cudaFree(B->f0); cudaFree(B->fsum);
    cudaFree(B->fin64); cudaFree(B->scr64); cudaFree(B->h); cudaFree(B->fsym); cudaFree(B->part_s);
    cudaFree(B->slots_dev); cudaFree(B->count_dev);
    if (B->host_stage) cudaFreeHost(B->host_stage);
    if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
}

bz_status upload_gsc(bz_batch &B) {
    const Plan &pl = *B.pl;
    std::vector<float> g((size_t)B.capacity * pl.N_rho);
    for (int b = 0; b < B.capacity; ++b)
        for (int i = 0; i < pl.N_rho; ++i)
            g[(size_t)b * pl.N_rho + i] = (float)std::pow(pl.terms.r[(size_t)i * pl.M], B.gamma[b] - pl.gamma);
    BZ_CUDA_TRY(cudaMemcpy(B.gsc, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice));
    return BZ_OK;
}

// Picks the terms per item: times one full batched collide of `trial` zero instances for each
// candidate and keeps the fastest.  part must hold trial * ceil(P / min candidate) fields.
int autotune_tb(bz_batch &B, int trial, cudaStream_t st) {
    const Plan &pl = *B.pl;
    const int cands[] = {16, 32, 64, 128, 256, 512};
    int best = -1;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<int> slots(trial);
    for (int b = 0; b < trial; ++b) slots[b] = b;
    stage_slots(B, trial, slots.data(), st);
    for (int tb : cands) {
        if (tb > B.units && best > 0) break;
        B.TB = tb < B.units ? tb : B.units;
        B.nblk = (B.units + B.TB - 1) / B.TB;
        ItemArgs a = item_args(B);
        launch_fused(pl, a, st);                      // warm-up
        cudaEventRecord(e0, st);
        launch_fused(pl, a, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) { best_ms = ms; best = B.TB; }
        if (B.TB == B.units) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return best;
}

}  // namespace
}  // namespace bz

using namespace bz;

namespace bz {
namespace {

bz_status check_slots(const bz_batch &B, int count, const int *slots) {
    if (count < 0 || count > B.capacity || (count > 0 && !slots)) return BZ_ERR_ARG;
    std::vector<char> seen(B.capacity, 0);
    for (int b = 0; b < count; ++b) {
        if (slots[b] < 0 || slots[b] >= B.capacity || seen[slots[b]]) return BZ_ERR_ARG;
        seen[slots[b]] = 1;
    }
    return BZ_OK;
}

// Chunked plans: each active slot through the plan's pipeline with the slot's radial scale.
bz_status chunked_collide(bz_batch &B, int count, const int *slots, const void *fhat, void *Qhat, int dtype,
                          cudaStream_t st) {
    bz_status s = check_slots(B, count, slots);
    if (s != BZ_OK) return s;
    Plan &pl = *B.pl;
    const size_t bytes = (size_t)pl.N * pl.N * pl.N * (dtype == BZ_C128 ? sizeof(double2) : sizeof(float2));
    int nl = 0;
    for (int b = 0; b < count && s == BZ_OK; ++b) {
        pl.gsc_cur = B.gsc + (size_t)slots[b] * pl.N_rho;
        s = collide_range(pl, 0, pl.P, (const char *)fhat + slots[b] * bytes, dtype, st, &nl);
        if (s == BZ_OK) s = write_output(pl, (char *)Qhat + slots[b] * bytes, dtype, st, &nl);
    }
    pl.gsc_cur = nullptr;
    pl.src = nullptr;
    B.last_launches = nl;
    return s;
}

// One RK4 step of one slot captured as a graph (the host then launches one graph per slot and
// step instead of some hundred kernels).
bz_status slot_graph(bz_batch &B, int slot, void *fhat_slot, int dtype, double dt, cudaGraphExec_t *out) {
    Plan &pl = *B.pl;
    const auto key = std::make_tuple(slot, dt, dtype, (const void *)fhat_slot);
    auto it = B.slot_graphs.find(key);
    if (it != B.slot_graphs.end()) {
        *out = it->second;
        return BZ_OK;
    }
    cudaGraph_t g = nullptr;
    BZ_CUDA_TRY(cudaStreamBeginCapture(B.cap_stream, cudaStreamCaptureModeThreadLocal));
    pl.gsc_cur = B.gsc + (size_t)slot * pl.N_rho;
    int nl = 0;
    const bz_status cs = rk4_steps(pl, fhat_slot, dtype, dt, 1, B.cap_stream, &nl);
    pl.gsc_cur = nullptr;
    pl.src = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(B.cap_stream, &g);
    if (cs != BZ_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cs != BZ_OK ? cs : BZ_ERR_CUDA;
    }
    cudaGraphExec_t ex = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return BZ_ERR_CUDA;
    B.slot_graphs.emplace(key, ex);
    B.slot_graph_launches = nl;
    *out = ex;
    return BZ_OK;
}

bz_status chunked_step_rk(bz_batch &B, int count, const int *slots, void *fhat, int dtype, double dt, int nsteps,
                          cudaStream_t st) {
    bz_status s = check_slots(B, count, slots);
    if (s != BZ_OK) return s;
    Plan &pl = *B.pl;
    const size_t bytes = (size_t)pl.N * pl.N * pl.N * (dtype == BZ_C128 ? sizeof(double2) : sizeof(float2));
    int nl = 0;
    if (pl.tm.on) {
        // per-kernel timing brackets every launch with events: no graphs
        for (int b = 0; b < count && s == BZ_OK; ++b) {
            pl.gsc_cur = B.gsc + (size_t)slots[b] * pl.N_rho;
            s = rk4_steps(pl, (char *)fhat + slots[b] * bytes, dtype, dt, nsteps, st, &nl);
        }
        pl.gsc_cur = nullptr;
        pl.src = nullptr;
        B.last_launches = nl;
        return s;
    }
    for (int b = 0; b < count && s == BZ_OK; ++b) {
        cudaGraphExec_t ex = nullptr;
        s = slot_graph(B, slots[b], (char *)fhat + slots[b] * bytes, dtype, dt, &ex);
        for (int k = 0; k < nsteps && s == BZ_OK; ++k) {
            if (cudaGraphLaunch(ex, st) != cudaSuccess) s = BZ_ERR_CUDA;
            nl += B.slot_graph_launches;
        }
    }
    B.last_launches = nl;
    return s;
}

}  // namespace
}  // namespace bz

extern "C" {

bz_status bz_batch_create(bz_batch **out, const bz_plan *plan, int capacity, int terms_per_item) {
    if (!out || !plan || capacity < 1) return BZ_ERR_ARG;
    *out = nullptr;
    Plan *pl = const_cast<Plan *>(plan_internal(plan));
    // batches: circular 3D plans; on the fused pipeline the real-data form needs h formed in FP64
    if (pl->Nin || pl->dim == 2 || (pl->use_fused && pl->real && !pl->h_fp64)) return BZ_ERR_UNSUPPORTED;
    bz_batch *B = new (std::nothrow) bz_batch();
    if (!B) return BZ_ERR_OOM;
    B->pl = pl;
    B->units = pl->real ? pl->P / 2 : pl->P;
    B->capacity = capacity;
    B->gamma.assign(capacity, pl->gamma);
    const size_t n3 = (size_t)pl->N * pl->N * pl->N;
    const size_t field = n3 * sizeof(float2);
    auto fail = [&](bz_status s) { free_batch(B); delete B; return s; };
    if (!pl->use_fused) {
        // chunked plans step their slots one after another through the plan's own pipeline
        // (each chunk kernel already fills the GPU); only the radial scales live in the batch
        B->chunked = true;
        if (cudaMalloc(&B->gsc, (size_t)capacity * pl->N_rho * sizeof(float)) != cudaSuccess ||
            cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return fail(BZ_ERR_OOM);
        }
        if (upload_gsc(*B) != BZ_OK) return fail(BZ_ERR_CUDA);
        B->TB = B->units;
        B->nblk = 1;
        *out = B;
        return BZ_OK;
    }
    if (cudaMalloc(&B->gsc, (size_t)capacity * pl->N_rho * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&B->fin, (size_t)capacity * field) != cudaSuccess ||
        cudaMalloc(&B->f0, (size_t)capacity * n3 * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&B->fsum, (size_t)capacity * n3 * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&B->fin64, (size_t)capacity * n3 * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&B->scr64, (size_t)capacity * n3 * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&B->h, (size_t)capacity * field) != cudaSuccess ||
        (pl->real && cudaMalloc(&B->fsym, (size_t)capacity * field) != cudaSuccess) ||
        cudaMalloc(&B->slots_dev, (size_t)capacity * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&B->count_dev, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&B->host_stage, (size_t)(capacity + 1) * sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(BZ_ERR_OOM);
    }
    if (upload_gsc(*B) != BZ_OK) return fail(BZ_ERR_CUDA);
    int tb = pl->real && terms_per_item > 0 ? (terms_per_item + 1) / 2 : terms_per_item;   // in units
    if (tb <= 0) {
        // autotune on a trial of up to 4 instances per resident cluster
        int trial = capacity < 4 * pl->fused_G ? capacity : 4 * pl->fused_G;
        int nblk_max = (B->units + 15) / 16;
        if (cudaMalloc(&B->part, (size_t)trial * nblk_max * field) != cudaSuccess ||
            (pl->real && cudaMalloc(&B->part_s, (size_t)trial * nblk_max * 3 * pl->N * pl->N * sizeof(float2)) !=
                             cudaSuccess)) {
            cudaGetLastError();
            return fail(BZ_ERR_OOM);
        }
        if (pl->real && cudaMemset(B->fsym, 0, (size_t)trial * field) != cudaSuccess) return fail(BZ_ERR_CUDA);
        if (cudaMemset(B->fin, 0, (size_t)trial * field) != cudaSuccess ||
            cudaMemset(B->h, 0, (size_t)trial * field) != cudaSuccess) return fail(BZ_ERR_CUDA);
        tb = autotune_tb(*B, trial, B->cap_stream);
        cudaStreamSynchronize(B->cap_stream);
        cudaFree(B->part);
        cudaFree(B->part_s);
        B->part = nullptr;
        B->part_s = nullptr;
        if (tb <= 0) return fail(BZ_ERR_CUDA);
    }
    B->TB = tb < B->units ? tb : B->units;
    B->nblk = (B->units + B->TB - 1) / B->TB;
    if (cudaMalloc(&B->part, (size_t)capacity * B->nblk * field) != cudaSuccess ||
        (pl->real && cudaMalloc(&B->part_s, (size_t)capacity * B->nblk * 3 * pl->N * pl->N * sizeof(float2)) !=
                         cudaSuccess)) {
        cudaGetLastError();
        return fail(BZ_ERR_OOM);
    }
    *out = B;
    return BZ_OK;
}

bz_status bz_batch_set_gamma(bz_batch *batch, int slot, double gamma) {
    if (!batch || slot < 0 || slot >= batch->capacity || !std::isfinite(gamma)) return BZ_ERR_ARG;
    batch->gamma[slot] = gamma;
    const Plan &pl = *batch->pl;
    std::vector<float> g(pl.N_rho);
    for (int i = 0; i < pl.N_rho; ++i) g[i] = (float)std::pow(pl.terms.r[(size_t)i * pl.M], gamma - pl.gamma);
    BZ_CUDA_TRY(cudaMemcpy(batch->gsc + (size_t)slot * pl.N_rho, g.data(), g.size() * sizeof(float),
                           cudaMemcpyHostToDevice));
    return BZ_OK;
}

bz_status bz_batch_info(const bz_batch *batch, int *capacity, int *terms_per_item, size_t *workspace_bytes) {
    if (!batch) return BZ_ERR_ARG;
    const size_t n3 = (size_t)batch->pl->N * batch->pl->N * batch->pl->N;
    if (capacity) *capacity = batch->capacity;
    if (terms_per_item) *terms_per_item = batch->TB * (batch->pl->real ? 2 : 1);
    if (workspace_bytes)
        *workspace_bytes = (size_t)batch->capacity * n3 * (sizeof(float2) * (1 + batch->nblk) + 2 * sizeof(double2));
    return BZ_OK;
}

bz_status bz_batch_collide(bz_batch *batch, int count, const int *slots, const void *fhat, void *Qhat, int dtype,
                           void *stream) {
    if (!batch || !fhat || !Qhat || fhat == Qhat) return BZ_ERR_ARG;
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    bz_batch &B = *batch;
    cudaStream_t st = (cudaStream_t)stream;
    if (B.chunked) return chunked_collide(B, count, slots, fhat, Qhat, dtype, st);
    bz_status s = stage_slots(B, count, slots, st);
    if (s != BZ_OK) return s;
    const int n3 = B.pl->N * B.pl->N * B.pl->N;
    if (!B.pl->real)
        k_batch_load<<<grid_for(B), 256, 0, st>>>(fhat, dtype, B.slots_dev, B.count_dev, n3, B.fin);
    if (B.pl->h_fp64) {                                   // (the real-data form's inputs come from the first pass)
        s = h64_launch(B.pl->N, fhat, dtype, B.slots_dev, B.count_dev, B.capacity, B.scr64, B.h, st, B.fsym);
        if (s != BZ_OK) return s;
    }
    s = launch_fused(*B.pl, item_args(B), st);
    if (s != BZ_OK) return s;
    if (B.pl->real)
        k_batch_out_real<<<grid_for(B), 256, 0, st>>>(B.part, B.part_s, B.nblk, B.slots_dev, B.count_dev, B.pl->N,
                                                     Qhat, dtype, nonfinite_flag(*B.pl));
    else
        k_batch_out<<<grid_for(B), 256, 0, st>>>(B.part, B.nblk, B.slots_dev, B.count_dev, n3, Qhat, dtype,
                                                nonfinite_flag(*B.pl));
    BZ_CUDA_TRY(cudaGetLastError());
    B.last_launches = (B.pl->real ? 2 : 3) + (B.pl->h_fp64 ? h64_launches(B.pl->N) : 0);
    return BZ_OK;
}

bz_status bz_batch_step_rk(bz_batch *batch, int count, const int *slots, void *fhat, int dtype, double dt,
                           int nsteps, void *stream) {
    if (!batch || !fhat || nsteps < 0 || !std::isfinite(dt)) return BZ_ERR_ARG;
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    bz_batch &B = *batch;
    cudaStream_t st = (cudaStream_t)stream;
    if (B.chunked) return chunked_step_rk(B, count, slots, fhat, dtype, dt, nsteps, st);
    bz_status s = stage_slots(B, count, slots, st);
    if (s != BZ_OK) return s;
    const int n3 = B.pl->N * B.pl->N * B.pl->N;
    auto it = B.graphs.find(dt);
    if (it == B.graphs.end()) {
        // capture one RK4 step: 4 x (fused items, stage update)
        cudaGraph_t g = nullptr;
        BZ_CUDA_TRY(cudaStreamBeginCapture(B.cap_stream, cudaStreamCaptureModeThreadLocal));
        bz_status cs = BZ_OK;
        for (int stage = 1; stage <= 4 && cs == BZ_OK; ++stage) {
            if (B.pl->h_fp64)
                cs = h64_launch(B.pl->N, B.fin64, BZ_C128, B.slots_dev, B.count_dev, B.capacity, B.scr64, B.h,
                                B.cap_stream, B.fsym);
            if (cs == BZ_OK) cs = launch_fused(*B.pl, item_args(B), B.cap_stream);
            if (B.pl->real)
                k_batch_rk_stage_real<<<grid_for(B), 256, 0, B.cap_stream>>>(B.part, B.part_s, B.nblk, B.slots_dev,
                                                                            B.count_dev, B.pl->N, B.f0, B.fsum,
                                                                            B.fin, B.fin64, stage, dt);
            else
                k_batch_rk_stage<<<grid_for(B), 256, 0, B.cap_stream>>>(B.part, B.nblk, B.slots_dev, B.count_dev, n3,
                                                                       B.f0, B.fsum, B.fin, B.fin64, stage, dt);
        }
        cudaError_t ce = cudaStreamEndCapture(B.cap_stream, &g);
        if (cs != BZ_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return cs != BZ_OK ? cs : BZ_ERR_CUDA;
        }
        cudaGraphExec_t ex = nullptr;
        ce = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return BZ_ERR_CUDA;
        it = B.graphs.emplace(dt, ex).first;
    }
    k_batch_rk_init<<<grid_for(B), 256, 0, st>>>(fhat, dtype, B.slots_dev, B.count_dev, n3, B.f0, B.fin, B.fin64);
    for (int step = 0; step < nsteps; ++step) BZ_CUDA_TRY(cudaGraphLaunch(it->second, st));
    k_batch_rk_out<<<grid_for(B), 256, 0, st>>>(B.f0, B.slots_dev, B.count_dev, n3, fhat, dtype, nonfinite_flag(*B.pl));
    BZ_CUDA_TRY(cudaGetLastError());
    B.last_launches = 2 + 4 * (2 + (B.pl->h_fp64 ? h64_launches(B.pl->N) : 0)) * nsteps;
    return BZ_OK;
}

bz_status bz_inhom_step(bz_batch *batch, int nx, double Lx, void *fcells, int dtype, double dt, int nsteps,
                        void *stream) {
    if (!batch || !fcells || nx < 1 || nx > batch->capacity || !(Lx > 0) || nsteps < 0 || !std::isfinite(dt))
        return BZ_ERR_ARG;
    if (dtype != BZ_C64 && dtype != BZ_C128) return BZ_ERR_ARG;
    const bz::Plan &pl = *batch->pl;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> slots(nx);
    for (int c = 0; c < nx; ++c) slots[c] = c;
    int launches = 0;
    for (int step = 0; step < nsteps; ++step) {
        // free streaming dt/2 before the first collision step, dt between two, dt/2 after the last
        bz_status s = bz::transport_x(pl.N, pl.L, nx, Lx, fcells, dtype, step == 0 ? 0.5 * dt : dt, st);
        if (s == BZ_OK) s = bz_batch_step_rk(batch, nx, slots.data(), fcells, dtype, dt, 1, stream);
        if (s != BZ_OK) return s;
        launches += 1 + batch->last_launches;
    }
    if (nsteps > 0) {
        bz_status s = bz::transport_x(pl.N, pl.L, nx, Lx, fcells, dtype, 0.5 * dt, st);
        if (s != BZ_OK) return s;
        ++launches;
    }
    batch->last_launches = launches;
    return BZ_OK;
}

int bz_batch_last_launches(const bz_batch *batch) { return batch ? batch->last_launches : 0; }

void bz_batch_destroy(bz_batch *batch) {
    if (!batch) return;
    free_batch(batch);
    delete batch;
}

}  // extern "C"

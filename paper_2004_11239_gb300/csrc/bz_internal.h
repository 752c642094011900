// Internal declarations shared by the translation units of libbz (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/bz.h"

#ifndef EXTRA_STREAMS
#define EXTRA_STREAMS 1
#endif

namespace bz {

// One radial node's part-II theta rule (Sec. 4.1): nodes t_n on [eps, pi] with
// weights W_n = w_n g(t_n), stored as (1 - cos t_n, sin t_n, W_n).
struct ThetaRule {
    std::vector<double> omc, sn, W;
};

struct HostTerms {
    std::vector<double> r, wr, q, wq, c;   // per term p = i*M + j; q is [P][3]
    std::vector<int> radial_index;          // i for each p
};

// Optional per-kernel CUDA-event timing (bz_plan_set_timing).
enum { TK_PLANE_INV = 0, TK_PENCIL = 1, TK_PLANE_FWD = 2, TK_REDUCE = 3, TK_OTHER = 4, TK_FUSED = 5, TK_COUNT = 6 };
struct Timing {
    bool on = false;
    std::vector<cudaEvent_t> ev;    // pairs (start, end)
    std::vector<int> kind;          // per pair
    size_t used = 0;                // pairs recorded since the last collect
    double ms[TK_COUNT] = {0, 0, 0, 0, 0, 0};
    long n[TK_COUNT] = {0, 0, 0, 0, 0, 0};
};

// Streams of the chunked pipeline beside the caller's.
constexpr int kExtraStreams = EXTRA_STREAMS;

struct Plan {
    // parameters
    int N = 0, N_rho = 0, M = 0, P = 0, kernel = 0, precision = 0, device = 0;
    int Nin = 0;                    // BZ_CONV_PADDED: the caller's modes per axis (N = 2 Nin); 0 = circular
    int dim = 3;                    // 3: the 3D operator; 2: the 2D operator on an N x N grid
    double L = 0, R = 0, gamma = 0, s = 0, eps = 0;
    double theta0 = 0;              // angular cutoff (0: none)
    double A[3] = {0, 0, 0};        // part I kernel moments
    double kc = 0;                  // kernel constant (c_s, 1/(4 pi), 5/(192 pi))
    HostTerms terms;
    std::vector<ThetaRule> rules;   // one per radial node
    // device tables
    float2 *alpha = nullptr;        // [P][N^3]  c_p F / N^3
    float2 *tw = nullptr;           // [P][3][N] exp(-i pi r q_d m / L)
    double *rule_buf = nullptr;     // concatenated (omc, sn, W) per radial node
    int *rule_off = nullptr;        // [N_rho + 1] node offsets
    int rule_max = 0;               // largest node count of one radial node
    double *term_dev = nullptr;     // [P][5]: r, q0, q1, q2, c
    // workspace
    int chunk = 0;                  // terms per chunk
    float2 *S = nullptr;            // [chunk][N^3]
    float2 *h = nullptr;            // [N^3]
    float2 *fin = nullptr;          // [N^3] FP32 input
    double2 *acc = nullptr;         // [N^3] FP64 accumulator (while a chunked collide runs, the same
                                    // bytes hold k_reduce's compensated FP32 state: s, c per mode pair)
    double2 *rk = nullptr;          // [3][N^3] RK4 state (f0, fsum) + spare
    double *mom = nullptr;          // moments scratch
    // fused cluster pipeline (N <= 32)
    int use_fused = 0;              // 1: bz_collide runs k_fused
    int fused_C = 0;                // CTAs per cluster
    int fused_G = 0;                // resident clusters (persistent grid)
    float fused_ms = 0.f;           // timed collide of the selected cluster size
    int h_fp64 = 1;                 // fused path: h formed in FP64 (1) or in FP32 in-kernel (0)
    double2 *fin64 = nullptr;       // [N^3] FP64 stage input (RK4) for the FP64 h pass
    double2 *scr64 = nullptr;       // [N^3] FP64 scratch of the h pass
    const void *src = nullptr;      // FP64-capable source of h for the next fused collide
    int src_dtype = BZ_C128;
    float2 *part = nullptr;         // [fused_G][N^3] per-cluster partial sums
    uint4 *wimg = nullptr;          // BZ_PREC_BF16X3: split DFT matrix (tensor-core B operand)
    // BZ_DATA_REAL: terms 2q and 2q + 1 share one pair of transforms
    int real = 0;
    int pair3 = 0;                  // N = 32: the three-CTA-per-SM pair kernel (k_pair3) instead of k_fused
    float2 *apair = nullptr;        // [P / 2][N^3] A = (alpha_2q - i alpha_2q+1) / 2
    float2 *cpair = nullptr;        // [P / 2][3][N][N] C = conj B(-k), B = (alpha_2q + i alpha_2q+1) / 2, on the
                                    // Nyquist planes (families k1 = -N/2, k2 = -N/2, k3 = -N/2), 0 elsewhere
    float2 *part_s = nullptr;       // [fused_G][3][N][N] per-item sums X on the Nyquist planes
    float2 *S_s = nullptr;          // chunked pipeline: [chunk][3][N][N] the chunk's Nyquist sums
    double2 *acc_s = nullptr;       // chunked pipeline: [3][N][N] FP64 sum of X
    // chunked pipeline on several streams: chunk i runs on lane i % (1 + xn), lane 0 the
    // caller's stream over S / acc, lane e > 0 the plan's stream xst[e - 1] over its own
    // scratch and accumulators; the lanes overlap and their sums are added at the end
    int xn = 0;                                      // extra streams in use
    cudaStream_t xst[kExtraStreams] = {};
    cudaEvent_t ev_fork = nullptr, xev_join[kExtraStreams] = {};
    float2 *xS[kExtraStreams] = {};                  // [chunk][N^3]
    float2 *xS_s[kExtraStreams] = {};                // [chunk][3][N][N] (BZ_DATA_REAL)
    double2 *xacc[kExtraStreams] = {};               // [N^3]
    double2 *xacc_s[kExtraStreams] = {};             // [3][N][N] (BZ_DATA_REAL)
    float2 *fsym = nullptr;         // [N^3] Hermitian part of fhat, Nyquist planes zero (FP32)
    double2 *fsym64 = nullptr;      // [N^3] the same in FP64 (source of h)
    const float *gsc_cur = nullptr; // chunked pipeline inside a batch call: the slot's radial scale
                                    // r_i^(gamma_slot - gamma) per radial node (null: none)
    int *dev_err = nullptr;         // device flags: [0] a bounded wait of a kernel gave up,
                                    // [1] a result written since the last check held NaN or Inf
    size_t ws_bytes = 0;
    int last_launches = 0;
    Timing tm;
};

// Raises the non-finite flag (Plan::dev_err[1]) if the value written is NaN or Inf.
#ifdef __CUDACC__
__device__ __forceinline__ void note_finite(double2 v, int *flag) {
    if (flag && !(isfinite(v.x) && isfinite(v.y))) atomicOr(flag, 1);
}
__device__ __forceinline__ void note_finite(float2 v, int *flag) {
    if (flag && !(isfinite(v.x) && isfinite(v.y))) atomicOr(flag, 1);
}
#endif
inline int *nonfinite_flag(const Plan &pl) { return pl.dev_err ? pl.dev_err + 1 : nullptr; }

// Fourier modes of one field: N^3 (3D) or N^2 (2D).
inline size_t modes(const Plan &pl) { return (size_t)pl.N * pl.N * (pl.dim == 2 ? 1 : pl.N); }

// Brackets one launch with events when timing is on (events are pre-created).
inline void tm_begin(Plan &pl, cudaStream_t st) {
    if (pl.tm.on && pl.tm.used < pl.tm.kind.size()) cudaEventRecord(pl.tm.ev[2 * pl.tm.used], st);
}
inline void tm_end(Plan &pl, cudaStream_t st, int kind) {
    if (pl.tm.on && pl.tm.used < pl.tm.kind.size()) {
        cudaEventRecord(pl.tm.ev[2 * pl.tm.used + 1], st);
        pl.tm.kind[pl.tm.used++] = kind;
    }
}

// bz_quad.cpp
int gauss_legendre(int n, double a, double b, std::vector<double> &x, std::vector<double> &w);
bz_status build_terms(Plan &pl, const double *sphere_xyz, const double *sphere_w);
bz_status build_kernel_constants(Plan &pl);
void build_theta_rules(Plan &pl);

// bz_ftable.cu
bz_status ftable_build(Plan &pl);
bz_status ftable_entries(Plan &pl, int count, const int *k_idx, const int *term, double *out);

// bz_collide.cu
bz_status collide_range(Plan &pl, int p0, int p1, const void *fhat, int in_dtype,
                        cudaStream_t st, int *launches);
bz_status write_output(Plan &pl, void *Qhat, int dtype, cudaStream_t st, int *launches);
bz_status load_input(Plan &pl, const void *fhat, int dtype, cudaStream_t st, int *launches);
bz_status collide_core(Plan &pl, int p0, int p1, cudaStream_t st, int *launches);
// pl.h = IFFT(fin) in FP32 (one plane pass and one pencil pass through pl.S; N = 8, 16, 32)
bz_status h_fp32(Plan &pl, const float2 *fin, cudaStream_t st);

// bz_fused.cu
// Arguments of the fused item kernel (see k_fused): item w = (instance w / nblk, term block
// w % nblk); instance b lives in array slot slots[b] (identity when slots is null).
struct ItemArgs {
    const float2 *fin = nullptr;     // [slots][N^3] FP32 inputs
    const float2 *tw = nullptr;      // [P][3][N]
    const float2 *alpha = nullptr;   // [P][N^3]
    const float *gsc = nullptr;      // [slots][N_rho] radial scale r_i^(gamma_b - gamma_plan), or null
    float2 *part = nullptr;          // [slots][nblk][N^3] per-item partial sums
    const float2 *hg = nullptr;      // [slots][N^3] h = IFFT(fhat), formed in FP64, stored FP32
    const int *slots = nullptr;      // device [count] or null
    const int *count_dev = nullptr;  // device instance count, or null (use count)
    int count = 1, p0 = 0, p1 = 0, TB = 1, nblk = 0, M = 1, N_rho = 1;
    int real = 0;                    // BZ_DATA_REAL: p0, p1 count term pairs, alpha = the pair table
    const float2 *cpair = nullptr;   // BZ_DATA_REAL: [pairs][3][N][N] Nyquist-plane table C
    float2 *part_s = nullptr;        // BZ_DATA_REAL: [slots][nblk][3][N][N] per-item sums X
};
int fused_candidates(int N, int *cs);
cudaError_t fused_setup(int N, int C, int *G, bool real);
bz_status launch_fused(const Plan &pl, const ItemArgs &a, cudaStream_t st);
// h[slot] = IFFT(f[slot]) computed in FP64 and stored FP32 for the active slots (N <= 32).
// Kernel launches of one h64_launch: three line passes (N = 32: the k3 and k2 passes as one).
inline int h64_launches(int N) { return N == 32 ? 2 : 3; }
// fsym (BZ_DATA_REAL, N a power of two): transform the Hermitian, Nyquist-free part of f and
// store that part in FP32 to fsym.
bz_status h64_launch(int N, const void *f, int dtype, const int *slots, const int *count_dev, int count,
                     double2 *scr, float2 *h, cudaStream_t st, float2 *fsym = nullptr);
bz_status collide_fused(Plan &pl, int p0, int p1, cudaStream_t st, int *launches);
// bz_real.cu (BZ_DATA_REAL): the pair table from alpha (after ftable_build); pl.fsym and
// pl.fsym64 from a c64 / c128 array
bz_status build_pair_table(Plan &pl);
bz_status sym_input(Plan &pl, const void *f, int dtype, cudaStream_t st);
// pl.acc <- Q from the nblk item sums of pl.part (V) and pl.part_s (X): one kernel
bz_status reduce_sym(Plan &pl, int nblk, cudaStream_t st);
// chunked pipeline: pl.acc (V, FP64) <- Q in place, with pl.acc_s (X)
bz_status sym_output(Plan &pl, cudaStream_t st);

// bz_pair3.cu (BZ_DATA_REAL, N = 32, FP64 h): resident clusters and launch of k_pair3
cudaError_t pair3_setup(int *G);
bz_status launch_pair3(const Plan &pl, const ItemArgs &a, cudaStream_t st);

// bz_mixed.cu (BZ_PREC_BF16X3, N = 32)
cudaError_t mixed_setup(int N, int *G);
bz_status mixed_upload(uint4 **wimg);
bz_status launch_mixed(const Plan &pl, const ItemArgs &a, cudaStream_t st);
// one bounded wait that nothing completes, giving up after `limit` clocks (bz_plan_wait_selftest)
bz_status wait_selftest(const Plan &pl, long long limit, cudaStream_t st);
cudaError_t collide_set_attributes(int N);
// bz_chunk64.cu: the plane and pencil passes of the chunked pipeline at N = 64 (radix 8 x 8)
cudaError_t chunk64_set_attributes();
void plane_inv64(const float2 *fin, const float2 *tw, float2 *S, int p0, int T, int use_tw, bool pair,
                 cudaStream_t st);
void plane_fwd64(float2 *S, const float2 *alpha, int p0, int T, const float2 *cpair, float2 *Ss, const float *gsc,
                 int M, bool pair, cudaStream_t st);
// pencil pass (axis 1) over T terms: mode 0 out = IFFT_1(S); 1 S = FFT_1(h . IFFT_1(S)); 2 as 1 with
// h real (N^3 packed floats); 3 out = Re IFFT_1(S) as N^3 packed floats
void pencil64(float2 *S, const float2 *h, float2 *out, int T, int mode, cudaStream_t st);
void reduce_parts(const float2 *part, int nblk, int n, double2 *acc, cudaStream_t st);
int chunk_terms_for(int N);          // after collide_set_attributes(N)
int supported_N(int N);

// bz_2d.cu (dim = 2)
cudaError_t setup_2d(Plan &pl);                       // persistent grid size (pl.fused_G)
bz_status collide_2d(Plan &pl, int p0, int p1, cudaStream_t st, int *launches);

// bz_inhom.cu: free streaming of nx cells (bz_transport_x)
bz_status transport_x(int N, double L, int nx, double Lx, void *f, int dtype, double t, cudaStream_t st);

// bz_rk.cu
bz_status rk4_steps(Plan &pl, void *fhat, int dtype, double dt, int nsteps, cudaStream_t st,
                    int *launches);
bz_status moments(Plan &pl, const void *fhat, int dtype, double out[5], cudaStream_t st);

}  // namespace bz

#define BZ_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return BZ_ERR_CUDA;          \
    } while (0)

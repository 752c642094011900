/*
 * bz -- fast Fourier spectral evaluation of the non-cutoff Boltzmann collision
 * operator (Hu & Qi, arXiv 2004.11239) on one NVIDIA GB300 (sm_103a).
 *
 * C ABI.  Plain pointers and sizes only.  Every function returns a bz_status;
 * nothing is thrown or printed.  Device pointers are CUDA device addresses on the
 * plan's device (for example torch.Tensor.data_ptr()); `stream` is a cudaStream_t
 * passed as void* (NULL = the legacy default stream).  Calls are asynchronous on
 * `stream` unless stated otherwise.  A plan is not re-entrant: do not run two calls
 * on one plan concurrently on different streams.
 *
 * Data layout.  A Fourier coefficient array (fhat, Qhat) holds N^3 complex values,
 * C-order [k1][k2][k3], FFT-natural index order: array index i along an axis is
 * the signed mode k = i for i < N/2 and k = i - N otherwise (the modes are
 * -N/2 .. N/2-1; Sec. 2 writes -N/2..N/2, read here as N modes).  The coefficients
 * follow Sec. 2: f_N(v) = sum_k fhat_k exp(i pi k.v / L) on [-L, L]^3.
 * dtype BZ_C64 = interleaved float (re, im); BZ_C128 = interleaved double.
 *
 * The operator (Sec. 4, eqs. GG1, approxG, realQ; terms p = i*M + j):
 *   Qhat_k = sum_p c_p F(k, r_i, qhat_j) sum_{l+m=k (mod N)} fhat_l beta_p(m) fhat_m,
 *   c_p = w_i w_j r_i^gamma r_i^2,  beta_p(m) = exp(-i pi r_i m.qhat_j / L),
 *   F(k,r,qhat) = int_{S^2} b(sigma.qhat) (exp(i pi r k.(qhat - sigma)/(2L)) - 1) dsigma
 *   (Sec. 2.1, eq. FF), computed by the split of Sec. 4.1 (Taylor part on [0, eps],
 *   quadrature on [eps, pi], exact phi integral).  The inner sum is the circular
 *   convolution computed by one inverse 3D FFT of beta_p fhat, a product with
 *   h = IFFT(fhat), and one forward 3D FFT per term (Sec. 4: "a few FFTs").
 */
#ifndef BZ_H
#define BZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BZ_OK = 0,
    BZ_ERR_ARG = 1,          /* invalid argument (sizes, pointers, aliasing)          */
    BZ_ERR_OOM = 2,          /* device or host allocation failed                      */
    BZ_ERR_CUDA = 3,         /* a CUDA runtime call failed                            */
    BZ_ERR_TIMEOUT = 4,      /* a bounded device or host wait ran out                 */
    BZ_ERR_NONFINITE = 5,    /* NaN or Inf detected in a result                       */
    BZ_ERR_BUSY = 6,         /* not admissible now / result not ready yet             */
    BZ_ERR_UNSUPPORTED = 7   /* parameter combination not implemented                 */
} bz_status;

enum { BZ_C64 = 0, BZ_C128 = 1 };

/* Angular kernels, given by g(theta) = sin(theta) b(cos theta):
 *   BZ_KERNEL_FAMILY: g = c_s sin^(-1-2s)(theta/2), 0 <= s < 1 (singularity theta^(-1-nu),
 *                     nu = 2s, Sec. 2.1 eq. bb); c_s = 1/(12 pi B(1-s, 3/2)) so that
 *                     lambda = 1/6 (Sec. 5.1).  s = 0 is eq. b6, s = 1/2 is eq. b7.
 *   BZ_KERNEL_B5:     b = 1/(4 pi), the cutoff kernel of eq. b5.
 *   BZ_KERNEL_B8:     b = 5 cos(theta/2) / (192 pi sin(theta) sin^(5/2)(theta/2)), eq. b8. */
enum { BZ_KERNEL_FAMILY = 0, BZ_KERNEL_B5 = 1, BZ_KERNEL_B8 = 2 };

/* BZ_KERNEL_DEBYE (3D, Sec. 5.4, eq. ApproximatedDebye): sin(theta) b = |log(2 sin(theta/2))| /
 * (2 sin(theta/2)), the angular part of the Debye-Yukawa kernel; its |v - v*| factor is
 * Phi(|q|) = |q|, i.e. gamma = 1.  Its part-I moments have no closed form and are computed by
 * Gauss-Legendre quadrature after t = eps u^2. */
enum { BZ_KERNEL_DEBYE = 7 };

/* 2D angular kernels (dim = 2; Sec. 5.2, eqs. b1-b4), b(cos theta) on theta in [0, 2 pi] with
 * the measure d theta on the circle, all with lambda = 1/8 (eq. KK2):
 *   BZ_KERNEL_B1: 1 / (2 pi) (cutoff);          BZ_KERNEL_B2: 3 / (32 sin(theta/2));
 *   BZ_KERNEL_B3: 1 / (8 pi sin^2(theta/2));     BZ_KERNEL_B4: 5 |cos(theta/2)| / (256 sin^(5/2)(theta/2)). */
enum { BZ_KERNEL_B1 = 3, BZ_KERNEL_B2 = 4, BZ_KERNEL_B3 = 5, BZ_KERNEL_B4 = 6 };

/* Arithmetic of the per-term transforms (Sec. 4, eq. realQ: two 3D FFTs per term).
 *   BZ_PREC_FP32:   FP32 register FFTs on the CUDA cores (every supported N).
 *   BZ_PREC_BF16X3: each one-axis transform is a DFT on the tensor cores with BF16 operands
 *                   split as x = x_hi + x_lo and the products x_hi w_hi + x_lo w_hi +
 *                   x_hi w_lo accumulated in FP32 (about 16 significant bits per product);
 *                   twiddles, the product with h, the alpha weighting and the sum over terms
 *                   stay FP32, h is formed in FP64.  Fused pipeline, N = 32 only; other N
 *                   or BZ_PIPE_CHUNKED give BZ_ERR_UNSUPPORTED.  Accuracy target: relative
 *                   L-infinity error 1e-3 of max |Qhat|. */
enum { BZ_PREC_FP32 = 0, BZ_PREC_BF16X3 = 1 };

/* Form of the inner sum over l + m = k (Sec. 2, eq. sum; Sec. 4, eq. realQ).
 *   BZ_CONV_CIRCULAR: l + m = k modulo N, the N-point FFT convolution the fast method
 *                     computes (eq. realQ).
 *   BZ_CONV_PADDED:   l + m = k without wrap-around, the literal Galerkin sum of eq. sum: the
 *                     plan runs the circular pipeline on a 2N grid (N = 8, 16 fused; 24, 32
 *                     chunked), the input embedded with the modes outside -N/2..N/2-1 zero,
 *                     alpha zero outside that range, and returns the N-range.  FP32 form;
 *                     bz_collide, bz_collide_terms, bz_moments and bz_ftable_entries take and
 *                     return N^3 arrays as for a circular plan; bz_step_rk, bz_plan_alpha,
 *                     bz_collide_noalloc and batches return BZ_ERR_UNSUPPORTED. */
enum { BZ_CONV_CIRCULAR = 0, BZ_CONV_PADDED = 1 };

/* Collide pipelines.  FUSED: one thread-block cluster per term keeps the whole field in
 * (distributed) shared memory from twiddle to weighted accumulation (N <= 32).  CHUNKED:
 * four kernels per chunk of terms over an L2-sized scratch buffer (every N).  AUTO picks
 * FUSED where it applies. */
enum { BZ_PIPE_AUTO = 0, BZ_PIPE_FUSED = 1, BZ_PIPE_CHUNKED = 2 };

/* Precision of h = IFFT(fhat) on the fused pipeline.  FP32 transforms leave a noise floor of
 * about eps max|h| over the grid, which the product h g_p turns into error where g_p is large
 * and h small; forming h in FP64 (from the caller's FP64 coefficients) removes that half of
 * the rounding error, at the cost of three short FP64 passes per collide.  FP32 forms h
 * inside the fused kernel.  AUTO = FP64. */
enum { BZ_H_AUTO = 0, BZ_H_FP64 = 1, BZ_H_FP32 = 2 };

/* Data of the operator (Sec. 2: f is a real distribution function, so fhat is Hermitian).
 *   BZ_DATA_COMPLEX: fhat is any complex array; the operator of eq. realQ as it stands.
 *   BZ_DATA_REAL:    f is real.  The plan takes the Hermitian part of fhat,
 *                    (fhat_k + conj fhat_{-k}) / 2, with every mode that has an index -N/2 (the
 *                    Nyquist planes) set to zero, and returns the operator of that band-limited
 *                    real f (every output mode).  For such f every g_p = IFFT(beta_p fhat) and h
 *                    are real, so two terms share one pair of 3D transforms: x = (beta_p +
 *                    i beta_p') fhat gives g_p + i g_p', and
 *                    with A = (alpha_p - i alpha_p') / 2 the pair adds W + conj(W(-k)),
 *                    W = A FFT(h (g_p + i g_p')); the sum of the W over pairs is symmetrised once
 *                    per collide.  On the Nyquist planes, where alpha_p(-k) != conj alpha_p(k), a
 *                    second sum with a 3 N^2 table per pair completes every mode, so for a real f
 *                    without Nyquist content the result is eq. realQ itself.  Half the transforms,
 *                    exchanges and (nearly) table bytes per term.  3D, FP32, circular, M even;
 *                    the fused pipeline for N = 8, 16, 32, the chunked one for N = 24, 48, 64
 *                    (BZ_PIPE_FUSED with those: BZ_ERR_UNSUPPORTED); bz_collide_terms takes even term bounds;
 *                    batches need h in FP64 (the default); bz_collide_noalloc returns
 *                    BZ_ERR_UNSUPPORTED. */
enum { BZ_DATA_COMPLEX = 0, BZ_DATA_REAL = 1 };

typedef struct bz_plan bz_plan;

typedef struct {
    int N;            /* modes per axis: 8, 16, 24, 32, 48 or 64                      */
    double L;         /* half-width of the periodic box [-L, L]^3 (Sec. 2)             */
    double R;         /* radius of the |q| ball, radial rule on [0, R] (Sec. 2, 4)     */
    double gamma;     /* Phi(|q|) = |q|^gamma (Sec. 1, eq. Bb)                        */
    double s;         /* BZ_KERNEL_FAMILY order, nu = 2 s                              */
    int N_rho;        /* Gauss-Legendre points in |q| (Sec. 4)                         */
    int M;            /* sphere points: 12 = icosahedron; 2n^2 or n^2 = product rule    */
    int kernel;       /* BZ_KERNEL_*                                                   */
    int precision;    /* BZ_PREC_*                                                     */
    double eps;       /* Taylor/quadrature split angle; <= 0 selects pi/1000 (Sec. 4.1) */
    const double *sphere_xyz;  /* optional host array [M][3] of unit vectors, or NULL  */
    const double *sphere_w;    /* optional host array [M] of weights (sum 4 pi)         */
    int chunk_terms;  /* terms per pipeline chunk; <= 0 selects automatically          */
    int pipeline;     /* BZ_PIPE_*; BZ_ERR_UNSUPPORTED if FUSED cannot run for this N     */
    int cluster;      /* FUSED: CTAs per cluster (N=16: 1|2, 24: 2|3, 32: 4|8); <= 0 times the
                         compiled sizes at creation and keeps the fastest                   */
    int h_precision;  /* BZ_H_*                                                            */
    int conv;         /* BZ_CONV_*                                                         */
    int dim;          /* 3 (or 0): the 3D operator; 2: the 2D operator of Sec. 4.1 (i) and Sec. 5.2 on
                         an N x N grid (N = 8, 16, 32 or 64; arrays [k1][k2]; kernels BZ_KERNEL_B1..B4;
                         M midpoint points phi_j = 2 pi (j + 1/2) / M on the circle, c_p = w_i w_j
                         r_i^gamma r_i; FP32, circular).  A 2D plan runs bz_collide, bz_collide_terms,
                         bz_step_rk, bz_ftable_entries (k_idx's third index ignored) and the
                         inspection calls; the others return BZ_ERR_UNSUPPORTED.                */
    double theta0;    /* angular cutoff: b = 0 for theta < theta0 (and theta > 2 pi - theta0 in 2D), as
                         eqs. ApproximatedDebyecutoff and b3cutoff; 0 = none, else eps <= theta0 < pi.
                         With a cutoff there is no Taylor part; the theta rule starts at theta0. */
    int data;         /* BZ_DATA_*                                                         */
    int ctas_per_sm;  /* fused pipeline, BZ_DATA_REAL at N = 32: 2 runs k_fused, 3 the three-CTA-
                         per-SM pair kernel k_pair3 (sum over pairs and fhat column in tensor
                         memory; with BZ_H_FP32 its h comes from one FP32 plane pass and one
                         pencil pass); <= 0 times both at creation and keeps the faster.  Any
                         other plan: must be <= 0 or 2, else BZ_ERR_UNSUPPORTED.              */
} bz_plan_desc;

/* Creates a plan: quadrature terms, the FP64 F table (computed on the device, stored
 * FP32 as alpha_p = c_p F / N^3), twiddle vectors and workspace, on the current CUDA
 * device.  Synchronous.  Sec. 4, eq. approxG; Sec. 4.1.
 * Errors: BZ_ERR_ARG for unsupported N, N_rho < 1, s outside [0, 1), a sphere rule
 * that does not exist for M; BZ_ERR_OOM; BZ_ERR_CUDA.  *out is NULL on error. */
bz_status bz_plan_create(bz_plan **out, int N, double L, double R, double gamma,
                         double s, int N_rho, int M);
bz_status bz_plan_create_ex(bz_plan **out, const bz_plan_desc *desc);
void bz_plan_destroy(bz_plan *plan);

/* Number of quadrature terms P = N_rho * M; bytes of the alpha table (with the pair table of a
 * BZ_DATA_REAL plan). */
bz_status bz_plan_info(const bz_plan *plan, int *P, size_t *alpha_bytes, size_t *workspace_bytes);

/* The collide pipeline the plan runs: *pipeline = BZ_PIPE_FUSED or BZ_PIPE_CHUNKED;
 * for FUSED, *cluster = CTAs per cluster, *clusters = resident clusters (persistent grid),
 * *tuned_ms = the timed collide that selected the cluster size.  Any pointer may be NULL. */
bz_status bz_plan_pipeline(const bz_plan *plan, int *pipeline, int *cluster, int *clusters, float *tuned_ms);

/* Name of the kernel that carries the plan's per-term work: "k_fused", "k_pair3" (the
 * three-CTA-per-SM pair kernel of a BZ_DATA_REAL plan at N = 32), "k_mixed", "k_collide_2d"
 * or "chunked"; NULL for a NULL plan.  The string is static. */
const char *bz_plan_kernel(const bz_plan *plan);

/* Copies the term list to host arrays of length P (any may be NULL):
 * r[p], w_r[p], qhat[3p..3p+2], w_q[p], c[p] = w_r w_q r^(gamma+2).  Synchronous. */
bz_status bz_plan_terms(const bz_plan *plan, double *r, double *w_r, double *qhat,
                        double *w_q, double *c);

/* Host only (no GPU needed).  The quadrature terms a plan with these parameters uses, in
 * term order p = i*M + j: radial Gauss-Legendre nodes and weights on [0, R], the sphere rule
 * (M = 12: icosahedron; M = 2n^2 or n^2: product rule), c_p = w_r w_q r^(gamma + 2)
 * (Sec. 4, eq. approxG).  Arrays of length N_rho * M (qhat: 3x), any may be NULL. */
bz_status bz_quadrature(int N_rho, double R, int M, double gamma, double *r, double *w_r, double *qhat,
                        double *w_q, double *c);

/* Host only (no GPU needed).  The terms one rank of a term-sharded collide evaluates.  The sum
 * over p in eq. realQ (Sec. 4) is a sum of independent terms, so `world` ranks can each
 * evaluate a contiguous range [*p0, *p1) with bz_collide_terms and add their N^3 results with
 * one all-reduce (sum); the ranges of ranks 0 .. world-1 are near-equal, in rank order, and
 * cover [0, P) exactly once.  data = BZ_DATA_REAL splits the P/2 term pairs so that both
 * terms of a pair (2q, 2q+1) stay on one rank (the bounds are even, as bz_collide_terms needs
 * for a real-data plan); a rank may get an empty range (*p0 == *p1) when world > P (or P/2).
 * Errors: BZ_ERR_ARG for NULL outputs, P < 0, world < 1, rank outside [0, world), an unknown
 * data form or an odd P with BZ_DATA_REAL. */
bz_status bz_partition_terms(int P, int data, int world, int rank, int *p0, int *p1);

/* Host only.  The angular kernel's normalisation c (g = sin(theta) b(cos theta), lambda = 1/6)
 * and the part-I moments A = (int g (1-cos), int g (1-cos)^2, int g sin^2) over [0, eps]
 * (Sec. 4.1; eps <= 0 selects pi/1000). */
bz_status bz_kernel_constants(int kernel, double s, double eps, double *c, double A[3]);

/* Qhat = Q(fhat, fhat) over all terms (eq. realQ).  fhat and Qhat are device arrays
 * of N^3 complex values of the given dtype; fhat != Qhat (BZ_ERR_ARG otherwise).
 * Arithmetic: FP32 FFTs and products, FP64 accumulation over terms. */
bz_status bz_collide(bz_plan *plan, const void *fhat, void *Qhat, int dtype, void *stream);

/* As bz_collide, restricted to terms p0 <= p < p1 (0 <= p0 <= p1 <= P). */
bz_status bz_collide_terms(bz_plan *plan, int p0, int p1, const void *fhat, void *Qhat,
                           int dtype, void *stream);

/* Classical RK4 (Sec. 5.2) for d fhat/dt = Q(fhat, fhat): nsteps steps of size dt,
 * fhat updated in place (device, dtype), *t (host, may be NULL) advanced by nsteps*dt.
 * The step state and the stage combination are FP64 on the device; each stage's
 * collide input is rounded to FP32.  workspace is reserved and may be NULL (the
 * plan's own workspace is used). */
bz_status bz_step_rk(bz_plan *plan, void *fhat, int dtype, double *t, double dt, int nsteps,
                     void *workspace, void *stream);

/* Moments of f_N over [-L, L]^3 in FP64: out[0] = mass = (2L)^3 Re fhat_0 (Sec. 4 remark),
 * out[1..3] = momentum, out[4] = energy int |v|^2 f_N dv (exact integrals of the
 * trigonometric basis).  out is a host array of 5 doubles; synchronous on stream. */
bz_status bz_moments(bz_plan *plan, const void *fhat, int dtype, double out[5], void *stream);

/* F(k, r_i, qhat_j) in FP64 for `count` entries (device arrays): k_idx[3e..3e+2] array
 * indices in [0, N), term[e] in [0, P); out[2e], out[2e+1] = re, im.  Uses the same
 * device code as the plan's table (before the FP32 store).  Synchronous. */
bz_status bz_ftable_entries(bz_plan *plan, int count, const int *k_idx, const int *term,
                            double *out);

/* Copies alpha_p (FP32 complex, c_p F / N^3) for terms p0 <= p < p1 into the device array
 * dst ((p1-p0) * N^3 complex64). */
bz_status bz_plan_alpha(const bz_plan *plan, int p0, int p1, void *dst, void *stream);

const char *bz_status_str(bz_status s);

/* Allocation-free collide.  The paper has no counterpart: this entry point exists for
 * callers that cannot let a library allocate device memory during a call (an application
 * whose device memory is reserved up front by its own pool allocator, a latency-critical
 * time loop that cannot pay the device synchronisation of cudaMalloc/cudaFree, a host
 * that forbids a library to grow its footprint after start-up).
 * It computes the operator bz_collide computes on the same plan: h = IFFT(fhat) is formed
 * the same way (in FP64 on the fused pipeline unless the plan asks for BZ_H_FP32, in FP32 on
 * the chunked one), the terms run through the chunked FP32 kernels and are summed in FP64;
 * results agree within the FP32 pipeline's rounding (the term chunking and summation order
 * differ).  Every scratch buffer lives in one file-scope device array of
 * BZ_NOALLOC_SCRATCH_BYTES that each GPU loading libbz holds until the process exits;
 * nothing is allocated or freed.  The plan must have been created beforehand on the
 * current device.
 *   - Size limit: the array holds the FP32 input copy and h (8 N^3 bytes each), the FP64
 *     accumulator (16 N^3), the FP64 h pass's scratch where h is formed in FP64 (16 N^3) and at
 *     least one term of 8 N^3 (each rounded up to 256-byte blocks).  N <= 48 fits (N = 48: five
 *     terms per chunk); N = 64 does not and returns BZ_ERR_ARG without touching Qhat.
 *   - Each call looks up the array's device address (cudaGetSymbolAddress) with the current
 *     device; the first lookup on a device may load the module there, so make the first
 *     call on each device before any stream capture begins.
 *   - All calls share the one array and it keeps the previous call's contents (the
 *     accumulator is cleared on the stream at the start of every call).  Calls whose work
 *     overlaps on the GPU (other streams, other host threads) race on the array: serialise them.
 * Errors: BZ_ERR_ARG for NULL or aliased arrays, a bad dtype, a plan of another device or a
 * plan too large for the array; BZ_ERR_UNSUPPORTED for padded, 2D, real-data (BZ_DATA_REAL)
 * and split-BF16 (BZ_PREC_BF16X3) plans, which bz_collide serves; BZ_ERR_CUDA if the address
 * lookup or a launch fails. */
#define BZ_NOALLOC_SCRATCH_BYTES (8u << 20)
bz_status bz_collide_noalloc(const bz_plan *plan, const void *fhat, void *Qhat, int dtype,
                             void *stream);

/* Non-finite results.  Every kernel that writes a result to the caller (the Qhat of bz_collide,
 * bz_collide_terms and batches, the fhat of bz_step_rk and batch RK steps) raises a device flag
 * of the plan when a value it writes is NaN or Inf.  This call waits for the device, returns
 * BZ_ERR_NONFINITE (and *nonfinite = 1) if the flag was raised since the last check, clears it,
 * and returns BZ_OK (*nonfinite = 0) otherwise; nonfinite may be NULL.  bz_moments returns
 * BZ_ERR_NONFINITE itself when a moment is NaN or Inf.  No counterpart in the paper. */
bz_status bz_plan_check_finite(bz_plan *plan, int *nonfinite);

/* Checkpoint and resume of an RK4 solve (Sec. 5.2).  The state between bz_step_rk calls is the
 * coefficient array and t.  bz_checkpoint_write waits for `stream`, copies fhat (device, dtype)
 * to the host and writes it as complex128 to `path` (through a temporary file renamed over it),
 * with t, every parameter of the plan's operator and its pipeline choices (pipeline, CTAs per
 * cluster, pair kernel, terms per chunk).  bz_checkpoint_plan_desc fills *desc (sphere_xyz and
 * sphere_w NULL: a plan built on a user sphere rule needs the same arrays again) and *t (may be
 * NULL) from the file, so that bz_plan_create_ex rebuilds a plan that makes the same choices.
 * bz_checkpoint_read checks that the file's operator equals the plan's (BZ_ERR_ARG otherwise),
 * writes the coefficients to fhat (device, dtype) and *t (may be NULL), and waits for `stream`.
 * With BZ_C128 state, steps taken after a resume on such a plan give the same bits as an
 * uninterrupted run (the RK state is FP64 and every sum has a fixed order); BZ_C64 state is
 * rounded to FP32 at every call boundary.  Errors: BZ_ERR_ARG for NULL arguments, a bad dtype,
 * a file that cannot be written or read or is not a checkpoint; BZ_ERR_CUDA.  No counterpart in
 * the paper. */
bz_status bz_checkpoint_write(const bz_plan *plan, const void *fhat, int dtype, double t, const char *path,
                              void *stream);
bz_status bz_checkpoint_plan_desc(const char *path, bz_plan_desc *desc, double *t);
bz_status bz_checkpoint_read(const bz_plan *plan, const char *path, void *fhat, int dtype, double *t, void *stream);

/* ---------------------------------------------------------------------------------------
 * Batches: many independent instances of one plan geometry (same N, L, R, kernel, N_rho, M
 * and F table; gamma per instance), standing in for the cells of a spatially
 * inhomogeneous solver.  Instance state lives in slots 0..capacity-1 of caller arrays of
 * capacity * N^3 complex values (dtype as above); every call names its active slots
 * (host array, distinct, in [0, capacity)), so instances can join and leave between calls.
 * gamma enters only through c_p (eq. approxG): slot b uses alpha_p r_i^(gamma_b - gamma_plan).
 * An instance's result does not depend on which other slots are active in the call.
 * On the fused pipeline (N <= 32) the active slots run as one batched kernel per RK stage; on
 * the chunked pipeline (N = 24 real data, 48, 64, or on request) they step one after another
 * through the plan's pipeline, each with its own gamma (padded and 2D plans, and fused
 * real-data plans with FP32 h, give BZ_ERR_UNSUPPORTED).  The plan must
 * outlive the batch.  Not re-entrant across streams.
 * --------------------------------------------------------------------------------------- */
typedef struct bz_batch bz_batch;

/* terms_per_item <= 0 autotunes the number of terms per work item (timed on the device at
 * creation).  Synchronous. */
bz_status bz_batch_create(bz_batch **out, const bz_plan *plan, int capacity, int terms_per_item);
void bz_batch_destroy(bz_batch *batch);
bz_status bz_batch_info(const bz_batch *batch, int *capacity, int *terms_per_item, size_t *workspace_bytes);
/* gamma of one slot (default: the plan's gamma).  Synchronous. */
bz_status bz_batch_set_gamma(bz_batch *batch, int slot, double gamma);
/* Qhat[slot] = Q(fhat[slot]) for each active slot (eq. realQ).  fhat != Qhat. */
bz_status bz_batch_collide(bz_batch *batch, int count, const int *slots, const void *fhat, void *Qhat,
                           int dtype, void *stream);
/* nsteps classical RK4 steps (Sec. 5.2) of size dt on each active slot of fhat, in place.  Each
 * step replays a CUDA graph captured on the first call with this dt (one fused launch and one
 * stage update per RK stage). */
bz_status bz_batch_step_rk(bz_batch *batch, int count, const int *slots, void *fhat, int dtype, double dt,
                           int nsteps, void *stream);
/* Kernel launches (graph nodes included) of the last batch call. */
int bz_batch_last_launches(const bz_batch *batch);

/* ---------------------------------------------------------------------------------------
 * Spatially inhomogeneous coupling: df/dt + v_1 df/dx = Q(f, f) on a periodic interval
 * [0, Lx) of nx cells, x_c = c Lx / nx, with the homogeneous operator as a black box per cell
 * (the paper's closing remark, Sec. 6; the splitting is this library's reading).  Cell arrays
 * are [nx][N][N][N] coefficients (c64 or c128, device), cell-major.
 * --------------------------------------------------------------------------------------- */

/* Free streaming df/dt + v_1 df/dx = 0 over time t (any sign), in place: exact at the velocity
 * nodes v_j = -L + 2 L j / N and spectral in x (x-DFT over the cells, phase
 * exp(-2 pi i kappa v_1 t / Lx) with the signed x-mode kappa, -nx/2 included, inverse x-DFT),
 * computed in FP64 along the k1 axis only (the phase depends on v_1 alone).  N and nx in
 * {8, 16, 24, 32}; BZ_ERR_UNSUPPORTED otherwise. */
bz_status bz_transport_x(int N, double L, int nx, double Lx, void *fcells, int dtype, double t, void *stream);

/* nsteps Strang steps of size dt: free streaming dt/2, one RK4 step (Sec. 5.2) of the collision
 * in every cell (the batch's slots 0 .. nx - 1, whose plan gives N and L), free streaming dt/2
 * (the half steps between two steps are taken as one).  nx <= the batch's capacity. */
bz_status bz_inhom_step(bz_batch *batch, int nx, double Lx, void *fcells, int dtype, double dt, int nsteps,
                        void *stream);

/* ---------------------------------------------------------------------------------------
 * Serving: a worker thread runs homogeneous relaxation solves (RK4 on d fhat/dt = Q) for
 * submitted requests with continuous batching.  Requests with equal geometry, data form,
 * precision and dt form a group with its own plan, batch (gamma per slot), stream and
 * completion event.  The worker admits queued requests in arrival order while the HBM budget
 * and group slots allow; a group whose step has completed (polled with cudaEventQuery: no group
 * waits for another) advances its requests by one RK4 step, retires the finished ones and
 * launches its next step, which requests admitted meanwhile join.  Groups on the fused pipeline
 * (N <= 32; N | 32 for BZ_DATA_REAL) step whenever idle; of the others (chunked pipeline) one
 * step is in flight at a time, the group with the shortest remaining work first (aged by its
 * wait).  State stays on the device from admission to completion.  A request's result does not
 * depend on the other requests in flight.
 * --------------------------------------------------------------------------------------- */
typedef struct bz_server bz_server;

typedef struct {
    int N; double L, R, gamma, s; int N_rho, M, kernel;   /* operator, as in bz_plan_desc   */
    const void *fhat0; int dtype;   /* host array of N^3 initial coefficients; copied by bz_submit */
    double t0, t_end, dt;           /* round((t_end - t0) / dt) RK4 steps of size dt              */
    double max_queue_s;             /* > 0: fail with BZ_ERR_TIMEOUT if not admitted in time      */
    int data;                       /* BZ_DATA_COMPLEX (0) or BZ_DATA_REAL (M even)               */
    int precision;                  /* BZ_PREC_FP32 (0) or BZ_PREC_BF16X3 (N = 32, complex data)  */
} bz_request;

typedef struct {
    int status;          /* BZ_OK, or the error that ended the request (BZ_ERR_NONFINITE: the
                            result held NaN or Inf; BZ_ERR_TIMEOUT: not admitted within
                            max_queue_s; BZ_ERR_OOM: larger than the whole budget)               */
    int steps;           /* RK4 steps taken                                                   */
    double t;            /* t0 + steps * dt                                                   */
    double latency_s;    /* submit to completion                                              */
    double queue_s;      /* submit to admission                                               */
} bz_result;

/* hbm_budget_bytes bounds the device memory of plans, batches and request state; max_batch
 * is the slot capacity of each batched group; terms_per_item <= 0 autotunes per group. */
bz_status bz_server_create(bz_server **out, size_t hbm_budget_bytes, int max_batch, int terms_per_item);
/* Queues a request (never blocks on the device).  *ticket identifies it for bz_poll.
 * Errors: BZ_ERR_ARG for an invalid request; BZ_ERR_UNSUPPORTED for BZ_DATA_REAL with M odd or
 * BZ_PREC_BF16X3 other than at N = 32 with complex data. */
bz_status bz_submit(bz_server *server, const bz_request *req, uint64_t *ticket);
/* Non-blocking.  BZ_ERR_BUSY while queued or running; otherwise fills *out, copies the
 * final coefficients to fhat_out (host, dtype; may be NULL) when out->status == BZ_OK,
 * forgets the ticket and returns BZ_OK.  BZ_ERR_ARG for an unknown ticket. */
bz_status bz_poll(bz_server *server, uint64_t ticket, bz_result *out, void *fhat_out, int dtype);
/* completed: requests retired; steps: RK4 steps completed, summed over requests; hbm_used:
 * bytes charged to the budget; queued / active: requests waiting / admitted.  Any may be NULL. */
bz_status bz_server_stats(bz_server *server, long *completed, long *steps, size_t *hbm_used, int *queued,
                          int *active);
/* Stops the worker after its current iteration and frees everything. */
void bz_server_destroy(bz_server *server);

/* Kernel kinds reported by bz_plan_timing. */
enum { BZ_K_PLANE_INV = 0, BZ_K_PENCIL = 1, BZ_K_PLANE_FWD = 2, BZ_K_REDUCE = 3, BZ_K_OTHER = 4,
       BZ_K_FUSED = 5 };

/* Per-kernel timing.  With max_launches > 0, the next max_launches pipeline launches of
 * this plan are each bracketed by a pair of CUDA events recorded on the launch stream
 * (events are created here, not during the launches); 0 turns timing off.  Resets the
 * totals.  Launches beyond max_launches are not timed. */
bz_status bz_plan_set_timing(bz_plan *plan, int max_launches);

/* Totals since bz_plan_set_timing for one kernel kind: number of timed launches and
 * their summed device time in milliseconds.  Waits for the recorded events. */
bz_status bz_plan_timing(bz_plan *plan, int kind, long *launches, double *ms);

/* Number of kernel launches issued by the last bz_collide / bz_collide_terms /
 * bz_step_rk call on this plan. */
int bz_plan_last_launches(const bz_plan *plan);

/* Device-side waits of the plan's kernels are bounded (BZ_PREC_BF16X3: the waits for
 * tensor-core completion).  *count = 1 if one gave up since the plan was created (the
 * results of that launch are invalid), else 0.  Waits for the device.  No counterpart in
 * the paper. */
bz_status bz_plan_device_errors(bz_plan *plan, int *count);

/* Exercises that path without a fault: one kernel on `stream` waits, through the same bounded
 * wait as the tensor-core kernels, on a shared-memory barrier that nothing completes, for at
 * most `cycles` SM clocks (1 .. 2^31); it then gives up, raises the plan's wait flag (which
 * bz_plan_device_errors reports from then on) and returns, with nothing left in flight.
 * Errors: BZ_ERR_ARG for a NULL plan or cycles outside the range; BZ_ERR_CUDA.  No counterpart
 * in the paper. */
bz_status bz_plan_wait_selftest(bz_plan *plan, long long cycles, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BZ_H */

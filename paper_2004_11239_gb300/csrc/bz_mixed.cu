// Split-BF16 tensor-core form of the fused per-term pipeline of eq. realQ (Sec. 4), N = 32.
//
// Each one-axis transform of a term is a DFT applied to 128 lines at once, written as one
// real GEMM on the 5th-generation tensor cores (tcgen05.mma, kind::f16, FP32 accumulators
// in tensor memory):
//     D[line][n] = sum_k A[line][k] B[n][k],   A = [Re x | Im x] (K = 64),
//     B[2 j] = [C_j, -S_j], B[2 j + 1] = [S_j, C_j], C_jk = cos(2 pi j k / N), S_jk = sin(..),
// so D[line] = (Re y_0, Im y_0, Re y_1, ...) with y_j = sum_k x_k exp(+2 pi i j k / N).  Every
// operand is split x = x_hi + x_lo into two BF16 numbers and the product is taken as
// A_hi B_hi + A_lo B_hi + A_hi B_lo (12 MMAs of 128 x 64 x 16); the dropped A_lo B_lo and
// the residue of the split are about 2^-17 of |x| |B|.  The forward transforms use the same
// B through FFT(u) = conj(IFFT(conj u)): the pipeline conjugates the product h g_p before
// the first forward pass and the result after the last.
//
// Work split as in the FP32 fused kernel: a cluster of 8 CTAs per term, CTA r owns planes
// k1 in [4r, 4r + 4) for the two plane-local axes and pencils j2 in [4r, 4r + 4) for the
// k1 axis; the two exchanges between the layouts are pushes (remote FP32 stores through
// distributed shared memory) into a pencil buffer X and a plane buffer Y, each followed by
// one cluster barrier.  Per term and CTA (128 threads, thread (w, l) = warp w, lane l):
//   1  A <- twiddle * fhat    rows (k1, k2), K = k3   MN-major   (fhat column from TMEM)
//   2  A <- D1                rows (k1, j3), K = k2   MN-major
//   -- push D2 into the pencil buffers X of the cluster, cluster barrier --
//   3  A <- pencil            rows (j2, j3), K = k1   K-major
//   4  A <- conj(D3 h)        rows (j2, j3), K = j1   K-major    (h column from TMEM)
//   -- push D4 into the plane buffers Y of the cluster, cluster barrier --
//   5  A <- plane rows        rows (k1, j2), K = j3   K-major
//   6  A <- D5                rows (k1, k3), K = j2   MN-major
//   acc += alpha_p * conj(D6)  (accumulator in TMEM)
// The MN-major passes take the previous result without a transpose: a thread holds one
// input index and 32 consecutive line indices, which is the 16-byte core-matrix row of an
// MN-major operand.  Tensor memory per CTA: D (64 columns), the accumulator (64), the
// thread's fhat column (64) and its h column (64); two CTAs per SM use all 512 columns.
#include "bz_cluster.cuh"
#include "bz_fft.cuh"
#include "bz_internal.h"

#include <cmath>
#include <cstring>

namespace bz {

namespace {

constexpr int XN = 32;                   // modes per axis
constexpr int XC = 8;                    // CTAs per cluster
constexpr int XP = XN / XC;              // planes (pencil rows) per CTA
constexpr int XT = XP * XN;              // threads = GEMM rows
constexpr uint32_t A_BYTES = 32768;      // A: 16 K-groups x 16 row-groups x 128 B
constexpr uint32_t A_KG = 2048;          // bytes between K-groups of A (LBO)
constexpr uint32_t A_LO = 8 * A_KG;      // the lo half of the split (K-groups 8..15)
constexpr uint32_t B_HALF = 8192;        // one split half of B: 8 K-groups x 8 row-groups x 128 B
constexpr uint32_t B_KG = 1024;          // bytes between K-groups of B (LBO)
constexpr uint32_t B_BYTES = 2 * B_HALF;
constexpr uint32_t X_BYTES = XP * XN * XN * 8;    // pencils [j2 - 4 rank][k1][j3], FP32
constexpr uint32_t Y_BYTES = XP * XN * XN * 8;    // planes [k1 - 4 rank][j2][j3 ^ (j2 & 15)], FP32
constexpr uint32_t X_SMEM = A_BYTES + B_BYTES + X_BYTES + Y_BYTES;
constexpr uint32_t TM_COLS = 256;        // D, acc, fhat column, h column
constexpr uint32_t TM_D = 0, TM_ACC = 64, TM_F = 128, TM_H = 192;
// at most two CTAs per SM may be resident, so that 2 x 256 tensor-memory columns always fit
static_assert(3 * (X_SMEM + 1024) > 228 * 1024, "a third CTA per SM would oversubscribe TMEM");
static_assert(2 * (X_SMEM + 1024 + 64) <= 228 * 1024, "two CTAs per SM");
static_assert(XT == 128, "one GEMM row per thread, M = 128");

// Instruction descriptor of tcgen05.mma kind::f16: FP32 D, BF16 A and B, M = 128, N = 64;
// A K-major (0) or MN-major (1), B K-major.
__host__ __device__ constexpr uint32_t idesc(int a_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((64u >> 3) << 17) |
           ((128u >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: LBO = bytes between core matrices along K,
// SBO = bytes between core matrices along M (or N); both 16-byte units.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t id, int accum) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem_d), "l"(ad), "l"(bd), "r"(id), "r"(accum) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                 ::"r"(mbar) : "memory");
}
__device__ __forceinline__ uint32_t mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    return ok;
}
// Wait for the phase of the given parity, for at most `limit` SM clocks (by default about one
// second); on time-out the device flag is raised, `dead` is set so that later waits return at
// once, and the pipeline carries on (every CTA still reaches every barrier; the results are
// invalid).
constexpr long long kWaitLimit = 1LL << 31;
__device__ __forceinline__ void mbar_wait(uint32_t mbar, uint32_t parity, int *err, bool &dead,
                                          long long limit = kWaitLimit) {
    if (dead) return;
    const long long t0 = clock64();
    while (!mbar_try(mbar, parity))
        if (clock64() - t0 > limit) {
            dead = true;
            if (err) atomicOr(err, 1);
            return;
        }
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// 16 consecutive 32-bit columns of the thread's own TMEM lane.
__device__ __forceinline__ void tm_ld16(uint32_t ta, float *v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(ta) : "memory");
    #pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tm_st16(uint32_t ta, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
                 ::"r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                   "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                   "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                   "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                   "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                   "r"(__float_as_uint(v[15])) : "memory");
}
// 64 columns = 32 complex values, stored (re, im) interleaved: v[2 i], v[2 i + 1].
__device__ __forceinline__ void tm_ld64(uint32_t ta, float *v) {
    #pragma unroll
    for (int c = 0; c < 4; ++c) tm_ld16(ta + 16 * c, v + 16 * c);
}
__device__ __forceinline__ void tm_st64(uint32_t ta, const float *v) {
    #pragma unroll
    for (int c = 0; c < 4; ++c) tm_st16(ta + 16 * c, v + 16 * c);
}

// Round-to-nearest BF16 pair (a in the low half) and the split of two floats.
__device__ __forceinline__ uint32_t bf2(float a, float b) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(r) : "f"(b), "f"(a));
    return r;
}
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    hi = bf2(a, b);
    lo = bf2(a - __uint_as_float(hi << 16), b - __uint_as_float(hi & 0xFFFF0000u));
}
// Eight values of one component -> their hi and lo 16-byte core-matrix rows.
__device__ __forceinline__ void split8_store(uint32_t s_hi, const float *v, int stride) {
    uint32_t h0, h1, h2, h3, l0, l1, l2, l3;
    split2(v[0], v[stride], h0, l0);
    split2(v[2 * stride], v[3 * stride], h1, l1);
    split2(v[4 * stride], v[5 * stride], h2, l2);
    split2(v[6 * stride], v[7 * stride], h3, l3);
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(s_hi), "r"(h0), "r"(h1), "r"(h2), "r"(h3) : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(s_hi + A_LO), "r"(l0), "r"(l1), "r"(l2), "r"(l3) : "memory");
}

// Operand A writers.  MN-major: the thread holds K index kk = comp * 32 + l and the values
// of rows 32 w + i (i = 0..31); rows 8 g .. 8 g + 7 form one 16-byte core-matrix row.
__device__ __forceinline__ void store_mn(uint32_t sA, const float *v, int w, int l) {
    #pragma unroll
    for (int g = 0; g < 4; ++g)
        #pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int kk = c * 32 + l;
            split8_store(sA + (uint32_t)(kk >> 3) * A_KG + (uint32_t)(4 * w + g) * 128 + (uint32_t)(kk & 7) * 16,
                         v + 16 * g + c, 2);
        }
}
// K-major: the thread holds row m and K indices comp * 32 + k (k = 0..31); k = 8 g .. 8 g + 7
// form one 16-byte core-matrix row.
__device__ __forceinline__ void store_k(uint32_t sA, const float *v, int m) {
    #pragma unroll
    for (int g = 0; g < 4; ++g)
        #pragma unroll
        for (int c = 0; c < 2; ++c)
            split8_store(sA + (uint32_t)(c * 4 + g) * A_KG + (uint32_t)m * 16, v + 16 * g + c, 2);
}

// Work items as in k_fused: item it = (instance it / nblk, term block it % nblk); the item's
// FP32 sum over its terms goes to part[slot * nblk + blk].
template <bool SCALED>
__global__ void __launch_bounds__(XT, 2) k_mixed(const ItemArgs a, const uint4 *__restrict__ wimg, int *err) {
    extern __shared__ __align__(128) uint8_t xsm[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
    const int rank = (int)cooperative_groups::this_cluster().block_rank();
    const int cid = blockIdx.x / XC, ncl = gridDim.x / XC;
    const uint32_t sA = (uint32_t)__cvta_generic_to_shared(xsm);
    const uint32_t sB = sA + A_BYTES;
    float2 *xpen = (float2 *)(xsm + A_BYTES + B_BYTES);                // X [XP][XN][XN]
    float2 *ypl = (float2 *)(xsm + A_BYTES + B_BYTES + X_BYTES);      // Y [XP][XN][XN]
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);

    for (int i = tid; i < (int)(B_BYTES / 16); i += XT) ((uint4 *)(xsm + A_BYTES))[i] = wimg[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"((uint32_t)__cvta_generic_to_shared(&s_tmem)), "n"(TM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    proxy_fence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t tl = tmem + ((uint32_t)(32 * w) << 16);      // this thread's lane, column 0
    uint32_t phase = 0;

    constexpr uint32_t SLAB = (uint32_t)(XN * XN * sizeof(float2));    // one [XN][XN] slab of X or Y
    // X element (j2 - 4 rr, k1 = 4 rank + w, j3 = l) and Y element (k1 - 4 rr, j2 = 4 rank + w,
    // j3 = l) in CTA rr, slab 0; slab (j2 % 4) resp. (k1 % 4) is SLAB bytes further
    const int jx = rank * XP + w;
    uint32_t xr[XC], yr[XC];
    #pragma unroll
    for (int r = 0; r < XC; ++r) {
        xr[r] = dsmem_addr(xpen + (size_t)jx * XN + l, (uint32_t)r);
        yr[r] = dsmem_addr(ypl + (size_t)jx * XN + (l ^ (jx & 15)), (uint32_t)r);
    }

    // One transform: 12 MMAs (A_hi B_hi, A_lo B_hi, A_hi B_lo over four K-slabs of 16)
    // into D, issued by one thread once every thread's operand writes are visible.
    auto run_pass = [&](int a_mn) {
        proxy_fence();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t id = a_mn ? idesc(1) : idesc(0);
            #pragma unroll
            for (int s = 0; s < 12; ++s) {
                const uint32_t q = (uint32_t)(s & 3);
                const uint32_t ao = (s >= 4 && s < 8 ? A_LO : 0u) + 2u * q * A_KG;
                const uint32_t bo = (s >= 8 ? B_HALF : 0u) + 2u * q * B_KG;
                mma_bf16(tmem + TM_D, sdesc(sA + ao, A_KG, 128), sdesc(sB + bo, B_KG, 128), id, s > 0);
            }
            mma_commit(mb);
        }
    };
    bool dead = false;
    auto wait_pass = [&]() {
        mbar_wait(mb, phase, err, dead);
        phase ^= 1u;
        tc_fence_after();
    };

    constexpr size_t N3 = (size_t)XN * XN * XN;
    const int count = a.count_dev ? *a.count_dev : a.count;
    const int nitems = count * a.nblk;
    cluster_barrier<XC>();                                       // every CTA of the cluster has started
    const int k1 = rank * XP + w;                                // plane of the plane-local passes
    const int j2 = rank * XP + w;                                // pencil row of the k1 passes

    for (int it = cid; it < nitems; it += ncl) {
        const int b = it / a.nblk, blk = it % a.nblk;
        const int slot = a.slots ? a.slots[b] : b;
        const int t0 = a.p0 + blk * a.TB;
        const int t1 = min(a.p1, t0 + a.TB);
        const float2 *fin = a.fin + (size_t)slot * N3;
        const float2 *hg = a.hg + (size_t)slot * N3;
        {
            // the thread's fhat column (k1, k2 = i, k3 = l), its h column (j1 = i, j2, j3 = l)
            // and a zero accumulator, in its tensor-memory lane
            float v[64];
            #pragma unroll
            for (int i = 0; i < XN; ++i) {
                const float2 f = fin[((size_t)k1 * XN + i) * XN + l];
                v[2 * i] = f.x; v[2 * i + 1] = f.y;
            }
            tm_st64(tl + TM_F, v);
            #pragma unroll
            for (int i = 0; i < XN; ++i) {
                const float2 h = hg[((size_t)i * XN + j2) * XN + l];
                v[2 * i] = h.x; v[2 * i + 1] = h.y;
            }
            tm_st64(tl + TM_H, v);
            #pragma unroll
            for (int i = 0; i < 64; ++i) v[i] = 0.f;
            tm_st64(tl + TM_ACC, v);
            tm_wait_st();
        }
        int ti = 0;
        for (int p = t0; p < t1; ++p, ++ti) {
            const float2 *alpha_p = a.alpha + ((size_t)p * XN + (size_t)rank * XP) * XN * XN;
            if (tid == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(alpha_p),
                             "r"((uint32_t)(XP * XN * XN * sizeof(float2))) : "memory");
            float sc = 1.f;
            if constexpr (SCALED) sc = a.gsc[(size_t)slot * a.N_rho + p / a.M];
            const float2 *tws = a.tw + (size_t)p * 3 * XN;            // L1-resident twiddles
            float v[64];

            // 1: beta_p fhat, rows (k1, k2), K = k3 = l
            tm_ld64(tl + TM_F, v);
            tm_wait_ld();
            {
                const float2 t13 = cmul(__ldg(tws + k1), __ldg(tws + 2 * XN + l));
                #pragma unroll
                for (int i = 0; i < XN; ++i) {
                    const float2 x = cmul(make_float2(v[2 * i], v[2 * i + 1]), cmul(t13, __ldg(tws + XN + i)));
                    v[2 * i] = x.x; v[2 * i + 1] = x.y;
                }
            }
            store_mn(sA, v, w, l);
            run_pass(1);
            wait_pass();
            // 2: D1 = row (k1, k2 = l) over j3 -> rows (k1, j3), K = k2 = l
            tm_ld64(tl + TM_D, v);
            tm_wait_ld();
            store_mn(sA, v, w, l);
            run_pass(1);
            wait_pass();
            // D2 = row (k1, j3 = l) over j2 -> X of the CTA that owns pencil row j2
            tm_ld64(tl + TM_D, v);
            tm_wait_ld();
            #pragma unroll
            for (int j = 0; j < XN; ++j)
                st_dsmem(xr[j / XP] + (uint32_t)(j % XP) * SLAB, make_float2(v[2 * j], v[2 * j + 1]));
            tc_fence_before();
            cluster_barrier<XC>();
            // 3: pencil (j2, j3 = l) over k1 from X, rows (j2, j3) = tid, K = k1
            #pragma unroll
            for (int k = 0; k < XN; ++k) {
                const float2 x = xpen[(size_t)(w * XN + k) * XN + l];
                v[2 * k] = x.x; v[2 * k + 1] = x.y;
            }
            store_k(sA, v, tid);
            run_pass(0);
            wait_pass();
            // 4: conj(h g_p) over j1, rows (j2, j3), K = j1
            {
                float hv[64];
                tm_ld64(tl + TM_D, v);
                tm_ld64(tl + TM_H, hv);
                tm_wait_ld();
                #pragma unroll
                for (int j = 0; j < XN; ++j) {
                    const float2 u = cmul(make_float2(v[2 * j], v[2 * j + 1]), make_float2(hv[2 * j], hv[2 * j + 1]));
                    v[2 * j] = u.x; v[2 * j + 1] = -u.y;
                }
            }
            store_k(sA, v, tid);
            run_pass(0);
            wait_pass();
            // D4 = pencil over k1 -> Y of the CTA that owns plane k1
            tm_ld64(tl + TM_D, v);
            tm_wait_ld();
            #pragma unroll
            for (int k = 0; k < XN; ++k)
                st_dsmem(yr[k / XP] + (uint32_t)(k % XP) * SLAB, make_float2(v[2 * k], v[2 * k + 1]));
            // this term's alpha_p(k1, k2 = i, k3 = l), loaded while the cluster catches up
            float2 al[XN];
            #pragma unroll
            for (int i = 0; i < XN; ++i) al[i] = alpha_p[(size_t)(w * XN + i) * XN + l];
            tc_fence_before();
            cluster_barrier<XC>();
            // 5: plane row (k1, j2 = l) over j3 from Y, rows (k1, j2) = tid, K = j3
            #pragma unroll
            for (int j = 0; j < XN; ++j) {
                const float2 x = ypl[(size_t)(w * XN + l) * XN + (j ^ (l & 15))];
                v[2 * j] = x.x; v[2 * j + 1] = x.y;
            }
            store_k(sA, v, tid);
            run_pass(0);
            wait_pass();
            // 6: D5 = row (k1, j2 = l) over k3 -> rows (k1, k3), K = j2 = l
            tm_ld64(tl + TM_D, v);
            tm_wait_ld();
            store_mn(sA, v, w, l);
            run_pass(1);
            wait_pass();
            // acc += alpha_p conj(D6): row (k1, k3 = l) over k2
            #pragma unroll
            for (int c = 0; c < 4; ++c) {
                float d[16], s[16];
                tm_ld16(tl + TM_D + 16 * c, d);
                tm_ld16(tl + TM_ACC + 16 * c, s);
                tm_wait_ld();
                #pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 A = al[8 * c + u];
                    const float xr = d[2 * u], xi = -d[2 * u + 1];
                    if constexpr (SCALED) {
                        s[2 * u] = fmaf(sc, xr * A.x - xi * A.y, s[2 * u]);
                        s[2 * u + 1] = fmaf(sc, xr * A.y + xi * A.x, s[2 * u + 1]);
                    } else {
                        s[2 * u] = fmaf(xr, A.x, fmaf(-xi, A.y, s[2 * u]));
                        s[2 * u + 1] = fmaf(xr, A.y, fmaf(xi, A.x, s[2 * u + 1]));
                    }
                }
                tm_st16(tl + TM_ACC + 16 * c, s);
            }
            tm_wait_st();
        }
        {
            float s[64];
            tm_ld64(tl + TM_ACC, s);
            tm_wait_ld();
            float2 *out = a.part + ((size_t)slot * a.nblk + blk) * N3 + (size_t)k1 * XN * XN;
            #pragma unroll
            for (int i = 0; i < XN; ++i) out[i * XN + l] = make_float2(s[2 * i], s[2 * i + 1]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(TM_COLS) : "memory");
}

}  // namespace

// ---- host side ----

static uint16_t bf16_rn(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static double bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

// B (row n = output column, K-major, no swizzle): row 2 j gives Re y_j = [C_j, -S_j], row
// 2 j + 1 gives Im y_j = [S_j, C_j], so that D holds (Re, Im) interleaved per output; hi half
// then lo half, split from the FP64 values.
static void build_w_image(std::vector<uint16_t> &img) {
    img.assign(B_BYTES / 2, 0);
    for (int n = 0; n < 2 * XN; ++n)
        for (int k = 0; k < 2 * XN; ++k) {
            const int j = n / 2, kk = k % XN;
            const double ang = 2.0 * M_PI * (double)((j * kk) % XN) / XN;
            const double c = std::cos(ang), s = std::sin(ang);
            const double val = (n & 1) == 0 ? (k < XN ? c : -s) : (k < XN ? s : c);
            const uint16_t hi = bf16_rn((float)val);
            const uint16_t lo = bf16_rn((float)(val - bf16_value(hi)));
            const size_t off = (size_t)(k >> 3) * B_KG + (size_t)(n >> 3) * 128 + (size_t)(n & 7) * 16 + (size_t)(k & 7) * 2;
            img[off / 2] = hi;
            img[(B_HALF + off) / 2] = lo;
        }
}

bz_status mixed_upload(uint4 **wimg) {
    std::vector<uint16_t> img;
    build_w_image(img);
    BZ_CUDA_TRY(cudaMalloc(wimg, B_BYTES));
    BZ_CUDA_TRY(cudaMemcpy(*wimg, img.data(), B_BYTES, cudaMemcpyHostToDevice));
    return BZ_OK;
}

static cudaLaunchConfig_t mixed_config(int G, cudaStream_t st, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = XC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(G * XC);
    cfg.blockDim = dim3(XT);
    cfg.dynamicSmemBytes = X_SMEM;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Resident 8-CTA clusters of the split-BF16 kernel (N = 32 only).  The occupancy query counts
// one CTA per SM for a kernel that allocates tensor memory, but two CTAs fit (2 x 256 of the
// 512 columns; shared memory admits no third): the grid takes the cluster count of the FP32
// kernel with the same cluster shape and two CTAs per SM when that is larger.
// One wait that nothing completes, through the bounded wait of the tensor-core kernels: one
// thread initialises an mbarrier that expects one arrival, no thread arrives, and the wait
// gives up after `limit` clocks, raising *err.  Nothing is in flight when it returns.
__global__ void k_wait_selftest(int *err, long long limit) {
    __shared__ __align__(8) unsigned long long mbar;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool dead = false;
        mbar_wait(mb, 0, err, dead, limit);
    }
}

bz_status wait_selftest(const Plan &pl, long long limit, cudaStream_t st) {
    k_wait_selftest<<<1, 32, 0, st>>>(pl.dev_err, limit);
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

cudaError_t mixed_setup(int N, int *G) {
    *G = 0;
    if (N != XN) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)X_SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = mixed_config(64, nullptr, attr);
    e = cudaOccupancyMaxActiveClusters(G, k_mixed<true>, &cfg);
    if (e != cudaSuccess) return e;
    int G2 = 0;
    if (fused_setup(XN, XC, &G2, false) == cudaSuccess && G2 > *G) *G = G2;
    cudaGetLastError();
    return *G > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

bz_status launch_mixed(const Plan &pl, const ItemArgs &a, cudaStream_t st) {
    if (pl.N != XN || !a.hg || !pl.wimg) return BZ_ERR_UNSUPPORTED;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = mixed_config(pl.fused_G, st, attr);
    if (a.gsc) BZ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_mixed<true>, a, (const uint4 *)pl.wimg, pl.dev_err));
    else BZ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_mixed<false>, a, (const uint4 *)pl.wimg, pl.dev_err));
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

}  // namespace bz

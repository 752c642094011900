// Term-pair kernel (BZ_DATA_REAL) at N = 32 with three CTAs per SM.
//
// The same pipeline as k_fused<32, 8, false, true> (phases A, B, C of a term pair with two
// cluster barriers; the Nyquist sums X; see bz_fused_kernel.cuh), with the per-thread state
// that limits k_fused to two CTAs per SM moved out of registers and shared memory:
//   * the sum over pairs (32 complex per thread) and the thread's fhat column (k1, k2 = 0..31,
//     k3 = lane) live in tensor memory (128 columns per CTA: 3 CTAs use 384 of 512), read and
//     written with tcgen05.ld / tcgen05.st on the thread's own lane;
//   * the pair table tile is not staged in shared memory: one thread prefetches the CTA's
//     32 KB of A to L2 when the pair starts and each thread loads its entries in the epilogue.
// At N = 32 with 8-CTA clusters a plane is one warp, so the two in-plane transposes of phases A
// and C need only __syncwarp: each warp stages its own Nyquist table rows (cp.async, waited
// by the warp) and reads the pair's twiddles through L1; the two cluster barriers per pair are
// the only block-wide synchronisation.  Shared memory: planes (33.8 KB), the real h slice
// (16 KB), X on the plane k1 = -N/2 (8 KB) and the pair's Nyquist table rows (10 KB).
#include "bz_cluster.cuh"
#include "bz_fft.cuh"
#include "bz_internal.h"

namespace bz {

namespace {

constexpr int PN = 32, PC = 8, PPP = PN / PC, PT = PN * PPP, PLD = PN + 1;
constexpr size_t P_PLANES = (size_t)PPP * PN * PLD * sizeof(float2);
constexpr size_t P_HS = (size_t)PPP * PN * PN * sizeof(float);
constexpr size_t P_XS1 = (size_t)PN * PN * sizeof(float2);
constexpr size_t P_CS = (size_t)(PN * PN + 2 * PPP * PN) * sizeof(float2);
constexpr size_t P_SMEM = P_PLANES + P_HS + P_XS1 + P_CS;
static_assert(PPP * PN == PT && PN == 32, "one warp per plane");
constexpr uint32_t P_TMEM_COLS = 128;          // acc (64 columns) + fhat column (64)
constexpr uint32_t TM_ACC = 0, TM_FH = 64;
static_assert(3 * (P_SMEM + 1024) <= 228 * 1024, "three CTAs per SM");
static_assert(4 * (P_SMEM + 1024) > 228 * 1024 || 4 * P_TMEM_COLS <= 512, "tensor memory never oversubscribed");

__device__ __forceinline__ void tfence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tfence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void t_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void t_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// 16 consecutive 32-bit columns of the thread's own lane.
__device__ __forceinline__ void t_ld16(uint32_t ta, float *v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(ta) : "memory");
    #pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void t_st16(uint32_t ta, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
                 ::"r"(ta), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                   "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                   "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                   "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                   "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                   "r"(__float_as_uint(v[15])) : "memory");
}

template <bool SCALED>
__global__ void __launch_bounds__(PT, 3) k_pair3(ItemArgs a) {
    constexpr int N = PN, C = PC, PPC = PPP, LD = PLD, TWN = 6 * N;
    extern __shared__ __align__(16) float2 smem[];
    __shared__ uint32_t s_tmem;
    float2 *planes = smem;                                            // [PPC][N][LD]
    float *shr = (float *)((char *)smem + P_PLANES);                  // real h slice [PPC][N][N]
    float2 *xs1 = (float2 *)((char *)shr + P_HS);                     // X on plane k1 = -N/2 [k2][k3]
    float2 *sc1 = xs1 + N * N;                                        // C on plane k1 = -N/2
    float2 *sc2 = sc1 + N * N;                                        // C rows, family k2 = -N/2 [pid][k3]
    float2 *sc3 = sc2 + PPC * N;                                      // C rows, family k3 = -N/2 [pid][k2]
    const int tid = threadIdx.x, w = tid >> 5;
    const int rank = (int)cooperative_groups::this_cluster().block_rank();
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    const int lane = tid % N, pid = tid / N;
    const int k1 = rank * PPC + pid, j2p = rank * PPC + pid;
    float2 *my = planes + (size_t)pid * N * LD;
    constexpr size_t N3 = (size_t)N * N * N;
    uint32_t pen[C];
    #pragma unroll
    for (int r = 0; r < C; ++r) pen[r] = dsmem_addr(planes + (size_t)j2p * LD + lane, (uint32_t)r);
    constexpr uint32_t PLANE_BYTES = (uint32_t)(N * LD * sizeof(float2));

    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"((uint32_t)__cvta_generic_to_shared(&s_tmem)), "n"(P_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tfence_before();
    __syncthreads();
    tfence_after();
    const uint32_t tl = s_tmem + ((uint32_t)(32 * w) << 16);          // this thread's lane, column 0

    const int count = a.count_dev ? *a.count_dev : a.count;
    const int nitems = count * a.nblk;

    for (int it_ = cid; it_ < nitems; it_ += ncl) {
        const int b = it_ / a.nblk, blk = it_ % a.nblk;
        const int slot = a.slots ? a.slots[b] : b;
        const int t0 = a.p0 + blk * a.TB;
        const int t1 = min(a.p1, t0 + a.TB);
        const float2 *fin = a.fin + (size_t)slot * N3;
        __syncthreads();                                              // the previous item is done
        {
            const float2 *hs = a.hg + (size_t)slot * N3;
            #pragma unroll 4
            for (int j = 0; j < N; ++j) shr[((size_t)pid * N + j) * N + lane] = hs[((size_t)j * N + j2p) * N + lane].x;
            // the thread's fhat column and a zero sum, in its tensor-memory lane
            float v[16];
            #pragma unroll
            for (int g = 0; g < 4; ++g) {
                #pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 f = fin[((size_t)k1 * N + 8 * g + u) * N + lane];
                    v[2 * u] = f.x;
                    v[2 * u + 1] = f.y;
                }
                t_st16(tl + TM_FH + 16 * g, v);
            }
            #pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
            #pragma unroll
            for (int g = 0; g < 4; ++g) t_st16(tl + TM_ACC + 16 * g, v);
            t_wait_st();
        }
        float2 x2 = make_float2(0.f, 0.f), x3 = make_float2(0.f, 0.f);
        if (k1 == N / 2) {
            #pragma unroll 8
            for (int i = 0; i < N; ++i) xs1[i * N + lane] = make_float2(0.f, 0.f);
        }
        for (int p = t0; p < t1; ++p) {
            const float2 *ap = a.alpha + ((size_t)p * N + (size_t)rank * PPC) * N * N;   // the CTA's A tile
            // batches: the instance's radial scale r_i^(gamma_b - gamma_plan) of the pair's node
            float sc = 1.f;
            if constexpr (SCALED) sc = a.gsc[(size_t)slot * a.N_rho + (2 * p) / a.M];
            if (tid == 0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(ap),
                             "r"((uint32_t)(PPC * N * N * sizeof(float2))) : "memory");
            {
                // this warp's Nyquist table rows: k2 = -N/2 family (lanes 0-15), k3 = -N/2 family
                // (lanes 16-31), and the whole plane k1 = -N/2 in the warp that holds it
                const float2 *cq = a.cpair + (size_t)p * 3 * N * N;
                const int l16 = lane & 15;
                __syncwarp();                                 // the warp is done with the previous rows
                if (lane < 16) cp_async16((char *)(sc2 + pid * N) + 16 * l16, (const char *)(cq + N * N + k1 * N) + 16 * l16);
                else cp_async16((char *)(sc3 + pid * N) + 16 * l16, (const char *)(cq + 2 * N * N + k1 * N) + 16 * l16);
                if (k1 == N / 2)
                    for (int c = lane; c < N * N * (int)sizeof(float2) / 16; c += 32)
                        cp_async16((char *)sc1 + 16 * c, (const char *)cq + 16 * c);
                cp_async_commit();
            }
            // A: x = (beta_p + i beta_p') fhat over k2, inverse over k2, then rows over k3
            {
                const float2 *tws = a.tw + (size_t)p * TWN;  // the pair's twiddles, through L1
                const float2 ta = cmul(__ldg(tws + k1), __ldg(tws + 2 * N + lane));
                const float2 tb = cmul(__ldg(tws + 3 * N + k1), __ldg(tws + 5 * N + lane));
                float2 x[N];
                #pragma unroll
                for (int g = 0; g < 4; ++g) t_ld16(tl + TM_FH + 16 * g, (float *)(x + 8 * g));
                t_wait_ld();
                #pragma unroll
                for (int i = 0; i < N; ++i) {
                    const float2 u = cmul(ta, __ldg(tws + N + i)), v = cmul(tb, __ldg(tws + 4 * N + i));
                    x[i] = cmul(x[i], make_float2(u.x - v.y, u.y + v.x));
                }
                fft_inplace<N, +1>(x);
                #pragma unroll
                for (int i = 0; i < N; ++i) my[i * LD + lane] = x[i];
                __syncwarp();                                 // the plane is this warp's
                #pragma unroll
                for (int j = 0; j < N; ++j) x[j] = my[lane * LD + j];
                fft_inplace<N, +1>(x);
                #pragma unroll
                for (int j = 0; j < N; ++j) my[lane * LD + j] = x[j];
            }
            cluster_barrier<C>();
            float2 x[N];
            // B: pencil (j2p, lane) over k1 from the cluster, times the real h, back
            #pragma unroll
            for (int k = 0; k < N; ++k) x[k] = ld_dsmem(pen[k / PPC] + (uint32_t)(k % PPC) * PLANE_BYTES);
            fft_inplace<N, +1>(x);
            #pragma unroll
            for (int j = 0; j < N; ++j) {
                const float hv = shr[((size_t)pid * N + j) * N + lane];
                x[j].x *= hv;
                x[j].y *= hv;
            }
            fft_inplace<N, -1>(x);
            #pragma unroll
            for (int k = 0; k < N; ++k) st_dsmem(pen[k / PPC] + (uint32_t)(k % PPC) * PLANE_BYTES, x[k]);
            cluster_barrier<C>();
            // C: rows over j3, columns over j2, then V += A Z and the Nyquist sums
            #pragma unroll
            for (int j = 0; j < N; ++j) x[j] = my[lane * LD + j];
            fft_inplace<N, -1>(x);
            #pragma unroll
            for (int j = 0; j < N; ++j) my[lane * LD + j] = x[j];
            cp_async_wait_all();                              // this warp's Nyquist rows
            __syncwarp();
            #pragma unroll
            for (int i = 0; i < N; ++i) x[i] = my[i * LD + lane];
            // the pair table entries (L2) are loaded one chunk of eight ahead of their use, the
            // first chunk during the last transform
            const float2 *apl = ap + (size_t)pid * N * N + lane;
            float2 an[8];
            #pragma unroll
            for (int u = 0; u < 8; ++u) an[u] = __ldg(apl + u * N);
            fft_inplace<N, -1>(x);
            #pragma unroll
            for (int g = 0; g < 4; ++g) {
                float2 al[8];
                #pragma unroll
                for (int u = 0; u < 8; ++u) al[u] = an[u];
                if (g < 3) {
                    #pragma unroll
                    for (int u = 0; u < 8; ++u) an[u] = __ldg(apl + (8 * (g + 1) + u) * N);
                }
                float s[16];
                t_ld16(tl + TM_ACC + 16 * g, s);
                t_wait_ld();
                #pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 z = x[8 * g + u];
                    const float2 A = make_float2(sc * al[u].x, sc * al[u].y);
                    s[2 * u] = fmaf(z.x, A.x, fmaf(-z.y, A.y, s[2 * u]));
                    s[2 * u + 1] = fmaf(z.x, A.y, fmaf(z.y, A.x, s[2 * u + 1]));
                }
                t_st16(tl + TM_ACC + 16 * g, s);
            }
            if (k1 == N / 2) {
                #pragma unroll
                for (int i = 0; i < N; ++i) {
                    const float2 c = make_float2(sc * sc1[i * N + lane].x, sc * sc1[i * N + lane].y);
                    float2 v = xs1[i * N + lane];
                    v.x = fmaf(x[i].x, c.x, fmaf(-x[i].y, c.y, v.x));
                    v.y = fmaf(x[i].x, c.y, fmaf(x[i].y, c.x, v.y));
                    xs1[i * N + lane] = v;
                }
            }
            float2 z3 = make_float2(0.f, 0.f);
            #pragma unroll
            for (int i = 0; i < N; ++i) {
                const float zr = __shfl_sync(0xffffffffu, x[i].x, N / 2, N);
                const float zi = __shfl_sync(0xffffffffu, x[i].y, N / 2, N);
                if (i == lane) z3 = make_float2(zr, zi);
            }
            const float2 c2 = make_float2(sc * sc2[pid * N + lane].x, sc * sc2[pid * N + lane].y);
            const float2 c3 = make_float2(sc * sc3[pid * N + lane].x, sc * sc3[pid * N + lane].y);
            const float2 zz = x[N / 2];
            x2.x = fmaf(zz.x, c2.x, fmaf(-zz.y, c2.y, x2.x));
            x2.y = fmaf(zz.x, c2.y, fmaf(zz.y, c2.x, x2.y));
            x3.x = fmaf(z3.x, c3.x, fmaf(-z3.y, c3.y, x3.x));
            x3.y = fmaf(z3.x, c3.y, fmaf(z3.y, c3.x, x3.y));
            t_wait_st();
        }
        cp_async_wait_all();
        float2 *out = a.part + ((size_t)slot * a.nblk + blk) * N3 + (size_t)k1 * N * N;
        #pragma unroll
        for (int g = 0; g < 4; ++g) {
            float s[16];
            t_ld16(tl + TM_ACC + 16 * g, s);
            t_wait_ld();
            #pragma unroll
            for (int u = 0; u < 8; ++u) out[(8 * g + u) * N + lane] = make_float2(s[2 * u], s[2 * u + 1]);
        }
        float2 *xo = a.part_s + ((size_t)slot * a.nblk + blk) * 3 * N * N;
        xo[N * N + k1 * N + lane] = x2;
        xo[2 * N * N + k1 * N + lane] = x3;
        if (k1 == N / 2) {
            #pragma unroll 8
            for (int i = 0; i < N; ++i) xo[i * N + lane] = xs1[i * N + lane];
        }
    }
    tfence_before();
    __syncthreads();
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(s_tmem), "n"(P_TMEM_COLS) : "memory");
}

// k_pair3's launch shape without tensor memory: the occupancy query counts its clusters at the
// residency its registers and shared memory allow (the query counts one CTA per SM for a kernel
// that allocates tensor memory).
__global__ void __launch_bounds__(PT, 3) k_pair3_shape(int *p) {
    if (p) p[threadIdx.x] = 0;
}

cudaLaunchConfig_t pair3_config(int G, cudaStream_t st, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = PC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(G * PC);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = P_SMEM;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace

cudaError_t pair3_setup(int *G) {
    *G = 0;
    for (const void *k : {(const void *)k_pair3<false>, (const void *)k_pair3<true>, (const void *)k_pair3_shape}) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair3_config(64, nullptr, attr);
    const cudaError_t e = cudaOccupancyMaxActiveClusters(G, k_pair3_shape, &cfg);
    if (e != cudaSuccess) return e;
    return *G > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

bz_status launch_pair3(const Plan &pl, const ItemArgs &a, cudaStream_t st) {
    if (pl.N != PN || !a.real || !a.hg) return BZ_ERR_UNSUPPORTED;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = pair3_config(pl.fused_G, st, attr);
    if (a.gsc) BZ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_pair3<true>, a));
    else BZ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_pair3<false>, a));
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

}  // namespace bz

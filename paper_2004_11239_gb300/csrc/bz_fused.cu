// Fused per-term pipeline of eq. realQ (Sec. 4) for N <= 32: one thread-block cluster keeps
// a term's whole N^3 field on chip from the twiddle to the weighted accumulation.
//
// A cluster of C CTAs owns PPC = N / C planes k1 each and loops over its share of the
// terms (persistent, cluster g takes terms p0 + g, p0 + g + G, ...).  Per term:
//   A  planes (own k1):   beta_p fhat -> IFFT over k2 (registers) -> IFFT over k3 (rows)
//                         (twiddles staged in shared memory one term ahead by cp.async)
//   -- cluster barrier --
//   B  pencils (own j2):  gather the k1 line from the cluster's shared memory (DSMEM),
//                         IFFT over k1, times h (held in shared memory), FFT over j1,
//                         scatter back
//   -- cluster barrier --
//   C  planes (own k1):   FFT over j3 (rows), FFT over j2 (registers), times alpha_p (tile
//                         prefetched by cp.async during A and B), accumulate in registers
// A prologue forms h = IFFT(fhat) for the CTA's pencils the same way (no twiddle, inverse
// only) straight into shared memory, so no separate h pass is launched.  DSMEM is reached
// with ld/st.shared::cluster on mapa addresses.  Each CTA ends with its plane slab of the
// cluster's partial sum (FP32 over the cluster's terms); a second kernel adds the G
// partials in FP64 in a fixed order (blocked summation, deterministic).  Global traffic per
// term is fhat (L2-resident) and alpha_p (HBM).
#include <cooperative_groups.h>

#include "bz_fft.cuh"
#include "bz_internal.h"

namespace cg = cooperative_groups;

namespace bz {

template <int N> struct FusedC;
template <> struct FusedC<8> { static constexpr int C = 1; };
template <> struct FusedC<16> { static constexpr int C = 1; };
template <> struct FusedC<24> { static constexpr int C = 2; };
template <> struct FusedC<32> { static constexpr int C = 4; };

template <int N> struct FK {
    static constexpr int C = FusedC<N>::C;
    static constexpr int PPC = N / C;                 // planes (and pencil rows) per CTA
    static constexpr int LD = N + 1;                  // padded plane row
    static constexpr int THREADS = N * PPC;
    static constexpr size_t PLANES = (size_t)PPC * N * LD * sizeof(float2);
    static constexpr size_t TILE = (size_t)PPC * N * N * sizeof(float2);   // alpha tile, h slice
    static constexpr size_t TW = (size_t)3 * N * sizeof(float2);           // one term's twiddles
    static constexpr size_t SMEM = PLANES + 2 * TILE + 2 * TW;
    static constexpr int MIN_BLOCKS = N <= 16 ? 2 : 1;   // N <= 16: two CTAs per SM fit
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Distributed shared memory through the shared::cluster window (32-bit addresses).
__device__ __forceinline__ uint32_t dsmem_addr(const void *local, uint32_t rank) {
    uint32_t a = (uint32_t)__cvta_generic_to_shared(local), r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_dsmem(uint32_t a) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_dsmem(uint32_t a, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}

template <int C> __device__ __forceinline__ void cluster_barrier() {
    if constexpr (C > 1) cg::this_cluster().sync();
    else __syncthreads();
}

// Phase A for plane k1 (column k3 = lane): x = twiddle * fhat over k2, IFFT over k2, store
// the column, then rows over k3.  tws == nullptr: no twiddle (the h prologue).
template <int N>
__device__ __forceinline__ void phase_a(const float2 *__restrict__ fin, const float2 *tws, float2 *my,
                                        int k1, int lane) {
    constexpr int LD = N + 1;
    const float2 *f = fin + (size_t)k1 * N * N;
    float2 x[N];
    if (tws) {
        const float2 t13 = cmul(tws[k1], tws[2 * N + lane]);
        #pragma unroll
        for (int i = 0; i < N; ++i) x[i] = cmul(f[i * N + lane], cmul(t13, tws[N + i]));
    } else {
        #pragma unroll
        for (int i = 0; i < N; ++i) x[i] = f[i * N + lane];
    }
    fft_inplace<N, +1>(x);                                    // k2 -> j2
    #pragma unroll
    for (int i = 0; i < N; ++i) my[i * LD + lane] = x[i];
    __syncthreads();
    #pragma unroll
    for (int j = 0; j < N; ++j) x[j] = my[lane * LD + j];
    fft_inplace<N, +1>(x);                                    // k3 -> j3 (row j2 = lane)
    #pragma unroll
    for (int j = 0; j < N; ++j) my[lane * LD + j] = x[j];
}

// Work item w: instance b = w / nblk (array slot slots[b]), term block blk = w % nblk covering
// terms [p0 + blk TB, min(p1, p0 + (blk + 1) TB)).  The item's FP32 sum over its terms goes to
// part[slot * nblk + blk]; it depends only on the instance and the block bounds, so a result
// does not depend on which other instances share the launch.
template <int N, bool SCALED>
__global__ void __launch_bounds__(FK<N>::THREADS, FK<N>::MIN_BLOCKS)
k_fused(ItemArgs a) {
    using K = FK<N>;
    constexpr int C = K::C, PPC = K::PPC, LD = K::LD, T = K::THREADS;
    extern __shared__ __align__(16) float2 smem[];
    float2 *planes = smem;                                   // [PPC][N][LD]
    float2 *sal = smem + (size_t)PPC * N * LD;               // alpha tile [PPC][N][N]
    float2 *shs = sal + (size_t)PPC * N * N;                 // h slice [PPC (j2)][N (j1)][N (j3)]
    float2 *stw = shs + (size_t)PPC * N * N;                 // twiddles, two buffers of [3][N]
    const int tid = threadIdx.x;
    int rank = 0;
    if constexpr (C > 1) rank = (int)cg::this_cluster().block_rank();
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    const int lane = tid % N, pid = tid / N;
    const int k1 = rank * PPC + pid;                         // plane phases
    const int j2p = rank * PPC + pid;                        // pencil phase: (j2p, lane)
    float2 *my = planes + (size_t)pid * N * LD;
    constexpr size_t N3 = (size_t)N * N * N;
    uint32_t pen[C];                                         // element (j2p, lane) of plane 0 in each CTA
    #pragma unroll
    for (int r = 0; r < C; ++r) pen[r] = dsmem_addr(planes + (size_t)j2p * LD + lane, (uint32_t)r);
    constexpr uint32_t PLANE_BYTES = (uint32_t)(N * LD * sizeof(float2));

    const int count = a.count_dev ? *a.count_dev : a.count;
    const int nitems = count * a.nblk;
    auto fetch_tw = [&](int p, int buf) {                    // one term's 3N twiddles, 16 B per copy
        if (p >= 0 && tid < (int)(K::TW / 16))
            cp_async16((char *)(stw + buf * 3 * N) + 16 * tid, (const char *)(a.tw + (size_t)p * 3 * N) + 16 * tid);
        cp_async_commit();
    };

    for (int w = cid; w < nitems; w += ncl) {
        const int b = w / a.nblk, blk = w % a.nblk;
        const int slot = a.slots ? a.slots[b] : b;
        const int t0 = a.p0 + blk * a.TB;
        const int t1 = min(a.p1, t0 + a.TB);
        const float2 *fin = a.fin + (size_t)slot * N3;
        // prologue: h = IFFT(fhat_b) for the pencils this CTA owns, into the h slice
        __syncthreads();                                      // the previous item is done with smem
        fetch_tw(t0, 0);
        phase_a<N>(fin, nullptr, my, k1, lane);
        cluster_barrier<C>();
        {
            float2 x[N];
            #pragma unroll
            for (int k = 0; k < N; ++k) x[k] = ld_dsmem(pen[k / PPC] + (uint32_t)(k % PPC) * PLANE_BYTES);
            fft_inplace<N, +1>(x);                            // k1 -> j1
            #pragma unroll
            for (int j = 0; j < N; ++j) shs[((size_t)pid * N + j) * N + lane] = x[j];
        }
        cluster_barrier<C>();                                 // planes free again in every CTA

        float2 acc[N];
        #pragma unroll
        for (int i = 0; i < N; ++i) acc[i] = make_float2(0.f, 0.f);
        int it = 0;
        for (int p = t0; p < t1; ++p, ++it) {
            const int buf = it & 1;
            cp_async_wait_all();                              // this term's twiddles have landed
            __syncthreads();                                  // ... for every thread; last term done
            {
                const char *ga = (const char *)(a.alpha + ((size_t)p * N + (size_t)rank * PPC) * N * N);
                char *sa = (char *)sal;
                for (int c = tid; c < (int)(K::TILE / 16); c += T) cp_async16(sa + 16 * c, ga + 16 * c);
                cp_async_commit();
            }
            fetch_tw(p + 1 < t1 ? p + 1 : -1, buf ^ 1);
            float sc = 1.f;
            if constexpr (SCALED) sc = a.gsc[(size_t)slot * a.N_rho + p / a.M];
            // A
            phase_a<N>(fin, stw + buf * 3 * N, my, k1, lane);
            cluster_barrier<C>();
            // B: pencil (j2p, lane) over k1, gathered from the cluster
            float2 x[N];
            #pragma unroll
            for (int k = 0; k < N; ++k) x[k] = ld_dsmem(pen[k / PPC] + (uint32_t)(k % PPC) * PLANE_BYTES);
            fft_inplace<N, +1>(x);                            // k1 -> j1
            #pragma unroll
            for (int j = 0; j < N; ++j) x[j] = cmul(x[j], shs[((size_t)pid * N + j) * N + lane]);
            fft_inplace<N, -1>(x);                            // j1 -> k1
            #pragma unroll
            for (int k = 0; k < N; ++k) st_dsmem(pen[k / PPC] + (uint32_t)(k % PPC) * PLANE_BYTES, x[k]);
            cluster_barrier<C>();
            // C: rows over j3, then column k3 = lane over j2, times alpha, accumulate
            #pragma unroll
            for (int j = 0; j < N; ++j) x[j] = my[lane * LD + j];
            fft_inplace<N, -1>(x);                            // j3 -> k3 (row j2 = lane)
            #pragma unroll
            for (int j = 0; j < N; ++j) my[lane * LD + j] = x[j];
            cp_async_wait_1();                                // alpha tile (the next twiddles may pend)
            __syncthreads();
            #pragma unroll
            for (int i = 0; i < N; ++i) x[i] = my[i * LD + lane];
            fft_inplace<N, -1>(x);                            // j2 -> k2
            #pragma unroll
            for (int i = 0; i < N; ++i) {
                float2 al = sal[((size_t)pid * N + i) * N + lane];
                if constexpr (SCALED) {
                    float2 t = cmul(x[i], al);
                    acc[i].x = fmaf(sc, t.x, acc[i].x);
                    acc[i].y = fmaf(sc, t.y, acc[i].y);
                } else {
                    acc[i].x = fmaf(x[i].x, al.x, fmaf(-x[i].y, al.y, acc[i].x));
                    acc[i].y = fmaf(x[i].x, al.y, fmaf(x[i].y, al.x, acc[i].y));
                }
            }
        }
        cp_async_wait_all();
        float2 *out = a.part + ((size_t)slot * a.nblk + blk) * N3 + (size_t)k1 * N * N;
        #pragma unroll
        for (int i = 0; i < N; ++i) out[i * N + lane] = acc[i];
    }
}

// acc[k] = sum over g of part[g][k] in FP64 with a fixed shape: thread (kk, s) of a 32 x 8
// block sums g = s, s + 8, ... for mode k = 32 blockIdx.x + kk; the eight slices are then
// added in order s = 0..7.
__global__ void __launch_bounds__(256) k_reduce_parts(const float2 *__restrict__ part, int G, int n3,
                                                     double2 *__restrict__ acc) {
    __shared__ double2 red[8][32];
    const int kk = threadIdx.x % 32, sl = threadIdx.x / 32;
    const int k = blockIdx.x * 32 + kk;
    double sr = 0.0, si = 0.0;
    if (k < n3) {
        for (int g = sl; g < G; g += 8) {
            float2 v = part[(size_t)g * n3 + k];
            sr += v.x;
            si += v.y;
        }
    }
    red[sl][kk] = make_double2(sr, si);
    __syncthreads();
    if (sl == 0 && k < n3) {
        double2 t = red[0][kk];
        #pragma unroll
        for (int u = 1; u < 8; ++u) { t.x += red[u][kk].x; t.y += red[u][kk].y; }
        acc[k] = t;
    }
}

template <int N, bool SC> static cudaError_t set_smem() {
    return cudaFuncSetAttribute(k_fused<N, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FK<N>::SMEM);
}

template <int N> static cudaError_t fused_setup_n(int *G) {
    using K = FK<N>;
    cudaError_t e = set_smem<N, false>();
    if (e == cudaSuccess) e = set_smem<N, true>();
    if (e != cudaSuccess) return e;
    if (K::C == 1) {
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused<N, true>, K::THREADS, K::SMEM);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        *G = per_sm * sms;
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = K::C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(K::C * 64);
        cfg.blockDim = dim3(K::THREADS);
        cfg.dynamicSmemBytes = K::SMEM;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(G, k_fused<N, true>, &cfg);
        if (e != cudaSuccess) return e;
    }
    return *G > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

// Number of resident clusters for the plan's N (0 when the fused path does not apply).
cudaError_t fused_setup(int N, int *G) {
    *G = 0;
    switch (N) {
        case 8: return fused_setup_n<8>(G);
        case 16: return fused_setup_n<16>(G);
        case 24: return fused_setup_n<24>(G);
        case 32: return fused_setup_n<32>(G);
    }
    return cudaErrorInvalidValue;
}

template <int N, bool SC> static bz_status launch_n(const Plan &pl, const ItemArgs &a, cudaStream_t st) {
    using K = FK<N>;
    const int G = pl.fused_G;
    if (K::C == 1) {
        k_fused<N, SC><<<G, K::THREADS, K::SMEM, st>>>(a);
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = K::C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(G * K::C);
        cfg.blockDim = dim3(K::THREADS);
        cfg.dynamicSmemBytes = K::SMEM;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        BZ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_fused<N, SC>, a));
    }
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

bz_status launch_fused(const Plan &pl, const ItemArgs &a, cudaStream_t st) {
    const bool sc = a.gsc != nullptr;
    switch (pl.N) {
        case 8: return sc ? launch_n<8, true>(pl, a, st) : launch_n<8, false>(pl, a, st);
        case 16: return sc ? launch_n<16, true>(pl, a, st) : launch_n<16, false>(pl, a, st);
        case 24: return sc ? launch_n<24, true>(pl, a, st) : launch_n<24, false>(pl, a, st);
        case 32: return sc ? launch_n<32, true>(pl, a, st) : launch_n<32, false>(pl, a, st);
    }
    return BZ_ERR_UNSUPPORTED;
}

// One instance (pl.fin), terms [p0, p1): one block of terms per resident cluster, then the
// fixed-order FP64 sum of the blocks into pl.acc.
bz_status collide_fused(Plan &pl, int p0, int p1, cudaStream_t st, int *launches) {
    const int n3 = pl.N * pl.N * pl.N;
    ItemArgs a;
    a.fin = pl.fin; a.tw = pl.tw; a.alpha = pl.alpha; a.part = pl.part;
    a.count = 1; a.p0 = p0; a.p1 = p1; a.M = pl.M; a.N_rho = pl.N_rho;
    const int nt = p1 - p0;
    a.TB = nt > 0 ? (nt + pl.fused_G - 1) / pl.fused_G : 1;
    a.nblk = nt > 0 ? (nt + a.TB - 1) / a.TB : 0;
    tm_begin(pl, st);
    bz_status s = launch_fused(pl, a, st);
    if (s != BZ_OK) return s;
    tm_end(pl, st, TK_FUSED);
    tm_begin(pl, st);
    k_reduce_parts<<<(n3 + 31) / 32, 256, 0, st>>>(pl.part, a.nblk, n3, pl.acc);
    tm_end(pl, st, TK_REDUCE);
    BZ_CUDA_TRY(cudaGetLastError());
    if (launches) *launches += 2;
    return BZ_OK;
}

}  // namespace bz

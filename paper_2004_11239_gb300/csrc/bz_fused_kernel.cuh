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
// h = IFFT(fhat) is formed beforehand in FP64 (k_h64_*) and each item's prologue loads the
// slice of h for the CTA's pencils into shared memory.  DSMEM is reached
// with ld/st.shared::cluster on mapa addresses.  Each CTA ends with its plane slab of the
// cluster's partial sum (FP32 over the cluster's terms); a second kernel adds the G
// partials in FP64 in a fixed order (blocked summation, deterministic).  Global traffic per
// term is fhat (L2-resident) and alpha_p (HBM).
#pragma once
// Device code of the fused kernel (the launch and the rest of the pipeline: bz_fused.cu).
#include <cooperative_groups.h>

#include "bz_cluster.cuh"
#include "bz_fft.cuh"
#include "bz_internal.h"

namespace bz {

namespace cg = cooperative_groups;

template <int N, int C_, bool R_ = false> struct FK {
    static constexpr int C = C_;
    static constexpr int PPC = N / C;                 // planes (and pencil rows) per CTA
    static constexpr int LD = N + 1;                  // padded plane row
    static constexpr int THREADS = N * PPC;
    static constexpr size_t PLANES = (size_t)PPC * N * LD * sizeof(float2);
    static constexpr size_t TILE = (size_t)PPC * N * N * sizeof(float2);   // alpha tile, h slice
    static constexpr size_t TW = (size_t)(R_ ? 6 : 3) * N * sizeof(float2);  // one term's (pair's) twiddles
    // pair form: h slice real (half a tile); X on the plane k1 = -N/2 and one pair's Nyquist
    // table C (that plane, then the CTA's rows of the k2 = -N/2 and k3 = -N/2 families)
    static constexpr size_t HS = R_ ? TILE / 2 : TILE;
    static constexpr size_t XS1 = R_ ? (size_t)N * N * sizeof(float2) : 0;
    static constexpr size_t CS = R_ ? (size_t)(N * N + 2 * PPC * N) * sizeof(float2) : 0;
    static constexpr size_t SMEM = PLANES + TILE + HS + 2 * TW + XS1 + CS;
    // two CTAs per SM where registers and shared memory allow it
    static constexpr int MIN_BLOCKS = (N <= 16 || N * N / C_ <= 128) ? 2 : 1;
};

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

// Phase A of a term pair (p, p') (BZ_DATA_REAL): x = (beta_p + i beta_p') fhat, whose inverse
// transform is g_p + i g_p' with both parts real; tws holds the two terms' [3][N] twiddles.
template <int N>
__device__ __forceinline__ void phase_a_pair(const float2 *__restrict__ fin, const float2 *tws, float2 *my,
                                             int k1, int lane) {
    constexpr int LD = N + 1;
    const float2 *f = fin + (size_t)k1 * N * N;
    const float2 ta = cmul(tws[k1], tws[2 * N + lane]);
    const float2 tb = cmul(tws[3 * N + k1], tws[5 * N + lane]);
    float2 x[N];
    #pragma unroll
    for (int i = 0; i < N; ++i) {
        const float2 u = cmul(ta, tws[N + i]), v = cmul(tb, tws[4 * N + i]);
        x[i] = cmul(f[i * N + lane], make_float2(u.x - v.y, u.y + v.x));       // u + i v
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
// REAL: the units are term pairs (BZ_DATA_REAL): a.alpha is the pair table A, h is real and
// the accumulated sum is V = sum of A Z over the pairs (symmetrised after the reduction).  On
// the Nyquist planes S a second sum X = sum of C Z is kept (a.cpair; C = 0 off S), one entry
// per mode of S in three families: k1 = -N/2 ([k2][k3], shared memory of the CTA owning that
// plane), else k3 = -N/2 ([k1][k2], one register per thread: the value of lane N/2 reaches lane
// k2 by shuffles), else k2 = -N/2 ([k1][k3], one register per thread); it goes to a.part_s.
template <int N, int CC, bool SCALED, bool REAL = false>
__global__ void __launch_bounds__(FK<N, CC, REAL>::THREADS, FK<N, CC, REAL>::MIN_BLOCKS)
k_fused(ItemArgs a) {
    static_assert(!REAL || 32 % N == 0, "the pair form shuffles within the lanes of one plane");
    using K = FK<N, CC, REAL>;
    constexpr int TWN = REAL ? 6 * N : 3 * N;                // twiddles per unit
    constexpr int C = K::C, PPC = K::PPC, LD = K::LD, T = K::THREADS;
    extern __shared__ __align__(16) float2 smem[];
    float2 *planes = smem;                                   // [PPC][N][LD]
    float2 *sal = smem + (size_t)PPC * N * LD;               // alpha tile [PPC][N][N]
    float2 *shs = sal + (size_t)PPC * N * N;                 // h slice [PPC (j2)][N (j1)][N (j3)]
    float *shr = (float *)shs;                               // REAL: the same, real
    float2 *stw = (float2 *)((char *)shs + K::HS);           // twiddles, two buffers of [TWN]
    float2 *xs1 = stw + 2 * TWN;                             // REAL: X on plane k1 = -N/2, [k2][k3]
    float2 *sc1 = xs1 + N * N;                               // REAL: C on plane k1 = -N/2 [k2][k3]
    float2 *sc2 = sc1 + N * N;                               // REAL: C rows k1 of family k2 = -N/2 [pid][k3]
    float2 *sc3 = sc2 + PPC * N;                             // REAL: C rows k1 of family k3 = -N/2 [pid][k2]
    const int tid = threadIdx.x;
    int rank = 0;
    if constexpr (C > 1) rank = (int)cg::this_cluster().block_rank();
    const bool owns_nyq = rank == (N / 2) / PPC;             // REAL: this CTA holds the plane k1 = -N/2
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
    auto fetch_tw = [&](int p, int buf) {                    // one unit's twiddles, 16 B per copy
        if (p >= 0 && tid < (int)(K::TW / 16))
            cp_async16((char *)(stw + buf * TWN) + 16 * tid, (const char *)(a.tw + (size_t)p * TWN) + 16 * tid);
        cp_async_commit();
    };

    for (int w = cid; w < nitems; w += ncl) {
        const int b = w / a.nblk, blk = w % a.nblk;
        const int slot = a.slots ? a.slots[b] : b;
        const int t0 = a.p0 + blk * a.TB;
        const int t1 = min(a.p1, t0 + a.TB);
        const float2 *fin = a.fin + (size_t)slot * N3;
        // prologue: the h slice of the pencils this CTA owns, either formed beforehand in FP64
        // (a.hg) or here in FP32 (no twiddle, inverse only) straight into shared memory
        __syncthreads();                                      // the previous item is done with smem
        fetch_tw(t0, 0);
        if (a.hg) {
            const float2 *hs = a.hg + (size_t)slot * N3;
            #pragma unroll 4
            for (int j = 0; j < N; ++j) {
                const float2 hv = hs[((size_t)j * N + j2p) * N + lane];
                if constexpr (REAL) shr[((size_t)pid * N + j) * N + lane] = hv.x;
                else shs[((size_t)pid * N + j) * N + lane] = hv;
            }
        } else {
            phase_a<N>(fin, nullptr, my, k1, lane);
            cluster_barrier<C>();
            float2 x[N];
            #pragma unroll
            for (int k = 0; k < N; ++k) x[k] = ld_dsmem(pen[k / PPC] + (uint32_t)(k % PPC) * PLANE_BYTES);
            fft_inplace<N, +1>(x);                            // k1 -> j1
            #pragma unroll
            for (int j = 0; j < N; ++j) {
                if constexpr (REAL) shr[((size_t)pid * N + j) * N + lane] = x[j].x;
                else shs[((size_t)pid * N + j) * N + lane] = x[j];
            }
            cluster_barrier<C>();                             // planes free again in every CTA
        }

        float2 acc[N];
        #pragma unroll
        for (int i = 0; i < N; ++i) acc[i] = make_float2(0.f, 0.f);
        float2 x2 = make_float2(0.f, 0.f), x3 = make_float2(0.f, 0.f);   // REAL: X at (k1, -N/2, lane), (k1, lane, -N/2)
        if constexpr (REAL) {
            if (k1 == N / 2) {
                #pragma unroll 8
                for (int i = 0; i < N; ++i) xs1[i * N + lane] = make_float2(0.f, 0.f);
            }
        }
        int it = 0;
        for (int p = t0; p < t1; ++p, ++it) {
            const int buf = it & 1;
            cp_async_wait_all();                              // this term's twiddles have landed
            __syncthreads();                                  // ... for every thread; last term done
            {
                const char *ga = (const char *)(a.alpha + ((size_t)p * N + (size_t)rank * PPC) * N * N);
                char *sa = (char *)sal;
                for (int c = tid; c < (int)(K::TILE / 16); c += T) cp_async16(sa + 16 * c, ga + 16 * c);
                if constexpr (REAL) {                         // this pair's Nyquist table rows
                    const float2 *cq = a.cpair + (size_t)p * 3 * N * N;
                    constexpr int ROW16 = PPC * N * (int)sizeof(float2) / 16;
                    if (tid < ROW16) {
                        cp_async16((char *)sc2 + 16 * tid, (const char *)(cq + N * N + rank * PPC * N) + 16 * tid);
                    } else if (tid < 2 * ROW16) {
                        const int c = tid - ROW16;
                        cp_async16((char *)sc3 + 16 * c, (const char *)(cq + 2 * N * N + rank * PPC * N) + 16 * c);
                    }
                    if (owns_nyq)
                        for (int c = tid; c < N * N * (int)sizeof(float2) / 16; c += T)
                            cp_async16((char *)sc1 + 16 * c, (const char *)cq + 16 * c);
                }
                cp_async_commit();
            }
            fetch_tw(p + 1 < t1 ? p + 1 : -1, buf ^ 1);
            float sc = 1.f;
            if constexpr (SCALED) sc = a.gsc[(size_t)slot * a.N_rho + (REAL ? 2 * p : p) / a.M];   // a pair shares its node
            // A
            if constexpr (REAL) phase_a_pair<N>(fin, stw + buf * TWN, my, k1, lane);
            else phase_a<N>(fin, stw + buf * TWN, my, k1, lane);
            cluster_barrier<C>();
            // B: pencil (j2p, lane) over k1, gathered from the cluster
            float2 x[N];
            #pragma unroll
            for (int k = 0; k < N; ++k) x[k] = ld_dsmem(pen[k / PPC] + (uint32_t)(k % PPC) * PLANE_BYTES);
            fft_inplace<N, +1>(x);                            // k1 -> j1
            if constexpr (REAL) {
                #pragma unroll
                for (int j = 0; j < N; ++j) {                 // h is real
                    const float hv = shr[((size_t)pid * N + j) * N + lane];
                    x[j].x *= hv;
                    x[j].y *= hv;
                }
            } else {
                #pragma unroll
                for (int j = 0; j < N; ++j) x[j] = cmul(x[j], shs[((size_t)pid * N + j) * N + lane]);
            }
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
            if constexpr (REAL) {
                if (k1 == N / 2) {                            // whole plane (warp-uniform)
                    #pragma unroll
                    for (int i = 0; i < N; ++i) {
                        float2 c = sc1[i * N + lane];
                        if constexpr (SCALED) { c.x *= sc; c.y *= sc; }
                        float2 v = xs1[i * N + lane];
                        v.x = fmaf(x[i].x, c.x, fmaf(-x[i].y, c.y, v.x));
                        v.y = fmaf(x[i].x, c.y, fmaf(x[i].y, c.x, v.y));
                        xs1[i * N + lane] = v;
                    }
                }
                float2 z3 = make_float2(0.f, 0.f);            // Z(k1, k2 = lane, -N/2) from lane N/2
                #pragma unroll
                for (int i = 0; i < N; ++i) {
                    const float zr = __shfl_sync(0xffffffffu, x[i].x, N / 2, N);
                    const float zi = __shfl_sync(0xffffffffu, x[i].y, N / 2, N);
                    if (i == lane) z3 = make_float2(zr, zi);
                }
                float2 c2 = sc2[pid * N + lane], c3 = sc3[pid * N + lane];
                if constexpr (SCALED) {                       // the pair's radial scale (one node per pair)
                    c2.x *= sc; c2.y *= sc; c3.x *= sc; c3.y *= sc;
                }
                const float2 z2 = x[N / 2];
                x2.x = fmaf(z2.x, c2.x, fmaf(-z2.y, c2.y, x2.x));
                x2.y = fmaf(z2.x, c2.y, fmaf(z2.y, c2.x, x2.y));
                x3.x = fmaf(z3.x, c3.x, fmaf(-z3.y, c3.y, x3.x));
                x3.y = fmaf(z3.x, c3.y, fmaf(z3.y, c3.x, x3.y));
            }
        }
        cp_async_wait_all();
        float2 *out = a.part + ((size_t)slot * a.nblk + blk) * N3 + (size_t)k1 * N * N;
        #pragma unroll
        for (int i = 0; i < N; ++i) out[i * N + lane] = acc[i];
        if constexpr (REAL) {
            float2 *xo = a.part_s + ((size_t)slot * a.nblk + blk) * 3 * N * N;
            xo[N * N + k1 * N + lane] = x2;
            xo[2 * N * N + k1 * N + lane] = x3;
            if (k1 == N / 2) {
                #pragma unroll 8
                for (int i = 0; i < N; ++i) xo[i * N + lane] = xs1[i * N + lane];
            }
        }
    }
}

}  // namespace bz

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
#include <cooperative_groups.h>

#include "bz_cluster.cuh"
#include "bz_fft.cuh"
#include "bz_internal.h"

namespace cg = cooperative_groups;

namespace bz {

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
    static_assert(!(SCALED && REAL), "the pair form has no per-instance radial scale");
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
            if constexpr (SCALED) sc = a.gsc[(size_t)slot * a.N_rho + p / a.M];
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
                        const float2 c = sc1[i * N + lane];
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
                const float2 c2 = sc2[pid * N + lane], c3 = sc3[pid * N + lane];
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

// h = IFFT(fhat) in FP64 (stored FP32) for the fused path.  FP32 transforms leave a noise
// floor of about eps max|h| over the whole grid, and the product h g_p turns that floor into
// errors where g_p is large and h is small; forming h in FP64 removes that half of the
// rounding error (the per-term g_p stay FP32).  FP64 throughput per SM is low on this GPU,
// so the transform runs as three line passes (axis 3, 2, 1) with eight lines per CTA: the
// N^2 lines of a pass spread over (nearly) every SM.
constexpr int kH64Lines = 8;

__device__ __forceinline__ double2 load_c(const void *f, int dtype, size_t i) {
    if (dtype == BZ_C128) return ((const double2 *)f)[i];
    float2 v = ((const float2 *)f)[i];
    return make_double2(v.x, v.y);
}

// AXIS 3: line (k1, k2) contiguous, from f into scr; AXIS 2: line (k1, k3) with stride N in
// scr; AXIS 1: line (j2, j3) with stride N^2, from scr into h (FP32).
template <int N, int AXIS>
__global__ void __launch_bounds__(kH64Lines)
k_h64_pass(const void *f, int dtype, const int *slots, const int *count_dev, double2 *scr, float2 *h) {
    constexpr int N2 = N * N;
    const int b = blockIdx.y;
    if (count_dev && b >= *count_dev) return;
    const int slot = slots ? slots[b] : b;
    const int line = blockIdx.x * kH64Lines + threadIdx.x;
    if (line >= N2) return;
    const size_t vol = (size_t)slot * N * N2;
    size_t base, stride;
    if (AXIS == 3) { base = vol + (size_t)line * N; stride = 1; }
    else if (AXIS == 2) { base = vol + (size_t)(line / N) * N2 + (line % N); stride = N; }
    else { base = vol + line; stride = N2; }
    double2 x[N];
    #pragma unroll
    for (int k = 0; k < N; ++k)
        x[k] = AXIS == 3 ? load_c(f, dtype, base + k * stride) : scr[base + k * stride];
    fft_inplace<N, +1>(x);
    if (AXIS == 1) {
        #pragma unroll
        for (int j = 0; j < N; ++j) h[base + j * stride] = make_float2((float)x[j].x, (float)x[j].y);
    } else {
        #pragma unroll
        for (int j = 0; j < N; ++j) scr[base + j * stride] = x[j];
    }
}

// Power-of-two N: one warp (N <= 16: a lane segment) per line, radix-2 decimation in
// frequency across lanes with shuffles, lane l ends with frequency bitrev(l).  Each lane's
// twiddles for the log2 N stages are read once.  32 lanes per line keep many more FP64
// operations in flight than one thread per line.
template <int N> __device__ __forceinline__ int bitrev_n(int l) {
    int r = 0;
    #pragma unroll
    for (int b = 1; b < N; b <<= 1) r = (r << 1) | ((l & b) ? 1 : 0);
    return r;
}

template <int N, int AXIS>
__global__ void __launch_bounds__(256)
k_h64_warp(const void *f, int dtype, const int *slots, const int *count_dev, double2 *scr, float2 *h) {
    constexpr int N2 = N * N, LPW = 32 / N, LINES = 8 * LPW;     // lines per warp, per CTA
    const int b = blockIdx.y;
    if (count_dev && b >= *count_dev) return;
    const int slot = slots ? slots[b] : b;
    const int lane = threadIdx.x & 31, l = lane % N;
    const int line = blockIdx.x * LINES + (threadIdx.x >> 5) * LPW + lane / N;
    if (line >= N2) return;                                   // whole segments exit together
    // twiddle of this lane at each stage (half-size hs): exp(+2 pi i (l mod hs) / (2 hs))
    double2 tw[16];
    int st = 0;
    #pragma unroll
    for (int hs = N / 2; hs >= 1; hs >>= 1, ++st) {
        const int j = (l % hs) * (N / (2 * hs));              // index into the length-N roots
        tw[st] = c_twd.v[tw_off<N>() + j];
    }
    const size_t vol = (size_t)slot * N * N2;
    size_t base, stride;
    if (AXIS == 3) { base = vol + (size_t)line * N; stride = 1; }
    else if (AXIS == 2) { base = vol + (size_t)(line / N) * N2 + (line % N); stride = N; }
    else { base = vol + line; stride = N2; }
    double2 v = AXIS == 3 ? load_c(f, dtype, base + (size_t)l * stride) : scr[base + (size_t)l * stride];
    st = 0;
    #pragma unroll
    for (int hs = N / 2; hs >= 1; hs >>= 1, ++st) {
        double2 p;
        p.x = __shfl_xor_sync(0xffffffffu, v.x, hs);
        p.y = __shfl_xor_sync(0xffffffffu, v.y, hs);
        if (l & hs) v = cmul(csub(p, v), tw[st]);
        else v = cadd(v, p);
    }
    const size_t o = base + (size_t)bitrev_n<N>(l) * stride;
    if (AXIS == 1) h[o] = make_float2((float)v.x, (float)v.y);
    else scr[o] = v;
}

template <int N>
static bz_status h64_n(const void *f, int dtype, const int *slots, const int *count_dev, int count, double2 *scr,
                       float2 *h, cudaStream_t st) {
    if constexpr ((N & (N - 1)) == 0) {
        constexpr int LINES = 8 * (32 / N);
        const dim3 grid((N * N + LINES - 1) / LINES, count);
        k_h64_warp<N, 3><<<grid, 256, 0, st>>>(f, dtype, slots, count_dev, scr, h);
        k_h64_warp<N, 2><<<grid, 256, 0, st>>>(f, dtype, slots, count_dev, scr, h);
        k_h64_warp<N, 1><<<grid, 256, 0, st>>>(f, dtype, slots, count_dev, scr, h);
    } else {
        const dim3 grid((N * N + kH64Lines - 1) / kH64Lines, count);
        k_h64_pass<N, 3><<<grid, kH64Lines, 0, st>>>(f, dtype, slots, count_dev, scr, h);
        k_h64_pass<N, 2><<<grid, kH64Lines, 0, st>>>(f, dtype, slots, count_dev, scr, h);
        k_h64_pass<N, 1><<<grid, kH64Lines, 0, st>>>(f, dtype, slots, count_dev, scr, h);
    }
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

bz_status h64_launch(int N, const void *f, int dtype, const int *slots, const int *count_dev, int count,
                     double2 *scr, float2 *h, cudaStream_t st) {
    if (count <= 0) return BZ_OK;
    switch (N) {
        case 8: return h64_n<8>(f, dtype, slots, count_dev, count, scr, h, st);
        case 16: return h64_n<16>(f, dtype, slots, count_dev, count, scr, h, st);
        case 24: return h64_n<24>(f, dtype, slots, count_dev, count, scr, h, st);
        case 32: return h64_n<32>(f, dtype, slots, count_dev, count, scr, h, st);
    }
    return BZ_ERR_UNSUPPORTED;
}

// acc[k] = sum over g of part[g][k] with a fixed shape: thread (kk, s) of a 32 x 8 block sums
// g = s, s + 8, ... for mode k = 32 blockIdx.x + kk with Kahan compensation in FP32, then the
// eight slices are added in order s = 0..7 (compensated).  FP32 pipes only.
struct Kahan2 {
    float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
    __device__ __forceinline__ void add(float vr, float vi) {
        float yr = vr - cr, yi = vi - ci;
        float tr = sr + yr, ti = si + yi;
        cr = (tr - sr) - yr;
        ci = (ti - si) - yi;
        sr = tr;
        si = ti;
    }
};

__global__ void __launch_bounds__(256) k_reduce_parts(const float2 *__restrict__ part, int G, int n3,
                                                     double2 *__restrict__ acc) {
    __shared__ float4 red[8][32];
    const int kk = threadIdx.x % 32, sl = threadIdx.x / 32;
    const int k = blockIdx.x * 32 + kk;
    Kahan2 s;
    if (k < n3) {
        for (int g = sl; g < G; g += 8) {
            float2 v = part[(size_t)g * n3 + k];
            s.add(v.x, v.y);
        }
    }
    red[sl][kk] = make_float4(s.sr, s.si, s.cr, s.ci);
    __syncthreads();
    if (sl == 0 && k < n3) {
        Kahan2 t;
        #pragma unroll
        for (int u = 0; u < 8; ++u) {
            float4 q = red[u][kk];
            t.add(q.x, q.y);
            t.add(-q.z, -q.w);
        }
        acc[k] = make_double2((double)t.sr - (double)t.cr, (double)t.si - (double)t.ci);
    }
}

template <int N, int C, bool SC, bool R> static cudaError_t set_smem() {
    return cudaFuncSetAttribute(k_fused<N, C, SC, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FK<N, C, R>::SMEM);
}

// Resident clusters (C > 1) or CTAs (C = 1) of the kernel that a plan of this form runs.
// The pair form (R) exists where the lanes of a plane share a warp (32 % N == 0).
template <int N> constexpr bool pair_form() { return 32 % N == 0; }

template <int N, int C, bool R> static cudaError_t occupancy(int *G) {
    using K = FK<N, C, R>;
    const void *kern;
    if constexpr (R) kern = (const void *)k_fused<N, C, false, true>;
    else kern = (const void *)k_fused<N, C, true, false>;
    cudaError_t e;
    if (C == 1) {
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, K::THREADS, K::SMEM);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        *G = per_sm * sms;
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(C * 64);
        cfg.blockDim = dim3(K::THREADS);
        cfg.dynamicSmemBytes = K::SMEM;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(G, kern, &cfg);
        if (e != cudaSuccess) return e;
    }
    return *G > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

template <int N, int C> static cudaError_t setup_nc(int *G, bool real) {
    cudaError_t e = set_smem<N, C, false, false>();
    if (e == cudaSuccess) e = set_smem<N, C, true, false>();
    if (e != cudaSuccess) return e;
    if constexpr (pair_form<N>()) {
        if (real) {
            e = set_smem<N, C, false, true>();
            return e == cudaSuccess ? occupancy<N, C, true>(G) : e;
        }
    } else {
        if (real) return cudaErrorInvalidValue;
    }
    return occupancy<N, C, false>(G);
}

// Cluster sizes compiled for each N (the plan times them and keeps the fastest).
int fused_candidates(int N, int *cs) {
    switch (N) {
        case 8: cs[0] = 1; return 1;
        case 16: cs[0] = 1; cs[1] = 2; return 2;
        case 24: cs[0] = 2; cs[1] = 3; return 2;
        case 32: cs[0] = 4; cs[1] = 8; return 2;
    }
    return 0;
}

// Resident clusters for (N, C) (0 when the fused path does not apply); real: the term-pair
// kernel of BZ_DATA_REAL.
cudaError_t fused_setup(int N, int C, int *G, bool real) {
    *G = 0;
    if (N == 8 && C == 1) return setup_nc<8, 1>(G, real);
    if (N == 16 && C == 1) return setup_nc<16, 1>(G, real);
    if (N == 16 && C == 2) return setup_nc<16, 2>(G, real);
    if (N == 24 && C == 2) return setup_nc<24, 2>(G, real);
    if (N == 24 && C == 3) return setup_nc<24, 3>(G, real);
    if (N == 32 && C == 4) return setup_nc<32, 4>(G, real);
    if (N == 32 && C == 8) return setup_nc<32, 8>(G, real);
    return cudaErrorInvalidValue;
}

template <int N, int C, bool SC, bool R> static bz_status launch_nc(const Plan &pl, const ItemArgs &a, cudaStream_t st) {
    using K = FK<N, C, R>;
    const int G = pl.fused_G;
    if (C == 1) {
        k_fused<N, C, SC, R><<<G, K::THREADS, K::SMEM, st>>>(a);
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(G * C);
        cfg.blockDim = dim3(K::THREADS);
        cfg.dynamicSmemBytes = K::SMEM;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        BZ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_fused<N, C, SC, R>, a));
    }
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

template <int N, int C> static bz_status launch_sc(const Plan &pl, const ItemArgs &a, cudaStream_t st) {
    if (a.real) {
        if constexpr (pair_form<N>()) return a.gsc ? BZ_ERR_UNSUPPORTED : launch_nc<N, C, false, true>(pl, a, st);
        else return BZ_ERR_UNSUPPORTED;
    }
    return a.gsc ? launch_nc<N, C, true, false>(pl, a, st) : launch_nc<N, C, false, false>(pl, a, st);
}

bz_status launch_fused(const Plan &pl, const ItemArgs &a, cudaStream_t st) {
    const int N = pl.N, C = pl.fused_C;
    if (pl.precision == BZ_PREC_BF16X3) return a.real ? BZ_ERR_UNSUPPORTED : launch_mixed(pl, a, st);
    if (N == 8 && C == 1) return launch_sc<8, 1>(pl, a, st);
    if (N == 16 && C == 1) return launch_sc<16, 1>(pl, a, st);
    if (N == 16 && C == 2) return launch_sc<16, 2>(pl, a, st);
    if (N == 24 && C == 2) return launch_sc<24, 2>(pl, a, st);
    if (N == 24 && C == 3) return launch_sc<24, 3>(pl, a, st);
    if (N == 32 && C == 4) return launch_sc<32, 4>(pl, a, st);
    if (N == 32 && C == 8) return launch_sc<32, 8>(pl, a, st);
    return BZ_ERR_UNSUPPORTED;
}

// acc[k] = sum over the nblk item partials of part (fixed order, compensated).
void reduce_parts(const float2 *part, int nblk, int n, double2 *acc, cudaStream_t st) {
    k_reduce_parts<<<(n + 31) / 32, 256, 0, st>>>(part, nblk, n, acc);
}

// One instance (pl.fin), terms [p0, p1): one block of terms per resident cluster, then the
// fixed-order FP64 sum of the blocks into pl.acc.  BZ_DATA_REAL: the input is first reduced to
// its Hermitian, Nyquist-free part, the blocks are of term pairs [p0 / 2, p1 / 2), and the sum
// is symmetrised at the end.
bz_status collide_fused(Plan &pl, int p0, int p1, cudaStream_t st, int *launches) {
    const int n3 = pl.N * pl.N * pl.N;
    ItemArgs a;
    a.fin = pl.fin; a.tw = pl.tw; a.alpha = pl.alpha; a.part = pl.part; a.hg = pl.h;
    a.count = 1; a.p0 = p0; a.p1 = p1; a.M = pl.M; a.N_rho = pl.N_rho;
    const void *src = pl.src ? pl.src : (const void *)pl.fin;
    int src_dtype = pl.src ? pl.src_dtype : BZ_C64;
    int nl = 0;
    bz_status s = BZ_OK;
    if (pl.real) {
        if ((p0 | p1) & 1) return BZ_ERR_ARG;
        tm_begin(pl, st);
        s = sym_input(pl, src, src_dtype, st);
        if (s != BZ_OK) return s;
        tm_end(pl, st, TK_OTHER);
        ++nl;
        src = pl.fsym64;
        src_dtype = BZ_C128;
        a.fin = pl.fsym; a.alpha = pl.apair; a.real = 1; a.cpair = pl.cpair; a.part_s = pl.part_s;
        a.p0 = p0 / 2; a.p1 = p1 / 2;
    }
    const int nt = a.p1 - a.p0;
    a.TB = nt > 0 ? (nt + pl.fused_G - 1) / pl.fused_G : 1;
    a.nblk = nt > 0 ? (nt + a.TB - 1) / a.TB : 0;
    if (pl.h_fp64 || pl.precision == BZ_PREC_BF16X3) {
        tm_begin(pl, st);
        s = h64_launch(pl.N, src, src_dtype, nullptr, nullptr, 1, pl.scr64, pl.h, st);
        if (s != BZ_OK) return s;
        tm_end(pl, st, TK_OTHER);
        nl += 3;
    } else {
        a.hg = nullptr;                                   // h formed in FP32 in the item prologue
    }
    tm_begin(pl, st);
    s = launch_fused(pl, a, st);
    if (s != BZ_OK) return s;
    tm_end(pl, st, TK_FUSED);
    tm_begin(pl, st);
    k_reduce_parts<<<(n3 + 31) / 32, 256, 0, st>>>(pl.part, a.nblk, n3, pl.acc);
    tm_end(pl, st, TK_REDUCE);
    BZ_CUDA_TRY(cudaGetLastError());
    nl += 2;
    if (pl.real) {
        tm_begin(pl, st);
        reduce_parts(pl.part_s, a.nblk, 3 * pl.N * pl.N, pl.acc_s, st);
        s = sym_output(pl, st);
        if (s != BZ_OK) return s;
        tm_end(pl, st, TK_OTHER);
        nl += 2;
    }
    if (launches) *launches += nl;
    return BZ_OK;
}

}  // namespace bz

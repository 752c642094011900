// The fused per-term pipeline (N <= 32): launch configuration, cluster-size setup, the FP64
// h passes and the fixed-order reduction of the items' partial sums.  The kernel itself is in
// bz_fused_kernel.cuh.
#include "bz_fused_kernel.cuh"

namespace bz {

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
k_h64_warp(const void *f, int dtype, const int *slots, const int *count_dev, double2 *scr, float2 *h,
           float2 *fsym) {
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
    double2 v;
    if (AXIS != 3) {
        v = scr[base + (size_t)l * stride];
    } else if (!fsym) {
        v = load_c(f, dtype, base + (size_t)l * stride);
    } else {
        // BZ_DATA_REAL: the Hermitian part (fhat_k + conj fhat_{-k}) / 2, zero where an index is
        // N/2; its FP32 copy is the fused kernel's input
        const int k1 = line / N, k2 = line % N, h2 = N / 2;
        v = make_double2(0.0, 0.0);
        if (k1 != h2 && k2 != h2 && l != h2) {
            const double2 a = load_c(f, dtype, base + l);
            const double2 c = load_c(f, dtype, vol + ((size_t)((N - k1) % N) * N + (N - k2) % N) * N + (N - l) % N);
            v = make_double2(0.5 * (a.x + c.x), 0.5 * (a.y - c.y));
        }
        fsym[base + l] = make_float2((float)v.x, (float)v.y);
    }
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

// One line transform of length 32 across the lanes of a warp (radix-2 decimation in frequency,
// as k_h64_warp): lane l holds x_l on entry and X_bitrev(l) on return.
__device__ __forceinline__ double2 warp_fft32(double2 v, int l) {
    int st = 0;
    #pragma unroll
    for (int hs = 16; hs >= 1; hs >>= 1, ++st) {
        const double2 tw = c_twd.v[tw_off<32>() + (l % hs) * (32 / (2 * hs))];
        double2 p;
        p.x = __shfl_xor_sync(0xffffffffu, v.x, hs);
        p.y = __shfl_xor_sync(0xffffffffu, v.y, hs);
        if (l & hs) v = cmul(csub(p, v), tw);
        else v = cadd(v, p);
    }
    return v;
}

// N = 32: the first two FP64 passes (axes k3 and k2, both inside a plane k1) in one kernel.  A
// cluster of 4 CTAs holds one plane: CTA r transforms the k3 lines of rows k2 = 8r .. 8r + 7 (one
// warp per line) into its shared memory, and after a cluster barrier the k2 lines of columns
// j3 = 8r .. 8r + 7, gathering each line from the four CTAs (DSMEM), into scr for the k1 pass.
// fsym: as k_h64_warp<N, 3>.  Grid (32 planes x 4, instances).
__global__ void __launch_bounds__(256) k_h64_plane32(const void *f, int dtype, const int *slots, const int *count_dev,
                                                    double2 *scr, float2 *fsym) {
    constexpr int N = 32, N2 = N * N;
    __shared__ double2 rows[8][N];                           // [k2 - 8r][j3]
    const int b = blockIdx.y;
    if (count_dev && b >= *count_dev) return;               // uniform over the cluster
    const int slot = slots ? slots[b] : b;
    const int r = (int)cooperative_groups::this_cluster().block_rank();
    const int k1 = blockIdx.x / 4, w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const size_t vol = (size_t)slot * N * N2;
    {                                                        // k3 line of row k2 = 8r + w
        const int k2 = 8 * r + w;
        const size_t base = vol + ((size_t)k1 * N + k2) * N;
        double2 v;
        if (!fsym) {
            v = load_c(f, dtype, base + l);
        } else {
            const int h2 = N / 2;
            v = make_double2(0.0, 0.0);
            if (k1 != h2 && k2 != h2 && l != h2) {
                const double2 a = load_c(f, dtype, base + l);
                const double2 c = load_c(f, dtype, vol + ((size_t)((N - k1) % N) * N + (N - k2) % N) * N + (N - l) % N);
                v = make_double2(0.5 * (a.x + c.x), 0.5 * (a.y - c.y));
            }
            fsym[base + l] = make_float2((float)v.x, (float)v.y);
        }
        rows[w][bitrev_n<N>(l)] = warp_fft32(v, l);
    }
    cooperative_groups::this_cluster().sync();
    {                                                        // k2 line of column j3 = 8r + w
        const int j3 = 8 * r + w;
        const uint32_t src = dsmem_addr(&rows[l % 8][j3], (uint32_t)(l / 8));   // element (k2 = l, j3)
        double2 v;
        asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];\n" : "=d"(v.x), "=d"(v.y) : "r"(src) : "memory");
        v = warp_fft32(v, l);
        scr[vol + ((size_t)k1 * N + bitrev_n<N>(l)) * N + j3] = v;
    }
    cooperative_groups::this_cluster().sync();               // no CTA leaves while its rows are read
}

template <int N>
static bz_status h64_n(const void *f, int dtype, const int *slots, const int *count_dev, int count, double2 *scr,
                       float2 *h, float2 *fsym, cudaStream_t st) {
    if constexpr ((N & (N - 1)) == 0) {
        constexpr int LINES = 8 * (32 / N);
        const dim3 grid((N * N + LINES - 1) / LINES, count);
        if constexpr (N == 32) {
            // axes k3 and k2 in one clustered pass, then the k1 pass
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 4;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(4 * N, count);
            cfg.blockDim = dim3(256);
            cfg.stream = st;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            BZ_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_h64_plane32, f, dtype, slots, count_dev, scr, fsym));
        } else {
            k_h64_warp<N, 3><<<grid, 256, 0, st>>>(f, dtype, slots, count_dev, scr, h, fsym);
            k_h64_warp<N, 2><<<grid, 256, 0, st>>>(f, dtype, slots, count_dev, scr, h, nullptr);
        }
        k_h64_warp<N, 1><<<grid, 256, 0, st>>>(f, dtype, slots, count_dev, scr, h, nullptr);
    } else {
        if (fsym) return BZ_ERR_UNSUPPORTED;
        const dim3 grid((N * N + kH64Lines - 1) / kH64Lines, count);
        k_h64_pass<N, 3><<<grid, kH64Lines, 0, st>>>(f, dtype, slots, count_dev, scr, h);
        k_h64_pass<N, 2><<<grid, kH64Lines, 0, st>>>(f, dtype, slots, count_dev, scr, h);
        k_h64_pass<N, 1><<<grid, kH64Lines, 0, st>>>(f, dtype, slots, count_dev, scr, h);
    }
    BZ_CUDA_TRY(cudaGetLastError());
    return BZ_OK;
}

bz_status h64_launch(int N, const void *f, int dtype, const int *slots, const int *count_dev, int count,
                     double2 *scr, float2 *h, cudaStream_t st, float2 *fsym) {
    if (count <= 0) return BZ_OK;
    switch (N) {
        case 8: return h64_n<8>(f, dtype, slots, count_dev, count, scr, h, fsym, st);
        case 16: return h64_n<16>(f, dtype, slots, count_dev, count, scr, h, fsym, st);
        case 24: return h64_n<24>(f, dtype, slots, count_dev, count, scr, h, fsym, st);
        case 32: return h64_n<32>(f, dtype, slots, count_dev, count, scr, h, fsym, st);
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
            if (e == cudaSuccess) e = set_smem<N, C, true, true>();
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
        if constexpr (pair_form<N>()) return a.gsc ? launch_nc<N, C, true, true>(pl, a, st) : launch_nc<N, C, false, true>(pl, a, st);
        else return BZ_ERR_UNSUPPORTED;
    }
    return a.gsc ? launch_nc<N, C, true, false>(pl, a, st) : launch_nc<N, C, false, false>(pl, a, st);
}

bz_status launch_fused(const Plan &pl, const ItemArgs &a, cudaStream_t st) {
    const int N = pl.N, C = pl.fused_C;
    if (pl.precision == BZ_PREC_BF16X3) return a.real ? BZ_ERR_UNSUPPORTED : launch_mixed(pl, a, st);
    if (pl.pair3 && a.real) return launch_pair3(pl, a, st);
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
        if (!(pl.h_fp64 || pl.precision == BZ_PREC_BF16X3)) {
            // h formed in FP32 in the kernel from the symmetrised copy (the FP64 pass writes it otherwise)
            tm_begin(pl, st);
            s = sym_input(pl, src, src_dtype, st);
            if (s != BZ_OK) return s;
            tm_end(pl, st, TK_OTHER);
            ++nl;
        }
        a.fin = pl.fsym; a.alpha = pl.apair; a.real = 1; a.cpair = pl.cpair; a.part_s = pl.part_s;
        a.p0 = p0 / 2; a.p1 = p1 / 2;
    }
    const int nt = a.p1 - a.p0;
    a.TB = nt > 0 ? (nt + pl.fused_G - 1) / pl.fused_G : 1;
    a.nblk = nt > 0 ? (nt + a.TB - 1) / a.TB : 0;
    if (pl.h_fp64 || pl.precision == BZ_PREC_BF16X3) {
        tm_begin(pl, st);
        s = h64_launch(pl.N, src, src_dtype, nullptr, nullptr, 1, pl.scr64, pl.h, st, pl.real ? pl.fsym : nullptr);
        if (s != BZ_OK) return s;
        tm_end(pl, st, TK_OTHER);
        nl += h64_launches(pl.N);
    } else if (pl.pair3) {
        // the pair kernel reads h: formed in FP32 from the symmetrised input by one plane pass
        // and one pencil pass of the chunked pipeline
        tm_begin(pl, st);
        s = h_fp32(pl, pl.fsym, st);
        if (s != BZ_OK) return s;
        tm_end(pl, st, TK_OTHER);
        nl += 2;
    } else {
        a.hg = nullptr;                                   // h formed in FP32 in the item prologue
    }
    tm_begin(pl, st);
    s = launch_fused(pl, a, st);
    if (s != BZ_OK) return s;
    tm_end(pl, st, TK_FUSED);
    tm_begin(pl, st);
    if (pl.real) {
        s = reduce_sym(pl, a.nblk, st);                   // sums of the blocks, symmetrised
        if (s != BZ_OK) return s;
    } else {
        k_reduce_parts<<<(n3 + 31) / 32, 256, 0, st>>>(pl.part, a.nblk, n3, pl.acc);
    }
    tm_end(pl, st, TK_REDUCE);
    BZ_CUDA_TRY(cudaGetLastError());
    nl += 2;
    if (launches) *launches += nl;
    return BZ_OK;
}

}  // namespace bz

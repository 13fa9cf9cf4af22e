// State management, initial states, FP64 reductions (norm, probabilities,
// entropy / Porter-Thomas moments) and sampling.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace {
thread_local char g_err[512] = "";

int sm_count_dev()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return qs_fail(e == cudaErrorMemoryAllocation ? QS_ENOMEM : QS_ECUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

#define QS_CUDA(call, what)                          \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

size_t amp_bytes(int dtype) { return dtype == QS_C128 ? 16 : 8; }

// ------------------------------------------------------------------ kernels

template <typename C, typename R>
__global__ void k_fill_uniform(C *psi, uint64_t N, R a)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        C z;
        z.x = a;
        z.y = 0;
        psi[i] = z;
    }
}

// zeros at every index outside the support {i : (i & ~free) == fix}
template <typename C>
__global__ void k_fill_outside(C *psi, uint64_t N, uint64_t free, uint64_t fix)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        if ((i & ~free) == fix) continue;
        C z;
        z.x = 0;
        z.y = 0;
        psi[i] = z;
    }
}

template <typename C>
__global__ void k_set_one(C *psi, uint64_t x)
{
    C o;
    o.x = 1;
    o.y = 0;
    psi[x] = o;
}

using qsd::prob;

template <typename C>
__global__ void k_probs(const C *__restrict__ psi, uint64_t first, uint64_t count, double *__restrict__ p)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        p[i] = prob(psi[first + i]);
}

using qsd::ff;
using qsd::ff_add;
using qsd::ff_from_double;
using qsd::ff_mul;
using qsd::ff_p_ln_p;
using qsd::ff_sqr_f;
using qsd::FFLogTable;
using qsd::ff_log_table_init;

// The float-float log tables, built once per device (k_fflog_init) and copied
// into shared memory by every block of the statistics kernel.
__device__ __align__(16) FFLogTable g_fflog;

__global__ void k_fflog_init() { ff_log_table_init(g_fflog); }

// Per-block FP64 partial sums of (p, -p ln p, p, p^2); NSTAT = 1 or 4.  The
// mean of N p equals the sum of p, and the mean of (N p)^2 is N sum p^2, so
// the moments cost one product per amplitude; the host applies the factor N.
// Everything runs in float-float on the FP32 pipe (GB300's FP64 pipe runs at
// 1/64 of its rate): complex128 amplitudes are split into float-float by bit
// manipulation (48 of their 53 bits), complex64 ones give p exactly (x^2 and
// y^2 with their FMA rounding errors).  p, p^2 and p ln p (table-driven log,
// ff_p_ln_p) are summed per thread in float-float; the rounding errors of
// those sums are random, about 2^-48 of the partial sum per step, so the
// total norm of a 30-qubit state carries an error near 1e-15.  p below 2^-79
// (where the low half of p's float-float form would leave the normal float
// range) takes p ln p from the FP64 math library, and complex128 amplitudes of
// 2^30 or more (unnormalised input) are summed in FP64 throughout; p below the
// normal double range contributes less than 1e-305 and is left out.
// Per-thread sums of the statistics; add() takes one amplitude, partials()
// reduces the block (every thread of the block calls it).
struct StatsAcc {
    double d0 = 0, d3 = 0, dent = 0;
    ff f0{0.f, 0.f}, f3{0.f, 0.f}, fent{0.f, 0.f};

    template <int NSTAT>
    __device__ __forceinline__ void add(const double2 a, const FFLogTable &lt)
    {
        // magnitude tests on the exponent fields (integer compares; FP64
        // compares would run on the FP64 pipe): field < 1053 is |v| < 2^30,
        // field >= 963 is |v| >= 2^-60
        const uint32_t ex = ((uint32_t)__double2hiint(a.x) >> 20) & 0x7FFu;
        const uint32_t ey = ((uint32_t)__double2hiint(a.y) >> 20) & 0x7FFu;
        if (ex < 1053u && ey < 1053u) {
            // x and y as float-float (values below 2^-60 add less than 2^-120
            // to p and count as zero), p and its sums in float-float
            const ff x = ex >= 963u ? ff_from_double(a.x) : ff{0.f, 0.f};
            const ff y = ey >= 963u ? ff_from_double(a.y) : ff{0.f, 0.f};
            const ff p = ff_add(ff_mul(x, x), ff_mul(y, y));
            f0 = ff_add(f0, p);
            if (NSTAT == 4) {
                f3 = ff_add(f3, ff_mul(p, p));
                if (p.hi >= 0x1p-79f) {
                    fent = ff_add(fent, ff_p_ln_p(lt, p));
                } else if (p.hi > 0.f) {
                    const double pd = (double)p.hi + (double)p.lo;
                    if (pd >= 2.2250738585072014e-308) dent += pd * log(pd);
                }
            }
        } else {
            // an amplitude of 2^30 or more (unnormalised input): FP64 throughout
            const double p = fma(a.x, a.x, a.y * a.y);
            d0 += p;
            if (NSTAT == 4) {
                d3 = fma(p, p, d3);
                dent += p * log(p);
            }
        }
    }

    template <int NSTAT>
    __device__ __forceinline__ void add(const float2 a, const FFLogTable &)
    {
        // complex64 amplitudes carry FP32 errors (2^-24 relative): p, p^2
        // and the logarithm of p are formed in FP32 (one rounding each, the
        // logarithm a few ulp), and the terms add up in float-float
        const float p = fmaf(a.x, a.x, __fmul_rn(a.y, a.y));
        f0 = ff_add_f(f0, p);
        if (NSTAT == 4) {
            f3 = ff_add_f(f3, __fmul_rn(p, p));
            if (p >= 0x1p-79f && p <= 0x1p100f) {
                fent = ff_add_f(fent, __fmul_rn(p, __logf(p)));
            } else if (p > 0.f) {
                const double pd = (double)p;
                if (pd >= 2.2250738585072014e-308) dent += pd * log(pd);
            }
        }
    }

    // part[blockIdx.x * NSTAT + j]: the block's sums of (p, -p ln p, p, p^2)
    template <int NSTAT>
    __device__ void partials(double *__restrict__ part) const
    {
        double acc[NSTAT];
        acc[0] = d0 + ((double)f0.hi + (double)f0.lo);
        if (NSTAT == 4) {
            acc[NSTAT > 1 ? 1 : 0] = -(dent + ((double)fent.hi + (double)fent.lo));
            acc[NSTAT > 2 ? 2 : 0] = acc[0];
            acc[NSTAT > 3 ? 3 : 0] = d3 + ((double)f3.hi + (double)f3.lo);
        }
        __shared__ double red[NSTAT][32];
#pragma unroll
        for (int j = 0; j < NSTAT; j++) {
            double v = acc[j];
            for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = v;
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            int nw = blockDim.x >> 5;
#pragma unroll
            for (int j = 0; j < NSTAT; j++) {
                double v = threadIdx.x < nw ? red[j][threadIdx.x] : 0.0;
                for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (threadIdx.x == 0) part[(size_t)blockIdx.x * NSTAT + j] = v;
            }
        }
    }
};

// The log tables into shared memory (complex128 statistics only).
template <typename C, int NSTAT>
__device__ __forceinline__ void load_fflog(FFLogTable &lt)
{
    if (NSTAT == 4 && sizeof(C) == 16) {
        const uint2 *src = reinterpret_cast<const uint2 *>(&g_fflog);
        uint2 *dst = reinterpret_cast<uint2 *>(&lt);
        for (int i = threadIdx.x; i < (int)(sizeof(FFLogTable) / sizeof(uint2)); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    }
}

// Per-block FP64 partial sums of (p, -p ln p, p, p^2); NSTAT = 1 or 4.  The
// mean of N p equals the sum of p, and the mean of (N p)^2 is N sum p^2, so
// the moments cost one product per amplitude; the host applies the factor N.
// Everything runs in float-float on the FP32 pipe (GB300's FP64 pipe runs at
// 1/64 of its rate): complex128 amplitudes are split into float-float by bit
// manipulation (48 of their 53 bits), complex64 ones give p exactly (x^2 and
// y^2 with their FMA rounding errors).  p, p^2 and p ln p (table-driven log,
// ff_p_ln_p) are summed per thread in float-float; the rounding errors of
// those sums are random, about 2^-48 of the partial sum per step, so the
// total norm of a 30-qubit state carries an error near 1e-15.  p below 2^-79
// (where the low half of p's float-float form would leave the normal float
// range) takes p ln p from the FP64 math library, and complex128 amplitudes of
// 2^30 or more (unnormalised input) are summed in FP64 throughout; p below the
// normal double range contributes less than 1e-305 and is left out.
template <typename C, int NSTAT>
__global__ void k_stats_partial(const C *__restrict__ psi, uint64_t N, double *__restrict__ part)
{
    constexpr bool c128 = sizeof(C) == 16;
    __shared__ __align__(16) FFLogTable lt;
    load_fflog<C, NSTAT>(lt);
    StatsAcc acc;
    // each thread loads kAhead amplitudes (block-strided, so every load of a
    // warp is contiguous) before it adds them up: more loads in flight
    constexpr int kAhead = c128 ? 4 : 8;
    const uint64_t span = (uint64_t)blockDim.x * kAhead;
    for (uint64_t base = (uint64_t)blockIdx.x * span; base < N; base += (uint64_t)gridDim.x * span) {
        C av[kAhead];
#pragma unroll
        for (int k = 0; k < kAhead; k++) {
            const uint64_t i = base + (uint64_t)k * blockDim.x + threadIdx.x;
            av[k] = i < N ? psi[i] : C{};   // a zero amplitude adds nothing
        }
#pragma unroll
        for (int k = 0; k < kAhead; k++) acc.add<NSTAT>(av[k], lt);
    }
    acc.partials<NSTAT>(part);
}

template <int NSTAT>
__global__ void k_stats_final(const double *__restrict__ part, int nblocks, double *__restrict__ out)
{
    // one warp; fixed order for reproducibility
    double acc[NSTAT];
#pragma unroll
    for (int j = 0; j < NSTAT; j++) acc[j] = 0;
    for (int b = threadIdx.x; b < nblocks; b += 32)
#pragma unroll
        for (int j = 0; j < NSTAT; j++) acc[j] += part[(size_t)b * NSTAT + j];
#pragma unroll
    for (int j = 0; j < NSTAT; j++) {
        double v = acc[j];
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) out[j] = v;
    }
}

std::mutex g_fflog_mu;
bool g_fflog_ready[64] = {false};

// Build the log tables on the current device once (one block, then a wait).
int ensure_fflog(cudaStream_t st)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return qs_fail(QS_EUNSUPPORTED, "statistics: no usable device");
    std::lock_guard<std::mutex> lock(g_fflog_mu);
    if (g_fflog_ready[dev]) return QS_OK;
    k_fflog_init<<<1, 1024, 0, st>>>();
    QS_CUDA(cudaGetLastError(), "log table launch");
    QS_CUDA(cudaStreamSynchronize(st), "log table");
    g_fflog_ready[dev] = true;
    return QS_OK;
}

// ------------------------------------------------------------------ sampling
// Pairwise sums over fixed power-of-two blocks: lane l of a warp reduces its
// contiguous len/32 values as a perfect binary tree, then the 32 lane results
// combine as the top five tree levels (lane pairs (0,1), (2,3), ... first).

template <typename C>
__device__ double load_p(const C *psi, uint64_t i) { return prob(psi[i]); }
__device__ double load_p(const double *v, uint64_t i) { return v[i]; }

template <typename T>
__device__ double tree_sum_serial(const T *src, uint64_t start, int len)
{
    double buf[32];
    for (int i = 0; i < len; i++) buf[i] = load_p(src, start + i);
    for (int w = len; w > 1; w >>= 1)
        for (int i = 0; i < w / 2; i++) buf[i] = buf[2 * i] + buf[2 * i + 1];
    return buf[0];
}

// The same pairwise tree over LEN values, unrolled: the loads are all issued
// first and the tree stays in registers (the runtime-length form above keeps
// its buffer in local memory).
template <int LEN, typename T>
__device__ __forceinline__ double tree_sum_fixed(const T *src, uint64_t start)
{
    double buf[LEN];
#pragma unroll
    for (int i = 0; i < LEN; i++) buf[i] = load_p(src, start + i);
#pragma unroll
    for (int w = LEN; w > 1; w >>= 1) {
#pragma unroll
        for (int i = 0; i < w / 2; i++) buf[i] = buf[2 * i] + buf[2 * i + 1];
    }
    return buf[0];
}

// One warp per segment of `len` (power of two, >= 32) values; PER > 0: len is
// 32 PER, summed by the unrolled tree.
template <typename T, int PER>
__global__ void k_segment_sums(const T *__restrict__ src, uint64_t nseg, int len, double *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int per = PER > 0 ? PER : len >> 5;
    for (uint64_t seg = warp; seg < nseg; seg += nwarps) {
        const uint64_t start = seg * (uint64_t)len + (uint64_t)lane * per;
        double v;
        if constexpr (PER > 0) v = tree_sum_fixed<PER>(src, start);
        else v = tree_sum_serial(src, start, per);
        for (int o = 1; o < 32; o <<= 1) {
            double w = __shfl_down_sync(0xffffffffu, v, o);
            if ((lane & (2 * o - 1)) == 0) v = v + w;
        }
        if (lane == 0) out[seg] = v;
    }
}

// Block sums of 1024 probabilities, as k_segment_sums<C, 32> (the same tree,
// built as the values arrive: one pending sum per level, each joined as the
// left operand of the next), and, from the same loads, the block's partial
// sums of the statistics as k_stats_partial<C, 4> forms them (in another
// order).  The block sums use the FP64 unit, the statistics the FP32 one
// (launched for complex64 states).
template <typename C>
__global__ void k_segment_sums_stats(const C *__restrict__ psi, uint64_t nseg, double *__restrict__ out,
                                     double *__restrict__ part)
{
    __shared__ __align__(16) FFLogTable lt;
    load_fflog<C, 4>(lt);
    StatsAcc acc;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t seg = warp; seg < nseg; seg += nwarps) {
        const C *src = psi + seg * 1024 + (uint64_t)lane * 32;
        double lvl[5];
        double v = 0.0;
#pragma unroll
        for (int i = 0; i < 32; i++) {
            const C a = src[i];
            acc.add<4>(a, lt);
            v = prob(a);
            // value i closes the subtrees of the levels where i has a one bit
#pragma unroll
            for (int l = 0; l < 5; l++) {
                if (!((i >> l) & 1)) {
                    lvl[l] = v;
                    break;
                }
                v = lvl[l] + v;
            }
        }
        for (int o = 1; o < 32; o <<= 1) {
            double w = __shfl_down_sync(0xffffffffu, v, o);
            if ((lane & (2 * o - 1)) == 0) v = v + w;
        }
        if (lane == 0) out[seg] = v;
    }
    acc.partials<4>(part);
}

// Segments shorter than a warp: one thread per segment.
template <typename T>
__global__ void k_segment_sums_small(const T *__restrict__ src, uint64_t nseg, int len, double *__restrict__ out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t seg = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; seg < nseg; seg += stride)
        out[seg] = tree_sum_serial(src, seg * (uint64_t)len, len);
}

// Q_0 = 0, Q_{s+1} = Q_s + T_s (one thread); R_{s,0} = Q_s, R_{s,j+1} = R_{s,j} + S_{sG+j}.
__global__ void k_prefix_super(const double *__restrict__ T, uint64_t ns, double *__restrict__ Q)
{
    double q = 0.0;
    for (uint64_t s = 0; s < ns; s++) {
        Q[s] = q;
        q = q + T[s];
    }
}

__global__ void k_prefix_blocks(const double *__restrict__ S, const double *__restrict__ Q, uint64_t ns,
                                uint64_t G, double *__restrict__ R)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += stride) {
        double r = Q[s];
        for (uint64_t j = 0; j < G; j++) {
            R[s * G + j] = r;
            r = r + S[s * G + j];
        }
    }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t j)
{
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// last index in [0, len) with a[idx] <= u (a non-decreasing, a[0] <= u)
__device__ uint64_t last_le(const double *a, uint64_t len, double u)
{
    uint64_t lo = 0, hi = len;   // invariant: a[lo] <= u, answer in [lo, hi)
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename C>
__global__ void k_draw(const C *__restrict__ psi, const double *__restrict__ Q, const double *__restrict__ R,
                       uint64_t ns, uint64_t G, uint64_t B, uint64_t seed, int64_t m, uint64_t *__restrict__ out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        double u = (double)(splitmix64(seed, (uint64_t)j) >> 11) * 0x1.0p-53;
        uint64_t s = last_le(Q, ns, u);
        uint64_t jb = last_le(R + s * G, G, u);
        uint64_t b = s * G + jb;
        double c = R[b];
        uint64_t i = B - 1;
        for (uint64_t x = 0; x < B; x++) {
            c = c + prob(psi[b * B + x]);
            if (c > u) { i = x; break; }
        }
        out[j] = b * B + i;
    }
}

// ---- draws by binary search over stored running sums (blocks of 1024)
//
// The per-draw scan above adds the probabilities of one block to R_b one
// after another until the sum passes u.  The same sums, in the same order,
// can be formed once for every block: c_{b,x} = R_b + p_{bB} + ... + p_{bB+x}
// (sequential FP64 additions).  They do not decrease (p >= 0 and rounding is
// monotone), so the scan's answer, the first x with c_{b,x} > u (B - 1 when
// there is none), is found by binary search: bit for bit the same outcome.

// Block sums of 1024 probabilities as k_segment_sums<C, 32> forms them, and the
// probabilities themselves stored (p[i] = prob(psi[i])).
template <typename C>
__global__ void k_block_sums_store(const C *__restrict__ psi, uint64_t nseg, double *__restrict__ out,
                                   double *__restrict__ p)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t seg = warp; seg < nseg; seg += nwarps) {
        const uint64_t start = seg * 1024 + (uint64_t)lane * 32;
        double buf[32];
#pragma unroll
        for (int i = 0; i < 32; i++) buf[i] = prob(psi[start + i]);
#pragma unroll
        for (int i = 0; i < 32; i += 2)
            *reinterpret_cast<double2 *>(p + start + i) = make_double2(buf[i], buf[i + 1]);
#pragma unroll
        for (int w = 32; w > 1; w >>= 1) {
#pragma unroll
            for (int i = 0; i < w / 2; i++) buf[i] = buf[2 * i] + buf[2 * i + 1];
        }
        double v = buf[0];
        for (int o = 1; o < 32; o <<= 1) {
            double w = __shfl_down_sync(0xffffffffu, v, o);
            if ((lane & (2 * o - 1)) == 0) v = v + w;
        }
        if (lane == 0) out[seg] = v;
    }
}

// In place: p[bB + x] <- c_{b,x} = R_b + p_{bB} + ... + p_{bB+x}.  Lane l of a
// warp owns block 32 w + l; the warp moves its 32 blocks through shared memory
// 32 values at a time, so every global access is a 256-byte run.
constexpr int kRunThreads = 128;

__global__ void __launch_bounds__(kRunThreads) k_running_sums(double *__restrict__ p, const double *__restrict__ R,
                                                              uint64_t nb)
{
    __shared__ double tile[kRunThreads / 32][32][33];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g * 32 < nb; g += nwarps) {
        const uint64_t b0 = g * 32;
        const int nblk = nb - b0 < 32 ? (int)(nb - b0) : 32;
        double c = lane < nblk ? R[b0 + lane] : 0.0;
        for (int x0 = 0; x0 < 1024; x0 += 32) {
            for (int r = 0; r < nblk; r++) tile[wl][r][lane] = p[(b0 + r) * 1024 + x0 + lane];
            __syncwarp();
            if (lane < nblk)
                for (int x = 0; x < 32; x++) {
                    c = c + tile[wl][lane][x];
                    tile[wl][lane][x] = c;
                }
            __syncwarp();
            for (int r = 0; r < nblk; r++) p[(b0 + r) * 1024 + x0 + lane] = tile[wl][r][lane];
            __syncwarp();
        }
    }
}

__global__ void k_draw_search(const double *__restrict__ c, const double *__restrict__ Q,
                              const double *__restrict__ R, uint64_t ns, uint64_t G, uint64_t seed, int64_t m,
                              uint64_t *__restrict__ out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const double u = (double)(splitmix64(seed, (uint64_t)j) >> 11) * 0x1.0p-53;
        const uint64_t s = last_le(Q, ns, u);
        const uint64_t b = s * G + last_le(R + s * G, G, u);
        const double *cb = c + b * 1024;
        uint64_t lo = 0, hi = 1024;          // first x with cb[x] > u, 1023 when none
        while (lo < hi) {
            const uint64_t mid = (lo + hi) / 2;
            if (cb[mid] > u) hi = mid; else lo = mid + 1;
        }
        out[j] = b * 1024 + (lo < 1024 ? lo : 1023);
    }
}

constexpr int kStatsBlocksPerSM = 16;

template <typename C>
int stats_impl(qs_state *s, double *out, int nstat)
{
    uint64_t N = 1ULL << s->n;
    const int block = 256;
    // 16 blocks of 256 per SM: the float-float work is latency-bound at lower
    // occupancy (30 qubits: 7.35 ms with 4 per SM, 6.64 ms with 16)
    int grid = (int)std::min<uint64_t>((N + block - 1) / block, (uint64_t)sm_count_dev() * kStatsBlocksPerSM);
    void *scr = nullptr;
    int rc = qs_state_scratch(s, sizeof(double) * (size_t)(grid + 1) * 4, &scr);
    if (rc) return rc;
    double *part = (double *)scr, *res = part + (size_t)grid * 4;
    cudaStream_t st = (cudaStream_t)s->stream;
    if (nstat == 4 && (rc = ensure_fflog(st))) return rc;
    if (nstat == 1) {
        k_stats_partial<C, 1><<<grid, block, 0, st>>>((const C *)s->amp, N, part);
        k_stats_final<1><<<1, 32, 0, st>>>(part, grid, res);
    } else {
        k_stats_partial<C, 4><<<grid, block, 0, st>>>((const C *)s->amp, N, part);
        k_stats_final<4><<<1, 32, 0, st>>>(part, grid, res);
    }
    QS_CUDA(cudaGetLastError(), "stats launch");
    QS_CUDA(cudaMemcpyAsync(out, res, sizeof(double) * nstat, cudaMemcpyDeviceToHost, st), "stats copy");
    QS_CUDA(cudaStreamSynchronize(st), "stats sync");
    if (nstat == 4) out[3] *= (double)N;   // mean of (N p)^2 = N sum p^2
    return QS_OK;
}

// The state's second stream and its fork/join events, made on first use.
int side_stream(qs_state *s, cudaStream_t *out)
{
    if (!s->side) {
        cudaStream_t ss;
        QS_CUDA(cudaStreamCreateWithFlags(&ss, cudaStreamNonBlocking), "side stream");
        cudaEvent_t e[2];
        for (int i = 0; i < 2; i++) {
            cudaError_t err = cudaEventCreateWithFlags(&e[i], cudaEventDisableTiming);
            if (err != cudaSuccess) {
                for (int j = 0; j < i; j++) cudaEventDestroy(e[j]);
                cudaStreamDestroy(ss);
                return cuda_fail(err, "side stream events");
            }
        }
        s->side = ss;
        s->side_ev[0] = e[0];
        s->side_ev[1] = e[1];
    }
    *out = (cudaStream_t)s->side;
    return QS_OK;
}

// stats (optional): also the statistics of qs_stats.  complex64 states with
// blocks of 1024 take them from the same pass over the state as the block sums
// (33.9 ms instead of 7.6 + 29.4 ms for 2^20 draws at 32 qubits).  complex128
// states with blocks of 1024 run the statistics pass (FP32 pipe) on a second
// stream beside the block sums (FP64 pipe), forked from and joined to the
// state's stream (one kernel doing both measured 28.6 ms against 7.2 + 19.7
// ms, its FP64 and FP32 work not overlapping); otherwise stats_impl runs
// first.
template <typename C>
int sample_impl(qs_state *s, uint64_t seed, int64_t m, uint64_t *out, double *stats)
{
    const uint64_t N = 1ULL << s->n;
    const uint64_t B = std::min<uint64_t>(N, 1024), nb = N / B;
    const uint64_t G = std::min<uint64_t>(nb, 1024), ns = nb / G;
    const int sms = sm_count_dev();
    const int gb = (int)std::min<uint64_t>((nb * 32 + 255) / 256, (uint64_t)sms * 16);
    constexpr bool c64 = sizeof(C) == 8;
    const bool fused = c64 && stats && B == 1024;
    const bool beside = !c64 && stats && B == 1024;
    if (stats && !fused && !beside)
        if (int rc = stats_impl<C>(s, stats, 4)) return rc;
    cudaStream_t st = (cudaStream_t)s->stream, ss = nullptr;
    if (fused || beside)
        if (int rc = ensure_fflog(st)) return rc;
    if (beside)
        if (int rc = side_stream(s, &ss)) return rc;
    const int sgrid = (int)std::min<uint64_t>((N + 255) / 256, (uint64_t)sms * kStatsBlocksPerSM);   // stats_impl's grid
    const size_t stats_bytes = beside ? sizeof(double) * ((size_t)sgrid + 1) * 4 : 0;
    const size_t m_slots = (size_t)std::max<int64_t>(m, 1);
    size_t bytes = sizeof(double) * (2 * nb + 2 * ns) + sizeof(uint64_t) * m_slots;
    if (fused) bytes += sizeof(double) * ((size_t)gb * 4 + 4);
    // complex128 with blocks of 1024: the running sums of every block are
    // stored (N doubles of scratch) and the draws search them; without room
    // for them, the draws scan the block as before (the same outcomes)
    bool search = !c64 && B == 1024 && m > 0;
    void *scr = nullptr;
    int rc = qs_state_scratch(s, bytes + stats_bytes + (search ? sizeof(double) * N : 0), &scr);
    if (rc && search) {
        cudaGetLastError();   // the failed allocation is not an error of the later launches
        search = false;
        rc = qs_state_scratch(s, bytes + stats_bytes, &scr);
    }
    if (rc) return rc;
    // the statistics' partial sums at the end of the scratch
    double *spart = (double *)((char *)scr + bytes + (search ? sizeof(double) * N : 0));
    double *sres = spart + (size_t)sgrid * 4;
    double *P = (double *)scr;                       // probabilities, then running sums
    if (search) scr = (void *)(P + N);
    double *S = (double *)scr, *R = S + nb, *T = R + nb, *Q = T + ns;
    uint64_t *dout = (uint64_t *)(Q + ns);
    double *part = (double *)(dout + m_slots), *res = part + (size_t)gb * 4;
    const C *psi = (const C *)s->amp;
    if (beside) {
        QS_CUDA(cudaEventRecord((cudaEvent_t)s->side_ev[0], st), "side fork");
        QS_CUDA(cudaStreamWaitEvent(ss, (cudaEvent_t)s->side_ev[0], 0), "side fork");
        k_stats_partial<C, 4><<<sgrid, 256, 0, ss>>>(psi, N, spart);
        k_stats_final<4><<<1, 32, 0, ss>>>(spart, sgrid, sres);
        QS_CUDA(cudaGetLastError(), "stats launch");
        QS_CUDA(cudaEventRecord((cudaEvent_t)s->side_ev[1], ss), "side join");
    }
    if (fused) {
        if constexpr (c64) k_segment_sums_stats<C><<<gb, 256, 0, st>>>(psi, nb, S, part);
        k_stats_final<4><<<1, 32, 0, st>>>(part, gb, res);
    } else if (search)
        k_block_sums_store<C><<<gb, 256, 0, st>>>(psi, nb, S, P);
    else if (B == 1024)
        k_segment_sums<C, 32><<<gb, 256, 0, st>>>(psi, nb, (int)B, S);
    else if (B >= 32)
        k_segment_sums<C, 0><<<gb, 256, 0, st>>>(psi, nb, (int)B, S);
    else
        k_segment_sums_small<C><<<1, 32, 0, st>>>(psi, nb, (int)B, S);
    const int gs = (int)std::min<uint64_t>((ns * 32 + 255) / 256, (uint64_t)sms * 16);
    if (G == 1024)
        k_segment_sums<double, 32><<<gs, 256, 0, st>>>(S, ns, (int)G, T);
    else if (G >= 32)
        k_segment_sums<double, 0><<<gs, 256, 0, st>>>(S, ns, (int)G, T);
    else
        k_segment_sums_small<double><<<1, 32, 0, st>>>(S, ns, (int)G, T);
    k_prefix_super<<<1, 1, 0, st>>>(T, ns, Q);
    k_prefix_blocks<<<(int)std::min<uint64_t>((ns + 127) / 128, 1024), 128, 0, st>>>(S, Q, ns, G, R);
    if (search) {
        const int gr = (int)std::min<uint64_t>((nb + kRunThreads - 1) / kRunThreads, (uint64_t)sms * 16);
        k_running_sums<<<gr, kRunThreads, 0, st>>>(P, R, nb);
        k_draw_search<<<(int)std::min<int64_t>((m + 255) / 256, (int64_t)sms * 16), 256, 0, st>>>(
            P, Q, R, ns, G, seed, m, dout);
    } else if (m > 0) {
        k_draw<C><<<(int)std::min<int64_t>((m + 255) / 256, (int64_t)sms * 16), 256, 0, st>>>(
            psi, Q, R, ns, G, B, seed, m, dout);
    }
    QS_CUDA(cudaGetLastError(), "sampling launch");
    if (m > 0)
        QS_CUDA(cudaMemcpyAsync(out, dout, sizeof(uint64_t) * m, cudaMemcpyDeviceToHost, st), "sample copy");
    if (fused)
        QS_CUDA(cudaMemcpyAsync(stats, res, sizeof(double) * 4, cudaMemcpyDeviceToHost, st), "stats copy");
    if (beside) {
        QS_CUDA(cudaStreamWaitEvent(st, (cudaEvent_t)s->side_ev[1], 0), "side join");
        QS_CUDA(cudaMemcpyAsync(stats, sres, sizeof(double) * 4, cudaMemcpyDeviceToHost, st), "stats copy");
    }
    QS_CUDA(cudaStreamSynchronize(st), "sampling sync");
    if (fused || beside) stats[3] *= (double)N;   // mean of (N p)^2 = N sum p^2
    return QS_OK;
}

int make_state(int n, int dtype, void *stream, void *ptr, bool owned, qs_state **out)
{
    qs_state *s = new (std::nothrow) qs_state();
    if (!s) return qs_fail(QS_ENOMEM, "out of host memory");
    s->n = n;
    s->dtype = dtype;
    s->amp = ptr;
    s->owned = owned;
    s->stream = stream;
    cudaGetDevice(&s->device);
    *out = s;
    return QS_OK;
}

}  // namespace

// ---------------------------------------------------------------- internals

int qs_fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int qs_state_scratch(qs_state *s, size_t bytes, void **out)
{
    if (bytes > s->scratch_bytes) {
        if (s->scratch) {
            cudaStreamSynchronize((cudaStream_t)s->stream);
            cudaFree(s->scratch);
            s->scratch = nullptr;
            s->scratch_bytes = 0;
        }
        size_t want = std::max<size_t>(bytes, 1 << 20);
        cudaError_t e = cudaMalloc(&s->scratch, want);
        if (e != cudaSuccess) {
            s->scratch = nullptr;
            return cuda_fail(e, "scratch allocation");
        }
        s->scratch_bytes = want;
    }
    *out = s->scratch;
    return QS_OK;
}

int qs_state_status(qs_state *s, int **out)
{
    if (!s->status) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, 256);
        if (e != cudaSuccess) return cuda_fail(e, "status word");
        e = cudaMemsetAsync(p, 0, 256, (cudaStream_t)s->stream);
        if (e != cudaSuccess) {
            cudaFree(p);
            return cuda_fail(e, "status word");
        }
        s->status = (int *)p;
    }
    *out = s->status;
    return QS_OK;
}

int qs_check_status(qs_state *s)
{
    if (!s->status) return QS_OK;
    int v = 0;
    cudaStream_t st = (cudaStream_t)s->stream;
    QS_CUDA(cudaMemcpyAsync(&v, s->status, sizeof(int), cudaMemcpyDeviceToHost, st), "status read");
    QS_CUDA(cudaStreamSynchronize(st), "status read");
    if (v) {
        cudaMemsetAsync(s->status, 0, sizeof(int), st);
        if (v & 1) return qs_fail(QS_ETIMEOUT, "a kernel's bounded wait ran out (status %d)", v);
        return qs_fail(QS_EINVAL, "amplitudes above ~2^1010 in magnitude: outside the complex128 tensor-core sweep's range");
    }
    return QS_OK;
}

// ------------------------------------------------------------------- C ABI

extern "C" const char *qs_last_error(void) { return g_err; }

extern "C" int qs_alloc(int n, int dtype, void *stream, qs_state **out)
{
    return qs_guard([&]() -> int {
        if (!out || n < 1 || n > QS_MAX_QUBITS || (dtype != QS_C64 && dtype != QS_C128))
            return qs_fail(QS_EINVAL, "qs_alloc: n = %d, dtype = %d not supported", n, dtype);
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, amp_bytes(dtype) << n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return qs_fail(QS_ENOMEM, "qs_alloc: %zu bytes: %s", amp_bytes(dtype) << n, cudaGetErrorString(e));
        }
        int rc = make_state(n, dtype, stream, p, true, out);
        if (rc) cudaFree(p);
        return rc;
    });
}

extern "C" int qs_wrap(void *dev_ptr, int n, int dtype, void *stream, qs_state **out)
{
    return qs_guard([&]() -> int {
        if (!out || !dev_ptr || ((uintptr_t)dev_ptr & 15) || n < 1 || n > QS_MAX_QUBITS ||
            (dtype != QS_C64 && dtype != QS_C128))
            return qs_fail(QS_EINVAL, "qs_wrap: bad pointer, n or dtype");
        return make_state(n, dtype, stream, dev_ptr, false, out);
    });
}

extern "C" void qs_free(qs_state *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize((cudaStream_t)s->stream);
    else cudaDeviceSynchronize();
    if (s->owned && s->amp) cudaFree(s->amp);
    if (s->scratch) cudaFree(s->scratch);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->status) cudaFree(s->status);
    if (s->side) {
        cudaStreamSynchronize((cudaStream_t)s->side);
        cudaStreamDestroy((cudaStream_t)s->side);
    }
    for (void *e : s->side_ev)
        if (e) cudaEventDestroy((cudaEvent_t)e);
    delete s;
}

extern "C" int qs_set_path(qs_state *s, int path)
{
    return qs_guard([&]() -> int {
        if (!s || path < QS_PATH_AUTO || path > QS_PATH_TENSOR) return qs_fail(QS_EINVAL, "qs_set_path");
        s->path = path;
        return QS_OK;
    });
}

extern "C" int qs_set_phase_fold(qs_state *s, int on)
{
    return qs_guard([&]() -> int {
        if (!s) return qs_fail(QS_EINVAL, "qs_set_phase_fold: null state");
        s->fold_phase = on != 0;
        return QS_OK;
    });
}

extern "C" int qs_num_qubits(const qs_state *s) { return s ? s->n : 0; }
extern "C" int qs_dtype(const qs_state *s) { return s ? s->dtype : -1; }
// the caller reads the buffer directly: the zeros outside the support first
extern "C" void *qs_device_ptr(const qs_state *s)
{
    if (!s) return nullptr;
    if (qs_guard([&]() { return qs_order_set(const_cast<qs_state *>(s), nullptr); })) return nullptr;
    if (qs_materialize(const_cast<qs_state *>(s))) return nullptr;
    return s->amp;
}
extern "C" int qs_set_stream(qs_state *s, void *stream)
{
    return qs_guard([&]() -> int {
        if (!s) return qs_fail(QS_EINVAL, "qs_set_stream: null state");
        if (stream != s->stream) {
            // the new stream starts after everything queued on the old one
            cudaEvent_t ev;
            QS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "qs_set_stream: event");
            cudaError_t e = cudaEventRecord(ev, (cudaStream_t)s->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent((cudaStream_t)stream, ev, 0);
            cudaEventDestroy(ev);
            if (e != cudaSuccess) return cuda_fail(e, "qs_set_stream");
        }
        s->stream = stream;
        return QS_OK;
    });
}

// |x>: one amplitude written, the support set to {x}; the zeros elsewhere are
// written by the first call that needs them (qs_materialize), and sweeps on
// the tensor cores never need them (Sec. 3.6 starts from a known state too).
// States on a caller's buffer (qs_wrap) get their zeros at once.
extern "C" int qs_init_basis(qs_state *s, uint64_t x)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp) return qs_fail(QS_EINVAL, "qs_init_basis: null state");
        if (x >> s->n) return qs_fail(QS_EINVAL, "qs_init_basis: index out of range");
        qs_loc_reset(s);   // fresh contents: every qubit at its own bit
        s->perm_invariant = false;
        cudaStream_t st = (cudaStream_t)s->stream;
        if (s->dtype == QS_C128)
            k_set_one<double2><<<1, 1, 0, st>>>((double2 *)s->amp, x);
        else
            k_set_one<float2><<<1, 1, 0, st>>>((float2 *)s->amp, x);
        QS_CUDA(cudaGetLastError(), "qs_init_basis");
        s->sup_free = 0;
        s->sup_fix = x;
        // a wrapped buffer can be read by its owner without a library call: its
        // zeros are written now
        return s->owned ? QS_OK : qs_materialize(s);
    });
}

int qs_basis_move(qs_state *s, uint64_t x)
{
    s->perm_invariant = false;
    cudaStream_t st = (cudaStream_t)s->stream;
    if (s->dtype == QS_C128)
        k_set_one<double2><<<1, 1, 0, st>>>((double2 *)s->amp, x);
    else
        k_set_one<float2><<<1, 1, 0, st>>>((float2 *)s->amp, x);
    QS_CUDA(cudaGetLastError(), "basis move");
    s->sup_free = 0;
    s->sup_fix = x;
    return QS_OK;
}

int qs_materialize(qs_state *s)
{
    if (qs_support_full(s)) return QS_OK;
    const uint64_t N = 1ULL << s->n, all = qs_index_mask(s->n);
    const uint64_t fr = s->sup_free & all, fx = s->sup_fix & ~fr & all;
    int grid = (int)std::min<uint64_t>((N + 255) / 256, (uint64_t)sm_count_dev() * 8);
    cudaStream_t st = (cudaStream_t)s->stream;
    if (s->dtype == QS_C128)
        k_fill_outside<double2><<<grid, 256, 0, st>>>((double2 *)s->amp, N, fr, fx);
    else
        k_fill_outside<float2><<<grid, 256, 0, st>>>((float2 *)s->amp, N, fr, fx);
    QS_CUDA(cudaGetLastError(), "fill outside the support");
    s->sup_free = ~0ULL;
    s->sup_fix = 0;
    return QS_OK;
}

extern "C" int qs_init_uniform(qs_state *s)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp) return qs_fail(QS_EINVAL, "qs_init_uniform: null state");
        qs_loc_reset(s);   // fresh contents: every qubit at its own bit
        uint64_t N = 1ULL << s->n;
        int grid = (int)std::min<uint64_t>((N + 255) / 256, (uint64_t)sm_count_dev() * 8);
        cudaStream_t st = (cudaStream_t)s->stream;
        // 2^{-n/2}: exact power of two for even n; sqrt(0.5) * 2^{-(n-1)/2} for odd n
        double a = (s->n % 2 == 0) ? ldexp(1.0, -s->n / 2) : sqrt(0.5) * ldexp(1.0, -(s->n - 1) / 2);
        if (s->dtype == QS_C128)
            k_fill_uniform<double2, double><<<grid, 256, 0, st>>>((double2 *)s->amp, N, a);
        else
            k_fill_uniform<float2, float><<<grid, 256, 0, st>>>((float2 *)s->amp, N, (float)a);
        QS_CUDA(cudaGetLastError(), "qs_init_uniform");
        s->sup_free = ~0ULL;
        s->sup_fix = 0;
        s->perm_invariant = true;   // every amplitude equal
        return QS_OK;
    });
}

extern "C" int qs_set_amplitudes(qs_state *s, const double *host)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp || !host) return qs_fail(QS_EINVAL, "qs_set_amplitudes: null argument");
        qs_loc_reset(s);   // fresh contents: every qubit at its own bit
        s->perm_invariant = false;
        uint64_t N = 1ULL << s->n;
        cudaStream_t st = (cudaStream_t)s->stream;
        if (s->dtype == QS_C128) {
            QS_CUDA(cudaMemcpyAsync(s->amp, host, 16 * N, cudaMemcpyHostToDevice, st), "qs_set_amplitudes");
        } else {
            // a host copy as large as the state (32 GiB at 32 qubits): no throw
            std::unique_ptr<float[]> f(new (std::nothrow) float[2 * N]);
            if (!f) return qs_fail(QS_ENOMEM, "qs_set_amplitudes: out of host memory");
            for (uint64_t i = 0; i < 2 * N; i++) f[i] = (float)host[i];
            QS_CUDA(cudaMemcpyAsync(s->amp, f.get(), 8 * N, cudaMemcpyHostToDevice, st), "qs_set_amplitudes");
        }
        QS_CUDA(cudaStreamSynchronize(st), "qs_set_amplitudes sync");
        s->sup_free = ~0ULL;
        s->sup_fix = 0;
        return QS_OK;
    });
}

extern "C" int qs_get_amplitudes(qs_state *s, double *host)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp || !host) return qs_fail(QS_EINVAL, "qs_get_amplitudes: null argument");
        if (int rc = qs_check_status(s)) return rc;
        if (int rc = qs_order_set(s, nullptr)) return rc;   // index order
        if (int rc = qs_materialize(s)) return rc;
        uint64_t N = 1ULL << s->n;
        cudaStream_t st = (cudaStream_t)s->stream;
        if (s->dtype == QS_C128) {
            QS_CUDA(cudaMemcpyAsync(host, s->amp, 16 * N, cudaMemcpyDeviceToHost, st), "qs_get_amplitudes");
            QS_CUDA(cudaStreamSynchronize(st), "qs_get_amplitudes sync");
        } else {
            std::unique_ptr<float[]> f(new (std::nothrow) float[2 * N]);
            if (!f) return qs_fail(QS_ENOMEM, "qs_get_amplitudes: out of host memory");
            QS_CUDA(cudaMemcpyAsync(f.get(), s->amp, 8 * N, cudaMemcpyDeviceToHost, st), "qs_get_amplitudes");
            QS_CUDA(cudaStreamSynchronize(st), "qs_get_amplitudes sync");
            for (uint64_t i = 0; i < 2 * N; i++) host[i] = (double)f[i];
        }
        return QS_OK;
    });
}

extern "C" int qs_get_amplitudes_at(qs_state *s, const uint64_t *idx, int64_t count, double *out)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp || count < 0 || (count > 0 && (!idx || !out)))
            return qs_fail(QS_EINVAL, "qs_get_amplitudes_at: bad arguments");
        if (int rc = qs_check_status(s)) return rc;
        if (int rc = qs_materialize(s)) return rc;
        const uint64_t N = 1ULL << s->n;
        cudaStream_t st = (cudaStream_t)s->stream;
        const bool moved = !qs_loc_identity(s);
        for (int64_t j = 0; j < count; j++) {
            if (idx[j] >= N) return qs_fail(QS_EINVAL, "qs_get_amplitudes_at: index %lld out of range", (long long)j);
            // the index in the state's bit order (qubits may sit at other bits)
            const uint64_t at = moved ? qs_loc_index(s, idx[j]) : idx[j];
            if (s->dtype == QS_C128) {
                QS_CUDA(cudaMemcpyAsync(out + 2 * j, (double2 *)s->amp + at, 16, cudaMemcpyDeviceToHost, st),
                        "qs_get_amplitudes_at");
            } else {
                float f[2];
                QS_CUDA(cudaMemcpyAsync(f, (float2 *)s->amp + at, 8, cudaMemcpyDeviceToHost, st), "qs_get_amplitudes_at");
                QS_CUDA(cudaStreamSynchronize(st), "qs_get_amplitudes_at");
                out[2 * j] = f[0];
                out[2 * j + 1] = f[1];
            }
        }
        QS_CUDA(cudaStreamSynchronize(st), "qs_get_amplitudes_at");
        return QS_OK;
    });
}

extern "C" int qs_norm(qs_state *s, double *out)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp || !out) return qs_fail(QS_EINVAL, "qs_norm: null argument");
        if (int rc = qs_check_status(s)) return rc;
        if (int rc = qs_materialize(s)) return rc;
        return s->dtype == QS_C128 ? stats_impl<double2>(s, out, 1) : stats_impl<float2>(s, out, 1);
    });
}

extern "C" int qs_stats(qs_state *s, double out[4])
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp || !out) return qs_fail(QS_EINVAL, "qs_stats: null argument");
        if (int rc = qs_check_status(s)) return rc;
        if (int rc = qs_materialize(s)) return rc;
        return s->dtype == QS_C128 ? stats_impl<double2>(s, out, 4) : stats_impl<float2>(s, out, 4);
    });
}

extern "C" int qs_probabilities(qs_state *s, double *out, int out_on_device)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp || !out) return qs_fail(QS_EINVAL, "qs_probabilities: null argument");
        if (int rc = qs_order_set(s, nullptr)) return rc;   // index order
        if (int rc = qs_materialize(s)) return rc;
        const uint64_t N = 1ULL << s->n;
        cudaStream_t st = (cudaStream_t)s->stream;
        const int sms = sm_count_dev();
        auto launch = [&](uint64_t first, uint64_t count, double *dst) {
            int grid = (int)std::min<uint64_t>((count + 255) / 256, (uint64_t)sms * 8);
            if (s->dtype == QS_C128)
                k_probs<double2><<<grid, 256, 0, st>>>((const double2 *)s->amp, first, count, dst);
            else
                k_probs<float2><<<grid, 256, 0, st>>>((const float2 *)s->amp, first, count, dst);
        };
        if (out_on_device) {
            launch(0, N, out);
            QS_CUDA(cudaGetLastError(), "qs_probabilities");
            return QS_OK;
        }
        // host output: chunks of at most 2^25 values through the scratch buffer
        const uint64_t chunk = std::min<uint64_t>(N, 1ULL << 25);
        void *scr = nullptr;
        int rc = qs_state_scratch(s, sizeof(double) * chunk, &scr);
        if (rc) return rc;
        for (uint64_t first = 0; first < N; first += chunk) {
            launch(first, chunk, (double *)scr);
            QS_CUDA(cudaGetLastError(), "qs_probabilities");
            QS_CUDA(cudaMemcpyAsync(out + first, scr, sizeof(double) * chunk, cudaMemcpyDeviceToHost, st),
                    "qs_probabilities copy");
        }
        QS_CUDA(cudaStreamSynchronize(st), "qs_probabilities sync");
        return QS_OK;
    });
}

extern "C" int qs_sample(qs_state *s, uint64_t seed, int64_t m, uint64_t *out)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp || m < 0 || (m > 0 && !out)) return qs_fail(QS_EINVAL, "qs_sample: bad arguments");
        if (int rc = qs_order_set(s, nullptr)) return rc;   // index order
        if (int rc = qs_materialize(s)) return rc;
        return s->dtype == QS_C128 ? sample_impl<double2>(s, seed, m, out, nullptr)
                                   : sample_impl<float2>(s, seed, m, out, nullptr);
    });
}

extern "C" int qs_sample_stats(qs_state *s, uint64_t seed, int64_t m, uint64_t *out, double *stats)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp || m < 0 || (m > 0 && !out) || !stats)
            return qs_fail(QS_EINVAL, "qs_sample_stats: bad arguments");
        if (int rc = qs_check_status(s)) return rc;
        if (int rc = qs_order_set(s, nullptr)) return rc;   // index order
        if (int rc = qs_materialize(s)) return rc;
        return s->dtype == QS_C128 ? sample_impl<double2>(s, seed, m, out, stats)
                                   : sample_impl<float2>(s, seed, m, out, stats);
    });
}

extern "C" int qs_synchronize(qs_state *s)
{
    return qs_guard([&]() -> int {
        if (!s) return qs_fail(QS_EINVAL, "qs_synchronize: null state");
        QS_CUDA(cudaStreamSynchronize((cudaStream_t)s->stream), "qs_synchronize");
        return qs_check_status(s);
    });
}

extern "C" int qs_selftest_timeout(qs_state *s)
{
    return qs_guard([&]() -> int {
        if (!s) return qs_fail(QS_EINVAL, "qs_selftest_timeout: null state");
        int rc = qs_launch_wait_selftest(s, 1000);
        if (rc) return rc;
        QS_CUDA(cudaStreamSynchronize((cudaStream_t)s->stream), "qs_selftest_timeout");
        return qs_check_status(s);
    });
}

// --------------------------------------------------------------------------
// Allocation-free statistics (no counterpart in the paper).
//
// For callers that must not allocate device memory: the partial sums live in a
// file-scope device array instead of the state's scratch.  Every call shares
// it, so calls whose kernels overlap on the GPU race on it.
// --------------------------------------------------------------------------
namespace {

constexpr int kStaticStatsBlocks = 1024;   // partial sums per statistic
// 4 statistics per block, plus 4 result slots: 4 * 1025 doubles = 32800 bytes.
static __device__ __align__(256) double g_stats_scratch[4 * (kStaticStatsBlocks + 1)];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double *g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_stats_scratch on the current device (looked up once per
// device, with that device current).
int static_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "qs_stats_static: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return qs_fail(QS_EUNSUPPORTED, "qs_stats_static: device %d", dev);
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_stats_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "qs_stats_static: cudaGetSymbolAddress");
        g_static_ptr[dev] = (double *)p;
    }
    *out = g_static_ptr[dev];
    return QS_OK;
}

template <typename C>
int stats_static_impl(const void *amp, int n, void *stream, double *out)
{
    double *scr;
    int rc = static_scratch(&scr);
    if (rc) return rc;
    const uint64_t N = 1ULL << n;
    const int block = 256;
    int grid = (int)std::min<uint64_t>((N + block - 1) / block, (uint64_t)sm_count_dev() * 4);
    grid = std::min(grid, kStaticStatsBlocks);
    double *part = scr, *res = scr + 4 * kStaticStatsBlocks;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ensure_fflog(st))) return rc;
    // every partial slot in [0, grid) and every result slot is written before it is read
    k_stats_partial<C, 4><<<grid, block, 0, st>>>((const C *)amp, N, part);
    k_stats_final<4><<<1, 32, 0, st>>>(part, grid, res);
    QS_CUDA(cudaGetLastError(), "qs_stats_static launch");
    QS_CUDA(cudaMemcpyAsync(out, res, sizeof(double) * 4, cudaMemcpyDeviceToHost, st), "qs_stats_static copy");
    QS_CUDA(cudaStreamSynchronize(st), "qs_stats_static sync");
    out[3] *= (double)N;   // mean of (N p)^2 = N sum p^2
    return QS_OK;
}

}  // namespace

extern "C" int qs_stats_static(const void *dev_amp, int n, int dtype, void *stream, double out[4])
{
    return qs_guard([&]() -> int {
        if (!dev_amp || !out) return qs_fail(QS_EINVAL, "qs_stats_static: null pointer");
        if (n < 1 || n > QS_MAX_QUBITS)
            return qs_fail(QS_EINVAL, "qs_stats_static: n = %d outside [1, %d]", n, QS_MAX_QUBITS);
        if (dtype != QS_C64 && dtype != QS_C128)
            return qs_fail(QS_EINVAL, "qs_stats_static: dtype %d", dtype);
        // the kernel loads whole amplitudes: aligned to their size
        if ((uintptr_t)dev_amp & (amp_bytes(dtype) - 1))
            return qs_fail(QS_EINVAL, "qs_stats_static: pointer not aligned to %zu bytes", amp_bytes(dtype));
        return dtype == QS_C128 ? stats_static_impl<double2>(dev_amp, n, stream, out)
                                : stats_static_impl<float2>(dev_amp, n, stream, out);
    });
}

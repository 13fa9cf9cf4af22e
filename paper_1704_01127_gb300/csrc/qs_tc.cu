// Tensor-core sweep for 5-qubit clusters (Sec. 3.2 with k = 5; the 2^{n-5}
// mat-vecs of one cluster form a dense GEMM).
//
// A tile of 128 groups is the matrix A[128 x 64]: row r holds the 32 complex
// amplitudes of group r as 64 reals (re, im interleaved, member x at columns
// 2x, 2x+1).  The cluster unitary in real form is B^T[64 x 64] with
//   B^T[2l][2x] = Re U[l][x],  B^T[2l][2x+1] = -Im U[l][x],
//   B^T[2l+1][2x] = Im U[l][x], B^T[2l+1][2x+1] = Re U[l][x],
// so D = A B (D[r][2l], D[r][2l+1] = Re, Im of (U v_r)_l) is the updated tile.
//
// complex64: every real is split into a tf32 head and a tf32 tail,
// a ~ a_h + a_t (a_h: a with its low 13 mantissa bits cleared, a_t: the rest
// rounded to the nearest tf32, so the split is unbiased), and
// D = A_h B_h + A_h B_t + A_t B_h accumulates in FP32 in tensor memory
// (tcgen05.mma kind::tf32, M = 128, N = 64, K = 8 per instruction).
//
// Operands sit in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, core matrices adjacent along K 128 B
// apart (leading byte offset), 8-row groups 2048 B apart (stride byte offset).
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "qs_internal.h"

namespace {

constexpr int kRows = 128;          // groups per tile (MMA M)
constexpr int kK = 64;              // reals per group (MMA K)
constexpr int kN = 64;              // output reals per group (MMA N)
constexpr uint32_t kLBO = 128;      // bytes between K-adjacent core matrices
constexpr uint32_t kSBO = 2048;     // bytes between 8-row groups (16 core matrices)
constexpr int kTmemCols = 64;
constexpr long kWaitLimit = 1L << 24;   // bounded mbarrier polling

// byte offset of fp32 element (row, k) in a K-major no-swizzle tile with 64 K
__host__ __device__ __forceinline__ uint32_t cm_off(int row, int k)
{
    return (uint32_t)((((row >> 3) * (kK / 4)) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor (tcgen05): start >> 4, LBO >> 4, SBO >> 4,
// version 1 at bit 46, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: D fp32 (bits 4-5 = 1), A/B tf32 (bits 7-9, 10-12 = 2),
// both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kN >> 3) << 17) |
                               ((uint32_t)(kRows >> 4) << 24);

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 16 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld()
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float tf32_head(float x)
{
    return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}
// the tail rounded to the nearest tf32 (the MMA would otherwise truncate it,
// which biases every sweep towards zero)
__device__ __forceinline__ float tf32_round(float x)
{
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

struct Targets5 {
    int q[5];
};

__device__ __forceinline__ uint64_t base5(uint64_t g, const Targets5 &t)
{
#pragma unroll
    for (int j = 0; j < 5; j++) {
        uint64_t lo = g & ((1ULL << t.q[j]) - 1);
        g = ((g ^ lo) << 1) | lo;
    }
    return g;
}

__device__ __forceinline__ uint64_t off5(int x, const Targets5 &t)
{
    uint64_t o = 0;
#pragma unroll
    for (int j = 0; j < 5; j++)
        if ((x >> j) & 1) o |= 1ULL << t.q[j];
    return o;
}

constexpr size_t kTileBytesF32 = (size_t)kRows * kK * 4;   // 32 KB
constexpr size_t kBBytesF32 = (size_t)kN * kK * 4;         // 16 KB
constexpr size_t kSmemF32 = 2 * kTileBytesF32 + 2 * kBBytesF32;

// One CTA of 128 threads; thread r owns row r (group) of each tile.  Tiles are
// taken in a grid-stride loop; warp 0 holds 64 TMEM columns for the CTA.
__global__ void __launch_bounds__(128, 2)
k_dense5_tc_c64(float2 *__restrict__ psi, uint64_t n_groups, Targets5 t, const float *__restrict__ bpack,
                int *__restrict__ status)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *A_h = smem;
    uint8_t *A_t = smem + kTileBytesF32;
    uint8_t *B_h = smem + 2 * kTileBytesF32;
    uint8_t *B_t = B_h + kBBytesF32;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base_s;

    const int tid = threadIdx.x, warp = tid >> 5;
    {
        const float4 *src = reinterpret_cast<const float4 *>(bpack);
        float4 *dst = reinterpret_cast<float4 *>(B_h);
        for (int i = tid; i < (int)(2 * kBBytesF32 / 16); i += blockDim.x) dst[i] = src[i];
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(&tmem_base_s), kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(smem_u32(&mbar), 1);
        fence_mbar_init();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const uint32_t mbar_a = smem_u32(&mbar);
    const uint32_t a_h = smem_u32(A_h), a_t = smem_u32(A_t), b_h = smem_u32(B_h), b_t = smem_u32(B_t);

    const uint64_t n_tiles = (n_groups + kRows - 1) / kRows;
    uint32_t parity = 0;
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint64_t g = tile * kRows + tid;
        const bool valid = g < n_groups;
        float2 *p = psi + (valid ? base5(g, t) : 0);
        // gather + split: members 2c and 2c+1 fill K columns 4c..4c+3
#pragma unroll
        for (int c = 0; c < 16; c++) {
            float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
            if (valid) {
                v0 = p[off5(2 * c, t)];
                v1 = p[off5(2 * c + 1, t)];
            }
            float4 h = make_float4(tf32_head(v0.x), tf32_head(v0.y), tf32_head(v1.x), tf32_head(v1.y));
            float4 tl = make_float4(tf32_round(v0.x - h.x), tf32_round(v0.y - h.y), tf32_round(v1.x - h.z),
                                    tf32_round(v1.y - h.w));
            *reinterpret_cast<float4 *>(A_h + cm_off(tid, 4 * c)) = h;
            *reinterpret_cast<float4 *>(A_t + cm_off(tid, 4 * c)) = tl;
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int ks = 0; ks < kK / 8; ks++) {
                const uint32_t koff = ks * 2 * kLBO;   // 8 tf32 = two core matrices along K
                mma_tf32(tmem, smem_desc(a_h + koff), smem_desc(b_h + koff), kIdescTf32, ks > 0);
                mma_tf32(tmem, smem_desc(a_h + koff), smem_desc(b_t + koff), kIdescTf32, 1);
                mma_tf32(tmem, smem_desc(a_t + koff), smem_desc(b_h + koff), kIdescTf32, 1);
            }
            mma_commit(mbar_a);
        }
        bool ok = false;
        for (long it = 0; it < kWaitLimit; it++)
            if (mbar_try_wait(mbar_a, parity)) {
                ok = true;
                break;
            }
        if (__syncthreads_or(!ok)) {
            // the MMAs did not complete in time: flag it, give them one more
            // bounded wait, and leave (TMEM is released below)
            if (tid == 0) {
                atomicExch(status, 1);
                for (long it = 0; it < kWaitLimit; it++)
                    if (mbar_try_wait(mbar_a, parity)) break;
            }
            break;
        }
        parity ^= 1;
        tc_fence_after();
        float r[kN];
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int c = 0; c < kN / 16; c++) tmem_ld16(lane_addr + c * 16, r + c * 16);
        tmem_wait_ld();
        if (valid) {
#pragma unroll
            for (int l = 0; l < 32; l++) p[off5(l, t)] = make_float2(r[2 * l], r[2 * l + 1]);
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

bool g_attr_set[64] = {false};

}  // namespace

// Host: real form of a sorted 32x32 complex matrix (interleaved FP64), split
// into tf32 head and fp32 tail, both in the canonical K-major layout.
std::vector<uint8_t> qs_pack_tc_c64(const std::vector<double> &M)
{
    std::vector<uint8_t> out(2 * kBBytesF32, 0);
    float *bh = reinterpret_cast<float *>(out.data());
    float *bt = reinterpret_cast<float *>(out.data() + kBBytesF32);
    auto put = [&](int n, int k, double v) {
        float f = (float)v;
        uint32_t u;
        std::memcpy(&u, &f, 4);
        u &= 0xFFFFE000u;
        float h;
        std::memcpy(&h, &u, 4);
        bh[cm_off(n, k) / 4] = h;
        float tail = (float)(v - (double)h);
        std::memcpy(&u, &tail, 4);
        u = (u + 0x1000u) & 0xFFFFE000u;   // nearest tf32
        std::memcpy(&tail, &u, 4);
        bt[cm_off(n, k) / 4] = tail;
    };
    for (int l = 0; l < 32; l++)
        for (int x = 0; x < 32; x++) {
            double re = M[2 * (l * 32 + x)], im = M[2 * (l * 32 + x) + 1];
            put(2 * l, 2 * x, re);
            put(2 * l, 2 * x + 1, -im);
            put(2 * l + 1, 2 * x, im);
            put(2 * l + 1, 2 * x + 1, re);
        }
    return out;
}

size_t qs_tc_pack_bytes(int dtype) { return dtype == QS_C64 ? 2 * kBBytesF32 : 0; }

int qs_launch_dense5_tc(qs_state *s, const int *sorted_qubits, const void *dev_pack)
{
    if (s->dtype != QS_C64) return qs_fail(QS_EUNSUPPORTED, "tensor-core sweep: complex64 only");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dev >= 0 && dev < 64 && !g_attr_set[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_dense5_tc_c64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemF32);
        if (e != cudaSuccess) return qs_fail(QS_ECUDA, "tc smem attribute: %s", cudaGetErrorString(e));
        g_attr_set[dev] = true;
    }
    Targets5 t;
    for (int j = 0; j < 5; j++) t.q[j] = sorted_qubits[j];
    const uint64_t groups = 1ULL << (s->n - 5);
    const uint64_t tiles = (groups + kRows - 1) / kRows;
    int grid = (int)std::min<uint64_t>(tiles, (uint64_t)sms * 2);
    int *status;
    int rc = qs_state_status(s, &status);
    if (rc) return rc;
    k_dense5_tc_c64<<<grid, kRows, kSmemF32, (cudaStream_t)s->stream>>>(
        (float2 *)s->amp, groups, t, (const float *)dev_pack, status);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "tc launch: %s", cudaGetErrorString(e));
}

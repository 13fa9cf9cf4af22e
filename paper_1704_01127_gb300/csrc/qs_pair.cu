// Two consecutive 5-qubit clusters in one sweep over a complex64 state: the
// GPU form of the paper's blocking, which applies several gates while a chunk
// of the state sits in fast memory (Fig. 2 caption; Sec. 4).
//
// With U = T1 u T2 the union of the two clusters' target qubits (u = |U| <= 10
// bits), the 2^u amplitudes that agree outside U form a super-group; both
// clusters act inside it (2^{u-5} groups each).  A tile is 4096 amplitudes,
// 2^{12-u} super-groups: 128 groups for either cluster, the M = 128 rows of
// one tensor-core product.  Per tile:
//   phase 1: thread r gathers group r of cluster 1 from HBM, the tile goes
//     through the same tf32 head/tail product as the one-cluster sweep
//     (qs_tc.cu), and the outputs land in a shared-memory copy X of the tile;
//   phase 2: thread r gathers group r of cluster 2 from X, the product with
//     cluster 2's operands runs, and the outputs are stored to HBM (with a
//     folded phase op, as in the one-cluster sweep).
// The state is read and written once for both clusters.  The numerics are
// those of two one-cluster sweeps: cluster 1's outputs are rounded to float
// before cluster 2 reads them, exactly as when they go through HBM.
//
// A CTA of 256 threads runs two independent sub-tiles of 128 threads (each
// with its own operand/X region, TMEM columns, mbarrier and named barrier),
// sharing the two clusters' operands; one CTA per SM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "qs_internal.h"
#include "qs_tcgen05.cuh"

namespace {

constexpr int kSub = 2;                                      // sub-tiles per CTA
constexpr int kPairThreads = kSub * kRows;                   // 256
constexpr size_t kPlaneF32 = (size_t)kRows * kK * 4;         // 32 KB: A head or tail
constexpr size_t kBPack = 2 * (size_t)kN * kK * 4;           // 32 KB: one cluster's head + tail
constexpr size_t kRegion = 2 * kPlaneF32;                    // per sub-tile: A head + tail (X aliases it)
constexpr size_t kSmemPair = 2 * kBPack + kSub * kRegion;    // 192 KB

// Where a super-group's amplitudes sit: local index l (u bits, U's qubits in
// ascending order) is at offset off_lo[l & 31] + off_hi[l >> 5] from the
// super-group's first amplitude; member m of group c of cluster j has local
// index grp[j][c] | mem[j][m].
struct PairLayout {
    uint64_t zmask;              // U's bits: zeros inserted there for a super-group's base
    uint64_t off_lo[32], off_hi[32];
    uint16_t mem[2][32], grp[2][32];
    int u;                       // |U|
};

struct PairSmem {
    uint64_t off_lo[32], off_hi[32];
    uint16_t mem[2][32], grp[2][32];
};

__device__ __forceinline__ uint64_t sg_base(uint64_t g, uint64_t zmask)
{
    for (uint64_t z = zmask; z; z &= z - 1) {
        const uint64_t lo = g & ((z & (0 - z)) - 1);
        g = ((g ^ lo) << 1) | lo;
    }
    return g;
}

// Slot of tile element i in X: the low four bits are mixed with a hash of the
// others (a bijection on 12-bit indices), so that the lanes of a warp, whose
// indices differ in the clusters' non-target bits, spread over the shared
// memory banks instead of landing on one.
__device__ __forceinline__ uint32_t xslot(uint32_t i)
{
    return i ^ (((i >> 4) * 0x9E3779B1u) >> 28);
}

__device__ __forceinline__ void bar_sub(int sub)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + sub), "r"(kRows) : "memory");
}
__device__ __forceinline__ bool bar_sub_or(int sub, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + sub), "r"(kRows)
        : "memory");
    return r != 0;
}

// tf32 head/tail split of one row's 32 members into the A planes
__device__ __forceinline__ void split_row(const float2 *v, uint8_t *A_h, uint8_t *A_t, int row)
{
#pragma unroll
    for (int c = 0; c < 16; c++) {
        const float2 v0 = v[2 * c], v1 = v[2 * c + 1];
        const float4 h = make_float4(tf32_head(v0.x), tf32_head(v0.y), tf32_head(v1.x), tf32_head(v1.y));
        const float4 tl = make_float4(tf32_round(v0.x - h.x), tf32_round(v0.y - h.y), tf32_round(v1.x - h.z),
                                      tf32_round(v1.y - h.w));
        *reinterpret_cast<float4 *>(A_h + cm_off(row, 4 * c)) = h;
        *reinterpret_cast<float4 *>(A_t + cm_off(row, 4 * c)) = tl;
    }
}

// head product and the two correction products, K = 64 in 8 steps
__device__ __forceinline__ void issue_pair_mma(uint32_t tmem, uint32_t a_h, uint32_t a_t, uint32_t b_h, uint32_t b_t)
{
#pragma unroll
    for (int ks = 0; ks < kK / 8; ks++) {
        const uint32_t koff = ks * 2 * kLBO;
        mma_tf32(tmem, smem_desc(a_h + koff), smem_desc(b_h + koff), kIdescTf32, ks > 0);
        mma_tf32(tmem + kN, smem_desc(a_h + koff), smem_desc(b_t + koff), kIdescTf32, ks > 0);
        mma_tf32(tmem + kN, smem_desc(a_t + koff), smem_desc(b_h + koff), kIdescTf32, 1);
    }
}

}  // namespace

namespace {

template <bool kPost>
__global__ void __launch_bounds__(kPairThreads, 1)
k_pair5_tc_c64(float2 *__restrict__ psi, uint64_t n_tiles, PairLayout lay, const float *__restrict__ pack1,
               const float *__restrict__ pack2, const qs_post_phase *__restrict__ post, int *__restrict__ status)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *B1 = smem, *B2 = smem + kBPack;
    __shared__ __align__(8) uint64_t mbar[kSub];
    __shared__ uint32_t tmem_base_s;
    __shared__ PairSmem ts;
    __shared__ PostSmem ps;

    const int tid = threadIdx.x, warp = tid >> 5, sub = tid >> 7, row = tid & (kRows - 1);
    {
        const float4 *s1 = reinterpret_cast<const float4 *>(pack1), *s2 = reinterpret_cast<const float4 *>(pack2);
        float4 *d1 = reinterpret_cast<float4 *>(B1), *d2 = reinterpret_cast<float4 *>(B2);
        for (int i = tid; i < (int)(kBPack / 16); i += blockDim.x) {
            d1[i] = s1[i];
            d2[i] = s2[i];
        }
        if (tid < 32) {
            ts.off_lo[tid] = lay.off_lo[tid];
            ts.off_hi[tid] = lay.off_hi[tid];
            for (int j = 0; j < 2; j++) {
                ts.mem[j][tid] = lay.mem[j][tid];
                ts.grp[j][tid] = lay.grp[j][tid];
            }
        }
        if constexpr (kPost) post_load(ps, post, tid, blockDim.x);
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(&tmem_base_s), kSub * kTmemCols);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < kSub; s++) mbar_init(smem_u32(&mbar[s]), 1);
        fence_mbar_init();
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const uint32_t tmem = tmem_base_s + (uint32_t)(sub * kTmemCols);
    const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    uint8_t *A_h = smem + 2 * kBPack + sub * kRegion, *A_t = A_h + kPlaneF32;
    float2 *X = reinterpret_cast<float2 *>(A_h);   // the tile between the two clusters
    const uint32_t a_h = smem_u32(A_h), a_t = smem_u32(A_t);
    const uint32_t b1h = smem_u32(B1), b1t = b1h + (uint32_t)(kBPack / 2);
    const uint32_t b2h = smem_u32(B2), b2t = b2h + (uint32_t)(kBPack / 2);
    const uint32_t mb = smem_u32(&mbar[sub]);
    const int gbits = lay.u - 5;
    // neighbouring rows take neighbouring super-groups (the lowest bits off
    // U), then the groups inside one
    const int sgl = row & ((1 << (7 - gbits)) - 1), grow = row >> (7 - gbits);
    const uint64_t per_tile = 1ULL << (12 - lay.u);
    const uint32_t xrow = (uint32_t)sgl << lay.u;
    const uint32_t g1 = ts.grp[0][grow], g2 = ts.grp[1][grow];
    auto off = [&](uint32_t l) { return ts.off_lo[l & 31] + ts.off_hi[l >> 5]; };

    uint32_t parity = 0;
    bool failed = false;
    // wait for this sub-tile's MMAs; on expiry flag it, give them one more
    // bounded wait, and leave
    auto wait_mma = [&]() -> bool {
        bool ok = false;
        for (long it = 0; it < kWaitLimit; it++)
            if (mbar_try_wait(mb, parity)) {
                ok = true;
                break;
            }
        if (bar_sub_or(sub, !ok)) {
            if (row == 0) {
                atomicExch(status, 1);
                for (long it = 0; it < kWaitLimit; it++)
                    if (mbar_try_wait(mb, parity)) break;
            }
            return false;
        }
        parity ^= 1;
        tc_fence_after();
        return true;
    };
    // head + corrections of output member m from TMEM (16 columns at a time)
    auto read_out = [&](float2 *o) {
#pragma unroll
        for (int c = 0; c < kN / 16; c++) {
            float r[16], q[16];
            tmem_ld16(lane_addr + c * 16, r);
            tmem_ld16(lane_addr + kN + c * 16, q);
            tmem_wait_ld();
#pragma unroll
            for (int l = 0; l < 8; l++) o[8 * c + l] = make_float2(r[2 * l] + q[2 * l], r[2 * l + 1] + q[2 * l + 1]);
        }
    };

    float2 v[32];
    uint64_t tile = (uint64_t)blockIdx.x * kSub + sub;
    const uint64_t tstride = (uint64_t)gridDim.x * kSub;
    auto load1 = [&](uint64_t tl) {
        if (tl < n_tiles) {
            const uint64_t base = sg_base(tl * per_tile + sgl, lay.zmask);
#pragma unroll
            for (int m = 0; m < 32; m++) v[m] = psi[base + off(g1 | ts.mem[0][m])];
        }
    };
    load1(tile);
    for (; tile < n_tiles && !failed; tile += tstride) {
        const uint64_t base = sg_base(tile * per_tile + sgl, lay.zmask);
        // ---- phase 1: cluster 1 from the registers
        split_row(v, A_h, A_t, row);
        fence_proxy_async();
        tc_fence_before();
        bar_sub(sub);
        tc_fence_after();
        if (row == 0) {
            issue_pair_mma(tmem, a_h, a_t, b1h, b1t);
            mma_commit(mb);
        }
        if (!wait_mma()) {
            failed = true;
            break;
        }
        read_out(v);
        tc_fence_before();
        bar_sub(sub);   // every thread has read A's products out of TMEM; the MMAs are done with A
#pragma unroll
        for (int m = 0; m < 32; m++) X[xslot(xrow | g1 | ts.mem[0][m])] = v[m];
        bar_sub(sub);
        // ---- phase 2: cluster 2 from the shared-memory tile
#pragma unroll
        for (int m = 0; m < 32; m++) v[m] = X[xslot(xrow | g2 | ts.mem[1][m])];
        bar_sub(sub);   // X read before the planes overwrite it
        split_row(v, A_h, A_t, row);
        fence_proxy_async();
        tc_fence_before();
        bar_sub(sub);
        tc_fence_after();
        if (row == 0) {
            issue_pair_mma(tmem, a_h, a_t, b2h, b2t);
            mma_commit(mb);
        }
        float2 o[32];
        load1(tile + tstride);   // the next tile's cluster-1 groups while the MMAs run
        if (!wait_mma()) {
            failed = true;
            break;
        }
        read_out(o);
        const uint64_t b2 = base + off(g2);
        uint32_t pe = 0, pf = 0;
        if constexpr (kPost) post_row(ps, b2, pe, pf);
#pragma unroll
        for (int m = 0; m < 32; m++) {
            float2 w = o[m];
            if constexpr (kPost) w = rot_i(w, post_member(pe, pf, m));
            psi[base + off(g2 | ts.mem[1][m])] = w;
        }
        tc_fence_before();
        bar_sub(sub);   // TMEM read out before the next tile's products
        tc_fence_after();
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem_base_s, kSub * kTmemCols);
}

bool g_pair_attr[2][64] = {};   // [folded phase][device]

}  // namespace

bool qs_pair_possible(const qs_state *s, const int *q1, const int *q2)
{
    if (s->dtype != QS_C64 || s->n < 12 || !qs_support_full(s)) return false;
    uint64_t u = 0;
    for (int j = 0; j < 5; j++) u |= (1ULL << q1[j]) | (1ULL << q2[j]);
    return __builtin_popcountll(u) <= 10;
}

int qs_launch_pair5_tc(qs_state *s, const int *q1, const void *pack1, const int *q2, const void *pack2,
                       const void *dev_post)
{
    s->perm_invariant = false;
    if (!qs_pair_possible(s, q1, q2)) return qs_fail(QS_EINVAL, "pair sweep: not applicable");
    PairLayout lay;
    std::memset(&lay, 0, sizeof(lay));
    int U[10], u = 0;
    uint64_t um = 0;
    for (int j = 0; j < 5; j++) um |= (1ULL << q1[j]) | (1ULL << q2[j]);
    for (int b = 0; b < s->n; b++)
        if ((um >> b) & 1) U[u++] = b;
    lay.u = u;
    lay.zmask = um;
    for (int x = 0; x < 32; x++) {
        for (int j = 0; j < 5 && j < u; j++)
            if ((x >> j) & 1) lay.off_lo[x] |= 1ULL << U[j];
        for (int j = 0; j < 5 && 5 + j < u; j++)
            if ((x >> j) & 1) lay.off_hi[x] |= 1ULL << U[5 + j];
    }
    const int *qs[2] = {q1, q2};
    for (int c = 0; c < 2; c++) {
        int tpos[5], lpos[5], nl = 0;
        for (int i = 0; i < u; i++) {
            int j = -1;
            for (int t = 0; t < 5; t++)
                if (qs[c][t] == U[i]) j = t;
            if (j >= 0) tpos[j] = i;       // targets come sorted: member bit j <-> local position
            else lpos[nl++] = i;
        }
        for (int m = 0; m < 32; m++) {
            uint32_t l = 0;
            for (int j = 0; j < 5; j++)
                if ((m >> j) & 1) l |= 1u << tpos[j];
            lay.mem[c][m] = (uint16_t)l;
        }
        for (int g = 0; g < (1 << nl); g++) {
            uint32_t l = 0;
            for (int i = 0; i < nl; i++)
                if ((g >> i) & 1) l |= 1u << lpos[i];
            lay.grp[c][g] = (uint16_t)l;
        }
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dev < 0 || dev >= 64) return qs_fail(QS_EUNSUPPORTED, "device %d", dev);
    const bool fold = dev_post != nullptr;
    if (!g_pair_attr[fold][dev]) {
        const void *fn = fold ? (const void *)k_pair5_tc_c64<true> : (const void *)k_pair5_tc_c64<false>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemPair);
        if (e != cudaSuccess) return qs_fail(QS_ECUDA, "pair smem attribute: %s", cudaGetErrorString(e));
        g_pair_attr[fold][dev] = true;
    }
    int *status;
    int rc = qs_state_status(s, &status);
    if (rc) return rc;
    const uint64_t n_tiles = 1ULL << (s->n - 12);
    const int grid = (int)std::min<uint64_t>((n_tiles + kSub - 1) / kSub, (uint64_t)sms);
    cudaStream_t st = (cudaStream_t)s->stream;
    const qs_post_phase *post = (const qs_post_phase *)dev_post;
    if (fold)
        k_pair5_tc_c64<true><<<grid, kPairThreads, kSmemPair, st>>>((float2 *)s->amp, n_tiles, lay,
                                                                   (const float *)pack1, (const float *)pack2,
                                                                   post, status);
    else
        k_pair5_tc_c64<false><<<grid, kPairThreads, kSmemPair, st>>>((float2 *)s->amp, n_tiles, lay,
                                                                    (const float *)pack1, (const float *)pack2,
                                                                    post, status);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "pair launch: %s", cudaGetErrorString(e));
}

// tcgen05 / mbarrier helpers and the tile layout shared by the tensor-core
// sweeps (qs_tc.cu: one 5-qubit cluster per sweep; qs_pair.cu: two clusters
// per sweep).  Inline PTX for sm_103a.  Everything sits in an unnamed
// namespace: each translation unit that includes this file gets its own copy.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "qs_internal.h"

namespace {

constexpr int kRows = 128;          // groups per tile (MMA M)
constexpr int kK = 64;              // reals per group (MMA K)
constexpr int kN = 64;              // output reals per group (MMA N)
constexpr uint32_t kLBO = 128;      // bytes between K-adjacent core matrices
constexpr uint32_t kSBO = 2048;     // bytes between 8-row groups (16 core matrices)
constexpr int kTmemCols = 128;     // complex64: head product and correction terms
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
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo = kSBO)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
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
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
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
// 4 consecutive 32-bit columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float *v)
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 4; i++) v[i] = __uint_as_float(r[i]);
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

// Where the members of a group sit for one 5-qubit sweep over the state's
// support (the indices that may hold nonzero amplitudes): group g's x = 0
// member is g with zeros inserted at the positions of zmask (the five targets
// and the support's fixed bits) and the fixed bits' values OR-ed in; member x
// adds the target bits of x.  Bit x of mmask is set when member x lies in the
// support before the sweep; the others are zero and are not read.  With the
// full support (full = 1): zeros at the targets only, fix = 0, every member
// read.  No arrays: an indexed parameter array would be copied to local memory.
struct TileLayout {
    int q[5];
    int full;
    uint32_t mmask;
    uint64_t fix;
    uint64_t zmask;
    int pairs;   // complex64: qubit 0 is a target and the buffer 16-byte aligned
};

__device__ __forceinline__ uint64_t tile_base(uint64_t g, const TileLayout &t)
{
    if (t.full) {
#pragma unroll
        for (int j = 0; j < 5; j++) {
            const uint64_t lo = g & ((1ULL << t.q[j]) - 1);
            g = ((g ^ lo) << 1) | lo;
        }
        return g;
    }
    for (uint64_t z = t.zmask; z; z &= z - 1) {
        const uint64_t lo = g & ((z & (0 - z)) - 1);      // bits below the lowest zero position
        g = ((g ^ lo) << 1) | lo;
    }
    return g | t.fix;
}

__device__ __forceinline__ uint64_t off5(int x, const TileLayout &t)
{
    uint64_t o = 0;
#pragma unroll
    for (int j = 0; j < 5; j++)
        if ((x >> j) & 1) o |= 1ULL << t.q[j];
    return o;
}

// A phase op folded into the sweep (qs_post_phase), copied to shared memory.
struct PostSmem {
    uint64_t c1, c2, tp[5];
    uint64_t part[QS_MAX_POST_TERMS];
    int a[QS_MAX_POST_TERMS];
    int n;
};

__device__ __forceinline__ void post_load(PostSmem &ps, const qs_post_phase *g, int tid, int nthr)
{
    const qs_phase_term *terms = reinterpret_cast<const qs_phase_term *>(g + 1);
    const int n = min(g->n_terms, QS_MAX_POST_TERMS);   // the host never packs more
    if (tid == 0) {
        ps.c1 = g->c1;
        ps.c2 = g->c2;
        for (int j = 0; j < 5; j++) ps.tp[j] = g->tp[j];
        ps.n = n;
    }
    for (int i = tid; i < n; i += nthr) {
        ps.part[i] = terms[i].partners;
        ps.a[i] = terms[i].a;
    }
}

// For the group with base index b: the exponent e of i (mod 4) and the mask of
// members whose sign flips (CZ partners off the sweep), as qs_post_phase
// defines them.
__device__ __forceinline__ void post_row(const PostSmem &ps, uint64_t b, uint32_t &e, uint32_t &flip)
{
    uint32_t x = (uint32_t)__popcll(b & ps.c1) + 2u * (uint32_t)__popcll(b & ps.c2);
    for (int i = 0; i < ps.n; i++)
        if ((b >> ps.a[i]) & 1) x += 2u * (uint32_t)__popcll(b & ps.part[i]);
    uint32_t f = 0;
#pragma unroll
    for (int j = 0; j < 5; j++) f |= ((uint32_t)__popcll(b & ps.tp[j]) & 1u) << j;
    e = x & 3u;
    flip = f;
}

// exponent of i for member m of a group with (e, flip)
__device__ __forceinline__ uint32_t post_member(uint32_t e, uint32_t flip, int m)
{
    return (e + 2u * (uint32_t)__popc((uint32_t)m & flip)) & 3u;
}

// (re + i im) i^r
__device__ __forceinline__ float2 rot_i(float2 v, uint32_t r)
{
    const float a = (r & 1u) ? v.y : v.x, b = (r & 1u) ? v.x : v.y;
    return make_float2(((r + 1u) & 2u) ? -a : a, (r & 2u) ? -b : b);
}

// the same on the two words of each FP64 value: a swap and sign-bit flips
__device__ __forceinline__ void rot_i_words(uint32_t &h0, uint32_t &l0, uint32_t &h1, uint32_t &l1, uint32_t r)
{
    if (r & 1u) {
        const uint32_t th = h0, tl = l0;
        h0 = h1;
        l0 = l1;
        h1 = th;
        l1 = tl;
    }
    h0 ^= ((r + 1u) & 2u) ? 0x80000000u : 0u;
    h1 ^= (r & 2u) ? 0x80000000u : 0u;
}

}  // namespace

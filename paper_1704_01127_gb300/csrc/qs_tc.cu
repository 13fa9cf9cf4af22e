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
// D = A_h B_h + (A_h B_t + A_t B_h) accumulates in FP32 in tensor memory, the
// head product and the correction in separate accumulators added once with
// round-to-nearest (tcgen05.mma kind::tf32, M = 128, N = 64, K = 8 per
// instruction).
//
// Operands sit in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, core matrices adjacent along K 128 B
// apart (leading byte offset), 8-row groups 2048 B apart (stride byte offset).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "qs_internal.h"
#include "qs_tcgen05.cuh"

namespace {
constexpr size_t kTileBytesF32 = (size_t)kRows * kK * 4;   // 32 KB
constexpr size_t kBBytesF32 = (size_t)kN * kK * 4;         // 16 KB
constexpr size_t kSmemF32 = 2 * kTileBytesF32 + 2 * kBBytesF32;

// One CTA of 128 threads; thread r owns row r (group) of each tile.  Tiles are
// taken in a grid-stride loop; warp 0 holds 128 TMEM columns for the CTA.
// kPost: a phase op folded into the sweep is applied to the outputs.
template <bool kPost>
__global__ void __launch_bounds__(128, 2)
k_dense5_tc_c64(float2 *__restrict__ psi, uint64_t n_groups, TileLayout t, const float *__restrict__ bpack,
                const qs_post_phase *__restrict__ post, int *__restrict__ status)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *A_h = smem;
    uint8_t *A_t = smem + kTileBytesF32;
    uint8_t *B_h = smem + 2 * kTileBytesF32;
    uint8_t *B_t = B_h + kBBytesF32;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base_s;
    __shared__ PostSmem ps;

    const int tid = threadIdx.x, warp = tid >> 5;
    {
        const float4 *src = reinterpret_cast<const float4 *>(bpack);
        float4 *dst = reinterpret_cast<float4 *>(B_h);
        for (int i = tid; i < (int)(2 * kBBytesF32 / 16); i += blockDim.x) dst[i] = src[i];
    }
    if constexpr (kPost) post_load(ps, post, tid, blockDim.x);
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
    // software pipeline: the next tile's amplitudes are loaded into registers
    // while the tensor cores work on the current one
    float2 v[32];
    uint64_t tile = blockIdx.x;
    bool valid = false;
    float2 *p = psi;
    auto load_tile = [&](uint64_t tl, float2 *vv, bool &val, float2 *&pp) {
        const uint64_t g = tl * kRows + tid;
        val = tl < n_tiles && g < n_groups;
        pp = psi + (val ? tile_base(g, t) : 0);
        if (t.pairs) {
            // members 2i and 2i+1 differ in qubit 0: one 16-byte load each
            // (a member outside the support is read but replaced by zero)
#pragma unroll
            for (int x = 0; x < 32; x += 2) {
                const float4 w = val ? *reinterpret_cast<const float4 *>(pp + off5(x, t)) : make_float4(0.f, 0.f, 0.f, 0.f);
                vv[x] = ((t.mmask >> x) & 1) ? make_float2(w.x, w.y) : make_float2(0.f, 0.f);
                vv[x + 1] = ((t.mmask >> (x + 1)) & 1) ? make_float2(w.z, w.w) : make_float2(0.f, 0.f);
            }
        } else {
#pragma unroll
            for (int x = 0; x < 32; x++) vv[x] = val && ((t.mmask >> x) & 1) ? pp[off5(x, t)] : make_float2(0.f, 0.f);
        }
    };
    load_tile(tile, v, valid, p);
    for (; tile < n_tiles; tile += gridDim.x) {
        // split: members 2c and 2c+1 fill K columns 4c..4c+3
#pragma unroll
        for (int c = 0; c < 16; c++) {
            const float2 v0 = v[2 * c], v1 = v[2 * c + 1];
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
                // head product and the two correction products in separate
                // accumulators: the tensor core's FP32 accumulation rounds
                // toward zero, so fewer steps on the large sum mean less drift
                mma_tf32(tmem, smem_desc(a_h + koff), smem_desc(b_h + koff), kIdescTf32, ks > 0);
                mma_tf32(tmem + kN, smem_desc(a_h + koff), smem_desc(b_t + koff), kIdescTf32, ks > 0);
                mma_tf32(tmem + kN, smem_desc(a_t + koff), smem_desc(b_h + koff), kIdescTf32, 1);
            }
            mma_commit(mbar_a);
        }
        float2 *const p_cur = p;
        const bool valid_cur = valid;
        load_tile(tile + gridDim.x, v, valid, p);
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
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        uint32_t pe = 0, pf = 0;
        if constexpr (kPost) post_row(ps, (uint64_t)(p_cur - psi), pe, pf);
        // output of member m: head + corrections, times the folded phase's factor
        auto out_of = [&](const float *r, const float *q, int l, int m) {
            float2 v = make_float2(r[2 * l] + q[2 * l], r[2 * l + 1] + q[2 * l + 1]);
            if constexpr (kPost) v = rot_i(v, post_member(pe, pf, m));
            return v;
        };
#pragma unroll
        for (int c = 0; c < kN / 16; c++) {
            float r[16], q[16];
            tmem_ld16(lane_addr + c * 16, r);
            tmem_ld16(lane_addr + kN + c * 16, q);
            tmem_wait_ld();
            if (valid_cur && t.pairs) {
#pragma unroll
                for (int l = 0; l < 8; l += 2) {
                    const float2 v0 = out_of(r, q, l, 8 * c + l), v1 = out_of(r, q, l + 1, 8 * c + l + 1);
                    *reinterpret_cast<float4 *>(p_cur + off5(8 * c + l, t)) = make_float4(v0.x, v0.y, v1.x, v1.y);
                }
            } else if (valid_cur) {
#pragma unroll
                for (int l = 0; l < 8; l++) p_cur[off5(8 * c + l, t)] = out_of(r, q, l, 8 * c + l);
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}


// ----------------------------------------------------------------------------
// complex128: exact integer slices on the fp16 tensor path.
//
// Each row r (group) is scaled by its largest exponent E_r and each column n of
// B^T by its largest exponent G_n; a value m 2^{e-1075} becomes the fixed-point
// integer F = round(m 2^{e-E-7}) (half to even, on the magnitude), |F| <= 2^46,
// so |F| = sum_{s<6} (b_s - 128) 2^{8(5-s)} with b_s the bytes of
// |F| + 0x808080808080, and the state digits are d_s = sigma (b_s - 128), sigma
// the value's sign (|d_s| <= 128, exact in fp16; the unitary's digits are the
// balanced bytes of its two's complement fixed point).  With A_i, B_j the
// digit planes and T = sum_{d<=6} D_d 2^{8(5-d)},
//   sum_k a_rk b_kn ~ 2^{E_r + G_n - 2096} T[r][n],  D_d = sum_{i+j=d} (A_i B_j^T),
// and the planes with i + j = d <= 6 are summed in accumulator D_d (TMEM; the
// dropped planes, d >= 7, weigh about 2^-51 of the result).  Every product of
// digits is an integer of magnitude <= 2^14 and a 64-term sum <= 2^20, so
// D_0..D_3 (at most four products) are exact integers of magnitude <= 2^22 in
// FP32; D_4..D_6 carry weight <= 2^-32 and are combined in FP32.  The FP64
// result is one int64 -> double conversion of T = P 2^32 + Q 2^16 + R
// (P = D_0 2^8 + D_1, Q = D_2 2^8 + D_3 exact in 32 bits, R the rounded low
// part), assembled in 32-bit halves, with the scale added to the exponent field.
// ----------------------------------------------------------------------------
constexpr int kSlices = 6;                                   // digit planes of A (the state)
constexpr int kSlicesB = 7;                                  // digit planes of B (the unitary)
constexpr int kDiags = 7;                                    // accumulators D_0 .. D_6
constexpr uint32_t kSBO16 = 1024;                            // 8 K-chunks x 128 B (16-bit elements)
constexpr size_t kPlaneA = (size_t)kRows * kK * 2;           // 16 KB per A digit plane
constexpr size_t kPlaneB = (size_t)kN * kK * 2;              // 8 KB per B digit plane
constexpr size_t kSmemC128 = kSlices * kPlaneA + kSlicesB * kPlaneB + 256;   // + column exponents
constexpr int kTmemCols128 = 512;

// byte offset of 16-bit element (row, k) in a K-major no-swizzle tile with 64 K
__host__ __device__ __forceinline__ uint32_t cm_off16(int row, int k)
{
    return (uint32_t)((((row >> 3) * (kK / 8)) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// |F| of a double relative to biased row exponent E, rounded half to even (the
// structured amplitudes of early circuit layers hit exact ties often, and
// rounding ties up would bias the norm), plus the digit bias 0x808080808080, as
// two 32-bit words; the high word also gets 0x6464 in its top bytes (|F| + bias
// < 2^48), the fp16 exponent byte its two digit planes pair with.  Members within 2^25 of the row's largest value (sh < 32;
// E7f = E + 7, or a value that sends every member to the general path when
// E < 25) take 32-bit funnel shifts: the round bit and the bits below it sit in
// x = lo << (32 - sh), and the increment is [x > 2^31 - lsb] (above half, or
// exactly half with an odd truncated value).
__device__ uint32_t g_qs_one = 1;   // read at run time, so the multiplies below stay on the FMA pipe

__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t imadhi(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ void mag48(double a, int E, int E7f, uint32_t one, uint32_t &flo, uint32_t &fhi)
{
    const uint32_t hi = (uint32_t)__double2hiint(a), lo = (uint32_t)__double2loint(a);
    // e = |hi| >> 20, sh = E7f - e, both on the FMA pipe
    const uint32_t e = imadhi(hi & 0x7FFFFFFFu, one << 12);
    const int sh = (int)imad(e, 0u - one, (uint32_t)E7f);
    if ((uint32_t)sh < 32u) {
        const uint32_t mh = (hi & 0x000FFFFFu) | 0x00100000u;
        const uint32_t tlo = __funnelshift_r(lo, mh, sh);
        const uint32_t thi = mh >> sh;
        const uint32_t x = lo << imad((uint32_t)sh, 0u - one, 32u);
        // carry of x + (2^31 - 1 + lsb) = [x > 2^31 - lsb]: the rounding
        // increment, added with the digit bias in one carry chain
        const uint32_t c1 = imad(tlo & 1u, one, 0x7FFFFFFFu);
        asm("{\n\t.reg .u32 t;\n\tadd.cc.u32 t, %2, %3;\n\taddc.cc.u32 %0, %4, 0x80808080;\n\taddc.u32 %1, %5, 0x64648080;\n\t}"
            : "=r"(flo), "=r"(fhi) : "r"(x), "r"(c1), "r"(tlo), "r"(thi));
    } else {
        const int ee = (int)((hi >> 20) & 0x7FF), shift = E + 7 - ee;
        uint64_t F = 0;
        if (ee != 0 && shift < 60) {
            const uint64_t m = ((uint64_t)(hi & 0x000FFFFFu) << 32 | lo) | (1ULL << 52);
            F = (m + (1ULL << (shift - 1)) - 1 + ((m >> shift) & 1)) >> shift;
        }
        F += 0x6464808080808080ULL;
        flo = (uint32_t)F;
        fhi = (uint32_t)(F >> 32);
    }
}

// The same from two words whose bytes 3 are 0x64 (the high words of |F| + bias)
__device__ __forceinline__ uint32_t f16x2_sdigits2(uint32_t w0, uint32_t w1, uint32_t sel, uint32_t sg, uint32_t nsg)
{
    uint32_t r;
    const uint32_t w = __byte_perm(w0, w1, sel);
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(w), "r"(sg), "r"(nsg));
    return r;
}

// Signed digit pair of one plane: the bytes (re, im) become fp16 1024 + b by a
// byte permute, and one f16x2 FMA with the amplitude's signs s (+-1 per half)
// gives s (b - 128): w s + (-1152 s).
__device__ __forceinline__ uint32_t f16x2_sdigits(uint32_t pairs, uint32_t sel, uint32_t sg, uint32_t nsg)
{
    uint32_t r;
    const uint32_t w = __byte_perm(pairs, 0x64646464u, sel);
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(w), "r"(sg), "r"(nsg));
    return r;
}

constexpr int kSplitThreads = 512;
constexpr int kEpiThreads = 384;                    // 3 warps per TMEM lane quarter
constexpr int kIssueThreads = 32;                   // one warp: issues the MMAs
constexpr int kC128Threads = kSplitThreads + kEpiThreads + kIssueThreads;
constexpr int kSplitParts = kSplitThreads / kRows;   // splitter threads per row
constexpr int kMPT = 32 / kSplitParts;               // amplitudes per splitter thread

__device__ __forceinline__ void bar_split() { asm volatile("bar.sync 1, %0;" ::"r"(kSplitThreads) : "memory"); }
__device__ __forceinline__ bool bar_split_or(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred p, 1, %2, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(kSplitThreads)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity)
{
    for (long it = 0; it < kWaitLimit; it++)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

// ----------------------------------------------------------------------------
// complex128 kernel: one CTA per SM, three warp-specialised groups:
//   splitters (512 threads, kSplitThreads / 128 per row, kMPT amplitudes
//     each): copy tile t+1 into a 64 KB stage while tile t is processed
//     (kBulk: full-state tiles whose member runs are 2 KB, as 32 bulk copies
//     from lane 0 of each splitter warp, halfway through its fixed point,
//     once an mbarrier shows that every splitter warp has read the stage;
//     otherwise 16-byte cp.async of each thread's own slots, which hold the
//     issuing warps up ~3K cycles a tile); find the row exponents (kBulk: the
//     four threads of a row are lanes of one warp, two shuffles; otherwise a
//     512-thread barrier) and the fixed-point values of tile t while the MMAs
//     of tile t-1 still read the digit planes, then write the planes;
//   issuer (one warp, one thread): issues the MMAs.  The tensor pipe takes
//     few instructions ahead, so the issuing thread waits about as long as
//     the MMAs run (~4K cycles a tile); on its own warp that wait holds up
//     no splitter (issued by splitter thread 0: 10.2 ms per 30-qubit sweep,
//     here 7.9 ms together with the arithmetic below and the bulk copies);
//   epilogue (384 threads, three warps per TMEM lane quarter, 3 + 3 + 2 and
//     2 + 3 + 3 four-column chunks of the two halves): rebuild FP64 results
//     from the accumulators and store them.
// The output columns come in two halves of 32, so that the tensor cores work
// on one half while the epilogue reads the other.
//   TMEM: half h holds D_0..D_6 for its 32 columns at columns 256 h + 32 d.
//   B:    4 KB blocks (half h, plane j) at (7 h + j) * 4 KB, so for A plane i
//         one MMA with N = 32 (7 - i) reads B planes 0..6-i of half h and
//         writes D_i..D_6 of that half (24 MMAs per half, 48 per tile).
// kSub (a sweep that widens the support: only M = 2^m of the 32 members of
// a group can be nonzero): those members take K positions 0 .. M-1 (B's K
// positions permuted to match when it is copied in), splitters whose K
// positions all lie past M keep zero planes and only join the barriers, and
// each half takes ceil(M / 8) K steps per A plane instead of 4.  Every
// accumulator sum is an exact integer, so the order of K changes no bit.
// kPost (a phase op folded into the sweep): the phase of a row splits into a
// part of its tile, formed one tile ahead by the issuing thread while it
// waits for the planes (four slots by tile index), and a part of its row,
// formed once per CTA (a table of 128); the epilogue combines the two.
// Hand-offs per tile: mbar_planes (splitter thread 0 after the planes are
// written), mbar_mma[h] (tcgen05.commit after half h's MMAs; half 1's also
// releases the A planes), mbar_free[h] (one arrival per epilogue thread when
// half h's accumulators are read).  All waits are bounded.
// ----------------------------------------------------------------------------
constexpr int kHalfN = 32;
constexpr int kEpiMaxChunks = 3;                          // 4-column chunks of a half per epilogue warp (3, 3, 2 / 2, 3, 3)
constexpr uint32_t kBlockB = (uint32_t)kHalfN * kK * 2;   // 4 KB: one plane of one half

// instruction descriptor: D fp32, A and B fp16 (format 0), both K-major,
// N >> 3 at bits 17-22, M >> 4 at bits 24-28
__host__ __device__ constexpr uint32_t idesc_f16_n(int n)
{
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ void issue_c128_half(uint32_t tmem, uint32_t a0, uint32_t b0, int h, int nks)
{
    const uint64_t da = smem_desc(a0, kSBO16), db = smem_desc(b0 + h * kSlicesB * kBlockB, kSBO16);
#pragma unroll
    for (int i = 0; i < kSlices; i++) {
#pragma unroll
        for (int ks = 0; ks < kK / 16; ks++) {
            if (ks >= nks) break;   // K columns past the support's members are zero
            const uint32_t koff = ks * 2 * kLBO;
            mma_f16(tmem + 256 * h + kHalfN * i, da + ((uint64_t)(i * kPlaneA + koff) >> 4),
                     db + ((uint64_t)koff >> 4), idesc_f16_n(kHalfN * (kDiags - i)), (i == 0 && ks == 0) ? 0u : 1u);
        }
    }
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

// 16-byte asynchronous global -> shared copy (zero fill when bytes = 0)
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *gptr, uint32_t bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(gptr), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr size_t kStageC128 = (size_t)kSplitThreads * kMPT * 16;   // raw next tile: 64 KB
constexpr size_t kSmemC128Pipe = kSmemC128 + kStageC128;

// The folded phase of a row (kPost) split into the part of its tile and the
// part of its row.  A row's base is b = H | l: H the base of the tile's first
// group, l the row's bits among the 7 lowest group positions (`low`).  Then
//   e(b) = popc(H & c1) + popc(l & c1) + 2 (q_H ^ q_l ^ parity(l & X_H))  (mod 4),
//   flip(b) = flip(H) ^ flip(l),
// where q_H, X_H depend on the tile alone (a term whose qubit a is set in H
// adds parity(H & partners) to q_H and its partners to X_H; a term whose qubit
// lies in `low` and whose partners meet H an odd number of times adds bit a to
// X_H) and q_l on the row alone (parity(l & c2) and the terms with both ends
// in the row's bits).  The tile's part is formed once per tile by the
// MMA-issuing thread, the row's part once per CTA for each of its 128 rows;
// X_H is kept as its bits at the `low` positions (bit k: the k-th lowest), so
// parity(l & X_H) = parity(r & X) for row r of the tile.
__device__ __forceinline__ void post_tile(const PostSmem &ps, uint64_t H, uint64_t low, uint32_t &X, uint32_t &C)
{
    uint32_t q = (uint32_t)__popcll(H & ps.c2) & 1u;
    uint64_t x = 0;
#pragma unroll 1
    for (int i = 0; i < ps.n; i++) {
        const uint64_t P = ps.part[i];
        const int a = ps.a[i];
        const uint32_t hp = (uint32_t)__popcll(H & P) & 1u;
        if ((H >> a) & 1) {
            q ^= hp;
            x ^= P;
        } else if (((low >> a) & 1) && hp) {
            x ^= 1ULL << a;
        }
    }
    uint32_t f = 0;
#pragma unroll
    for (int j = 0; j < 5; j++) f |= ((uint32_t)__popcll(H & ps.tp[j]) & 1u) << j;
    uint32_t xc = 0;
    int k = 0;
    for (uint64_t w = low; w; w &= w - 1, k++) xc |= (uint32_t)((x >> (__ffsll((long long)w) - 1)) & 1) << k;
    X = xc;
    C = ((uint32_t)__popcll(H & ps.c1) & 3u) | q << 2 | f << 3;
}
__device__ __forceinline__ uint32_t post_rowpart(const PostSmem &ps, uint64_t l)
{
    uint32_t q = (uint32_t)__popcll(l & ps.c2) & 1u;
#pragma unroll 1
    for (int i = 0; i < ps.n; i++)
        if ((l >> ps.a[i]) & 1) q ^= (uint32_t)__popcll(l & ps.part[i]) & 1u;
    uint32_t f = 0;
#pragma unroll
    for (int j = 0; j < 5; j++) f |= ((uint32_t)__popcll(l & ps.tp[j]) & 1u) << j;
    return ((uint32_t)__popcll(l & ps.c1) & 3u) | q << 2 | f << 3;
}

template <bool kPost, bool kBulk, bool kSub>
__global__ void __launch_bounds__(kC128Threads, 1)
k_dense5_tc_c128_pipe(double2 *__restrict__ psi, uint64_t n_groups, TileLayout t, const uint8_t *__restrict__ bpack,
                      const qs_post_phase *__restrict__ post, int *__restrict__ status)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *A = smem;
    uint8_t *B = smem + kSlices * kPlaneA;
    uint4 *stage = reinterpret_cast<uint4 *>(smem + kSmemC128);   // [8][512] x 16 B
    __shared__ __align__(8) uint64_t mbar_mma[2], mbar_free[2], mbar_planes, mbar_full, mbar_used;
    __shared__ uint64_t moff[32];         // offset of member x within a group
    __shared__ uint64_t ioff[32];         // kSub: offset of the member at K position x (support members first)
    __shared__ int perm[32];              // kSub: member at K position x
    __shared__ uint32_t tmem_base_s;
    __shared__ int rowexp[kSplitParts][kRows];
    // exponent-field terms, added modulo 2^32 (only the sum must fit):
    __shared__ uint32_t rowX[2][kRows];   // (E_r - 2096) << 20 of the last two tiles
    __shared__ int gext[2];               // smallest and largest G_n
    __shared__ uint32_t colX[kN];         // G_n << 20
    __shared__ volatile int abort_flag;
    __shared__ PostSmem ps;               // a phase op folded into the sweep (kPost)
    __shared__ uint32_t postX[4];         // kPost: the tile's part of the folded phase (X_H; by tile index mod 4)
    __shared__ uint32_t postC[4];         // kPost: popc(H & c1) mod 4, q_H, flip(H)
    __shared__ uint8_t postR[kRows];      // kPost: the same for the row part, by row of the tile

    const int tid = threadIdx.x, warp = tid >> 5;
    // kSub: M = 2^m of the 32 members lie in the support (the others read as
    // zero); they take K positions 0 .. M-1, in order, and the rows of B^T
    // follow them, so only the first M K positions of A can be nonzero
    const int M = kSub ? __popc(t.mmask) : 32;
    if constexpr (kSub) {
        if (tid < 32) {
            const uint32_t below = (1u << tid) - 1u;
            perm[(t.mmask >> tid) & 1 ? __popc(t.mmask & below) : M + __popc(~t.mmask & below)] = tid;
        }
        __syncthreads();
        if (tid < 32) ioff[tid] = off5(perm[tid], t);
        // plane-major pack -> half-major blocks, K positions permuted (a
        // member's two reals are one 4-byte word)
        const uint32_t *src = reinterpret_cast<const uint32_t *>(bpack);
        uint32_t *dst = reinterpret_cast<uint32_t *>(B);
        for (int i = tid; i < kSlicesB * 2 * 1024; i += blockDim.x) {
            const int blk = i >> 10, n = (i >> 5) & 31, x = i & 31;   // source block 2 j + h, row n, K position x
            const int j = blk >> 1, h = blk & 1;
            dst[((h * kSlicesB + j) * kBlockB + cm_off16(n, 2 * x)) >> 2] = src[(blk * kBlockB + cm_off16(n, 2 * perm[x])) >> 2];
        }
    } else {
        // plane-major pack (plane j = halves 0, 1) -> half-major blocks
        const uint4 *src = reinterpret_cast<const uint4 *>(bpack);
        uint4 *dst = reinterpret_cast<uint4 *>(B);
        constexpr int kPerBlock = (int)(kBlockB / 16);
        for (int i = tid; i < kSlicesB * 2 * kPerBlock; i += blockDim.x) {
            const int blk = i / kPerBlock, w = i - blk * kPerBlock;   // source block 2 j + h
            const int j = blk >> 1, h = blk & 1;
            dst[(h * kSlicesB + j) * kPerBlock + w] = src[i];
        }
    }
    {
        const int *G = reinterpret_cast<const int *>(bpack + kSlicesB * kPlaneB);
        if (tid < kN) colX[tid] = (uint32_t)G[tid] << 20;
        if (tid == 0) {
            int lo = 2047, hi = 0;
            for (int n = 0; n < kN; n++) {
                lo = min(lo, G[n]);
                hi = max(hi, G[n]);
            }
            gext[0] = lo;
            gext[1] = hi;
        }
        if (tid < 32) moff[tid] = off5(tid, t);
        if constexpr (kPost) post_load(ps, post, tid, blockDim.x);
    }
    if (warp == 0) {
        tmem_alloc(smem_u32(&tmem_base_s), kTmemCols128);
        tmem_relinquish();
    }
    if (tid == 0) {
        for (int h = 0; h < 2; h++) {
            mbar_init(smem_u32(&mbar_mma[h]), 1);
            mbar_init(smem_u32(&mbar_free[h]), kEpiThreads);
        }
        mbar_init(smem_u32(&mbar_planes), 1);
        mbar_init(smem_u32(&mbar_full), kSplitThreads / 32);
        mbar_init(smem_u32(&mbar_used), kSplitThreads / 32);
        fence_mbar_init();
        abort_flag = 0;
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;
    const uint64_t n_tiles = (n_groups + kRows - 1) / kRows;
    if constexpr (kPost) {
        // the folded phase's row part, row by row (the same in every tile), and
        // the tile part of this CTA's first tile
        if (tid < kRows) postR[tid] = (uint8_t)post_rowpart(ps, tile_base(tid, t) ^ tile_base(0, t));
        if (tid == kRows && blockIdx.x < n_tiles)
            post_tile(ps, tile_base((uint64_t)blockIdx.x * kRows, t), tile_base(kRows - 1, t) ^ tile_base(0, t), postX[0], postC[0]);
        __syncthreads();
    }

    if (kSub && tid < kSplitThreads && kMPT * (tid >> 7) >= M) {
        // ------------------------------------------------- idle splitters (kSub)
        // K positions kMPT part .. + kMPT-1 are past M: zero planes, written
        // once; then only the splitters' barriers, tile by tile
        const int row = tid & (kRows - 1), part = tid >> 7;
        for (int c = 0; c < kMPT / 4; c++)
            for (int sl = 0; sl < kSlices; sl++)
                *reinterpret_cast<uint4 *>(A + cm_off16(row, 2 * kMPT * part + 8 * c) + sl * kPlaneA) = make_uint4(0u, 0u, 0u, 0u);
        fence_proxy_async();
        for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            rowexp[part][row] = 0;
            bar_split();
            if (bar_split_or(abort_flag)) break;
        }
    } else if (tid < kSplitThreads) {
        // ------------------------------------------------------------ splitters
        // kBulk: the four threads of a row are lanes r, r+8, r+16, r+24 of one
        // warp (warp w: rows 8w .. 8w+7), so the row's exponent is two warp
        // shuffles; otherwise thread tid is row tid & 127, part tid >> 7
        const int row = kBulk ? 8 * (tid >> 5) + (tid & 7) : tid & (kRows - 1);
        const int part = kBulk ? (tid >> 3) & 3 : tid >> 7;
        const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
        const uint32_t one = *(volatile uint32_t *)&g_qs_one;
        const uint32_t stage_a = smem_u32(stage) + 16u * tid;
        // this thread's kMPT amplitudes of tile tl into its own stage slots
        // (slot x at x * kSplitThreads + tid): asynchronous, a whole iteration ahead
        auto prefetch = [&](uint64_t tl) {
            const uint64_t g = tl * kRows + row;
            const bool val = tl < n_tiles && g < n_groups;
            const double2 *pp = psi + (val ? tile_base(g, t) : 0);
#pragma unroll
            for (int x = 0; x < kMPT; x++) {
                // kSub: K positions past M are members outside the support (zero)
                const bool vx = val && (!kSub || kMPT * part + x < M);
                cp_async16(stage_a + 16u * kSplitThreads * x, vx ? pp + (kSub ? ioff : moff)[kMPT * part + x] : psi, vx ? 16u : 0u);
            }
            cp_async_commit();
        };
        // full-state tiles whose rows are 128 consecutive amplitudes (every
        // target >= 7): member m is one 2 KB run, copied by lane 0 of splitter
        // warp m >> 1 into slots (m & 7) of splitters 128 (m >> 3) .. + 127
        // (kBulk: the launcher checked that every tile is such a full-state tile)
        constexpr bool bulk = kBulk;
        const uint32_t mfull = smem_u32(&mbar_full), stage_s = smem_u32(stage);
        auto fill = [&](uint64_t tl) {
            if ((tid & 31) == 0) {
                const double2 *tb = psi + tile_base(tl * kRows, t);
                mbar_arrive_expect_tx(mfull, 4096u);
                for (int m = 2 * (tid >> 5); m < 2 * (tid >> 5) + 2; m++)
                    bulk_g2s(stage_s + 8192u * (m & 7) + 2048u * (m >> 3), tb + moff[m], 2048u, mfull);
            }
        };
        int pending = -1;   // tile whose bulk copies are in flight
        if constexpr (bulk) {
            fill(blockIdx.x);
            pending = 0;
        } else {
            prefetch(blockIdx.x);
        }
        int it = 0;
        for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, it++) {
            bool full_ok = true;
            if constexpr (bulk) {
                full_ok = mbar_wait_bounded(mfull, it & 1);
                if (full_ok) pending = -1;
            } else {
                cp_async_wait_all();
            }
            double2 v[kMPT];
#pragma unroll
            for (int x = 0; x < kMPT; x++) {
                const uint4 w = stage[kSplitThreads * x + (kBulk ? kRows * part + row : tid)];
                v[x] = make_double2(__hiloint2double((int)w.y, (int)w.x), __hiloint2double((int)w.w, (int)w.z));
            }
            uint32_t emax = 0;
#pragma unroll
            for (int x = 0; x < kMPT; x++) {
                emax = max(emax, (uint32_t)__double2hiint(v[x].x) & 0x7FF00000u);
                emax = max(emax, (uint32_t)__double2hiint(v[x].y) & 0x7FF00000u);
            }
            // emax depends on every slot read above, so the shared loads are
            // complete before the next tile's copies may overwrite the slots
            asm volatile("" ::"r"(emax) : "memory");
            int E;
            if constexpr (bulk) {
                // this warp has read its stage slots; the row's exponent from
                // the four lanes that hold the row
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(smem_u32(&mbar_used));
                emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, 8));
                emax = max(emax, __shfl_xor_sync(0xFFFFFFFFu, emax, 16));
                E = (int)(emax >> 20);
                if (!full_ok) {
                    if ((tid & 31) == 0) atomicExch(status, 1);
                    abort_flag = 1;
                }
            } else {
                prefetch(tile + gridDim.x);
                rowexp[part][row] = (int)(emax >> 20);
                bar_split();
                E = rowexp[0][row];
#pragma unroll
                for (int q = 1; q < kSplitParts; q++) E = max(E, rowexp[q][row]);
            }
            // a result's exponent field is that of T (1023 .. 1085 for T != 0)
            // plus E + G_n - 2096.  Rows below ~2^-970 take E >= 1074 - min G_n
            // (no result leaves the normal range; they keep fewer bits, an
            // absolute error near 2^-1015); rows whose results could pass
            // 2^1024 (magnitudes above ~2^1010) are flagged, status bit 2
            E = max(E, 1074 - ((volatile int *)gext)[0]);
            if (part == 0 && E + ((volatile int *)gext)[1] > 3057) atomicOr(status, 2);
            const int E7f = E >= 25 ? E + 7 : 0x40000000;
            uint32_t glo[2 * kMPT], ghi[2 * kMPT], sgn[kMPT];
#pragma unroll
            for (int x = 0; x < kMPT; x++) {
                if (bulk && x == kMPT / 2 && full_ok && tile + gridDim.x < n_tiles) {
                    // every splitter warp has read the stage (by now, as a rule):
                    // the next tile's runs
                    if ((tid & 31) == 0) {
                        if (mbar_wait_bounded(smem_u32(&mbar_used), it & 1)) {
                            fill(tile + gridDim.x);
                            pending = it + 1;
                        } else {
                            atomicExch(status, 1);
                            abort_flag = 1;
                        }
                    }
                }
                mag48(v[x].x, E, E7f, one, glo[2 * x], ghi[2 * x]);
                mag48(v[x].y, E, E7f, one, glo[2 * x + 1], ghi[2 * x + 1]);
                // sign bits of re (bit 15) and im (bit 31)
                sgn[x] = __byte_perm((uint32_t)__double2hiint(v[x].x), (uint32_t)__double2hiint(v[x].y), 0x7632u) & 0x80008000u;
            }
            // tile it-1's MMAs (both halves) must have finished reading the planes
            const bool ok = it == 0 || mbar_wait_bounded(smem_u32(&mbar_mma[1]), (it - 1) & 1);
            // tile it-1's half-1 MMAs were issued after the epilogue had read
            // tile it-2's scale, so slot it & 1 is free
            if (part == 0) rowX[it & 1][row] = (uint32_t)(E - 2096) << 20;
#pragma unroll
            for (int c = 0; c < kMPT / 4; c++) {
                uint8_t *dst = A + cm_off16(row, 2 * kMPT * part + 8 * c);
                uint32_t pl[6][4];                     // [plane][member of the chunk]
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int x = 4 * c + j;           // words 2x (re), 2x+1 (im)
                    const uint32_t y23 = __byte_perm(glo[2 * x], glo[2 * x + 1], 0x7632u);
                    const uint32_t y01 = __byte_perm(glo[2 * x], glo[2 * x + 1], 0x5410u);
                    const uint32_t sg = sgn[x] | 0x3C003C00u, nsg = sgn[x] ^ 0xE480E480u;   // +-1, -+1152
                    // the high words carry 0x64 in their top bytes: bytes 5 and 4
                    // of |F| pair with it directly
                    pl[0][j] = f16x2_sdigits2(ghi[2 * x], ghi[2 * x + 1], 0x7531u, sg, nsg);   // byte 5 of |F|
                    pl[1][j] = f16x2_sdigits2(ghi[2 * x], ghi[2 * x + 1], 0x7430u, sg, nsg);   // byte 4
                    pl[2][j] = f16x2_sdigits(y23, 0x4341u, sg, nsg);   // byte 3
                    pl[3][j] = f16x2_sdigits(y23, 0x4240u, sg, nsg);   // byte 2
                    pl[4][j] = f16x2_sdigits(y01, 0x4341u, sg, nsg);   // byte 1
                    pl[5][j] = f16x2_sdigits(y01, 0x4240u, sg, nsg);   // byte 0
                }
#pragma unroll
                for (int sl = 0; sl < kSlices; sl++)
                    *reinterpret_cast<uint4 *>(dst + sl * kPlaneA) = make_uint4(pl[sl][0], pl[sl][1], pl[sl][2], pl[sl][3]);
            }
            fence_proxy_async();
            // every splitter has written its planes (and seen tile it-1's MMAs
            // finish, or the abort)
            if (bar_split_or(!ok || abort_flag)) {
                if (tid == 0) atomicExch(status, 1);
                break;
            }
            if (tid == 0) mbar_arrive(smem_u32(&mbar_planes));   // planes of tile it are written
        }
        cp_async_wait_all();
        // bulk copies still in flight land before the CTA leaves
        if (pending >= 0) mbar_wait_bounded(mfull, pending & 1);
    } else if (tid >= kSplitThreads + kEpiThreads) {
        // ---------------------------------------------------------------- issuer
        if (tid == kSplitThreads + kEpiThreads) {
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
            const uint64_t low = tile_base(kRows - 1, t) ^ tile_base(0, t);
            int it = 0;
            for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, it++) {
                // the folded phase's tile part for tile it+1, while the planes of
                // tile it are written: slot (it+1) & 3 last held tile it-3's, which
                // the epilogue read before releasing tile it-2's half 0 (waited for
                // by tile it-1's MMAs); it reads tile it+1's after the last MMAs of
                // tile it complete (committed after this write)
                if (kPost && tile + gridDim.x < n_tiles)
                    post_tile(ps, tile_base((tile + gridDim.x) * kRows, t), low, postX[(it + 1) & 3], postC[(it + 1) & 3]);
                if (!mbar_wait_bounded(smem_u32(&mbar_planes), it & 1) || abort_flag) {
                    atomicExch(status, 1);
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                // half h of tile it-1 must have been read out before half h of tile it
                bool ok = true;
                for (int h = 0; h < 2 && ok; h++) {
                    if (it > 0 && !mbar_wait_bounded(smem_u32(&mbar_free[h]), (it - 1) & 1)) {
                        atomicExch(status, 1);
                        abort_flag = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    issue_c128_half(tmem, a0, b0, h, (M + 7) >> 3);
                    mma_commit(smem_u32(&mbar_mma[h]));
                }
                if (!ok) break;
            }
            // leave only after the last MMAs are complete (they read this CTA's planes)
            if (it > 0 && !abort_flag) mbar_wait_bounded(smem_u32(&mbar_mma[1]), (it - 1) & 1);
        }
    } else {
        // ------------------------------------------------------------- epilogue
        const int ew = warp - kSplitThreads / 32;                 // 0 .. 11
        const int row = 32 * (warp & 3) + (tid & 31), ej = ew >> 2;   // warp ej of its lane quarter
        const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        int it = 0;
        bool failed = false;
        for (uint64_t tile = blockIdx.x; tile < n_tiles && !failed; tile += gridDim.x, it++) {
            const uint64_t g = tile * kRows + row;
            const bool valid = g < n_groups;
            double2 *p = psi + (valid ? tile_base(g, t) : 0);
            uint32_t pe = 0, pf = 0;
            if constexpr (kPost) {
                // i^pe (-1)^popc(m & pf) for member m of this row
                const uint32_t X = postX[it & 3], C = postC[it & 3], Crow = postR[row];
                const uint32_t sq = ((C ^ Crow) >> 2) ^ (uint32_t)__popc((uint32_t)row & X);
                pe = ((C & 3u) + (Crow & 3u) + 2u * (sq & 1u)) & 3u;
                pf = ((C ^ Crow) >> 3) & 31u;
            }
            for (int h = 0; h < 2; h++) {
                if (!mbar_wait_bounded(smem_u32(&mbar_mma[h]), it & 1) || abort_flag) {
                    atomicExch(status, 1);
                    abort_flag = 1;
                    failed = true;
                    break;
                }
                tc_fence_after();
                const uint32_t Xr = rowX[it & 1][row];
                // the half's accumulators reduced to the exact partial sums P, Q and
                // the rounded low part, then the half is released to the next
                // tile's MMAs before the FP64 rebuild and the stores
                // this warp's chunks of the half: 3, 3, 2 (half 0) and 2, 3, 3 (half 1)
                const int c0 = h == 0 ? 3 * ej : (ej == 0 ? 0 : 3 * ej - 1);
                const int nc = h == 0 ? (ej < 2 ? 3 : 2) : (ej == 0 ? 2 : 3);
                int Pv[kEpiMaxChunks][4], Qv[kEpiMaxChunks][4], Rv[kEpiMaxChunks][4];
#pragma unroll
                for (int c = 0; c < kEpiMaxChunks; c++) {
                    if (c >= nc) break;
                    const int col = 4 * (c0 + c);
                    float D[kDiags][4];
#pragma unroll
                    for (int d = 0; d < 4; d++) tmem_ld4(lane_addr + 256 * h + kHalfN * d + col, D[d]);
                    tmem_wait_ld();
                    // T = P 2^32 + Q 2^16 + r with P = D_0 2^8 + D_1 and
                    // Q = D_2 2^8 + D_3 exact in 32 bits (|D_d| <= 2^22)
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        // raw words 0x4B400000 + D_d; P and Q carry 257 * 0x4B400000
                        Pv[c][q] = (int)((uint32_t)__float_as_int(D[0][q] + 12582912.0f) * 256u + (uint32_t)__float_as_int(D[1][q] + 12582912.0f));
                        Qv[c][q] = (int)((uint32_t)__float_as_int(D[2][q] + 12582912.0f) * 256u + (uint32_t)__float_as_int(D[3][q] + 12582912.0f));
                    }
#pragma unroll
                    for (int d = 4; d < kDiags; d++) tmem_ld4(lane_addr + 256 * h + kHalfN * d + col, D[d]);
                    tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        Rv[c][q] = __float2int_rn(fmaf(D[4][q], 256.0f, fmaf(D[6][q], 0.00390625f, D[5][q])));
                    }
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&mbar_free[h]));   // the half's accumulators are read
#pragma unroll
                for (int c = 0; c < kEpiMaxChunks; c++) {
                    if (c >= nc) break;
                    const int col = 4 * (c0 + c);              // column within the half
                    uint32_t hw[4], lw[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        // T = (P - K) 2^32 + (Q - K) 2^16 + R, K = 257 * 0x4B400000 = 0x8B400000 (mod 2^32)
                        const int R = Rv[c][q];
                        const int Qt = (int)((uint32_t)Qv[c][q] - 0x8B400000u);
                        uint32_t tl, th;
                        asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, %5;"
                            : "=r"(tl), "=r"(th)
                            : "r"((uint32_t)Qt << 16), "r"((uint32_t)R), "r"((uint32_t)Pv[c][q] + (uint32_t)(Qt >> 16)),
                              "r"((uint32_t)(R >> 31) - 0x8B400000u));
                        const double dv = __ll2double_rn((long long)((uint64_t)th << 32 | tl));
                        const uint32_t hi = (uint32_t)__double2hiint(dv);
                        // T = 0 gives +0.0 (hi = 0); otherwise add the scale to the exponent
                        hw[q] = hi == 0 ? 0u : hi + Xr + colX[kHalfN * h + col + q];
                        lw[q] = (uint32_t)__double2loint(dv);
                    }
                    const int m0 = (kHalfN * h + col) >> 1;   // columns 2m, 2m+1: re, im of member m
                    if constexpr (kPost) {
                        rot_i_words(hw[0], lw[0], hw[1], lw[1], post_member(pe, pf, m0));
                        rot_i_words(hw[2], lw[2], hw[3], lw[3], post_member(pe, pf, m0 + 1));
                    }
                    if (valid) {
                        p[moff[m0]] = make_double2(__hiloint2double((int)hw[0], (int)lw[0]),
                                                   __hiloint2double((int)hw[1], (int)lw[1]));
                        p[moff[m0 + 1]] = make_double2(__hiloint2double((int)hw[2], (int)lw[2]),
                                                       __hiloint2double((int)hw[3], (int)lw[3]));
                    }
                }
            }
        }
    }
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols128);
}

// The bounded-wait failure path on its own: one thread waits on an mbarrier
// that nothing arrives on, gives up after `polls` tries, records the expiry
// in the status word and returns (the tensor-core sweeps do the same when
// their MMAs or partner warps never answer).
__global__ void k_wait_selftest(int *__restrict__ status, long polls)
{
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x != 0) return;
    mbar_init(smem_u32(&mbar), 1);
    fence_mbar_init();
    bool done = false;
    for (long it = 0; it < polls && !done; it++) done = mbar_try_wait(smem_u32(&mbar), 0);
    if (!done) atomicExch(status, 1);
}

bool g_attr_c64[2][64] = {};       // [folded phase][device]
bool g_attr_c128[2][3][64] = {};   // [folded phase][staging mode][device]
using C128Kernel = void (*)(double2 *, uint64_t, TileLayout, const uint8_t *, const qs_post_phase *, int *);

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

// Host: digit planes of the real-form matrix for the complex128 path.  Per
// column n of B^T the largest biased exponent G_n; a value becomes
// F' = round(m 2^{e-G_n+1}), |F'| <= 2^54, = sum_{j<7} e_j 2^{8(6-j)} with
// balanced digits, i.e. the same scale as the state's digits (weight
// 2^{8(5-j)} of 2^{G_n-1068}) plus one extra plane, so the unitary is carried
// to about 2^-55; fp16 planes in the canonical layout, then the 64 exponents.
// fp16 encoding of an integer |d| <= 2048 (exact): the fp32 encoding with the
// exponent rebased from 127 to 15 and the mantissa cut to 10 bits
static uint16_t f16_of_small_int(int d)
{
    if (d == 0) return 0;
    float f = (float)d;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t sign = (u >> 16) & 0x8000u, ex = ((u >> 23) & 0xFFu) - 127u + 15u;
    return (uint16_t)(sign | (ex << 10) | ((u >> 13) & 0x3FFu));
}

std::vector<uint8_t> qs_pack_tc_c128(const std::vector<double> &M)
{
    std::vector<uint8_t> out(kSlicesB * kPlaneB + 256, 0);
    double bt[kN][kK];
    for (int l = 0; l < 32; l++)
        for (int x = 0; x < 32; x++) {
            double re = M[2 * (l * 32 + x)], im = M[2 * (l * 32 + x) + 1];
            bt[2 * l][2 * x] = re;
            bt[2 * l][2 * x + 1] = -im;
            bt[2 * l + 1][2 * x] = im;
            bt[2 * l + 1][2 * x + 1] = re;
        }
    int *Gcol = reinterpret_cast<int *>(out.data() + kSlicesB * kPlaneB);
    for (int n = 0; n < kN; n++) {
        int G = 0;
        for (int k = 0; k < kK; k++) {
            uint64_t b;
            std::memcpy(&b, &bt[n][k], 8);
            G = std::max(G, (int)((b >> 52) & 0x7FF));
        }
        Gcol[n] = G;
        for (int k = 0; k < kK; k++) {
            uint64_t b;
            std::memcpy(&b, &bt[n][k], 8);
            int e = (int)((b >> 52) & 0x7FF), shift = G - 1 - e;
            uint64_t F = 0;
            if (e != 0 && shift < 60) {
                uint64_t m = (b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
                F = shift < 0    ? (m << -shift)
                    : shift == 0 ? m
                                 : (m + (1ULL << (shift - 1)) - 1 + ((m >> shift) & 1)) >> shift;   // half to even
                if (b >> 63) F = 0 - F;
            }
            uint64_t Gb = F + 0x80808080808080ULL;
            for (int sl = 0; sl < kSlicesB; sl++) {
                int dig = (int)((Gb >> (8 * (6 - sl))) & 0xFF) - 128;
                uint16_t h = f16_of_small_int(dig);
                std::memcpy(out.data() + sl * kPlaneB + cm_off16(n, k), &h, 2);
            }
        }
    }
    return out;
}

size_t qs_tc_pack_bytes(int dtype) { return dtype == QS_C64 ? 2 * kBBytesF32 : kSlicesB * kPlaneB + 256; }

int qs_launch_dense5_tc(qs_state *s, const int *sorted_qubits, const void *dev_pack, uint64_t grow,
                        const void *dev_post)
{
    s->perm_invariant = false;
    const bool c64 = s->dtype == QS_C64, fold = dev_post != nullptr;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (dev < 0 || dev >= 64) return qs_fail(QS_EUNSUPPORTED, "device %d", dev);
    if (c64 && !g_attr_c64[fold][dev]) {
        const void *fn = fold ? (const void *)k_dense5_tc_c64<true> : (const void *)k_dense5_tc_c64<false>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemF32);
        if (e != cudaSuccess) return qs_fail(QS_ECUDA, "tc smem attribute: %s", cudaGetErrorString(e));
        g_attr_c64[fold][dev] = true;
    }
    // the sweep covers the support after it: the support's free bits plus the
    // targets; groups enumerate the free bits that are not targets
    const uint64_t all = qs_index_mask(s->n);
    const uint64_t fr = s->sup_free & all, fx = s->sup_fix & ~fr & all;
    TileLayout t;
    uint64_t tm = 0;
    for (int j = 0; j < 5; j++) {
        t.q[j] = sorted_qubits[j];
        tm |= 1ULL << t.q[j];
    }
    t.mmask = 0;
    for (int x = 0; x < 32; x++) {
        bool in = true;
        for (int j = 0; j < 5; j++)
            if (!((fr >> t.q[j]) & 1) && (uint64_t)((x >> j) & 1) != ((fx >> t.q[j]) & 1)) in = false;
        if (in) t.mmask |= 1u << x;
    }
    const uint64_t G = fr & ~tm;
    t.zmask = all & ~G;
    t.fix = fx & ~tm;
    t.full = fr == all;
    t.pairs = c64 && t.q[0] == 0 && ((uintptr_t)s->amp & 15) == 0;
    const uint64_t groups = 1ULL << __builtin_popcountll(G);
    const uint64_t tiles = (groups + kRows - 1) / kRows;
    // complex128 tiles of 128 consecutive amplitudes per member (no inserted
    // bit below bit 7), all members read: bulk copies of the stage
    const bool bulk = !c64 && (t.zmask & 0x7Full) == 0 && groups % kRows == 0 && t.mmask == 0xFFFFFFFFu;
    // complex128 staging: 0 cp.async (every member in the support), 1 bulk
    // copies, 2 members outside the support (compacted, fewer K steps)
    const int mode = bulk ? 1 : t.mmask != 0xFFFFFFFFu ? 2 : 0;
    C128Kernel c128 = nullptr;
    if (!c64) {
        static const C128Kernel fns[2][3] = {
            {k_dense5_tc_c128_pipe<false, false, false>, k_dense5_tc_c128_pipe<false, true, false>,
             k_dense5_tc_c128_pipe<false, false, true>},
            {k_dense5_tc_c128_pipe<true, false, false>, k_dense5_tc_c128_pipe<true, true, false>,
             k_dense5_tc_c128_pipe<true, false, true>}};
        c128 = fns[fold][mode];
        if (!g_attr_c128[fold][mode][dev]) {
            cudaError_t e = cudaFuncSetAttribute((const void *)c128, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kSmemC128Pipe);
            if (e != cudaSuccess) return qs_fail(QS_ECUDA, "tc smem attribute: %s", cudaGetErrorString(e));
            g_attr_c128[fold][mode][dev] = true;
        }
    }
    int *status;
    int rc = qs_state_status(s, &status);
    if (rc) return rc;
    const qs_post_phase *post = (const qs_post_phase *)dev_post;
    cudaStream_t st = (cudaStream_t)s->stream;
    if (c64) {
        int grid = (int)std::min<uint64_t>(tiles, (uint64_t)sms * 2);
        if (fold)
            k_dense5_tc_c64<true><<<grid, kRows, kSmemF32, st>>>((float2 *)s->amp, groups, t,
                                                                (const float *)dev_pack, post, status);
        else
            k_dense5_tc_c64<false><<<grid, kRows, kSmemF32, st>>>((float2 *)s->amp, groups, t,
                                                                 (const float *)dev_pack, post, status);
    } else {
        int grid = (int)std::min<uint64_t>(tiles, (uint64_t)sms);
        c128<<<grid, kC128Threads, kSmemC128Pipe, st>>>((double2 *)s->amp, groups, t, (const uint8_t *)dev_pack,
                                                       post, status);
    }
    // amplitudes on the padding targets of an embedded cluster keep their
    // fixed values (U (x) 1 leaves zero inputs zero), so only the cluster's own
    // qubits join the support
    s->sup_free = (fr | (grow & tm)) == all ? ~0ULL : (fr | (grow & tm));
    s->sup_fix = fx & ~(grow & tm);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "tc launch: %s", cudaGetErrorString(e));
}

int qs_launch_wait_selftest(qs_state *s, long polls)
{
    int *status;
    int rc = qs_state_status(s, &status);
    if (rc) return rc;
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)s->stream>>>(status, polls);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "wait self-test launch: %s", cudaGetErrorString(e));
}

// Qubit swaps as one sweep over the state: the local bit swaps of Sec. 3.4 and
// the bit-location remapping of Sec. 3.6.  Swapping qubit a_j with qubit b_j
// (j < m) moves amplitude i to P(i), where P exchanges bits a_j and b_j of the
// index; P is its own inverse, so the sweep can run in place.
//
// Two kernels:
//   k_swap_pairs: every swapped bit is at least kPairLow.  Thread i exchanges
//     amplitudes i and P(i) when P(i) > i.  P leaves the low bits alone, so
//     neighbouring threads touch neighbouring amplitudes on both sides.
//   k_swap_tiled: some swapped bit is low.  With c = the lowest bit count that
//     covers the low swapped bits (at least kRunBits, so that every access is a
//     contiguous run of 2^c amplitudes) and H the swapped bits at c and above,
//     the 2^{c+|H|} amplitudes with the other bits fixed form a block that P
//     maps onto itself.  A CTA reads a block's 2^{|H|} runs into shared memory
//     and writes them back permuted (position table built once per CTA).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "qs_internal.h"

namespace {

constexpr int kPairLow = 3;          // k_swap_pairs when every swapped bit is >= 3
constexpr int kMaxBlockBits = 11;    // tiled blocks of at most 2^11 amplitudes
constexpr int kSwapThreads = 256;
constexpr int kMaxPairs = 32;        // one sweep: up to 32 exchanges (a state has at most 36 qubits)
constexpr size_t kTiledBytes = 32768; // amplitudes a tiled pass holds in shared memory

struct SwapPlan {
    uint64_t amask, bmask;           // bits a_j, b_j
    int a[kMaxPairs], b[kMaxPairs];
    int m;
    int c;                           // tiled: low run bits
    int h;                           // tiled: number of swapped bits >= c
    int hb[2 * kMaxPairs];           // tiled: those bits, ascending
    uint64_t zmask;                  // tiled: bits that do not enumerate blocks (low run + H)
    int lnb;                         // tiled: log2 of the blocks one pass holds
};

__host__ __device__ __forceinline__ uint64_t swap_bits(uint64_t i, const SwapPlan &p)
{
    uint64_t r = i & ~(p.amask | p.bmask);
    for (int j = 0; j < p.m; j++) {
        r |= ((i >> p.a[j]) & 1ULL) << p.b[j];
        r |= ((i >> p.b[j]) & 1ULL) << p.a[j];
    }
    return r;
}

template <typename C>
__global__ void __launch_bounds__(kSwapThreads)
k_swap_pairs(C *__restrict__ psi, uint64_t N, SwapPlan p)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        const uint64_t j = swap_bits(i, p);
        if (j > i) {
            const C x = psi[i], y = psi[j];
            psi[i] = y;
            psi[j] = x;
        }
    }
}

// block index -> index of its first amplitude: zeros inserted at zmask's bits
__device__ __forceinline__ uint64_t block_base(uint64_t g, uint64_t zmask)
{
    for (uint64_t z = zmask; z; z &= z - 1) {
        const uint64_t lo = g & ((z & (0 - z)) - 1);
        g = ((g ^ lo) << 1) | lo;
    }
    return g;
}

template <typename C>
__global__ void __launch_bounds__(kSwapThreads)
k_swap_tiled(C *__restrict__ psi, uint64_t n_blocks, SwapPlan p)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    constexpr int VEC = sizeof(C) == 8 ? 2 : 1;
    const int lb = p.c + p.h, B = 1 << lb, run = 1 << p.c;
    // nb consecutive blocks per pass (32 KB of amplitudes), so that every
    // thread has several loads in flight before the barrier
    const int lnb = p.lnb, nb = 1 << lnb;
    // buf holds each run with one element of padding, so that the permuted
    // reads (runs 2^c elements apart) fall in different banks
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int prun = run + 1;
    uint64_t *jdep = reinterpret_cast<uint64_t *>(smem_raw + sizeof(C) * ((size_t)prun << (p.h + lnb)));
    uint64_t *hoff = jdep + nb;                 // offset of run s: its H bits
    uint16_t *src = reinterpret_cast<uint16_t *>(hoff + (1 << p.h));
    // position q = (s, t) of a block (run s, offset t) holds, after the sweep,
    // the amplitude from position src[q]: P applied to q's index bits
    for (int q = threadIdx.x; q < B; q += blockDim.x) {
        const int s = q >> p.c, t = q & (run - 1);
        uint64_t idx = (uint64_t)t;
        for (int j = 0; j < p.h; j++) idx |= (uint64_t)((s >> j) & 1) << p.hb[j];
        const uint64_t from = swap_bits(idx, p);
        int fs = 0;
        for (int j = 0; j < p.h; j++) fs |= (int)((from >> p.hb[j]) & 1ULL) << j;
        src[q] = (uint16_t)((fs << p.c) | (int)(from & (uint64_t)(run - 1)));
    }
    for (int s = threadIdx.x; s < (1 << p.h); s += blockDim.x) {
        uint64_t o = 0;
        for (int j = 0; j < p.h; j++) o |= (uint64_t)((s >> j) & 1) << p.hb[j];
        hoff[s] = o;
    }
    // block pass * nb + j starts at block_base(pass * nb) + block_base(j): the
    // low lnb bits of a block index come from j alone
    for (int j = threadIdx.x; j < nb; j += blockDim.x) jdep[j] = block_base((uint64_t)j, p.zmask);
    const uint64_t n_pass = (n_blocks + nb - 1) >> lnb;
    for (uint64_t pass = blockIdx.x; pass < n_pass; pass += gridDim.x) {
        const uint64_t pbase = block_base(pass << lnb, p.zmask);
        __syncthreads();   // the previous pass's writes have read buf; the tables are ready
        // VEC neighbouring elements of a run per thread (16-byte global accesses
        // for complex64; a run is at least 8 elements)
        for (int e = threadIdx.x * VEC; e < (B << lnb); e += blockDim.x * VEC) {
            const int j = e >> lb, q = e & (B - 1);
            if ((pass << lnb) + (uint64_t)j >= n_blocks) continue;
            const C *g = psi + pbase + jdep[j] + hoff[q >> p.c] + (uint64_t)(q & (run - 1));
            C *d = buf + ((j << p.h) + (q >> p.c)) * prun + (q & (run - 1));
            if constexpr (VEC == 2) {
                const float4 w = *reinterpret_cast<const float4 *>(g);
                d[0] = make_float2(w.x, w.y);
                d[1] = make_float2(w.z, w.w);
            } else {
                d[0] = g[0];
            }
        }
        __syncthreads();
        for (int e = threadIdx.x * VEC; e < (B << lnb); e += blockDim.x * VEC) {
            const int j = e >> lb, q = e & (B - 1);
            if ((pass << lnb) + (uint64_t)j >= n_blocks) continue;
            C *g = psi + pbase + jdep[j] + hoff[q >> p.c] + (uint64_t)(q & (run - 1));
            const int f0 = src[q];
            const C v0 = buf[((j << p.h) + (f0 >> p.c)) * prun + (f0 & (run - 1))];
            if constexpr (VEC == 2) {
                const int f1 = src[q + 1];
                const C v1 = buf[((j << p.h) + (f1 >> p.c)) * prun + (f1 & (run - 1))];
                *reinterpret_cast<float4 *>(g) = make_float4(v0.x, v0.y, v1.x, v1.y);
            } else {
                g[0] = v0;
            }
        }
    }
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

int qs_launch_swap(qs_state *s, const int *a, const int *b, int m)
{
    s->perm_invariant = false;
    if (m == 0) return QS_OK;
    if (m > kMaxPairs) return qs_fail(QS_EINVAL, "swap: %d pairs", m);
    int rc = qs_materialize(s);
    if (rc) return rc;
    SwapPlan p;
    std::memset(&p, 0, sizeof(p));
    p.m = m;
    int lowest_low = -1;
    for (int j = 0; j < m; j++) {
        p.a[j] = a[j];
        p.b[j] = b[j];
        p.amask |= 1ULL << a[j];
        p.bmask |= 1ULL << b[j];
        const int lo = std::min(a[j], b[j]);
        if (lo < kPairLow) lowest_low = std::max(lowest_low, lo);
    }
    const uint64_t N = 1ULL << s->n;
    const bool c128 = s->dtype == QS_C128;
    cudaStream_t st = (cudaStream_t)s->stream;
    const int sms = sm_count();
    bool tiled = false;
    size_t smem = 0;
    if (lowest_low >= 0) {
        // run bits: cover every swapped bit below kPairLow (and any swapped bit
        // just above, which would otherwise count towards H), at least 5 bits
        // for complex128 (512-byte runs) and 6 for complex64
        int c = std::max(c128 ? 5 : 6, lowest_low + 1);
        c = std::min(c, s->n);
        int h = 0;
        for (int j = 0; j < m; j++) {
            if (a[j] >= c) p.hb[h++] = a[j];
            if (b[j] >= c) p.hb[h++] = b[j];
        }
        std::sort(p.hb, p.hb + h);
        if (c + h <= kMaxBlockBits) {
            tiled = true;
            p.c = c;
            p.h = h;
            p.zmask = (1ULL << c) - 1;
            for (int j = 0; j < h; j++) p.zmask |= 1ULL << p.hb[j];
            const size_t B = (size_t)1 << (c + h), asz = c128 ? 16 : 8;
            const size_t nb = std::max<size_t>(1, kTiledBytes / asz / B);
            p.lnb = __builtin_ctzll(nb);
            smem = asz * (((size_t)1 << c) + 1) * ((size_t)1 << h) * nb + 8 * nb + 8 * ((size_t)1 << h) + 2 * B;
        }
    }
    if (tiled) {
        const uint64_t n_blocks = N >> (p.c + p.h);
        const uint64_t nb = 1ULL << p.lnb;
        const int grid = (int)std::min<uint64_t>((n_blocks + nb - 1) / nb, (uint64_t)sms * 5);
        if (c128)
            k_swap_tiled<double2><<<grid, kSwapThreads, smem, st>>>((double2 *)s->amp, n_blocks, p);
        else
            k_swap_tiled<float2><<<grid, kSwapThreads, smem, st>>>((float2 *)s->amp, n_blocks, p);
    } else {
        const int grid = (int)std::min<uint64_t>((N + kSwapThreads - 1) / kSwapThreads, (uint64_t)sms * 8);
        if (c128)
            k_swap_pairs<double2><<<grid, kSwapThreads, 0, st>>>((double2 *)s->amp, N, p);
        else
            k_swap_pairs<float2><<<grid, kSwapThreads, 0, st>>>((float2 *)s->amp, N, p);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "swap launch: %s", cudaGetErrorString(e));
}

// Host side of the same permutation (used to map indices between orders).
uint64_t qs_swap_index(uint64_t i, const int *a, const int *b, int m)
{
    uint64_t amask = 0, bmask = 0;
    for (int j = 0; j < m; j++) {
        amask |= 1ULL << a[j];
        bmask |= 1ULL << b[j];
    }
    uint64_t r = i & ~(amask | bmask);
    for (int j = 0; j < m; j++) {
        r |= ((i >> a[j]) & 1ULL) << b[j];
        r |= ((i >> b[j]) & 1ULL) << a[j];
    }
    return r;
}

int qs_order_set(qs_state *s, const int *want)
{
    int target[64];
    bool same = true;
    for (int q = 0; q < s->n; q++) {
        target[q] = want ? want[q] : q;
        same = same && target[q] == s->loc[q];
    }
    if (same) return QS_OK;
    if (s->perm_invariant) {
        // every amplitude equal: the qubits change places without moving data
        for (int q = 0; q < s->n; q++) s->loc[q] = target[q];
        return QS_OK;
    }
    if (s->sup_free == 0) {
        // the lazily written basis state: its one amplitude moves, nothing else
        const uint64_t x = qs_loc_index(s, s->sup_fix);      // index in qubit order
        for (int q = 0; q < s->n; q++) s->loc[q] = target[q];
        return qs_basis_move(s, qs_loc_index(s, x));
    }
    // undo the present exchanges, then make the wanted ones
    int a[kMaxPairs], b[kMaxPairs], m = 0;
    for (int q = 0; q < s->n; q++)
        if (s->loc[q] > q) {
            a[m] = q;
            b[m++] = s->loc[q];
        }
    int rc = qs_launch_swap(s, a, b, m);
    if (rc) return rc;
    for (int q = 0; q < s->n; q++) s->loc[q] = q;
    m = 0;
    for (int q = 0; q < s->n; q++)
        if (target[q] > q) {
            a[m] = q;
            b[m++] = target[q];
        }
    if ((rc = qs_launch_swap(s, a, b, m))) return rc;
    for (int q = 0; q < s->n; q++) s->loc[q] = target[q];
    return QS_OK;
}

extern "C" int qs_swap_qubits(qs_state *s, const int *a, const int *b, int m)
{
    return qs_guard([&]() -> int {
        if (!s || !s->amp) return qs_fail(QS_EINVAL, "qs_swap_qubits: null state");
        if (m < 0 || m > QS_MAX_SWAP || (m > 0 && (!a || !b)))
            return qs_fail(QS_EINVAL, "qs_swap_qubits: m = %d outside [0, %d]", m, QS_MAX_SWAP);
        uint64_t seen = 0;
        for (int j = 0; j < m; j++) {
            for (int q : {a[j], b[j]}) {
                if (q < 0 || q >= s->n) return qs_fail(QS_EINVAL, "qs_swap_qubits: qubit %d outside [0, %d)", q, s->n);
                if ((seen >> q) & 1) return qs_fail(QS_EINVAL, "qs_swap_qubits: qubit %d named twice", q);
                seen |= 1ULL << q;
            }
        }
        // the qubits' present bit locations
        int pa[QS_MAX_SWAP], pb[QS_MAX_SWAP];
        for (int j = 0; j < m; j++) {
            pa[j] = qs_loc(s, a[j]);
            pb[j] = qs_loc(s, b[j]);
        }
        return qs_launch_swap(s, pa, pb, m);
    });
}

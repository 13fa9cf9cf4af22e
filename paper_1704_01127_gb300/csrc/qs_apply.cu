// State sweeps of the hot path: dense k-qubit cluster apply (Sec. 3.2), table
// diagonals and CZ/T phase products (Sec. 2, Sec. 3.5), and the schedule runner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace {

using qsd::cplx;
using qsd::Targets;
using qsd::group_base;
using qsd::member_offset;
using qsd::rotate8;

int g_sms = 0;
int sm_count()
{
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    return g_sms;
}

// Dense k-qubit cluster: one thread per group c, the 2^K amplitudes gathered at
// strides 2^{q_j} into registers, v <- U v, scattered back in place.  Each
// complex multiply-accumulate is the pair of real FMA updates of Eqs. (2)-(3):
// acc += (v_R m_R, v_I m_R) then acc += (-v_I m_I, v_R m_I).  U (row-major,
// ascending qubit order) is staged once per CTA in shared memory and read as a
// warp-uniform broadcast.  Consecutive threads take consecutive groups, so for
// targets above bit 4 every gathered row of a warp is one contiguous segment.
template <typename R, int K>
__global__ void __launch_bounds__(128)
k_dense(typename cplx<R>::t *__restrict__ psi, uint64_t n_groups, Targets t,
        const R *__restrict__ Ug)
{
    using C = typename cplx<R>::t;
    constexpr int D = 1 << K;
    __shared__ C Us[D * D];
    for (int i = threadIdx.x; i < D * D; i += blockDim.x)
        Us[i] = reinterpret_cast<const C *>(Ug)[i];
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_groups; g += stride)
        qsd::dense_group<R, K, false>(psi + group_base<K>(g, t), t, Us);
}

// Table diagonal on up to QS_MAX_DIAG_K qubits: psi_i *= d[x(i)].
template <typename R>
__global__ void k_diag(typename cplx<R>::t *__restrict__ psi, uint64_t N, int k, const int *__restrict__ qg,
                       const R *__restrict__ dg)
{
    using C = typename cplx<R>::t;
    __shared__ int q[QS_MAX_DIAG_K];
    if (threadIdx.x < k) q[threadIdx.x] = qg[threadIdx.x];
    __syncthreads();
    const C *d = reinterpret_cast<const C *>(dg);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
        int x = 0;
        for (int j = 0; j < k; j++) x |= (int)((i >> q[j]) & 1) << j;
        C m = __ldg(&d[x]);
        C a = psi[i], o;
        o.x = a.x * m.x - a.y * m.y;
        o.y = a.x * m.y + a.y * m.x;
        psi[i] = o;
    }
}

// Product of T-type phases and CZ signs (Sec. 2, Sec. 3.5): amplitude i gets
// e^{i pi m(i)/4}, m(i) = sum_q c_q i_q + 4 sum_a i_a popc(i & P_a) mod 8, with
// P_a the CZ partners b > a of qubit a.  The index splits into low bits l
// (below L) and high bits h.  The low part m_lo(l) (the c_q and partner pairs
// inside the low bits) is a table built once per CTA in shared memory; every
// chunk of 2^L amplitudes shares h, so m_hi(h) and the mask M_h of low qubits
// whose partner set meets h an odd number of times are computed once per
// chunk:  m(i) = m_lo(l) + m_hi(h) + 4 popc(l & M_h).  CZ-only ops cost no
// floating-point work.
constexpr int kPhaseLowBits = 14;

template <typename R>
__global__ void __launch_bounds__(256)
k_phase(typename cplx<R>::t *__restrict__ psi, int n, const qs_phase_dev *__restrict__ ph, int n_act)
{
    using C = typename cplx<R>::t;
    __shared__ uint8_t tab[1 << kPhaseLowBits];
    __shared__ uint64_t part[64];
    __shared__ int act[64];
    const int L = n < kPhaseLowBits ? n : kPhaseLowBits;
    const uint64_t c0 = ph->cmask[0], c1 = ph->cmask[1], c2 = ph->cmask[2];
    const qs_phase_term *terms = reinterpret_cast<const qs_phase_term *>(ph + 1);
    for (int i = threadIdx.x; i < n_act; i += blockDim.x) {
        part[i] = terms[i].partners;
        act[i] = terms[i].a;
    }
    __syncthreads();
    const uint64_t cm[3] = {c0, c1, c2};
    for (int l = threadIdx.x; l < (1 << L); l += blockDim.x) tab[l] = qsd::phase_low((uint64_t)l, cm, act, part, n_act, L);
    __syncthreads();
    const uint64_t n_chunks = 1ULL << (n - L);
    for (uint64_t ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
        const uint64_t h = ch << L;
        uint64_t Mh;
        const int mh = qsd::phase_high(h, cm, act, part, n_act, L, Mh);
        C *base = psi + h;
        for (int l = threadIdx.x; l < (1 << L); l += blockDim.x) {
            const int m = (tab[l] + mh + 4 * __popcll((uint64_t)l & Mh)) & 7;
            if (m) base[l] = rotate8<C, R>(base[l], m);
        }
    }
}

int grid_for(uint64_t work, int block, int per_sm)
{
    uint64_t want = (work + block - 1) / block;
    uint64_t cap = (uint64_t)sm_count() * per_sm;
    if (want < 1) want = 1;
    return (int)std::min<uint64_t>(want, cap);
}

template <typename R, int K>
int launch_dense_t(qs_state *s, const int *q, const void *U)
{
    Targets t;
    for (int j = 0; j < K; j++) t.q[j] = q[j];
    uint64_t groups = 1ULL << (s->n - K);
    const int block = 128;
    int grid = grid_for(groups, block, 8);
    k_dense<R, K><<<grid, block, 0, (cudaStream_t)s->stream>>>(
        reinterpret_cast<typename cplx<R>::t *>(s->amp), groups, t, reinterpret_cast<const R *>(U));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "k_dense launch: %s", cudaGetErrorString(e));
}

template <typename R>
int launch_dense_r(qs_state *s, const int *q, int k, const void *U)
{
    switch (k) {
    case 1: return launch_dense_t<R, 1>(s, q, U);
    case 2: return launch_dense_t<R, 2>(s, q, U);
    case 3: return launch_dense_t<R, 3>(s, q, U);
    case 4: return launch_dense_t<R, 4>(s, q, U);
    case 5: return launch_dense_t<R, 5>(s, q, U);
    default: return qs_fail(QS_EINVAL, "dense cluster of %d qubits", k);
    }
}

}  // namespace

// complex64: clusters of 4 and 5 qubits (a 4-qubit cluster embedded in 5 on
// the tensor cores measured 11.3 ms at 32 qubits against 16.1 ms for the FP32
// CUDA-core sweep, which is FMA-bound there); complex128: every cluster of 2 or
// more qubits (native FP64 runs at 1/58 of the FP32 rate).  Tensor-core sweeps
// need n >= 5.
bool qs_tc_wanted(int dtype, int k, int n)
{
    if (n < 5) return false;
    return dtype == QS_C64 ? k >= 4 : k >= 2;
}

int qs_launch_dense(qs_state *s, const int *sorted_qubits, int k, const void *dev_matrix,
                    const void *dev_tc)
{
    s->perm_invariant = false;
    if (k == 5 && dev_tc) return qs_launch_dense5_tc(s, sorted_qubits, dev_tc, ~0ULL);
    int rc = qs_materialize(s);   // the CUDA-core sweeps read every amplitude
    if (rc) return rc;
    return s->dtype == QS_C128 ? launch_dense_r<double>(s, sorted_qubits, k, dev_matrix)
                               : launch_dense_r<float>(s, sorted_qubits, k, dev_matrix);
}

int qs_launch_diag(qs_state *s, const int *dev_qubits, int k, const void *dev_table)
{
    s->perm_invariant = false;
    int rc = qs_materialize(s);
    if (rc) return rc;
    uint64_t N = 1ULL << s->n;
    const int block = 256;
    int grid = grid_for(N, block, 8);
    cudaStream_t st = (cudaStream_t)s->stream;
    if (s->dtype == QS_C128)
        k_diag<double><<<grid, block, 0, st>>>((double2 *)s->amp, N, k, dev_qubits, (const double *)dev_table);
    else
        k_diag<float><<<grid, block, 0, st>>>((float2 *)s->amp, N, k, dev_qubits, (const float *)dev_table);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "k_diag launch: %s", cudaGetErrorString(e));
}

int qs_launch_phase(qs_state *s, const void *dev_phase, int n_act)
{
    s->perm_invariant = false;
    int rc = qs_materialize(s);
    if (rc) return rc;
    const int L = s->n < kPhaseLowBits ? s->n : kPhaseLowBits;
    const uint64_t chunks = 1ULL << (s->n - L);
    const int block = 256;
    int grid = (int)std::min<uint64_t>(chunks, (uint64_t)sm_count() * 8);
    cudaStream_t st = (cudaStream_t)s->stream;
    if (s->dtype == QS_C128)
        k_phase<double><<<grid, block, 0, st>>>((double2 *)s->amp, s->n, (const qs_phase_dev *)dev_phase, n_act);
    else
        k_phase<float><<<grid, block, 0, st>>>((float2 *)s->amp, s->n, (const qs_phase_dev *)dev_phase, n_act);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "k_phase launch: %s", cudaGetErrorString(e));
}

// ------------------------------------------------------------------ host side

namespace {

// Sorted copy of (qubits, matrix): ascending qubit order, the matrix permuted so
// that bit j of its index belongs to the j-th smallest qubit (Sec. 3.2).
void sort_targets(const int *qubits, int k, const double *U, bool dense, int *qs_out,
                  std::vector<double> &M)
{
    int perm[QS_MAX_DIAG_K];
    for (int j = 0; j < k; j++) perm[j] = j;
    std::sort(perm, perm + k, [&](int a, int b) { return qubits[a] < qubits[b]; });
    for (int j = 0; j < k; j++) qs_out[j] = qubits[perm[j]];
    auto remap = [&](int xn) {
        int xo = 0;
        for (int j = 0; j < k; j++) xo |= ((xn >> j) & 1) << perm[j];
        return xo;
    };
    const int d = 1 << k;
    if (dense) {
        M.resize(2 * d * d);
        for (int r = 0; r < d; r++)
            for (int c = 0; c < d; c++) {
                int ro = remap(r), co = remap(c);
                M[2 * (r * d + c)] = U[2 * (ro * d + co)];
                M[2 * (r * d + c) + 1] = U[2 * (ro * d + co) + 1];
            }
    } else {
        M.resize(2 * d);
        for (int x = 0; x < d; x++) {
            M[2 * x] = U[2 * remap(x)];
            M[2 * x + 1] = U[2 * remap(x) + 1];
        }
    }
}

// Pack FP64 values into the state's real type.
std::vector<uint8_t> to_real(const std::vector<double> &v, int dtype)
{
    std::vector<uint8_t> out;
    if (dtype == QS_C128) {
        out.resize(v.size() * sizeof(double));
        std::memcpy(out.data(), v.data(), out.size());
    } else {
        out.resize(v.size() * sizeof(float));
        float *f = reinterpret_cast<float *>(out.data());
        for (size_t i = 0; i < v.size(); i++) f[i] = (float)v[i];
    }
    return out;
}


int check_state(qs_state *s, const char *who)
{
    if (!s || !s->amp) return qs_fail(QS_EINVAL, "%s: null state", who);
    return QS_OK;
}

// Stage a small operand block in the state's scratch (stream-ordered: the copy
// runs after earlier kernels on the stream have finished reading the slot).
int stage(qs_state *s, const void *host, size_t bytes, void **dev)
{
    void *p = nullptr;
    int rc = qs_state_scratch(s, bytes, &p);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(p, host, bytes, cudaMemcpyHostToDevice, (cudaStream_t)s->stream);
    if (e != cudaSuccess) return qs_fail(QS_ECUDA, "operand copy: %s", cudaGetErrorString(e));
    *dev = p;
    return QS_OK;
}

int check_qubits(qs_state *s, const int *qubits, int k, int kmax, const char *who)
{
    if (!qubits || k < 1 || k > kmax || k > s->n)
        return qs_fail(QS_EINVAL, "%s: k = %d not in [1, %d] or above n", who, k, kmax);
    uint64_t seen = 0;
    for (int j = 0; j < k; j++) {
        if (qubits[j] < 0 || qubits[j] >= s->n)
            return qs_fail(QS_EINVAL, "%s: qubit %d out of range", who, qubits[j]);
        if ((seen >> qubits[j]) & 1) return qs_fail(QS_EINVAL, "%s: qubit %d repeated", who, qubits[j]);
        seen |= 1ULL << qubits[j];
    }
    return QS_OK;
}

// Which dense clusters go to the tensor cores (qs_tc_wanted): complex64 clusters
// of 4 and 5 qubits, complex128 clusters of 2 or more; smaller ones are
// embedded in 5 qubits.
bool tc_wanted(int dtype, int k, int n) { return qs_tc_wanted(dtype, k, n); }

// U (x) 1: a k-qubit cluster (sorted qubits q, sorted matrix M) as a 5-qubit
// one on q plus the highest qubits not in q; output sorted as well.
void embed5(const int *q, int k, const std::vector<double> &M, int n, std::array<int, 5> &q5,
            std::vector<double> &M5)
{
    uint64_t used = 0;
    for (int j = 0; j < k; j++) used |= 1ULL << q[j];
    // pad with the highest free qubits: low qubits as targets would make the
    // tile gather touch one amplitude per group instead of runs of groups
    uint64_t all = used;
    for (int b = n - 1; b >= 0 && __builtin_popcountll(all) < 5; b--) all |= 1ULL << b;
    int pos[5], j5 = 0;
    for (int b = 0; b < n; b++)
        if ((all >> b) & 1) q5[j5++] = b;
    // position of each original target within q5
    for (int j = 0; j < k; j++)
        for (int i = 0; i < 5; i++)
            if (q5[i] == q[j]) pos[j] = i;
    uint32_t extra = 0;
    for (int i = 0; i < 5; i++)
        if (!((used >> q5[i]) & 1)) extra |= 1u << i;
    const int d = 1 << k;
    M5.assign(2 * 32 * 32, 0.0);
    for (int r5 = 0; r5 < 32; r5++)
        for (int c5 = 0; c5 < 32; c5++) {
            if ((r5 & extra) != (c5 & extra)) continue;
            int r = 0, c = 0;
            for (int j = 0; j < k; j++) {
                r |= ((r5 >> pos[j]) & 1) << j;
                c |= ((c5 >> pos[j]) & 1) << j;
            }
            M5[2 * (r5 * 32 + c5)] = M[2 * (r * d + c)];
            M5[2 * (r5 * 32 + c5) + 1] = M[2 * (r * d + c) + 1];
        }
}

std::vector<uint8_t> tc_pack_for(int dtype, const std::vector<double> &M5)
{
    return dtype == QS_C64 ? qs_pack_tc_c64(M5) : qs_pack_tc_c128(M5);
}

// Fold of phase op ph into the tensor-core sweep on the sorted qubits q5 with
// matrix M5 (qs_post_phase): M5f = D M5, D the diagonal of the phase terms on
// q5 (coefficients and CZ pairs with both ends in q5, Sec. 2), and desc the
// rest: CZ pairs with one or no end in q5 and the coefficients off q5, which
// act on each group as a conditional Z on a target or a phase of the group
// (Sec. 3.5).  False when a coefficient off q5 is odd (its factor is not a
// power of i) or there are more CZ terms off q5 than the kernel holds.
bool fold_phase(int n, const std::array<int, 5> &q5, const std::vector<double> &M5, const qs_op_host &ph,
                std::vector<double> &M5f, std::vector<uint8_t> &desc)
{
    int pos[64];
    std::fill(pos, pos + 64, -1);
    for (int j = 0; j < 5; j++) pos[q5[j]] = j;
    qs_post_phase hdr;
    std::memset(&hdr, 0, sizeof(hdr));
    int cq[5] = {0, 0, 0, 0, 0};        // coefficient of qubit q5[j]
    for (int q = 0; q < n; q++) {
        const int c = ((ph.coeff[q] % 8) + 8) % 8;
        if (pos[q] >= 0) {
            cq[pos[q]] = c;
        } else {
            if (c & 1) return false;
            if (c & 2) hdr.c1 |= 1ULL << q;
            if (c & 4) hdr.c2 |= 1ULL << q;
        }
    }
    uint32_t inner[5] = {0, 0, 0, 0, 0};   // bit j' of inner[j]: CZ (q5[j], q5[j']), j < j', mod 2
    std::vector<uint64_t> partners(n, 0);
    for (const auto &e : ph.edges) {
        const int a = std::min(e.first, e.second), b = std::max(e.first, e.second);
        const int ja = pos[a], jb = pos[b];
        if (ja >= 0 && jb >= 0) inner[ja] ^= 1u << jb;
        else if (ja >= 0) hdr.tp[ja] ^= 1ULL << b;
        else if (jb >= 0) hdr.tp[jb] ^= 1ULL << a;
        else partners[a] ^= 1ULL << b;
    }
    std::vector<qs_phase_term> terms;
    for (int a = 0; a < n; a++)
        if (partners[a]) terms.push_back({partners[a], a, 0});
    if ((int)terms.size() > QS_MAX_POST_TERMS) return false;
    hdr.n_terms = (int32_t)terms.size();
    // row m of M5 times w^{s(m)}, w = e^{i pi / 4}: exact for even s
    const double r = std::sqrt(0.5);
    const double wr[8] = {1, r, 0, -r, -1, -r, 0, r}, wi[8] = {0, r, 1, r, 0, -r, -1, -r};
    M5f.assign(M5.size(), 0.0);
    for (int m = 0; m < 32; m++) {
        int sm = 0;
        for (int j = 0; j < 5; j++)
            if ((m >> j) & 1) sm += cq[j] + 4 * __builtin_popcount(inner[j] & (uint32_t)m);
        sm &= 7;
        for (int x = 0; x < 32; x++) {
            const double a = M5[2 * (m * 32 + x)], b = M5[2 * (m * 32 + x) + 1];
            M5f[2 * (m * 32 + x)] = a * wr[sm] - b * wi[sm];
            M5f[2 * (m * 32 + x) + 1] = a * wi[sm] + b * wr[sm];
        }
    }
    desc.resize(sizeof(hdr) + terms.size() * sizeof(qs_phase_term));
    std::memcpy(desc.data(), &hdr, sizeof(hdr));
    if (!terms.empty()) std::memcpy(desc.data() + sizeof(hdr), terms.data(), terms.size() * sizeof(qs_phase_term));
    return true;
}

// Append bytes to an op's data at a 256-byte boundary; returns their offset.
size_t append_aligned(std::vector<uint8_t> &part, const std::vector<uint8_t> &bytes)
{
    const size_t at = (part.size() + 255) & ~(size_t)255;
    part.resize(at + bytes.size());
    std::memcpy(part.data() + at, bytes.data(), bytes.size());
    return at;
}

// Device image of a schedule for one dtype: every op's data, 256-byte aligned.
std::vector<uint8_t> schedule_blob(const qs_schedule *sc, int dtype, qs_dev_sched &d)
{
    std::vector<uint8_t> blob;
    const size_t nops = sc->ops.size();
    std::vector<size_t> &offset = d.offset, &tc_off = d.tc_off;
    std::vector<std::array<int, 5>> &tc_q = d.tc_q;
    offset.assign(nops, 0);
    d.n_act.assign(nops, 0);
    tc_off.assign(nops, 0);
    d.fold_off.assign(nops, 0);
    d.post_off.assign(nops, 0);
    tc_q.assign(nops, std::array<int, 5>{{0, 0, 0, 0, 0}});
    std::vector<int> &n_act = d.n_act;
    for (size_t i = 0; i < sc->ops.size(); i++) {
        const qs_op_host &op = sc->ops[i];
        std::vector<uint8_t> part;
        if (op.kind == QS_OP_PHASE) {
            part = qs_pack_phase(sc->n, op.coeff, op.edges, &n_act[i]);
        } else if (op.kind == QS_OP_DIAG) {
            std::vector<uint8_t> tab = to_real(op.matrix, dtype);
            part.resize(64 + tab.size());
            std::memcpy(part.data(), op.qubits, sizeof(int) * op.k);
            std::memcpy(part.data() + 64, tab.data(), tab.size());
        } else {
            part = to_real(op.matrix, dtype);
            if (sc->n >= 5) {   // tensor-core operands for every dense op (any path may run it)
                std::vector<double> M5;
                if (op.k == 5) {
                    for (int j = 0; j < 5; j++) tc_q[i][j] = op.qubits[j];
                    M5 = op.matrix;
                } else {
                    embed5(op.qubits, op.k, op.matrix, sc->n, tc_q[i], M5);
                }
                tc_off[i] = append_aligned(part, tc_pack_for(dtype, M5));
                // a phase op right after it can run inside its sweep
                std::vector<double> M5f;
                std::vector<uint8_t> desc;
                if (i + 1 < nops && sc->ops[i + 1].kind == QS_OP_PHASE &&
                    fold_phase(sc->n, tc_q[i], M5, sc->ops[i + 1], M5f, desc)) {
                    d.fold_off[i] = append_aligned(part, tc_pack_for(dtype, M5f));
                    d.post_off[i] = append_aligned(part, desc);
                }
            }
        }
        size_t at = (blob.size() + 255) & ~(size_t)255;
        blob.resize(at + part.size());
        std::memcpy(blob.data() + at, part.data(), part.size());
        offset[i] = at;
    }
    if (blob.empty()) blob.resize(256);
    return blob;
}

int ensure_dev_schedule(qs_state *s, const qs_schedule *csc)
{
    qs_schedule *sc = const_cast<qs_schedule *>(csc);
    qs_dev_sched &d = sc->dev[s->dtype];
    int dev = 0;
    cudaGetDevice(&dev);
    if (d.pool && d.device == dev) return QS_OK;
    if (d.pool) {
        cudaFree(d.pool);
        d.pool = nullptr;
    }
    std::vector<uint8_t> blob = schedule_blob(sc, s->dtype, d);
    cudaError_t e = cudaMalloc(&d.pool, blob.size());
    if (e != cudaSuccess) {
        d.pool = nullptr;
        return qs_fail(QS_ENOMEM, "schedule upload: %s", cudaGetErrorString(e));
    }
    // copied on a stream of its own that waits for nothing, so an upload made
    // ahead of time does not wait for kernels running on other streams
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.pool, blob.data(), blob.size(), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaFree(d.pool);
        d.pool = nullptr;
        return qs_fail(QS_ECUDA, "schedule upload: %s", cudaGetErrorString(e));
    }
    d.bytes = blob.size();
    d.device = dev;
    return QS_OK;
}

// Kernel path of a dense op: the state's setting if not AUTO, else the op's
// planned path if any, else the default policy.  *folded: the phase op after
// it ran inside its tensor-core sweep.
int path_of(const qs_state *s, const qs_op_host &op)
{
    return s->path != QS_PATH_AUTO ? s->path
           : op.path != QS_PATH_AUTO ? op.path
           : (tc_wanted(s->dtype, op.k, s->n) ? QS_PATH_TENSOR : QS_PATH_CUDA_CORES);
}

// Dense ops i and i + 1 as one sweep (qs_pair.cu) when both run on the tensor
// cores and their target qubits fit one super-group; *skip = the ops after i
// that ran inside it (the second cluster, and a phase op folded into it).
bool try_pair(qs_state *s, const qs_schedule *sc, const qs_dev_sched &d, size_t i, int *rc, int *skip)
{
    if (!s->pair_sweeps || s->dtype != QS_C64 || i + 1 >= sc->ops.size()) return false;
    const qs_op_host &a = sc->ops[i], &b = sc->ops[i + 1];
    if (a.kind != QS_OP_DENSE || b.kind != QS_OP_DENSE || !d.tc_off[i] || !d.tc_off[i + 1]) return false;
    if (path_of(s, a) != QS_PATH_TENSOR || path_of(s, b) != QS_PATH_TENSOR) return false;
    if (!qs_pair_possible(s, d.tc_q[i].data(), d.tc_q[i + 1].data())) return false;
    const uint8_t *da = (const uint8_t *)d.pool + d.offset[i], *db = (const uint8_t *)d.pool + d.offset[i + 1];
    const bool fold = s->fold_phase && d.fold_off[i + 1];
    *rc = qs_launch_pair5_tc(s, d.tc_q[i].data(), da + d.tc_off[i], d.tc_q[i + 1].data(),
                             db + (fold ? d.fold_off[i + 1] : d.tc_off[i + 1]), fold ? db + d.post_off[i + 1] : nullptr);
    *skip = fold ? 2 : 1;
    return true;
}

int launch_op_dense(qs_state *s, const qs_dev_sched &d, size_t i, const qs_op_host &op, const uint8_t *data,
                    bool *folded)
{
    *folded = false;
    int path = path_of(s, op);
    if (path == QS_PATH_TENSOR && d.tc_off[i]) {
        uint64_t grow = 0;
        for (int j = 0; j < op.k; j++) grow |= 1ULL << op.qubits[j];
        if (s->fold_phase && d.fold_off[i]) {
            *folded = true;
            return qs_launch_dense5_tc(s, d.tc_q[i].data(), data + d.fold_off[i], grow, data + d.post_off[i]);
        }
        return qs_launch_dense5_tc(s, d.tc_q[i].data(), data + d.tc_off[i], grow);
    }
    return qs_launch_dense(s, op.qubits, op.k, data, nullptr);
}

}  // namespace

extern "C" int qs_apply_cluster(qs_state *s, const int *qubits, int k, const double *U)
{
    return qs_guard([&]() -> int {
        int rc = check_state(s, "qs_apply_cluster");
        if (rc) return rc;
        if ((rc = check_qubits(s, qubits, k, QS_MAX_K, "qs_apply_cluster"))) return rc;
        if (!U) return qs_fail(QS_EINVAL, "qs_apply_cluster: null matrix");
        int lq[QS_MAX_K], q[QS_MAX_K];
        for (int j = 0; j < k; j++) lq[j] = qs_loc(s, qubits[j]);   // the qubits' index bits
        std::vector<double> M;
        sort_targets(lq, k, U, true, q, M);
        const bool tc = s->path == QS_PATH_TENSOR ? s->n >= 5
                                                  : s->path == QS_PATH_AUTO && tc_wanted(s->dtype, k, s->n);
        if (tc) {
            std::array<int, 5> q5;
            std::vector<double> M5;
            if (k == 5) {
                for (int j = 0; j < 5; j++) q5[j] = q[j];
                M5 = M;
            } else {
                embed5(q, k, M, s->n, q5, M5);
            }
            std::vector<uint8_t> p = tc_pack_for(s->dtype, M5);
            void *dp = nullptr;
            if ((rc = stage(s, p.data(), p.size(), &dp))) return rc;
            uint64_t grow = 0;
            for (int j = 0; j < k; j++) grow |= 1ULL << q[j];
            return qs_launch_dense5_tc(s, q5.data(), dp, grow);
        }
        std::vector<uint8_t> packed = to_real(M, s->dtype);
        void *dU = nullptr;
        if ((rc = stage(s, packed.data(), packed.size(), &dU))) return rc;
        return qs_launch_dense(s, q, k, dU, nullptr);
    });
}

extern "C" int qs_apply_diag(qs_state *s, const int *qubits, int k, const double *d)
{
    return qs_guard([&]() -> int {
        int rc = check_state(s, "qs_apply_diag");
        if (rc) return rc;
        if ((rc = check_qubits(s, qubits, k, QS_MAX_DIAG_K, "qs_apply_diag"))) return rc;
        if (!d) return qs_fail(QS_EINVAL, "qs_apply_diag: null table");
        int lq[QS_MAX_DIAG_K], q[QS_MAX_DIAG_K];
        for (int j = 0; j < k; j++) lq[j] = qs_loc(s, qubits[j]);   // the qubits' index bits
        std::vector<double> M;
        sort_targets(lq, k, d, false, q, M);
        std::vector<uint8_t> tab = to_real(M, s->dtype);
        std::vector<uint8_t> blob(64 + tab.size());
        std::memcpy(blob.data(), q, sizeof(int) * k);
        std::memcpy(blob.data() + 64, tab.data(), tab.size());
        void *dev = nullptr;
        if ((rc = stage(s, blob.data(), blob.size(), &dev))) return rc;
        return qs_launch_diag(s, (const int *)dev, k, (const uint8_t *)dev + 64);
    });
}

extern "C" int qs_apply_phase(qs_state *s, const int *coeff, int n_edges, const int *edges)
{
    return qs_guard([&]() -> int {
        int rc = check_state(s, "qs_apply_phase");
        if (rc) return rc;
        if (!coeff || n_edges < 0 || (n_edges > 0 && !edges))
            return qs_fail(QS_EINVAL, "qs_apply_phase: bad arguments");
        // coefficients and CZ pairs on the qubits' index bits
        std::vector<int32_t> c(s->n);
        for (int q = 0; q < s->n; q++) c[qs_loc(s, q)] = coeff[q];
        std::vector<std::pair<int, int>> e;
        for (int i = 0; i < n_edges; i++) {
            int a = edges[2 * i], b = edges[2 * i + 1];
            if (a < 0 || a >= s->n || b < 0 || b >= s->n || a == b)
                return qs_fail(QS_EINVAL, "qs_apply_phase: bad edge %d", i);
            e.push_back({qs_loc(s, a), qs_loc(s, b)});
        }
        int n_act;
        std::vector<uint8_t> blob = qs_pack_phase(s->n, c, e, &n_act);
        void *dev = nullptr;
        if ((rc = stage(s, blob.data(), blob.size(), &dev))) return rc;
        return qs_launch_phase(s, dev, n_act);
    });
}

extern "C" int qs_run_circuit(qs_state *s, const qs_schedule *sc)
{
    return qs_guard([&]() -> int {
        int rc = check_state(s, "qs_run_circuit");
        if (rc) return rc;
        if (!sc || sc->n != s->n) return qs_fail(QS_EINVAL, "qs_run_circuit: schedule/state qubit mismatch");
        if ((rc = ensure_dev_schedule(s, sc))) return rc;
        // the schedule's ops name index bits: put the qubits where it expects them
        if ((rc = qs_order_set(s, sc->remap.empty() ? nullptr : sc->remap.data()))) return rc;
        const qs_dev_sched &d = sc->dev[s->dtype];
        for (size_t i = 0; i < sc->ops.size(); i++) {
            const qs_op_host &op = sc->ops[i];
            const uint8_t *data = (const uint8_t *)d.pool + d.offset[i];
            int skip = 0;
            if (op.kind == QS_OP_DENSE && try_pair(s, sc, d, i, &rc, &skip)) {
                i += skip;         // the ops after it that ran inside the pair's sweep
            } else if (op.kind == QS_OP_DENSE) {
                bool folded;
                rc = launch_op_dense(s, d, i, op, data, &folded);
                if (folded) i++;   // the phase op after it ran inside the sweep
            } else if (op.kind == QS_OP_DIAG) {
                rc = qs_launch_diag(s, (const int *)data, op.k, data + 64);
            } else {
                rc = qs_launch_phase(s, data, d.n_act[i]);
            }
            if (rc) return rc;
        }
        return QS_OK;
    });
}

extern "C" int qs_run_circuit_timed(qs_state *s, const qs_schedule *sc, float *op_ms)
{
    return qs_guard([&]() -> int {
        int rc = check_state(s, "qs_run_circuit_timed");
        if (rc) return rc;
        if (!sc || sc->n != s->n || !op_ms)
            return qs_fail(QS_EINVAL, "qs_run_circuit_timed: bad schedule or output");
        if ((rc = ensure_dev_schedule(s, sc))) return rc;
        // the schedule's ops name index bits (any exchange sweep is not timed)
        if ((rc = qs_order_set(s, sc->remap.empty() ? nullptr : sc->remap.data()))) return rc;
        const qs_dev_sched &d = sc->dev[s->dtype];
        cudaStream_t st = (cudaStream_t)s->stream;
        size_t nops = sc->ops.size();
        std::vector<cudaEvent_t> ev(nops + 1);
        std::vector<char> skipped(nops, 0);
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) return qs_fail(QS_ECUDA, "event create");
        cudaEventRecord(ev[0], st);
        for (size_t i = 0; i < nops && !rc; i++) {
            const qs_op_host &op = sc->ops[i];
            const uint8_t *data = (const uint8_t *)d.pool + d.offset[i];
            bool folded = false;
            int skip = 0;
            if (op.kind == QS_OP_DENSE && try_pair(s, sc, d, i, &rc, &skip)) {
                // the second cluster (and a phase op folded into it) ran inside the sweep
            } else if (op.kind == QS_OP_DENSE) {
                rc = launch_op_dense(s, d, i, op, data, &folded);
                skip = folded ? 1 : 0;   // the phase op after it ran inside the sweep
            } else if (op.kind == QS_OP_DIAG) {
                rc = qs_launch_diag(s, (const int *)data, op.k, data + 64);
            } else {
                rc = qs_launch_phase(s, data, d.n_act[i]);
            }
            cudaEventRecord(ev[i + 1], st);
            for (int j = 0; j < skip; j++) {
                skipped[++i] = 1;
                cudaEventRecord(ev[i + 1], st);
            }
        }
        if (!rc) {
            cudaError_t e = cudaEventSynchronize(ev[nops]);
            if (e != cudaSuccess) rc = qs_fail(QS_ECUDA, "qs_run_circuit_timed: %s", cudaGetErrorString(e));
            for (size_t i = 0; i < nops && !rc; i++) {
                if (skipped[i]) op_ms[i] = -1.0f;
                else cudaEventElapsedTime(&op_ms[i], ev[i], ev[i + 1]);
            }
        }
        for (auto &e : ev) cudaEventDestroy(e);
        return rc;
    });
}

extern "C" int64_t qs_schedule_upload_bytes(const qs_schedule *sc, int dtype)
{
    int64_t bytes = 0;
    const int rc = qs_guard([&]() -> int {
        if (!sc || (dtype != QS_C64 && dtype != QS_C128)) return qs_fail(QS_EINVAL, "qs_schedule_upload_bytes");
        qs_dev_sched tmp;
        bytes = (int64_t)schedule_blob(sc, dtype, tmp).size();
        return QS_OK;
    });
    return rc == QS_OK ? bytes : rc;
}

extern "C" int qs_set_pair_sweeps(qs_state *s, int on)
{
    return qs_guard([&]() -> int {
        if (!s) return qs_fail(QS_EINVAL, "qs_set_pair_sweeps: null state");
        s->pair_sweeps = on != 0;
        return QS_OK;
    });
}

extern "C" int qs_schedule_remap(qs_schedule *sc, const int *loc)
{
    return qs_guard([&]() -> int {
        if (!sc || !loc) return qs_fail(QS_EINVAL, "qs_schedule_remap: null argument");
        if (!sc->remap.empty()) return qs_fail(QS_EINVAL, "qs_schedule_remap: schedule already remapped");
        const int n = sc->n;
        for (int q = 0; q < n; q++)
            if (loc[q] < 0 || loc[q] >= n || loc[loc[q]] != q)
                return qs_fail(QS_EINVAL, "qs_schedule_remap: loc is not a set of exchanges at qubit %d", q);
        for (qs_op_host &op : sc->ops) {
            if (op.kind == QS_OP_PHASE) {
                std::vector<int32_t> c(n);
                for (int q = 0; q < n; q++) c[loc[q]] = op.coeff[q];
                op.coeff = c;
                for (auto &e : op.edges) e = {loc[e.first], loc[e.second]};
                continue;
            }
            int lq[QS_MAX_DIAG_K], q[QS_MAX_DIAG_K];
            for (int j = 0; j < op.k; j++) lq[j] = loc[op.qubits[j]];
            std::vector<double> M;
            sort_targets(lq, op.k, op.matrix.data(), op.kind == QS_OP_DENSE, q, M);
            for (int j = 0; j < op.k; j++) op.qubits[j] = q[j];
            op.matrix = M;
        }
        for (auto &d : sc->dev) {   // device images describe the old ops
            if (d.pool) cudaFree(d.pool);
            d = qs_dev_sched();
        }
        sc->remap.assign(loc, loc + n);
        return QS_OK;
    });
}

extern "C" int qs_schedule_get_remap(const qs_schedule *sc, int *loc)
{
    return qs_guard([&]() -> int {
        if (!sc || !loc) return qs_fail(QS_EINVAL, "qs_schedule_get_remap: null argument");
        for (int q = 0; q < sc->n; q++) loc[q] = sc->remap.empty() ? q : sc->remap[q];
        return QS_OK;
    });
}

extern "C" int qs_schedule_choose_remap(const qs_schedule *sc, int dtype, int *loc)
{
    return qs_guard([&]() -> int {
        if (!sc || !loc || (dtype != QS_C64 && dtype != QS_C128))
            return qs_fail(QS_EINVAL, "qs_schedule_choose_remap: bad arguments");
        const int n = sc->n;
        for (int q = 0; q < n; q++) loc[q] = q;
        // the index bits whose sweeps cost more (measured): 0-1 for complex128,
        // 0-4 for complex64
        const int nlow = std::min(n, dtype == QS_C128 ? 2 : 5);
        if (n < 5 + nlow) return QS_OK;
        // weight of each qubit: the dense sweeps it is a target of, each
        // counted by the share of the state it covers from |0...0> (the support
        // grows by every dense cluster's qubits)
        std::vector<double> w(n, 0.0);
        uint64_t sup = 0;
        for (const qs_op_host &op : sc->ops) {
            if (op.kind != QS_OP_DENSE) continue;
            for (int j = 0; j < op.k; j++) sup |= 1ULL << op.qubits[j];
            const double share = std::ldexp(1.0, __builtin_popcountll(sup) - n);
            for (int j = 0; j < op.k; j++) w[op.qubits[j]] += share;
        }
        // the nlow lightest qubits go to the low bits (ties: a qubit already
        // there, then the lower qubit)
        std::vector<int> order(n);
        for (int q = 0; q < n; q++) order[q] = q;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            if (w[a] != w[b]) return w[a] < w[b];
            return (a < nlow) > (b < nlow);
        });
        std::vector<char> chosen(n, 0);
        for (int i = 0; i < nlow; i++) chosen[order[i]] = 1;
        std::vector<int> in, out;              // chosen qubits above, low bits to free
        for (int q = nlow; q < n; q++)
            if (chosen[q]) in.push_back(q);
        for (int b = 0; b < nlow; b++)
            if (!chosen[b]) out.push_back(b);
        for (size_t i = 0; i < in.size() && i < out.size(); i++) {
            loc[in[i]] = out[i];
            loc[out[i]] = in[i];
        }
        return QS_OK;
    });
}

extern "C" int qs_schedule_upload(const qs_schedule *sc, int dtype)
{
    return qs_guard([&]() -> int {
        if (!sc || (dtype != QS_C64 && dtype != QS_C128)) return qs_fail(QS_EINVAL, "qs_schedule_upload");
        qs_state probe;
        probe.n = sc->n;
        probe.dtype = dtype;
        return ensure_dev_schedule(&probe, sc);
    });
}

extern "C" int qs_set_device(int device)
{
    return qs_guard([&]() -> int {
        cudaError_t e = cudaSetDevice(device);
        return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "qs_set_device(%d): %s", device, cudaGetErrorString(e));
    });
}

extern "C" void qs_schedule_free(qs_schedule *sc)
{
    if (!sc) return;
    for (auto &d : sc->dev)
        if (d.pool) cudaFree(d.pool);
    delete sc;
}

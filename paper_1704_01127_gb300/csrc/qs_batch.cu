// Batched simulation of many small circuits in one persistent launch.
//
// Every circuit keeps its own state (2^n amplitudes) in one device buffer.  A
// thread-block cluster of C CTAs owns one circuit at a time (static
// round-robin over circuits sorted by descending cost) and applies all of its
// ops in order; the CTAs of a cluster split each sweep and meet at a hardware
// cluster barrier between ops, so a circuit's ops stay ordered and no CTA ever
// waits on another cluster.  The per-group arithmetic is the single-state
// kernels' (qs_device.cuh), so a batch reproduces single-state CUDA-core runs
// bit for bit.  The launch configuration (C, threads per CTA) and the cluster
// bound k_max of the scheduler are chosen by a timing autotuner; a launch can
// be captured once in a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "qs_device.cuh"
#include "qs_internal.h"

namespace {

using qsd::cplx;
using qsd::Targets;

struct BatchOp {
    int32_t kind;      // QS_OP_DENSE or QS_OP_PHASE
    int32_t k;
    int32_t n_act;
    int32_t q[5];
    uint64_t data;     // byte offset into the pool
};

struct BatchCirc {
    int32_t n;
    int32_t n_ops;
    int64_t op_first;
    int64_t amp_off;   // in amplitudes
};

constexpr int kBatchLowBits = 12;

__device__ __forceinline__ void cluster_sync_all(int C)
{
    if (C == 1) {
        __syncthreads();
        return;
    }
    __threadfence();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <typename R, int K>
__device__ __forceinline__ void dense_sweep(typename cplx<R>::t *psi, uint64_t N, const Targets &t,
                                            const typename cplx<R>::t *Us, uint64_t g0, uint64_t gstride)
{
    const uint64_t G = N >> K;
    for (uint64_t g = g0; g < G; g += gstride) qsd::dense_group<R, K, true>(psi + qsd::group_base<K>(g, t), t, Us);
}

template <typename R>
__global__ void __launch_bounds__(512)
k_batch(const BatchCirc *__restrict__ circ, const int *__restrict__ order, int n_circ, const BatchOp *__restrict__ ops,
        const uint8_t *__restrict__ pool, typename cplx<R>::t *__restrict__ amp, int C)
{
    using C2 = typename cplx<R>::t;
    __shared__ __align__(16) C2 Us[32 * 32];
    __shared__ uint8_t tab[1 << kBatchLowBits];
    __shared__ uint64_t part[64];
    __shared__ int act[64];
    __shared__ uint64_t cm[3];
    const int rank = blockIdx.x % C, cid = blockIdx.x / C, ncl = gridDim.x / C;
    const uint64_t gi0 = (uint64_t)rank * blockDim.x + threadIdx.x, gstride = (uint64_t)C * blockDim.x;
    for (int w = cid; w < n_circ; w += ncl) {
        const BatchCirc cc = circ[order[w]];
        C2 *psi = amp + cc.amp_off;
        const uint64_t N = 1ULL << cc.n;
        for (uint64_t i = gi0; i < N; i += gstride) {
            C2 z;
            z.x = i == 0 ? (R)1 : (R)0;
            z.y = 0;
            psi[i] = z;
        }
        cluster_sync_all(C);
        for (int o = 0; o < cc.n_ops; o++) {
            const BatchOp op = ops[cc.op_first + o];
            if (op.kind == QS_OP_DENSE) {
                const int D = 1 << op.k;
                const C2 *U = reinterpret_cast<const C2 *>(pool + op.data);
                for (int i = threadIdx.x; i < D * D; i += blockDim.x) Us[i] = U[i];
                __syncthreads();
                Targets t;
#pragma unroll
                for (int j = 0; j < 5; j++) t.q[j] = op.q[j];
                switch (op.k) {
                case 1: dense_sweep<R, 1>(psi, N, t, Us, gi0, gstride); break;
                case 2: dense_sweep<R, 2>(psi, N, t, Us, gi0, gstride); break;
                case 3: dense_sweep<R, 3>(psi, N, t, Us, gi0, gstride); break;
                case 4: dense_sweep<R, 4>(psi, N, t, Us, gi0, gstride); break;
                default: dense_sweep<R, 5>(psi, N, t, Us, gi0, gstride); break;
                }
            } else {
                const qs_phase_dev *ph = reinterpret_cast<const qs_phase_dev *>(pool + op.data);
                const qs_phase_term *terms = reinterpret_cast<const qs_phase_term *>(ph + 1);
                if (threadIdx.x < 3) cm[threadIdx.x] = ph->cmask[threadIdx.x];
                for (int i = threadIdx.x; i < op.n_act; i += blockDim.x) {
                    part[i] = terms[i].partners;
                    act[i] = terms[i].a;
                }
                __syncthreads();
                const int L = cc.n < kBatchLowBits ? cc.n : kBatchLowBits;
                for (int l = threadIdx.x; l < (1 << L); l += blockDim.x)
                    tab[l] = qsd::phase_low((uint64_t)l, cm, act, part, op.n_act, L);
                __syncthreads();
                const uint64_t n_chunks = N >> L;
                for (uint64_t ch = rank; ch < n_chunks; ch += C) {
                    const uint64_t h = ch << L;
                    uint64_t Mh;
                    const int mh = qsd::phase_high(h, cm, act, part, op.n_act, L, Mh);
                    C2 *base = psi + h;
                    for (int l = threadIdx.x; l < (1 << L); l += blockDim.x) {
                        const int m = (tab[l] + mh + 4 * __popcll((uint64_t)l & Mh)) & 7;
                        if (m) base[l] = qsd::rotate8<C2, R>(qsd::ld<true>(base + l), m);
                    }
                }
            }
            cluster_sync_all(C);
        }
    }
}

// Per-circuit FP64 statistics: one CTA per circuit.
template <typename R>
__global__ void __launch_bounds__(256)
k_batch_stats(const BatchCirc *__restrict__ circ, const typename cplx<R>::t *__restrict__ amp, double *__restrict__ out)
{
    __shared__ qsd::LogTable lt;
    __shared__ double red[4][8];
    static_assert(sizeof(qsd::LogTable) + sizeof(red) < 48 * 1024, "static shared memory");
    qsd::log_table_init(lt);
    __syncthreads();
    const BatchCirc cc = circ[blockIdx.x];
    const uint64_t N = 1ULL << cc.n;
    const double Nd = (double)N;
    double a[4] = {0, 0, 0, 0};
    for (uint64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double p = qsd::prob(amp[cc.amp_off + i]);
        a[0] += p;
        if (p >= 2.2250738585072014e-308) a[1] -= p * qsd::log_tab(lt, p);
        a[3] = fma(p, p, a[3]);
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        double v = a[j];
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        // sum p, entropy, mean of N p (= sum p), mean of (N p)^2 (= N sum p^2)
        const int src = threadIdx.x == 2 ? 0 : threadIdx.x;
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[src][w];
        out[4 * blockIdx.x + threadIdx.x] = threadIdx.x == 3 ? v * Nd : v;
    }
}

uint64_t splitmix64(uint64_t seed, uint64_t j)
{
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

}  // namespace

struct qs_batch {
    int dtype = QS_C64;
    int n_circ = 0;
    void *stream = nullptr;
    void *amp = nullptr;
    void *ops = nullptr, *circ = nullptr, *order = nullptr, *pool = nullptr, *stats = nullptr;
    std::vector<int> nq;
    std::vector<uint64_t> amp_off;
    int cluster = 1, block = 256;
    cudaGraphExec_t exec = nullptr;
    int exec_cluster = 0, exec_block = 0;
};

namespace {

template <typename T>
int upload(void **dst, const std::vector<T> &v)
{
    size_t bytes = std::max<size_t>(v.size() * sizeof(T), 16);
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) {
        *dst = nullptr;
        return qs_fail(QS_ENOMEM, "batch upload: %s", cudaGetErrorString(e));
    }
    if (!v.empty() && (e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess)
        return qs_fail(QS_ECUDA, "batch upload: %s", cudaGetErrorString(e));
    return QS_OK;
}

int launch_batch(qs_batch *b, int C, int block)
{
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = b->dtype == QS_C128
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<double>, block, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<float>, block, 0);
    if (e != cudaSuccess || occ < 1) occ = 1;
    int clusters = std::max(1, std::min(b->n_circ, sms * occ / C));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * C);
    cfg.blockDim = dim3(block);
    cfg.stream = (cudaStream_t)b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const BatchCirc *circ = (const BatchCirc *)b->circ;
    const int *order = (const int *)b->order;
    const BatchOp *ops = (const BatchOp *)b->ops;
    const uint8_t *pool = (const uint8_t *)b->pool;
    if (b->dtype == QS_C128)
        e = cudaLaunchKernelEx(&cfg, k_batch<double>, circ, order, b->n_circ, ops, pool, (double2 *)b->amp, C);
    else
        e = cudaLaunchKernelEx(&cfg, k_batch<float>, circ, order, b->n_circ, ops, pool, (float2 *)b->amp, C);
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "batch launch: %s", cudaGetErrorString(e));
}

bool valid_config(int C, int block)
{
    return (C == 1 || C == 2 || C == 4 || C == 8) && (block == 128 || block == 256 || block == 512);
}

}  // namespace

extern "C" int qs_batch_circuit_params(uint64_t seed, int *rows, int *cols, int *cz_cycles)
{
    return qs_guard([&]() -> int {
        if (!rows || !cols || !cz_cycles) return qs_fail(QS_EINVAL, "qs_batch_circuit_params: null output");
        static const int grids[3][2] = {{4, 4}, {4, 5}, {3, 7}};
        const uint64_t r = splitmix64(seed ^ 0x6A09E667F3BCC909ULL, 0);
        const int g = (int)(r % 3);
        *rows = grids[g][0];
        *cols = grids[g][1];
        *cz_cycles = 8 + (int)((r >> 32) % 33);
        return QS_OK;
    });
}

extern "C" int qs_batch_create(int n_circ, const qs_schedule *const *scheds, int dtype, void *stream, qs_batch **out)
{
    return qs_guard([&]() -> int {
        if (!out || n_circ < 1 || !scheds || (dtype != QS_C64 && dtype != QS_C128))
            return qs_fail(QS_EINVAL, "qs_batch_create: bad arguments");
        const size_t rsz = dtype == QS_C128 ? 8 : 4;
        std::vector<BatchCirc> circ(n_circ);
        std::vector<BatchOp> ops;
        std::vector<uint8_t> pool;
        std::vector<double> cost(n_circ, 0.0);
        qs_batch *b = new (std::nothrow) qs_batch();
        if (!b) return qs_fail(QS_ENOMEM, "qs_batch_create: out of host memory");
        b->dtype = dtype;
        b->n_circ = n_circ;
        b->stream = stream;
        uint64_t amp_total = 0;
        for (int c = 0; c < n_circ; c++) {
            const qs_schedule *sc = scheds[c];
            if (!sc || sc->n < 1 || sc->n > 26) {
                delete b;
                return qs_fail(QS_EINVAL, "qs_batch_create: circuit %d must have 1..26 qubits", c);
            }
            if (!sc->remap.empty()) {
                delete b;
                return qs_fail(QS_EINVAL, "qs_batch_create: circuit %d has a remapped schedule", c);
            }
            circ[c].n = sc->n;
            circ[c].n_ops = (int32_t)sc->ops.size();
            circ[c].op_first = (int64_t)ops.size();
            circ[c].amp_off = (int64_t)amp_total;
            b->nq.push_back(sc->n);
            b->amp_off.push_back(amp_total);
            amp_total += ((1ULL << sc->n) + 31) & ~31ULL;   // 256-byte aligned states
            for (const qs_op_host &op : sc->ops) {
                BatchOp bo;
                std::memset(&bo, 0, sizeof(bo));
                bo.kind = op.kind;
                bo.k = op.k;
                size_t at = (pool.size() + 255) & ~(size_t)255;
                if (op.kind == QS_OP_DENSE) {
                    for (int j = 0; j < op.k; j++) bo.q[j] = op.qubits[j];
                    pool.resize(at + op.matrix.size() * rsz);
                    for (size_t i = 0; i < op.matrix.size(); i++) {
                        if (dtype == QS_C128) std::memcpy(pool.data() + at + 8 * i, &op.matrix[i], 8);
                        else {
                            float f = (float)op.matrix[i];
                            std::memcpy(pool.data() + at + 4 * i, &f, 4);
                        }
                    }
                    cost[c] += (double)(1ULL << sc->n) * (1 + (1 << op.k) / 8.0);
                } else if (op.kind == QS_OP_PHASE) {
                    int n_act = 0;
                    std::vector<uint8_t> ph = qs_pack_phase(sc->n, op.coeff, op.edges, &n_act);
                    bo.n_act = n_act;
                    pool.resize(at + ph.size());
                    std::memcpy(pool.data() + at, ph.data(), ph.size());
                    cost[c] += (double)(1ULL << sc->n);
                } else {
                    delete b;
                    return qs_fail(QS_EUNSUPPORTED, "qs_batch_create: table diagonals are not batched");
                }
                bo.data = at;
                ops.push_back(bo);
            }
        }
        std::vector<int> order(n_circ);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cost[a] > cost[c]; });
        int rc = QS_OK;
        cudaError_t e = cudaMalloc(&b->amp, amp_total * 2 * rsz);
        if (e != cudaSuccess) rc = qs_fail(QS_ENOMEM, "qs_batch_create: states: %s", cudaGetErrorString(e));
        if (!rc) rc = upload(&b->ops, ops);
        if (!rc) rc = upload(&b->circ, circ);
        if (!rc) rc = upload(&b->order, order);
        if (!rc) rc = upload(&b->pool, pool);
        if (!rc && (e = cudaMalloc(&b->stats, sizeof(double) * 4 * n_circ)) != cudaSuccess)
            rc = qs_fail(QS_ENOMEM, "qs_batch_create: stats: %s", cudaGetErrorString(e));
        if (rc) {
            qs_batch_free(b);
            return rc;
        }
        *out = b;
        return QS_OK;
    });
}

extern "C" void qs_batch_free(qs_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize((cudaStream_t)b->stream);
    else cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (void *p : {b->amp, b->ops, b->circ, b->order, b->pool, b->stats})
        if (p) cudaFree(p);
    delete b;
}

extern "C" int qs_batch_set_config(qs_batch *b, int cluster_ctas, int threads)
{
    return qs_guard([&]() -> int {
        if (!b || !valid_config(cluster_ctas, threads)) return qs_fail(QS_EINVAL, "qs_batch_set_config");
        b->cluster = cluster_ctas;
        b->block = threads;
        return QS_OK;
    });
}

extern "C" int qs_batch_get_config(const qs_batch *b, int *cluster_ctas, int *threads)
{
    return qs_guard([&]() -> int {
        if (!b || !cluster_ctas || !threads) return qs_fail(QS_EINVAL, "qs_batch_get_config");
        *cluster_ctas = b->cluster;
        *threads = b->block;
        return QS_OK;
    });
}

extern "C" int qs_batch_run(qs_batch *b)
{
    return qs_guard([&]() -> int {
        if (!b) return qs_fail(QS_EINVAL, "qs_batch_run: null batch");
        return launch_batch(b, b->cluster, b->block);
    });
}

extern "C" int qs_batch_run_graph(qs_batch *b)
{
    return qs_guard([&]() -> int {
        if (!b) return qs_fail(QS_EINVAL, "qs_batch_run_graph: null batch");
        cudaStream_t st = (cudaStream_t)b->stream;
        if (!st) return qs_fail(QS_EINVAL, "qs_batch_run_graph: needs a non-default stream");
        if (!b->exec || b->exec_cluster != b->cluster || b->exec_block != b->block) {
            if (b->exec) {
                cudaGraphExecDestroy(b->exec);
                b->exec = nullptr;
            }
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return qs_fail(QS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
            int rc = launch_batch(b, b->cluster, b->block);
            e = cudaStreamEndCapture(st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return qs_fail(QS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&b->exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->exec = nullptr;
                return qs_fail(QS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
            }
            b->exec_cluster = b->cluster;
            b->exec_block = b->block;
        }
        cudaError_t e = cudaGraphLaunch(b->exec, st);
        return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "graph launch: %s", cudaGetErrorString(e));
    });
}

extern "C" int qs_batch_stats(qs_batch *b, double *out)
{
    return qs_guard([&]() -> int {
        if (!b || !out) return qs_fail(QS_EINVAL, "qs_batch_stats: bad arguments");
        cudaStream_t st = (cudaStream_t)b->stream;
        if (b->dtype == QS_C128)
            k_batch_stats<double><<<b->n_circ, 256, 0, st>>>((const BatchCirc *)b->circ, (const double2 *)b->amp,
                                                             (double *)b->stats);
        else
            k_batch_stats<float><<<b->n_circ, 256, 0, st>>>((const BatchCirc *)b->circ, (const float2 *)b->amp,
                                                            (double *)b->stats);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, b->stats, sizeof(double) * 4 * b->n_circ, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "qs_batch_stats: %s", cudaGetErrorString(e));
    });
}

extern "C" int qs_batch_get_amplitudes(qs_batch *b, int i, double *host)
{
    return qs_guard([&]() -> int {
        if (!b || !host || i < 0 || i >= b->n_circ) return qs_fail(QS_EINVAL, "qs_batch_get_amplitudes: bad arguments");
        const uint64_t N = 1ULL << b->nq[i];
        cudaStream_t st = (cudaStream_t)b->stream;
        cudaError_t e;
        if (b->dtype == QS_C128) {
            e = cudaMemcpyAsync(host, (double2 *)b->amp + b->amp_off[i], 16 * N, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        } else {
            std::vector<float> f(2 * N);
            e = cudaMemcpyAsync(f.data(), (float2 *)b->amp + b->amp_off[i], 8 * N, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            for (uint64_t j = 0; j < 2 * N; j++) host[j] = f[j];
        }
        return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "qs_batch_get_amplitudes: %s", cudaGetErrorString(e));
    });
}

// Time every launch configuration (cluster of 1, 2, 4, 8 CTAs x 128, 256, 512
// threads), keep the fastest in the batch and report it.
extern "C" int qs_batch_tune(qs_batch *b, int *cluster_ctas, int *threads, float *ms)
{
    return qs_guard([&]() -> int {
        if (!b) return qs_fail(QS_EINVAL, "qs_batch_tune: null batch");
        cudaStream_t st = (cudaStream_t)b->stream;
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
            return qs_fail(QS_ECUDA, "qs_batch_tune: events");
        float best = 1e30f;
        int bc = 1, bt = 256, rc = QS_OK;
        for (int C : {1, 2, 4, 8})
            for (int T : {128, 256, 512}) {
                if ((rc = launch_batch(b, C, T))) break;   // warm-up
                cudaEventRecord(e0, st);
                for (int r = 0; r < 2 && !rc; r++) rc = launch_batch(b, C, T);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = qs_fail(QS_ECUDA, "qs_batch_tune: sync");
                    break;
                }
                float t = 0;
                cudaEventElapsedTime(&t, e0, e1);
                t /= 2;
                if (t < best) {
                    best = t;
                    bc = C;
                    bt = T;
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        b->cluster = bc;
        b->block = bt;
        if (cluster_ctas) *cluster_ctas = bc;
        if (threads) *threads = bt;
        if (ms) *ms = best;
        return QS_OK;
    });
}

// Autotune the whole batched path: schedules with k_max in {3, 4, 5}, each
// batch tuned over its launch configurations; the fastest triple is returned.
extern "C" int qs_batch_autotune(int n_circ, const int *n_qubits, const qs_gate *const *gates, const int *n_gates,
                                 int dtype, void *stream, int *k_max, int *cluster_ctas, int *threads, float *ms)
{
    return qs_guard([&]() -> int {
        if (n_circ < 1 || !n_qubits || !gates || !n_gates || !k_max || !cluster_ctas || !threads)
            return qs_fail(QS_EINVAL, "qs_batch_autotune: bad arguments");
        float best = 1e30f;
        int rc = QS_OK;
        for (int km : {3, 4, 5}) {
            std::vector<qs_schedule *> sc(n_circ, nullptr);
            qs_sched_opts o = {km, 1, 1, 0, 1, 1, 1, 1, 0};
            for (int c = 0; c < n_circ && !rc; c++) rc = qs_schedule_build(n_qubits[c], gates[c], n_gates[c], &o, &sc[c]);
            qs_batch *b = nullptr;
            if (!rc) rc = qs_batch_create(n_circ, sc.data(), dtype, stream, &b);
            int C = 1, T = 256;
            float t = 0;
            if (!rc) rc = qs_batch_tune(b, &C, &T, &t);
            if (!rc && t < best) {
                best = t;
                *k_max = km;
                *cluster_ctas = C;
                *threads = T;
            }
            qs_batch_free(b);
            for (qs_schedule *s : sc) qs_schedule_free(s);
            if (rc) return rc;
        }
        if (ms) *ms = best;
        return QS_OK;
    });
}

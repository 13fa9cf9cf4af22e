// Cost models for the scheduler (Sec. 3.3: which k to use depends on the
// machine; Sec. 3.6: the scheduler trades clusters against their cost):
//  * op features (cluster size, target bit positions, dtype, diagonal flag,
//    kernel path, state size);
//  * an analytic model, max(bytes / HBM bandwidth, flops / arithmetic peak);
//  * a timing harness that runs random clusters on the device;
//  * a 2 x 64 tanh MLP on log-time, trained on the GPU in FP64 by this file's
//    forward, backward and Adam kernels;
//  * the planner: per circuit, the cluster bound k_max and each dense op's
//    kernel path that minimise the predicted time.  The MLP is used only when
//    it beats the analytic model on held-out timings and the op's features lie
//    inside the training range; otherwise the analytic model decides.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "qs_internal.h"

namespace {

constexpr int kF = QS_NFEAT;      // features per op
constexpr int kH = 64;            // hidden width

uint64_t splitmix64(uint64_t seed, uint64_t j)
{
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

struct Rng {
    uint64_t seed, j = 0;
    explicit Rng(uint64_t s) : seed(s) {}
    uint64_t next() { return splitmix64(seed, j++); }
    double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }
    int below(int m) { return (int)(next() % (uint64_t)m); }
};

// ------------------------------------------------------------------ features

void op_features(int n, int dtype, int kind, int k, const int *q, int path, int n_act, int odd, double *f)
{
    std::memset(f, 0, sizeof(double) * kF);
    f[0] = n / 32.0;
    f[1] = dtype == QS_C128 ? 1.0 : 0.0;
    f[2] = kind == QS_OP_PHASE ? 1.0 : 0.0;
    f[9] = (n + std::log2(dtype == QS_C128 ? 16.0 : 8.0)) / 40.0;
    if (kind == QS_OP_PHASE) {
        f[10] = n_act / (double)n;
        f[11] = odd ? 1.0 : 0.0;
        return;
    }
    f[3] = k / 5.0;
    f[4] = path == QS_PATH_TENSOR ? 1.0 : 0.0;
    int lo = q[0], hi = q[0], b5 = 0, b3 = 0;
    for (int j = 0; j < k; j++) {
        lo = std::min(lo, q[j]);
        hi = std::max(hi, q[j]);
        b5 += q[j] < 5;
        b3 += q[j] < 3;
    }
    f[5] = lo / (double)n;
    f[6] = hi / (double)n;
    f[7] = b5 / 5.0;
    f[8] = b3 / 3.0;
}

// max(2 bytes(state) / HBM bandwidth, flops / peak) + launch overhead, in ms.
// Peaks: FP32 70 TFLOP/s and FP64 1.2 TFLOP/s (the CUDA-core sweeps); the
// tensor-core sweeps are taken as HBM-bound.
double analytic_ms(const double *f, double hbm_gbs)
{
    const int n = (int)std::lround(f[0] * 32), k = (int)std::lround(f[3] * 5);
    const bool c128 = f[1] > 0.5, phase = f[2] > 0.5, tc = f[4] > 0.5;
    const double amps = std::ldexp(1.0, n);
    const double t_mem = 2.0 * amps * (c128 ? 16 : 8) / (hbm_gbs * 1e9) * 1e3;
    double flops = 0, peak = c128 ? 1.2e12 : 70e12;
    if (!phase && !tc) flops = amps * (8.0 * (1 << k) - 2);
    if (phase && c128 && f[11] > 0.5) flops = amps * 2.0;
    const double t_flop = flops / peak * 1e3;
    return std::max(t_mem, t_flop) + 0.005;
}

// -------------------------------------------------------------- MLP kernels
// Parameters, one FP64 array: W1[F][H], b1[H], W2[H][H], b2[H], w3[H], b3.
constexpr int kP = kF * kH + kH + kH * kH + kH + kH + 1;
constexpr int oW1 = 0, ob1 = kF * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, ow3 = ob2 + kH, ob3 = ow3 + kH;

__global__ void k_mlp_fwd(const double *__restrict__ X, int B, const double *__restrict__ W, double *__restrict__ A1,
                          double *__restrict__ A2, double *__restrict__ out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double a1[kH];
#pragma unroll 4
    for (int j = 0; j < kH; j++) {
        double z = W[ob1 + j];
        for (int f = 0; f < kF; f++) z = fma(X[(size_t)b * kF + f], W[oW1 + f * kH + j], z);
        a1[j] = tanh(z);
        A1[(size_t)b * kH + j] = a1[j];
    }
    double y = W[ob3];
    for (int j = 0; j < kH; j++) {
        double z = W[ob2 + j];
        for (int i = 0; i < kH; i++) z = fma(a1[i], W[oW2 + i * kH + j], z);
        const double a2 = tanh(z);
        A2[(size_t)b * kH + j] = a2;
        y = fma(a2, W[ow3 + j], y);
    }
    out[b] = y;
}

// loss = mean over the batch of (out - y)^2: per-sample deltas
__global__ void k_mlp_delta(const double *__restrict__ A1, const double *__restrict__ A2, const double *__restrict__ out,
                            const double *__restrict__ Y, int B, const double *__restrict__ W, double *__restrict__ D1,
                            double *__restrict__ D2, double *__restrict__ dy)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double g = 2.0 * (out[b] - Y[b]) / B;
    dy[b] = g;
    double d2[kH];
    for (int j = 0; j < kH; j++) {
        const double a2 = A2[(size_t)b * kH + j];
        d2[j] = g * W[ow3 + j] * (1.0 - a2 * a2);
        D2[(size_t)b * kH + j] = d2[j];
    }
    for (int i = 0; i < kH; i++) {
        double s = 0;
        for (int j = 0; j < kH; j++) s = fma(d2[j], W[oW2 + i * kH + j], s);
        const double a1 = A1[(size_t)b * kH + i];
        D1[(size_t)b * kH + i] = s * (1.0 - a1 * a1);
    }
}

// one thread per parameter, samples summed in index order (deterministic)
__global__ void k_mlp_grad(const double *__restrict__ X, const double *__restrict__ A1, const double *__restrict__ A2,
                           const double *__restrict__ D1, const double *__restrict__ D2, const double *__restrict__ dy,
                           int B, double *__restrict__ G)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kP) return;
    double s = 0;
    if (p < ob1) {
        const int f = p / kH, j = p % kH;
        for (int b = 0; b < B; b++) s = fma(X[(size_t)b * kF + f], D1[(size_t)b * kH + j], s);
    } else if (p < oW2) {
        const int j = p - ob1;
        for (int b = 0; b < B; b++) s += D1[(size_t)b * kH + j];
    } else if (p < ob2) {
        const int i = (p - oW2) / kH, j = (p - oW2) % kH;
        for (int b = 0; b < B; b++) s = fma(A1[(size_t)b * kH + i], D2[(size_t)b * kH + j], s);
    } else if (p < ow3) {
        const int j = p - ob2;
        for (int b = 0; b < B; b++) s += D2[(size_t)b * kH + j];
    } else if (p < ob3) {
        const int j = p - ow3;
        for (int b = 0; b < B; b++) s = fma(A2[(size_t)b * kH + j], dy[b], s);
    } else {
        for (int b = 0; b < B; b++) s += dy[b];
    }
    G[p] = s;
}

// Adam (Kingma & Ba 2015), bias-corrected step size lr_t
__global__ void k_adam(double *__restrict__ W, const double *__restrict__ G, double *__restrict__ m,
                       double *__restrict__ v, double lr_t, double beta1, double beta2, double eps)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= kP) return;
    m[p] = beta1 * m[p] + (1 - beta1) * G[p];
    v[p] = beta2 * v[p] + (1 - beta2) * G[p] * G[p];
    W[p] -= lr_t * m[p] / (sqrt(v[p]) + eps);
}

}  // namespace

// ----------------------------------------------------------------- the MLP

struct qs_mlp {
    double *W = nullptr, *G = nullptr, *m = nullptr, *v = nullptr;
    // batch buffers, grown on demand
    double *X = nullptr, *Y = nullptr, *A1 = nullptr, *A2 = nullptr, *D1 = nullptr, *D2 = nullptr, *out = nullptr,
           *dy = nullptr;
    int cap = 0;
};

namespace {

int mlp_reserve(qs_mlp *M, int B)
{
    if (B <= M->cap) return QS_OK;
    for (double *p : {M->X, M->Y, M->A1, M->A2, M->D1, M->D2, M->out, M->dy})
        if (p) cudaFree(p);
    cudaError_t e = cudaSuccess;
    auto al = [&](double **p, size_t n) {
        if (e == cudaSuccess) e = cudaMalloc(p, sizeof(double) * n);
    };
    al(&M->X, (size_t)B * kF);
    al(&M->Y, B);
    al(&M->A1, (size_t)B * kH);
    al(&M->A2, (size_t)B * kH);
    al(&M->D1, (size_t)B * kH);
    al(&M->D2, (size_t)B * kH);
    al(&M->out, B);
    al(&M->dy, B);
    if (e != cudaSuccess) {
        M->cap = 0;
        return qs_fail(QS_ENOMEM, "mlp buffers: %s", cudaGetErrorString(e));
    }
    M->cap = B;
    return QS_OK;
}

int mlp_upload(qs_mlp *M, const double *X, const double *Y, int B)
{
    int rc = mlp_reserve(M, B);
    if (rc) return rc;
    cudaError_t e = cudaMemcpy(M->X, X, sizeof(double) * B * kF, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && Y) e = cudaMemcpy(M->Y, Y, sizeof(double) * B, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "mlp upload: %s", cudaGetErrorString(e));
}

void mlp_fwd(qs_mlp *M, int B) { k_mlp_fwd<<<(B + 127) / 128, 128>>>(M->X, B, M->W, M->A1, M->A2, M->out); }

void mlp_grad(qs_mlp *M, int B)
{
    mlp_fwd(M, B);
    k_mlp_delta<<<(B + 127) / 128, 128>>>(M->A1, M->A2, M->out, M->Y, B, M->W, M->D1, M->D2, M->dy);
    k_mlp_grad<<<(kP + 127) / 128, 128>>>(M->X, M->A1, M->A2, M->D1, M->D2, M->dy, B, M->G);
}

}  // namespace

extern "C" int qs_mlp_create(uint64_t seed, qs_mlp **out)
{
    return qs_guard([&]() -> int {
        if (!out) return qs_fail(QS_EINVAL, "qs_mlp_create: null output");
        qs_mlp *M = new (std::nothrow) qs_mlp();
        if (!M) return qs_fail(QS_ENOMEM, "qs_mlp_create");
        std::vector<double> w(kP, 0.0);
        Rng r(seed);
        // Glorot-uniform weights, zero biases
        auto fill = [&](int off, int fan_in, int fan_out, int count) {
            const double a = std::sqrt(6.0 / (fan_in + fan_out));
            for (int i = 0; i < count; i++) w[off + i] = (2 * r.uniform() - 1) * a;
        };
        fill(oW1, kF, kH, kF * kH);
        fill(oW2, kH, kH, kH * kH);
        fill(ow3, kH, 1, kH);
        cudaError_t e = cudaSuccess;
        for (double **p : {&M->W, &M->G, &M->m, &M->v})
            if (e == cudaSuccess) e = cudaMalloc(p, sizeof(double) * kP);
        if (e == cudaSuccess) e = cudaMemcpy(M->W, w.data(), sizeof(double) * kP, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(M->m, 0, sizeof(double) * kP);
        if (e == cudaSuccess) e = cudaMemset(M->v, 0, sizeof(double) * kP);
        if (e != cudaSuccess) {
            qs_mlp_free(M);
            return qs_fail(QS_ENOMEM, "qs_mlp_create: %s", cudaGetErrorString(e));
        }
        *out = M;
        return QS_OK;
    });
}

extern "C" void qs_mlp_free(qs_mlp *M)
{
    if (!M) return;
    for (double *p : {M->W, M->G, M->m, M->v, M->X, M->Y, M->A1, M->A2, M->D1, M->D2, M->out, M->dy})
        if (p) cudaFree(p);
    delete M;
}

extern "C" int qs_mlp_num_params(void) { return kP; }

extern "C" int qs_mlp_get_params(const qs_mlp *M, double *out)
{
    return qs_guard([&]() -> int {
        if (!M || !out) return qs_fail(QS_EINVAL, "qs_mlp_get_params");
        cudaError_t e = cudaMemcpy(out, M->W, sizeof(double) * kP, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "qs_mlp_get_params: %s", cudaGetErrorString(e));
    });
}

extern "C" int qs_mlp_set_params(qs_mlp *M, const double *in)
{
    return qs_guard([&]() -> int {
        if (!M || !in) return qs_fail(QS_EINVAL, "qs_mlp_set_params");
        cudaError_t e = cudaMemcpy(M->W, in, sizeof(double) * kP, cudaMemcpyHostToDevice);
        return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "qs_mlp_set_params: %s", cudaGetErrorString(e));
    });
}

extern "C" int qs_mlp_forward(qs_mlp *M, const double *X, int B, double *out)
{
    return qs_guard([&]() -> int {
        if (!M || !X || !out || B < 1) return qs_fail(QS_EINVAL, "qs_mlp_forward");
        int rc = mlp_upload(M, X, nullptr, B);
        if (rc) return rc;
        mlp_fwd(M, B);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(out, M->out, sizeof(double) * B, cudaMemcpyDeviceToHost);
        return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "qs_mlp_forward: %s", cudaGetErrorString(e));
    });
}

extern "C" int qs_mlp_gradient(qs_mlp *M, const double *X, const double *Y, int B, double *grad, double *loss)
{
    return qs_guard([&]() -> int {
        if (!M || !X || !Y || !grad || B < 1) return qs_fail(QS_EINVAL, "qs_mlp_gradient");
        int rc = mlp_upload(M, X, Y, B);
        if (rc) return rc;
        mlp_grad(M, B);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpy(grad, M->G, sizeof(double) * kP, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && loss) {
            std::vector<double> o(B);
            e = cudaMemcpy(o.data(), M->out, sizeof(double) * B, cudaMemcpyDeviceToHost);
            double s = 0;
            for (int b = 0; b < B; b++) s += (o[b] - Y[b]) * (o[b] - Y[b]);
            *loss = s / B;
        }
        return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "qs_mlp_gradient: %s", cudaGetErrorString(e));
    });
}

extern "C" int qs_mlp_train(qs_mlp *M, const double *X, const double *Y, int B, int epochs, double lr, double *loss)
{
    return qs_guard([&]() -> int {
        if (!M || !X || !Y || B < 1 || epochs < 0 || !(lr > 0)) return qs_fail(QS_EINVAL, "qs_mlp_train");
        int rc = mlp_upload(M, X, Y, B);
        if (rc) return rc;
        cudaMemset(M->m, 0, sizeof(double) * kP);
        cudaMemset(M->v, 0, sizeof(double) * kP);
        const double b1 = 0.9, b2 = 0.999;
        double p1 = 1, p2 = 1;
        for (int t = 1; t <= epochs; t++) {
            mlp_grad(M, B);
            p1 *= b1;
            p2 *= b2;
            const double lr_t = lr * std::sqrt(1 - p2) / (1 - p1);
            k_adam<<<(kP + 127) / 128, 128>>>(M->W, M->G, M->m, M->v, lr_t, b1, b2, 1e-8);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return qs_fail(QS_ECUDA, "qs_mlp_train: %s", cudaGetErrorString(e));
        if (loss) {
            mlp_fwd(M, B);
            std::vector<double> o(B);
            e = cudaMemcpy(o.data(), M->out, sizeof(double) * B, cudaMemcpyDeviceToHost);
            double s = 0;
            for (int b = 0; b < B; b++) s += (o[b] - Y[b]) * (o[b] - Y[b]);
            *loss = s / B;
        }
        return e == cudaSuccess ? QS_OK : qs_fail(QS_ECUDA, "qs_mlp_train: %s", cudaGetErrorString(e));
    });
}

// ----------------------------------------------------------- cost model

struct qs_cost_model {
    double hbm_gbs = 6696.8;
    qs_mlp *mlp = nullptr;
    bool use_mlp = false;
    double fmu[kF], fsd[kF], fmin[kF], fmax[kF];
    double ymu = 0, ysd = 1;
};

extern "C" int qs_cost_model_create(double hbm_gbs, qs_cost_model **out)
{
    return qs_guard([&]() -> int {
        if (!out || !(hbm_gbs > 0)) return qs_fail(QS_EINVAL, "qs_cost_model_create");
        qs_cost_model *c = new (std::nothrow) qs_cost_model();
        if (!c) return qs_fail(QS_ENOMEM, "qs_cost_model_create");
        c->hbm_gbs = hbm_gbs;
        for (int f = 0; f < kF; f++) {
            c->fmu[f] = 0;
            c->fsd[f] = 1;
            c->fmin[f] = c->fmax[f] = 0;
        }
        *out = c;
        return QS_OK;
    });
}

extern "C" void qs_cost_model_free(qs_cost_model *c)
{
    if (!c) return;
    qs_mlp_free(c->mlp);
    delete c;
}

namespace {

bool in_range(const qs_cost_model *c, const double *f)
{
    for (int j = 0; j < kF; j++)
        if (f[j] < c->fmin[j] - 1e-9 || f[j] > c->fmax[j] + 1e-9) return false;
    return true;
}

int mlp_predict_ms(const qs_cost_model *c, const double *feats, int count, double *ms)
{
    std::vector<double> z((size_t)count * kF);
    for (int i = 0; i < count; i++)
        for (int f = 0; f < kF; f++) z[(size_t)i * kF + f] = (feats[(size_t)i * kF + f] - c->fmu[f]) / c->fsd[f];
    std::vector<double> y(count);
    int rc = qs_mlp_forward(c->mlp, z.data(), count, y.data());
    if (rc) return rc;
    for (int i = 0; i < count; i++) ms[i] = std::exp(y[i] * c->ysd + c->ymu);
    return QS_OK;
}

double median_abs(std::vector<double> v)
{
    if (v.empty()) return 0;
    std::nth_element(v.begin(), v.begin() + v.size() / 2, v.end());
    return v[v.size() / 2];
}

}  // namespace

extern "C" int qs_cost_model_fit(qs_cost_model *c, const double *feats, const double *ms, int count, int epochs,
                                 uint64_t seed, double report[4])
{
    return qs_guard([&]() -> int {
        if (!c || !feats || !ms || count < 20 || epochs < 1) return qs_fail(QS_EINVAL, "qs_cost_model_fit");
        for (int i = 0; i < count; i++)
            if (!(ms[i] > 0)) return qs_fail(QS_EINVAL, "qs_cost_model_fit: timing %d not positive", i);
        // held-out split: every fifth sample (by a seeded hash) is kept for validation
        std::vector<int> tr, ho;
        for (int i = 0; i < count; i++) (splitmix64(seed, (uint64_t)i) % 5 == 0 ? ho : tr).push_back(i);
        if (tr.size() < 10 || ho.empty()) return qs_fail(QS_EINVAL, "qs_cost_model_fit: too few samples");
        for (int f = 0; f < kF; f++) {
            double s = 0, s2 = 0, lo = 1e300, hi = -1e300;
            for (int i : tr) {
                const double x = feats[(size_t)i * kF + f];
                s += x;
                s2 += x * x;
                lo = std::min(lo, x);
                hi = std::max(hi, x);
            }
            const double mu = s / tr.size(), var = s2 / tr.size() - mu * mu;
            c->fmu[f] = mu;
            c->fsd[f] = var > 1e-12 ? std::sqrt(var) : 1.0;
            c->fmin[f] = lo;
            c->fmax[f] = hi;
        }
        double s = 0, s2 = 0;
        for (int i : tr) {
            const double y = std::log(ms[i]);
            s += y;
            s2 += y * y;
        }
        c->ymu = s / tr.size();
        c->ysd = std::max(1e-6, std::sqrt(std::max(0.0, s2 / tr.size() - c->ymu * c->ymu)));
        std::vector<double> X(tr.size() * kF), Y(tr.size());
        for (size_t a = 0; a < tr.size(); a++) {
            for (int f = 0; f < kF; f++) X[a * kF + f] = (feats[(size_t)tr[a] * kF + f] - c->fmu[f]) / c->fsd[f];
            Y[a] = (std::log(ms[tr[a]]) - c->ymu) / c->ysd;
        }
        if (!c->mlp) {
            int rc = qs_mlp_create(seed, &c->mlp);
            if (rc) return rc;
        }
        double loss = 0;
        int rc = qs_mlp_train(c->mlp, X.data(), Y.data(), (int)tr.size(), epochs, 3e-3, &loss);
        if (rc) return rc;
        // held-out errors of both models on log-time
        std::vector<double> hf(ho.size() * kF), pm(ho.size());
        for (size_t a = 0; a < ho.size(); a++)
            for (int f = 0; f < kF; f++) hf[a * kF + f] = feats[(size_t)ho[a] * kF + f];
        if ((rc = mlp_predict_ms(c, hf.data(), (int)ho.size(), pm.data()))) return rc;
        std::vector<double> em, ea;
        for (size_t a = 0; a < ho.size(); a++) {
            const double t = ms[ho[a]];
            em.push_back(std::fabs(std::log(pm[a] / t)));
            ea.push_back(std::fabs(std::log(analytic_ms(&hf[a * kF], c->hbm_gbs) / t)));
        }
        const double mlp_err = median_abs(em), an_err = median_abs(ea);
        c->use_mlp = mlp_err < an_err;
        if (report) {
            report[0] = loss;
            report[1] = mlp_err;
            report[2] = an_err;
            report[3] = c->use_mlp ? 1.0 : 0.0;
        }
        return QS_OK;
    });
}

extern "C" int qs_cost_model_predict(const qs_cost_model *c, const double *feats, int count, int which, double *ms)
{
    return qs_guard([&]() -> int {
        if (!c || !feats || !ms || count < 0 || which < QS_COST_AUTO || which > QS_COST_MLP)
            return qs_fail(QS_EINVAL, "qs_cost_model_predict");
        if (count == 0) return QS_OK;
        if (which == QS_COST_MLP && !c->mlp) return qs_fail(QS_EINVAL, "qs_cost_model_predict: model not trained");
        std::vector<double> mlp(count, 0.0);
        const bool want_mlp = which == QS_COST_MLP || (which == QS_COST_AUTO && c->use_mlp && c->mlp);
        if (want_mlp) {
            int rc = mlp_predict_ms(c, feats, count, mlp.data());
            if (rc) return rc;
        }
        for (int i = 0; i < count; i++) {
            const double *f = feats + (size_t)i * kF;
            const bool use = which == QS_COST_MLP || (want_mlp && in_range(c, f));
            ms[i] = use ? mlp[i] : analytic_ms(f, c->hbm_gbs);
        }
        return QS_OK;
    });
}

// ----------------------------------------------------------- timing harness

namespace {

// a dense unitary for timing (values do not change the kernels' work): a
// product of random single-qubit rotations on each of the k qubits
std::vector<double> timing_unitary(int k, Rng &r)
{
    const int d = 1 << k;
    std::vector<double> U(2 * d * d, 0.0);
    for (int i = 0; i < d; i++) U[2 * (i * d + i)] = 1.0;
    for (int j = 0; j < k; j++) {
        const double a = 6.283185307179586 * r.uniform(), c = std::cos(a), s = std::sin(a);
        std::vector<double> V(U);
        for (int row = 0; row < d; row++) {
            if ((row >> j) & 1) continue;
            const int r1 = row | (1 << j);
            for (int col = 0; col < d; col++) {
                const double x0 = U[2 * (row * d + col)], y0 = U[2 * (row * d + col) + 1];
                const double x1 = U[2 * (r1 * d + col)], y1 = U[2 * (r1 * d + col) + 1];
                V[2 * (row * d + col)] = c * x0 - s * x1;
                V[2 * (row * d + col) + 1] = c * y0 - s * y1;
                V[2 * (r1 * d + col)] = s * x0 + c * x1;
                V[2 * (r1 * d + col) + 1] = s * y0 + c * y1;
            }
        }
        U.swap(V);
    }
    return U;
}

}  // namespace

extern "C" int qs_cost_sample(int n_min, int n_max, int dtype, int count, uint64_t seed, double max_ms,
                              double *feats, double *ms)
{
    return qs_guard([&]() -> int {
        if (n_min < 5 || n_max < n_min || n_max > 33 || (dtype != QS_C64 && dtype != QS_C128) || count < 1 || !feats ||
            !ms || !(max_ms > 0))
            return qs_fail(QS_EINVAL, "qs_cost_sample: bad arguments");
        qs_state *big = nullptr;
        int rc = qs_alloc(n_max, dtype, nullptr, &big);
        if (rc) return rc;
        rc = qs_init_uniform(big);
        Rng r(seed);
        std::vector<qs_state *> views(n_max + 1, nullptr);
        for (int n = n_min; n <= n_max && !rc; n++) rc = qs_wrap(big->amp, n, dtype, nullptr, &views[n]);
        long attempts = 0;
        for (int i = 0; i < count && !rc;) {
            if (++attempts > 100L * count + 1000) {
                rc = qs_fail(QS_EINVAL, "qs_cost_sample: max_ms %.3g rejects almost every op", max_ms);
                break;
            }
            const int n = n_min + r.below(n_max - n_min + 1);
            qs_schedule sc;
            sc.n = n;
            qs_op_host op;
            int path = QS_PATH_AUTO, n_act = 0, odd = 0;
            if (r.uniform() < 0.15) {
                op.kind = QS_OP_PHASE;
                op.coeff.assign(n, 0);
                odd = r.uniform() < 0.5;
                for (int q = 0; q < n; q++) op.coeff[q] = 2 * r.below(4) + (odd && r.uniform() < 0.3 ? 1 : 0);
                if (odd) op.coeff[r.below(n)] |= 1;
                const int ne = r.below(2 * n + 1);
                for (int e = 0; e < ne; e++) {
                    int a = r.below(n), b = r.below(n);
                    if (a != b) op.edges.push_back({std::min(a, b), std::max(a, b)});
                }
                int na;
                qs_pack_phase(n, op.coeff, op.edges, &na);
                n_act = na;
            } else {
                op.kind = QS_OP_DENSE;
                op.k = 1 + r.below(5);
                std::vector<int> perm(n);
                for (int q = 0; q < n; q++) perm[q] = q;
                for (int j = 0; j < op.k; j++) std::swap(perm[j], perm[j + r.below(n - j)]);
                std::sort(perm.begin(), perm.begin() + op.k);
                for (int j = 0; j < op.k; j++) op.qubits[j] = perm[j];
                op.matrix = timing_unitary(op.k, r);
                path = r.uniform() < 0.5 ? QS_PATH_CUDA_CORES : QS_PATH_TENSOR;
                op.path = path;
            }
            double f[kF];
            op_features(n, dtype, op.kind, op.k, op.qubits, path, n_act, odd, f);
            if (analytic_ms(f, 6696.8) > max_ms) continue;   // skip ops known to be far too slow to time
            sc.ops.push_back(op);
            float t[2] = {0, 0};
            rc = qs_run_circuit_timed(views[n], &sc, &t[0]);   // first run uploads the op
            if (!rc) rc = qs_run_circuit_timed(views[n], &sc, &t[1]);
            for (auto &dv : sc.dev)
                if (dv.pool) cudaFree(dv.pool);
            if (rc) break;
            std::memcpy(feats + (size_t)i * kF, f, sizeof(f));
            ms[i] = std::max(t[1], 1e-4f);
            i++;
        }
        for (qs_state *v : views) qs_free(v);
        qs_free(big);
        return rc;
    });
}

// ----------------------------------------------------------------- planner

constexpr int kCandidates = 8;   // search runs the planner predicts per k_max

// Predicted time of a schedule's ops (ms) with the qubits moved to the bits
// loc names (nullable: as they are), and each dense op's cheaper kernel path.
// From |0...0> the tensor-core sweeps cover only the support so far (the
// qubits of the dense ops before and including them): their features take
// that support's size as the state size.  A phase op right after a
// tensor-core sweep is folded into it (no time of its own).
static int plan_cost(const qs_schedule *sc, int dtype, const qs_cost_model *c, int which, const int *loc,
                     double *total, std::vector<int> *paths)
{
    const int n = sc->n;
    std::vector<double> F;
    std::vector<int> owner, cand_path;
    uint64_t sup = 0;
    const uint64_t all = n >= 64 ? ~0ULL : ((1ULL << n) - 1);
    bool prev_tc = false;
    for (size_t i = 0; i < sc->ops.size(); i++) {
        const qs_op_host &op = sc->ops[i];
        double f[kF];
        if (op.kind == QS_OP_PHASE) {
            if (prev_tc) {
                prev_tc = false;
                continue;                      // folded into the sweep before it
            }
            int na;
            qs_pack_phase(n, op.coeff, op.edges, &na);
            int odd = 0;
            for (int q = 0; q < n; q++) odd |= op.coeff[q] & 1;
            op_features(n, dtype, op.kind, 0, op.qubits, 0, na, odd, f);
            F.insert(F.end(), f, f + kF);
            owner.push_back((int)i);
            cand_path.push_back(QS_PATH_AUTO);
            sup = all;                         // phase sweeps cover the whole state
            continue;
        }
        int q[QS_MAX_DIAG_K];
        for (int j = 0; j < op.k; j++) q[j] = loc ? loc[op.qubits[j]] : op.qubits[j];
        std::sort(q, q + op.k);
        uint64_t grown = sup;
        for (int j = 0; j < op.k; j++) grown |= 1ULL << q[j];
        for (int path : {QS_PATH_CUDA_CORES, QS_PATH_TENSOR}) {
            if (path == QS_PATH_TENSOR && n < 5) continue;
            // a tensor-core sweep on a partial support works on 2^|support| amplitudes
            const int neff = (path == QS_PATH_TENSOR && grown != all) ? std::max(5, __builtin_popcountll(grown)) : n;
            op_features(neff, dtype, op.kind, op.k, q, path, 0, 0, f);
            F.insert(F.end(), f, f + kF);
            owner.push_back((int)i);
            cand_path.push_back(path);
        }
        sup = grown;
        prev_tc = n >= 5;
    }
    std::vector<double> t(owner.size());
    if (!owner.empty()) {
        int rc = qs_cost_model_predict(c, F.data(), (int)owner.size(), which, t.data());
        if (rc) return rc;
    }
    std::vector<double> op_t(sc->ops.size(), 0.0);
    std::vector<char> seen(sc->ops.size(), 0);
    if (paths) paths->assign(sc->ops.size(), QS_PATH_AUTO);
    for (size_t a = 0; a < owner.size(); a++) {
        const int i = owner[a];
        if (!seen[i] || t[a] < op_t[i]) {
            op_t[i] = t[a];
            seen[i] = 1;
            if (paths) (*paths)[i] = cand_path[a];
        }
    }
    double sum = 0;
    for (double x : op_t) sum += x;
    *total = sum;
    return QS_OK;
}

extern "C" int qs_plan_circuit(int n, const qs_gate *gates, int n_gates, int dtype, const qs_cost_model *c, int which,
                               qs_schedule **out, int *k_max_out, double *predicted_ms)
{
    return qs_guard([&]() -> int {
        if (!out || !c || (dtype != QS_C64 && dtype != QS_C128)) return qs_fail(QS_EINVAL, "qs_plan_circuit");
        qs_schedule *best = nullptr;
        double best_t = 1e300;
        int best_k = 0;
        std::vector<int> best_loc;
        std::vector<int> best_paths;
        for (int km = 2; km <= QS_MAX_K; km++) {
            // the clustering search of qs_schedule_build's defaults; its best
            // kCandidates distinct runs by analytic cost are each predicted
            qs_sched_opts o = {km, 1, 1, 0, 1, 13, 1, 16, 5};
            std::vector<qs_schedule *> cands;
            int rc = qs_schedule_build_ranked(n, gates, n_gates, &o, kCandidates, cands);
            if (rc) {
                for (qs_schedule *x : cands) qs_schedule_free(x);
                qs_schedule_free(best);
                return rc;
            }
          for (size_t ci = 0; ci < cands.size(); ci++) {
            qs_schedule *sc = cands[ci];
            double t0 = 0, t1 = 0;
            std::vector<int> paths0, paths1;
            if ((rc = plan_cost(sc, dtype, c, which, nullptr, &t0, &paths0))) {
                for (size_t cj = ci; cj < cands.size(); cj++) qs_schedule_free(cands[cj]);
                qs_schedule_free(best);
                return rc;
            }
            // the same schedule with its qubits moved off the costly low bits
            // (qs_schedule_choose_remap), kept if the model predicts it faster
            std::vector<int> loc(n);
            bool moved = false;
            if ((rc = qs_schedule_choose_remap(sc, dtype, loc.data()))) {
                for (size_t cj = ci; cj < cands.size(); cj++) qs_schedule_free(cands[cj]);
                qs_schedule_free(best);
                return rc;
            }
            for (int q = 0; q < n; q++) moved = moved || loc[q] != q;
            bool use_loc = false;
            if (moved) {
                if ((rc = plan_cost(sc, dtype, c, which, loc.data(), &t1, &paths1))) {
                    for (size_t cj = ci; cj < cands.size(); cj++) qs_schedule_free(cands[cj]);
                    qs_schedule_free(best);
                    return rc;
                }
                use_loc = t1 < t0 * (1.0 - 1e-9);
            }
            const double t = use_loc ? t1 : t0;
            if (t < best_t) {
                qs_schedule_free(best);
                best = sc;
                best_t = t;
                best_k = km;
                best_loc = use_loc ? loc : std::vector<int>();
                best_paths = use_loc ? paths1 : paths0;
            } else {
                qs_schedule_free(sc);
            }
            cands[ci] = nullptr;
          }
        }
        for (size_t i = 0; i < best->ops.size(); i++)
            if (best->ops[i].kind == QS_OP_DENSE) best->ops[i].path = best_paths[i];
        if (!best_loc.empty()) {
            int rc = qs_schedule_remap(best, best_loc.data());
            if (rc) {
                qs_schedule_free(best);
                return rc;
            }
        }
        *out = best;
        if (k_max_out) *k_max_out = best_k;
        if (predicted_ms) *predicted_ms = best_t;
        return QS_OK;
    });
}

extern "C" int qs_op_features(int n, int dtype, int kind, int k, const int *qubits, int path, int n_act, int odd,
                              double *out)
{
    return qs_guard([&]() -> int {
        if (!out || n < 1 || (kind == QS_OP_DENSE && (!qubits || k < 1 || k > QS_MAX_K)))
            return qs_fail(QS_EINVAL, "qs_op_features");
        op_features(n, dtype, kind, k, qubits, path, n_act, odd, out);
        return QS_OK;
    });
}

extern "C" double qs_cost_analytic_ms(const double *features, double hbm_gbs)
{
    return features ? analytic_ms(features, hbm_gbs) : -1.0;
}

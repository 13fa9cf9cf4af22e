/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow, gate-by-gate complex128 state-vector arithmetic, written from the
 * definitions in Sec. 2 (state vector, Kronecker-embedded gates) and Sec. 3.2
 * (gather / mat-vec / scatter form of a k-qubit gate) of Haener & Steiger,
 * "0.5 Petabyte Simulation of a 45-Qubit Quantum Circuit".  Only the tests, the
 * package's smoke check and the CPU-baseline leg of the benchmark may load it.
 * It shares no code, header or constant with the CUDA library.
 *
 * Conventions (Sec. 2): the state holds 2^n amplitudes alpha_i; qubit q is bit q
 * of the index i (qubit 0 = least significant bit).  Storage is interleaved
 * (re, im) doubles: psi[2*i] = Re alpha_i, psi[2*i+1] = Im alpha_i.
 *
 * Build with -ffp-contract=off: every product and sum is rounded on its own, so
 * x86-64 and aarch64 hosts give bit-identical results.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads.  The element-wise loops below (one gate, one phase product, the
 * probabilities) update every index, or index pair, on its own, so splitting
 * their iterations over OpenMP threads gives the serial loop's result bit for
 * bit.  The reductions (norm, statistics, sampling sums) stay serial: their
 * order of additions is part of their definition here. */
void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* (a + ib)(c + id) written out; kept as a helper so every complex product in
 * this file is the textbook formula. */
static inline void cmul(double ar, double ai, double br, double bi, double *cr, double *ci)
{
    *cr = ar * br - ai * bi;
    *ci = ar * bi + ai * br;
}

/* Sec. 2: U on qubit q is 1 (x) ... (x) U (x) ... (x) 1 with U in position q
 * counted from the right.  For every index pair (i0, i1) differing only in bit
 * q (bit q of i0 is 0):  (a0, a1) <- (u00 a0 + u01 a1, u10 a0 + u11 a1).
 * u: 2x2 row-major complex, interleaved (re, im). */
void or_apply_1q(double *psi, int n, int q, const double *u)
{
    uint64_t dim = (uint64_t)1 << n, bit = (uint64_t)1 << q;
#pragma omp parallel for schedule(static)
    for (uint64_t i0 = 0; i0 < dim; i0++) {
        if (i0 & bit) continue;
        uint64_t i1 = i0 | bit;
        double a0r = psi[2 * i0], a0i = psi[2 * i0 + 1];
        double a1r = psi[2 * i1], a1i = psi[2 * i1 + 1];
        double t0r, t0i, t1r, t1i, t2r, t2i, t3r, t3i;
        cmul(u[0], u[1], a0r, a0i, &t0r, &t0i);
        cmul(u[2], u[3], a1r, a1i, &t1r, &t1i);
        cmul(u[4], u[5], a0r, a0i, &t2r, &t2i);
        cmul(u[6], u[7], a1r, a1i, &t3r, &t3i);
        psi[2 * i0] = t0r + t1r;  psi[2 * i0 + 1] = t0i + t1i;
        psi[2 * i1] = t2r + t3r;  psi[2 * i1 + 1] = t2i + t3i;
    }
}

/* Sec. 2: CZ = diag(1, 1, 1, -1) adds a -1 phase to the |11> component of
 * qubits a and b; it is symmetric in a and b. */
void or_apply_cz(double *psi, int n, int a, int b)
{
    uint64_t dim = (uint64_t)1 << n;
    uint64_t ma = (uint64_t)1 << a, mb = (uint64_t)1 << b;
#pragma omp parallel for schedule(static)
    for (uint64_t i = 0; i < dim; i++) {
        if ((i & ma) && (i & mb)) {
            psi[2 * i] = -psi[2 * i];
            psi[2 * i + 1] = -psi[2 * i + 1];
        }
    }
}

/* Sec. 3.2: a k-qubit gate on qubits i_0..i_{k-1} (given in any order).  Every
 * index whose target bits are all zero starts one group c; the 2^k members of
 * the group are base + sum_j x_j 2^{i_j}, and x = x_{i_{k-1}} ... x_{i_0} is the
 * member's position in the temporary vector v.  v is gathered, multiplied by
 * the 2^k x 2^k matrix U (row-major complex, interleaved) and scattered back.
 * There are 2^{n-k} such mat-vecs. */
int or_apply_kq(double *psi, int n, const int *qubits, int k, const double *U)
{
    if (k < 1 || k > 12 || k > n) return -1;
    uint64_t dim = (uint64_t)1 << n, tmask = 0, K = (uint64_t)1 << k;
    for (int j = 0; j < k; j++) {
        if (qubits[j] < 0 || qubits[j] >= n) return -1;
        if (tmask & ((uint64_t)1 << qubits[j])) return -1;
        tmask |= (uint64_t)1 << qubits[j];
    }
    double *v = (double *)malloc(sizeof(double) * 2 * K);
    double *w = (double *)malloc(sizeof(double) * 2 * K);
    uint64_t *idx = (uint64_t *)malloc(sizeof(uint64_t) * K);
    if (!v || !w || !idx) { free(v); free(w); free(idx); return -2; }
    for (uint64_t base = 0; base < dim; base++) {
        if (base & tmask) continue;
        for (uint64_t x = 0; x < K; x++) {
            uint64_t i = base;
            for (int j = 0; j < k; j++)
                if ((x >> j) & 1) i |= (uint64_t)1 << qubits[j];
            idx[x] = i;
            v[2 * x] = psi[2 * i];
            v[2 * x + 1] = psi[2 * i + 1];
        }
        for (uint64_t l = 0; l < K; l++) {
            double sr = 0.0, si = 0.0;
            for (uint64_t x = 0; x < K; x++) {
                double pr, pi;
                cmul(U[2 * (l * K + x)], U[2 * (l * K + x) + 1], v[2 * x], v[2 * x + 1], &pr, &pi);
                sr += pr;
                si += pi;
            }
            w[2 * l] = sr;
            w[2 * l + 1] = si;
        }
        for (uint64_t x = 0; x < K; x++) {
            psi[2 * idx[x]] = w[2 * x];
            psi[2 * idx[x] + 1] = w[2 * x + 1];
        }
    }
    free(v); free(w); free(idx);
    return 0;
}

/* Exchange of qubits a[j] and b[j], j < m (the local bit swaps of Sec. 3.4):
 * amplitude i moves to the index with bits a[j] and b[j] of i exchanged.
 * Written as the permutation itself, through a copy of the state. */
int or_apply_swap(double *psi, int n, const int *a, const int *b, int m)
{
    uint64_t dim = (uint64_t)1 << n;
    for (int j = 0; j < m; j++)
        if (a[j] < 0 || a[j] >= n || b[j] < 0 || b[j] >= n) return -1;
    double *old = (double *)malloc(sizeof(double) * 2 * dim);
    if (!old) return -2;
    memcpy(old, psi, sizeof(double) * 2 * dim);
    for (uint64_t i = 0; i < dim; i++) {
        uint64_t t = i;
        for (int j = 0; j < m; j++) {
            uint64_t ba = (i >> a[j]) & 1, bb = (i >> b[j]) & 1;
            t &= ~(((uint64_t)1 << a[j]) | ((uint64_t)1 << b[j]));
            t |= (ba << b[j]) | (bb << a[j]);
        }
        psi[2 * t] = old[2 * i];
        psi[2 * t + 1] = old[2 * i + 1];
    }
    free(old);
    return 0;
}

/* A diagonal k-qubit gate: amplitude i is multiplied by d[x], x gathered from
 * the bits of i at qubits[0..k-1] exactly as in or_apply_kq. */
int or_apply_diag(double *psi, int n, const int *qubits, int k, const double *d)
{
    if (k < 1 || k > 20 || k > n) return -1;
    uint64_t dim = (uint64_t)1 << n;
    for (int j = 0; j < k; j++)
        if (qubits[j] < 0 || qubits[j] >= n) return -1;
#pragma omp parallel for schedule(static)
    for (uint64_t i = 0; i < dim; i++) {
        uint64_t x = 0;
        for (int j = 0; j < k; j++) x |= ((i >> qubits[j]) & 1) << j;
        double r, m;
        cmul(d[2 * x], d[2 * x + 1], psi[2 * i], psi[2 * i + 1], &r, &m);
        psi[2 * i] = r;
        psi[2 * i + 1] = m;
    }
    return 0;
}

/* e^{i pi m / 4} for m = 0..7, written from its definition with the exact
 * values of cos and sin at multiples of pi/4. */
static void omega_pow(int m, double *re, double *im)
{
    const double r = 0.70710678118654752440; /* 1/sqrt(2) */
    static const double tr[8] = {1, 1, 0, -1, -1, -1, 0, 1};
    static const double ti[8] = {0, 1, 1, 1, 0, -1, -1, -1};
    m &= 7;
    *re = (m & 1) ? tr[m] * r : tr[m];
    *im = (m & 1) ? ti[m] * r : ti[m];
}

/* A product of diagonal gates from the supremacy gate set: T_q contributes
 * e^{i pi/4} when bit q is set (Sec. 2), CZ(a,b) contributes -1 = e^{i pi 4/4}
 * when bits a and b are both set.  Amplitude i is multiplied by
 * e^{i pi m(i)/4} with m(i) = sum_q c[q] i_q + 4 sum_{(a,b)} i_a i_b  (mod 8).
 * c: n coefficients; edges: n_edges pairs (a, b). */
int or_apply_phase(double *psi, int n, const int *c, int n_edges, const int *edges)
{
    uint64_t dim = (uint64_t)1 << n;
    for (int e = 0; e < 2 * n_edges; e++)
        if (edges[e] < 0 || edges[e] >= n) return -1;
#pragma omp parallel for schedule(static)
    for (uint64_t i = 0; i < dim; i++) {
        int m = 0;
        for (int q = 0; q < n; q++)
            if ((i >> q) & 1) m += c[q];
        for (int e = 0; e < n_edges; e++)
            if (((i >> edges[2 * e]) & 1) && ((i >> edges[2 * e + 1]) & 1)) m += 4;
        double wr, wi, r, im;
        omega_pow(((m % 8) + 8) % 8, &wr, &wi);
        cmul(wr, wi, psi[2 * i], psi[2 * i + 1], &r, &im);
        psi[2 * i] = r;
        psi[2 * i + 1] = im;
    }
    return 0;
}

/* Sec. 2: measuring gives outcome i with probability p_i = |alpha_i|^2.  Each
 * product and the sum are rounded separately (no fused multiply-add). */
void or_probabilities(const double *psi, int n, double *p)
{
    uint64_t dim = (uint64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (uint64_t i = 0; i < dim; i++) {
        double a = psi[2 * i] * psi[2 * i];
        double b = psi[2 * i + 1] * psi[2 * i + 1];
        p[i] = a + b;
    }
}

/* Sum of p_i, sequential in index order. */
double or_norm(const double *psi, int n)
{
    uint64_t dim = (uint64_t)1 << n;
    double s = 0.0;
    for (uint64_t i = 0; i < dim; i++)
        s += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
    return s;
}

/* Output-distribution statistics (Sec. 4.2 computes the entropy with a final
 * reduction): out[0] = sum p, out[1] = -sum p ln p (terms with p = 0 dropped),
 * out[2] = mean of N p, out[3] = mean of (N p)^2, with N = 2^n. */
void or_stats(const double *psi, int n, double *out)
{
    uint64_t dim = (uint64_t)1 << n;
    double N = (double)dim, s = 0, h = 0, m1 = 0, m2 = 0;
    for (uint64_t i = 0; i < dim; i++) {
        double p = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
        s += p;
        if (p > 0) h -= p * log(p);
        m1 += N * p;
        m2 += (N * p) * (N * p);
    }
    out[0] = s;
    out[1] = h;
    out[2] = m1 / N;
    out[3] = m2 / N;
}

/* ---------------------------------------------------------------------------
 * Sampling.  The paper samples nothing, so the procedure is this project's
 * reading, fixed so that two implementations given the same amplitudes draw the
 * same outcomes:
 *   u_j  = (splitmix64 output j of `seed`) >> 11, times 2^-53;
 *   p_x  = fl(fl(re^2) + fl(im^2))                       (or_probabilities);
 *   S_b  = pairwise sum of the p_x of block b (B = 1024 outcomes, or 2^n if
 *          smaller): sum(v[0,2m)) = sum(v[0,m)) + sum(v[m,2m));
 *   T_s  = pairwise sum of the S_b of super-block s (G = 1024 blocks, or all);
 *   Q_0 = 0, Q_{s+1} = Q_s + T_s                          (sequential);
 *   R_{s,0} = Q_s, R_{s,j+1} = R_{s,j} + S_{sG+j}         (sequential);
 *   c_0 = R_{s,j}, c_{i+1} = c_i + p_{bB+i}               (sequential);
 *   s* = largest s with Q_s <= u, j* = largest j with R_{s*,j} <= u,
 *   i* = smallest i with c_{i+1} > u (B-1 if none); the outcome is b*B + i*.
 * ------------------------------------------------------------------------- */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the j-th output (j >= 0) of the
 * generator seeded with `seed` mixes seed + (j+1) * 0x9E3779B97F4A7C15. */
uint64_t or_splitmix64(uint64_t seed, uint64_t j)
{
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double pairwise(const double *v, uint64_t len)
{
    if (len == 1) return v[0];
    uint64_t h = len / 2;
    return pairwise(v, h) + pairwise(v + h, len - h);
}

int or_sample(const double *psi, int n, uint64_t seed, int64_t m, uint64_t *out)
{
    uint64_t dim = (uint64_t)1 << n;
    uint64_t B = dim < 1024 ? dim : 1024;
    uint64_t nb = dim / B;
    uint64_t G = nb < 1024 ? nb : 1024;
    uint64_t ns = nb / G;
    double *p = (double *)malloc(sizeof(double) * dim);
    double *S = (double *)malloc(sizeof(double) * nb);
    double *T = (double *)malloc(sizeof(double) * ns);
    double *Q = (double *)malloc(sizeof(double) * ns);
    double *R = (double *)malloc(sizeof(double) * nb);
    if (!p || !S || !T || !Q || !R) { free(p); free(S); free(T); free(Q); free(R); return -2; }
    or_probabilities(psi, n, p);
    for (uint64_t b = 0; b < nb; b++) S[b] = pairwise(p + b * B, B);
    for (uint64_t s = 0; s < ns; s++) T[s] = pairwise(S + s * G, G);
    Q[0] = 0.0;
    for (uint64_t s = 0; s + 1 < ns; s++) Q[s + 1] = Q[s] + T[s];
    for (uint64_t s = 0; s < ns; s++) {
        R[s * G] = Q[s];
        for (uint64_t j = 0; j + 1 < G; j++) R[s * G + j + 1] = R[s * G + j] + S[s * G + j];
    }
    for (int64_t t = 0; t < m; t++) {
        double u = (double)(or_splitmix64(seed, (uint64_t)t) >> 11) * 0x1.0p-53;
        uint64_t s = 0;
        for (uint64_t q = 0; q < ns; q++) if (Q[q] <= u) s = q;
        uint64_t jb = 0;
        for (uint64_t j = 0; j < G; j++) if (R[s * G + j] <= u) jb = j;
        uint64_t b = s * G + jb;
        double c = R[b];
        uint64_t i = B - 1;
        for (uint64_t x = 0; x < B; x++) {
            c = c + p[b * B + x];
            if (c > u) { i = x; break; }
        }
        out[t] = b * B + i;
    }
    free(p); free(S); free(T); free(Q); free(R);
    return 0;
}

/*
 * qs -- GB300 (sm_103a) state-vector simulator for fused k-qubit cluster sweeps
 * over low-depth random ("supremacy") circuits, after Haener & Steiger,
 * "0.5 Petabyte Simulation of a 45-Qubit Quantum Circuit".
 *
 * C ABI.  All functions return QS_OK (0) or a negative QS_E* code and never
 * abort; qs_last_error() gives a thread-local message for the last failure.
 * Pointers are host pointers unless a parameter says "device".  Every call is
 * ordered on the state's CUDA stream; calls that return results to host memory
 * (qs_norm, qs_stats, qs_probabilities to host, qs_sample, qs_get_amplitudes)
 * synchronise that stream before returning.  The caller keeps ownership of every
 * array it passes; the library copies what it needs before returning.
 *
 * State layout (Sec. 2): 2^n amplitudes alpha_i, qubit q = bit q of the index i
 * (qubit 0 least significant), stored contiguously in device memory as
 * interleaved (re, im) pairs: double2 for QS_C128, float2 for QS_C64.
 */
#ifndef QS_H
#define QS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    QS_OK = 0,
    QS_EINVAL = -1,        /* bad argument (range, duplicate qubit, size) */
    QS_ENOMEM = -2,        /* device or host allocation failed */
    QS_ECUDA = -3,         /* a CUDA runtime call failed */
    QS_ETIMEOUT = -4,      /* a bounded device wait ran out */
    QS_EUNSUPPORTED = -5   /* valid request this build does not handle */
};

enum { QS_C64 = 0, QS_C128 = 1 };   /* amplitude type: complex float / double */

#define QS_MAX_K 5          /* largest dense cluster (2^5 x 2^5 unitary) */
#define QS_MAX_DIAG_K 12    /* largest table diagonal */
#define QS_MAX_SWAP 16      /* most qubit pairs one qs_swap_qubits call exchanges */
#define QS_MAX_QUBITS 36    /* largest state this build addresses */

typedef struct qs_state qs_state;   /* opaque, owned by the library */

const char *qs_last_error(void);

/* Allocate a state of 2^n amplitudes of the given dtype on the current CUDA
 * device (Sec. 2; in place, one buffer, Sec. 3.2).  stream: a cudaStream_t or
 * NULL for the legacy default stream.  Contents are undefined until an init
 * call.  Errors: QS_EINVAL (n < 1 or n > QS_MAX_QUBITS, bad dtype),
 * QS_ENOMEM (cudaMalloc failed, e.g. more than the free device memory).
 *
 * No entry point lets a C++ exception escape: a host allocation that fails
 * inside any call returns QS_ENOMEM, any other internal exception QS_EINVAL,
 * with the message in qs_last_error(). */
int qs_alloc(int n, int dtype, void *stream, qs_state **out);

/* Adopt an existing device buffer of 2^n amplitudes (e.g. a torch tensor's
 * storage; 16-byte aligned).  The library never frees dev_ptr.  Errors as
 * qs_alloc, plus QS_EINVAL for a NULL or misaligned pointer. */
int qs_wrap(void *dev_ptr, int n, int dtype, void *stream, qs_state **out);

/* Release a state and the library's scratch buffers (not a wrapped buffer).
 * NULL is ignored. */
void qs_free(qs_state *s);

/* Make `device` the current CUDA device of the calling thread for later
 * qs_alloc / qs_wrap calls.  QS_ECUDA if the device does not exist. */
int qs_set_device(int device);

/* Which kernels apply dense clusters.  The tensor-core sweep handles 5-qubit
 * clusters (smaller ones embedded as U (x) 1 on extra qubits; n >= 5):
 * complex64 by a tf32 head/tail split with FP32 accumulation, complex128 by
 * exact 8-bit integer digit planes on the fp16 path rebuilt in integer
 * arithmetic.  QS_PATH_AUTO: tensor cores for complex64 clusters of 4 and 5
 * qubits and for complex128 clusters of 2..5 qubits, CUDA cores otherwise;
 * QS_PATH_TENSOR: tensor cores for every dense cluster (n >= 5);
 * QS_PATH_CUDA_CORES: the FP32 / FP64 CUDA-core kernel for every cluster. */
enum { QS_PATH_AUTO = 0, QS_PATH_CUDA_CORES = 1, QS_PATH_TENSOR = 2 };
int qs_set_path(qs_state *s, int path);

/* Phase folding in qs_run_circuit (on by default).  A phase op (merged CZ / T
 * run, Sec. 2) that directly follows a dense op run by the tensor-core sweep
 * is applied inside that sweep, saving its own HBM sweep.  The phase terms on
 * the sweep's five qubits are multiplied into the cluster matrix (FP64, before
 * packing).  A CZ with one end off those qubits acts on each group as a Z on
 * the other end or not, and one with both ends off as a phase of the whole
 * group (the specialisation Sec. 3.5 makes for CZ on global qubits); these and
 * the coefficients off the sweep's qubits become a power of i per group and a
 * sign per member, applied to the sweep's outputs.  The fold is taken only
 * where every coefficient off the sweep's qubits is even (a power of i;
 * CZ-only layers always qualify); other phase ops run as their own sweep.
 * on = 0 turns folding off.  Results agree with the unfolded run to rounding;
 * bit for bit (up to the sign of zeros) when no phase term lies on the
 * sweep's qubits, as the matrix is then unchanged.  QS_EINVAL for a null
 * state. */
int qs_set_phase_fold(qs_state *s, int on);

/* Pair sweeps in qs_run_circuit (off by default: measured slower than two
 * separate sweeps on GB300, 1.63 against 1.40 ms for two 28-qubit clusters
 * sharing two qubits, 3.4 ms against 1.4 ms for disjoint high targets).  On:
 * for complex64 states of 12 or
 * more qubits with every amplitude reachable, two consecutive dense ops that
 * both run on the tensor cores and whose (padded) target qubits number at most
 * 10 are applied in one sweep.  The GPU form of applying several gates while
 * a chunk of the state sits in fast memory (Fig. 2 caption, Sec. 4): the
 * 2^{|T1 u T2|} amplitudes that agree off both clusters' targets pass through
 * shared memory between the two products, so the state is read and written
 * once for both.  Results equal the two separate sweeps' bit for bit (the
 * first cluster's outputs are rounded to float in between, as in HBM).  A
 * phase op after the second cluster is folded into it as usual;
 * qs_run_circuit_timed reports the pair's time on the first op and -1 on the
 * ops that ran inside it.  on = 1 turns pairing on.  QS_EINVAL for a null
 * state. */
int qs_set_pair_sweeps(qs_state *s, int on);

int qs_num_qubits(const qs_state *s);
int qs_dtype(const qs_state *s);
/* Device pointer to amplitude 0, holding the whole state: zeros the library
 * has not written yet (see qs_init_basis) are written first, on the state's
 * stream.  NULL for a null state or when that write fails. */
void *qs_device_ptr(const qs_state *s);

/* Order later calls on `stream` (a cudaStream_t or NULL for the legacy default
 * stream) instead of the state's current stream.  Work already queued on the
 * old stream (sweeps, the state's scratch and status words) is finished first:
 * the new stream waits on an event recorded on the old one, so the next call
 * on the new stream never runs beside earlier calls on the old one.  The host
 * does not block.  QS_EINVAL for a null state, QS_ECUDA if the event cannot
 * be recorded or waited on. */
int qs_set_stream(qs_state *s, void *stream);

/* |x>: amplitude x = 1, all others 0 (Sec. 2).  QS_EINVAL if x >= 2^n.
 * On a state from qs_alloc only amplitude x is written now.  Tensor-core
 * cluster sweeps then work on the indices the circuit so far can reach
 * (targets of the clusters applied since, other bits as in x) and give the same
 * result as on the zero-filled state; every other call writes the remaining
 * zeros first.  A state on the caller's buffer (qs_wrap) is written in full. */
int qs_init_basis(qs_state *s, uint64_t x);

/* (2^{-n/2}, ..., 2^{-n/2}): the state after the H layer of cycle 0, which a
 * simulator may prepare directly (Sec. 3.6). */
int qs_init_uniform(qs_state *s);

/* Copy 2^n complex128 amplitudes (interleaved re, im; host memory) into the
 * state, rounding to the state's dtype; and back (widening for QS_C64). */
int qs_set_amplitudes(qs_state *s, const double *host_c128);
int qs_get_amplitudes(qs_state *s, double *host_c128);
/* Amplitudes at `count` indices (each < 2^n) as complex128 (host memory; out:
 * 2*count doubles), for spot checks of states too large to copy whole. */
int qs_get_amplitudes_at(qs_state *s, const uint64_t *indices, int64_t count, double *out);

/* Apply a dense k-qubit gate in place (Sec. 3.2): for every assignment c of the
 * n-k other bits, the 2^k amplitudes whose target bits spell x (x_j = bit
 * qubits[j] of the index) form a vector v, replaced by U v.  There are 2^{n-k}
 * such products.  qubits: k distinct values in [0, n), any order; the library
 * permutes U to ascending qubit order (Sec. 3.2).  U: 2^k x 2^k row-major,
 * complex128 interleaved (re, im), FP64 for both dtypes (rounded to float for
 * QS_C64).  1 <= k <= QS_MAX_K.  Errors: QS_EINVAL. */
int qs_apply_cluster(qs_state *s, const int *qubits, int k, const double *U);

/* Apply a diagonal k-qubit gate: amplitude i is multiplied by d[x], x gathered
 * from the bits qubits[0..k-1] of i as in qs_apply_cluster.  d: 2^k complex128
 * interleaved.  1 <= k <= QS_MAX_DIAG_K. */
int qs_apply_diag(qs_state *s, const int *qubits, int k, const double *d);

/* Exchange qubit a[j] with qubit b[j] for j < m (the local bit swaps of Sec.
 * 3.4, used by the bit-location remapping of Sec. 3.6): amplitude i moves to
 * the index with bits a[j] and b[j] of i exchanged, i.e. the product of the m
 * SWAP gates (a[j], b[j]).  One sweep over the state in place; swaps that
 * involve qubits 0-2 go through shared memory so that every global access is
 * a contiguous run of at least 512 bytes.  The 2m qubits are distinct and in
 * [0, n); 0 <= m <= QS_MAX_SWAP.  Errors: QS_EINVAL. */
int qs_swap_qubits(qs_state *s, const int *a, const int *b, int m);

/* Apply a product of T-type phases and CZ gates (Sec. 2, Sec. 3.5: both are
 * diagonal): amplitude i is multiplied by e^{i pi m(i)/4} with
 *   m(i) = sum_q coeff[q] i_q + 4 sum_{e < n_edges} i_{edges[2e]} i_{edges[2e+1]}
 * (mod 8).  coeff: n integers (taken mod 8); edges: 2*n_edges qubit indices in
 * [0, n) (a pair may repeat; a == b is rejected). */
int qs_apply_phase(qs_state *s, const int *coeff, int n_edges, const int *edges);

/* sum_i |alpha_i|^2, accumulated in FP64 (Sec. 2).  out: host double. */
int qs_norm(qs_state *s, double *out);

/* p_i = |alpha_i|^2 in FP64, each product and the sum rounded separately
 * (Sec. 2).  out: 2^n doubles, device memory if out_on_device, else host. */
int qs_probabilities(qs_state *s, double *out, int out_on_device);

/* Output-distribution statistics in FP64 (Sec. 4.2 computes the entropy with a
 * final reduction): out[0] = sum p, out[1] = -sum p ln p, out[2] = mean of N p,
 * out[3] = mean of (N p)^2 (N = 2^n; Porter-Thomas gives 1 and 2). */
int qs_stats(qs_state *s, double out[4]);

/* Draw m outcomes (not in the paper; this library's rule): u_j = (SplitMix64
 * output j of seed >> 11) * 2^-53 and outcome j = the first x whose cumulative
 * probability exceeds u_j, the cumulative sums taken in FP64 in a fixed order
 * (pairwise within blocks of 1024 outcomes and super-blocks of 1024 blocks,
 * sequential across them).  out: m uint64 in host memory.  m >= 0. */
int qs_sample(qs_state *s, uint64_t seed, int64_t m, uint64_t *out);

/* qs_stats and qs_sample in one call (not in the paper): the same draws, bit
 * for bit, and the same statistics up to the order of their float-float sums
 * (relative differences near 1e-15).  For complex64 states of 10 qubits or
 * more one pass over the state forms both the block sums of the draws and the
 * statistics; complex128 states of 10 qubits or more run qs_stats' pass on a
 * second stream of the state beside the block sums (forked from and joined to
 * the state's stream before the call returns; the statistics then equal
 * qs_stats' exactly); smaller states take the statistics first.  out: m
 * uint64 in host memory; stats: 4 host doubles as qs_stats.  Errors as
 * qs_stats. */
int qs_sample_stats(qs_state *s, uint64_t seed, int64_t m, uint64_t *out, double stats[4]);

/* qs_stats without any allocation.  The paper has no counterpart: this entry
 * exists for callers that may not allocate device memory, for example code that
 * runs while a framework's caching allocator owns the device memory, or code
 * that cannot afford the device-wide synchronisation a cudaMalloc implies.
 * dev_amp: 2^n amplitudes of the given dtype in device memory (interleaved
 * re, im), aligned to one amplitude (16 bytes for QS_C128, 8 for QS_C64; a
 * view starting at any amplitude of a state qualifies, anything else is
 * QS_EINVAL), read only; out: 4 doubles in host memory, as
 * qs_stats.  The partial sums use a fixed 32,800-byte array compiled into the
 * library (one per GPU that loads it, held until the process exits); the
 * kernels use at most 1024 blocks, so every n in [1, QS_MAX_QUBITS] fits and
 * anything else is rejected with QS_EINVAL.  The first call on a device looks
 * up that array's device address; make that first call before any stream
 * capture.  Calls share the array: calls whose kernels overlap on the GPU (on
 * different streams) race and must be serialised by the caller.  Calls no
 * cudaMalloc / cudaFree; synchronises `stream` before returning. */
int qs_stats_static(const void *dev_amp, int n, int dtype, void *stream, double out[4]);

/* Wait for all work queued on the state's stream; QS_ETIMEOUT (once, the word
 * is cleared) if a tensor-core kernel's bounded wait ran out since the last
 * check; QS_EINVAL (once) if a complex128 tensor-core sweep met amplitudes
 * above ~2^1010 in magnitude, whose results could pass the double range (its
 * outputs are then not meaningful).  Rows below ~2^-970 are swept with their
 * scale raised, so no result leaves the normal range (absolute error
 * ~2^-1015). */
int qs_synchronize(qs_state *s);

/* Exercises the failure path of the bounded waits: one thread waits on an
 * mbarrier nothing arrives on, gives up after 1000 tries (microseconds to
 * milliseconds), records the expiry in the state's status word and returns.
 * Returns QS_ETIMEOUT and clears the word; the state and the context stay
 * usable.  No GPU fault or hang.  QS_EINVAL for a null state. */
int qs_selftest_timeout(qs_state *s);

/* ------------------------------------------------------------------------
 * Circuits (Fig. 1 caption; Sec. 3.6).
 * ---------------------------------------------------------------------- */
enum {
    QS_GATE_H = 0, QS_GATE_T = 1, QS_GATE_SQRT_X = 2, QS_GATE_SQRT_Y = 3,
    QS_GATE_CZ = 4, QS_GATE_X = 5, QS_GATE_TDG = 6, QS_GATE_SQRT_XDG = 7,
    QS_GATE_SQRT_YDG = 8
};

typedef struct {
    int32_t cycle;   /* clock cycle (0 = H layer) */
    int32_t kind;    /* QS_GATE_* */
    int32_t q0;      /* qubit */
    int32_t q1;      /* second qubit of CZ, else -1 */
} qs_gate;

/* Generate a supremacy circuit on a rows x cols grid with some sites removed
 * (removed_rc: n_removed (row, col) pairs), cz_cycles CZ cycles after the H
 * layer, seed for the single-qubit gate choices.  Fig. 1 caption: H on every
 * qubit in cycle 0; eight staggered CZ layouts repeated; a qubit that left a CZ
 * gets T first, later a uniform choice among {T, X^1/2, Y^1/2} minus its
 * previous gate.  Readings where the paper is silent: qubit = row-major index of
 * the remaining sites; layouts H(1,0) V(0,0) H(0,0) V(1,0) V(0,1) H(1,1) V(1,1)
 * H(0,1), where H(a,b) couples (r,c)-(r,c+1) with c%2 == a, r%2 == b and V(a,b)
 * couples (r,c)-(r+1,c) with r%2 == a, c%2 == b; choice j takes the
 * ((SplitMix64 output j) >> 63)-th allowed gate.  Gates are written to
 * gates[0..max_gates); *n_gates receives the count (QS_EINVAL, with *n_gates
 * set, if max_gates is too small).  *n_qubits receives the qubit count. */
int qs_supremacy_circuit(int rows, int cols, const int *removed_rc, int n_removed,
                         int cz_cycles, uint64_t seed, int *n_qubits,
                         qs_gate *gates, int max_gates, int *n_gates);

/* ------------------------------------------------------------------------
 * Schedules (Sec. 3.6 step 2: clusters of k <= k_max qubits; Sec. 3.2 matrix
 * pre-permutation; Sec. 3.5 diagonal gates).
 * ---------------------------------------------------------------------- */
typedef struct qs_schedule qs_schedule;   /* opaque, owned by the library */

enum { QS_OP_DENSE = 0, QS_OP_PHASE = 1, QS_OP_DIAG = 2 };

typedef struct {
    int32_t k_max;        /* 2..QS_MAX_K when fuse != 0 */
    int32_t fuse;         /* 0: one op per gate (plain form); 1: greedy clusters */
    int32_t merge_phase;  /* 1: merge neighbouring all-diagonal ops into one phase op */
    int32_t drop_final_diagonal;  /* 1: leave out the trailing all-diagonal ops.  They
                                   * change phases only, not |amplitude|^2, so the
                                   * output distribution, its statistics and samples
                                   * are those of the full circuit (Sec. 3.6 skips the
                                   * last CZ layer this way); amplitudes differ by
                                   * those phases.  0: keep every gate. */
    int32_t commute_diagonal;     /* 1: diagonal gates (T, T^dagger, CZ) may pass one
                                   * another on a qubit while clusters are formed:
                                   * diagonal matrices commute, so the product is the
                                   * same, and runs of them no longer split clusters
                                   * (30-qubit 5x6 depth 25: 28-29 dense clusters at
                                   * k_max 5 instead of 36).  0: every qubit keeps its
                                   * gate order (the paper's rule, Sec. 3.6). */
    int32_t search_runs;          /* 0..64; with commute_diagonal: 0 or 1, the greedy
                                   * rule alone; R > 1, the best of R runs: run 0
                                   * the greedy rule, run s >= 1 choosing, while the
                                   * dense clusters taken so far leave some qubit
                                   * out, among the clusters within
                                   * search_slack0 + s - 1 gates of the largest the
                                   * one adding the fewest qubits to them (then the
                                   * greedy rank).  The run of
                                   * lowest cost wins, then the fewest clusters,
                                   * then the lower r; cost = the number of dense
                                   * clusters, or with search_from_basis each dense
                                   * cluster weighted by 2^(|support| - n), the
                                   * support growing by its qubits from none (the
                                   * sweep sizes after qs_init_basis).  Runs go on
                                   * host threads (at most 32). */
    int32_t search_from_basis;    /* 1: the state will start as a basis state (see
                                   * search_runs); 0: any state. */
    int32_t search_first;         /* 0..16; 0 or 1: each run takes its first cluster
                                   * by its own rule; F > 1: each of the R runs is
                                   * made F times, the f-th time (f = 1..F-1) with
                                   * its first cluster the one of rank f among the
                                   * clusters grown from all seeds (the last one
                                   * when there are fewer) -- where the support
                                   * starts; R x F runs compete as above, run index
                                   * f * R + r. */
    int32_t search_slack0;        /* 0..64: the slack of support-aware run 1 (see
                                   * search_runs); 0 gives slacks 0..R-2. */
} qs_sched_opts;

/* Build a schedule for an n-qubit gate list.  With fuse, gates are packed into
 * clusters by the greedy closure rule (each cluster: the gates that can run on a
 * qubit set S, S grown from a seed gate while |S| <= k_max, the largest cluster
 * taken first; with commute_diagonal, diagonal gates may pass one another on a
 * qubit), an all-diagonal cluster becomes a phase op, and every dense
 * cluster's unitary is the FP64 product of its gates in ascending qubit order.
 * With drop_final_diagonal the trailing phase ops are left out (see the field).
 * Errors: QS_EINVAL (bad gate, opts). */
int qs_schedule_build(int n, const qs_gate *gates, int n_gates, const qs_sched_opts *opts,
                      qs_schedule **out);

/* A schedule from explicit ops (the caller's own clustering): op i is dense
 * (kinds[i] = QS_OP_DENSE: ks[i] qubits in qubits[5i..5i+ks[i]), unitary at
 * pool[offsets[i]], 2^k x 2^k complex128 interleaved), a table diagonal
 * (QS_OP_DIAG, 2^k complex128 at pool[offsets[i]]) or a phase op (QS_OP_PHASE,
 * Sec. 2: amplitude x times e^{i pi s(x) / 4}, s(x) = sum_q c_q x_q +
 * 4 sum_pairs x_a x_b; ks[i] = number of CZ pairs, qubits[] unused; at
 * pool[offsets[i]] the n coefficients c_q, then the 2 ks[i] qubits of the
 * pairs, all integers stored as doubles; coefficients are taken mod 8).
 * QS_EINVAL for a bad kind, qubit, pair, non-integer entry or a read past the
 * pool. */
int qs_schedule_from_ops(int n, int n_ops, const int *kinds, const int *ks,
                         const int *qubits, const int64_t *offsets,
                         const double *pool, int64_t pool_len, qs_schedule **out);

void qs_schedule_free(qs_schedule *sc);

/* Bytes qs_run_circuit copies host -> device the first time it runs this
 * schedule on a state of the given dtype (op matrices, tables, phase masks). */
int64_t qs_schedule_upload_bytes(const qs_schedule *sc, int dtype);

/* Bit-location remapping (Sec. 3.6: map qubits to index bits so that the
 * kernels' targets avoid the costly positions; the paper's local bit swaps,
 * Sec. 3.4, move the data).  loc: n entries, qubit q to index bit loc[q], a set
 * of exchanges (loc[loc[q]] == q).  qs_schedule_remap relabels every op of the
 * schedule (dense and diagonal ops get their qubits mapped and their matrices
 * permuted to ascending order; phase ops their coefficients and CZ pairs), so
 * qs_schedule_op then reports index bits.  qs_run_circuit first brings the
 * state's qubits to those bits: free after qs_init_basis (the one amplitude
 * is written at its new index), one or two exchange sweeps otherwise.  The
 * state remembers where its qubits are: calls that name qubits or indices
 * (qs_apply_*, qs_swap_qubits, qs_get_amplitudes_at) translate them, and
 * calls whose result follows the index order (qs_get_amplitudes,
 * qs_probabilities, qs_sample, qs_sample_stats, qs_device_ptr) first move
 * the qubits back to their own bits (one exchange sweep); qs_norm and
 * qs_stats do not depend on the order.  qs_init_*, qs_set_amplitudes start in
 * the identity order.  A remapped schedule cannot join a batch.  QS_EINVAL for
 * a bad loc or a schedule remapped before.
 * qs_schedule_choose_remap picks loc for a schedule started from |0...0>:
 * the qubits that are targets of the least dense-sweep work (each sweep
 * weighted by the share of the state it covers, the support growing by every
 * dense cluster's qubits) go to index bits 0-1 (complex128) or 0-4
 * (complex64), exchanged with the qubits there; measured on GB300, 5-qubit
 * sweeps with targets among those bits take 25-30% longer. */
int qs_schedule_remap(qs_schedule *sc, const int *loc);
int qs_schedule_choose_remap(const qs_schedule *sc, int dtype, int *loc);
/* The schedule's qubit-to-bit map: n entries, the identity for a schedule
 * never remapped.  QS_EINVAL for null arguments. */
int qs_schedule_get_remap(const qs_schedule *sc, int *loc);

/* Stages for a state held as 2^n_global parts (Sec. 3.4, Sec. 3.6 steps 1 and
 * 3): the top n_global index bits of a stage hold its global qubits, on which
 * the stage applies no gate except diagonal ones (CZ, T; Sec. 3.5 applies
 * those as conditional phases of a part).  The gate list is split greedily in
 * its order: a gate joins the present stage unless it is a non-diagonal gate
 * on a global qubit or shares a qubit with a gate left for later; the next
 * stage's global qubits are the n_global whose next non-diagonal gate comes
 * last.  Each stage is clustered with opts (qs_schedule_build) and remapped
 * (qs_schedule_remap) so that its global qubits sit at the top bits; running
 * the stages in order with qs_run_circuit moves the qubits between stages,
 * the global-to-local swap: on one GPU one or two exchange sweeps
 * (qs_swap_qubits), where a multi-GPU form would exchange the parts' data
 * (Sec. 3.4 all-to-all).  stages: room for max_stages schedules, each freed
 * with qs_schedule_free; *n_stages stages made; stage_of_gate (nullable):
 * n_gates entries, the stage of every gate.  Errors: QS_EINVAL (bad arguments,
 * more than max_stages stages, no gate runnable with n_global global
 * qubits). */
int qs_plan_stages(int n, const qs_gate *gates, int n_gates, int n_global, const qs_sched_opts *opts,
                   qs_schedule **stages, int max_stages, int *n_stages, int *stage_of_gate);

/* Build the schedule's device image for `dtype` (every op's matrix in the
 * dtype, tensor-core operand planes, folded phase descriptors) and copy it to
 * the calling thread's current device now, instead of at the first
 * qs_run_circuit there.  The copy goes through a stream of its own, so a host
 * thread can prepare the next circuit while kernels of the current one run on
 * other streams.  A schedule must not be uploaded and run on the same device
 * from two threads at once.  Errors: QS_EINVAL, QS_ENOMEM, QS_ECUDA. */
int qs_schedule_upload(const qs_schedule *sc, int dtype);

/* Most host threads the clustering search of qs_schedule_build uses (0, the
 * default: one per hardware thread).  A caller that launches kernels while a
 * second thread builds the next schedule can leave cores to the launching
 * thread.  QS_EINVAL for n < 0. */
int qs_set_host_threads(int n);
int qs_schedule_num_qubits(const qs_schedule *sc);
int qs_schedule_num_ops(const qs_schedule *sc);

typedef struct {
    int32_t kind;                /* QS_OP_* */
    int32_t k;                   /* qubits touched (dense/diag); phase: qubits in its support */
    int32_t qubits[QS_MAX_K];    /* ascending (dense/diag) */
    int32_t n_gates;             /* gates of the circuit in this op */
    int32_t n_edges;             /* phase: CZ pairs */
    int32_t reserved;
} qs_op_info;

/* Describe op i.  Optional outputs (NULL to skip): matrix (dense: 2^{2k}
 * complex128 interleaved, qubits[j] <-> bit j; diag: 2^k), gate_idx (n_gates
 * circuit indices in the order multiplied), coeff (phase: n integers mod 8),
 * edges (phase: 2*n_edges). */
int qs_schedule_op(const qs_schedule *sc, int i, qs_op_info *info, double *matrix,
                   int32_t *gate_idx, int32_t *coeff, int32_t *edges);

/* Apply every op of a schedule, in order, to the state (one HBM sweep per op). */
int qs_run_circuit(qs_state *s, const qs_schedule *sc);

/* As qs_run_circuit, recording a CUDA event before and after every op on the
 * state's stream; waits for the stream and writes op i's device time in
 * milliseconds to op_ms[i] (host, qs_schedule_num_ops entries).  An op that
 * runs inside the sweep before it launches nothing and gets op_ms[i] = -1:
 * a phase op folded into a tensor-core sweep (qs_set_phase_fold) or the
 * second cluster of a pair sweep (qs_set_pair_sweeps); its time is part of
 * the previous op's. */
int qs_run_circuit_timed(qs_state *s, const qs_schedule *sc, float *op_ms);

/* ------------------------------------------------------------------------
 * Batched simulation of many small circuits (one persistent launch).
 * ---------------------------------------------------------------------- */
typedef struct qs_batch qs_batch;   /* opaque, owned by the library */

/* Grid and depth of the batched workload's circuit `seed` (this library's
 * reading of "grids uniform over 4x4, 4x5, 3x7, depth uniform over 8..40"):
 * r = SplitMix64 output 0 of (seed ^ 0x6A09E667F3BCC909); grid = r mod 3 in
 * that order, cz_cycles = 8 + (r >> 32) mod 33.  The circuit itself is
 * qs_supremacy_circuit(rows, cols, none removed, cz_cycles, seed). */
int qs_batch_circuit_params(uint64_t seed, int *rows, int *cols, int *cz_cycles);

/* One state per schedule (1..26 qubits, dense and phase ops), all in one
 * device allocation, plus the packed op list.  Each run starts every state at
 * |0...0> and applies its schedule; a cluster of CTAs owns one circuit at a
 * time (ops in order, a cluster barrier between ops), circuits sorted by
 * descending cost.  stream: cudaStream_t (non-NULL for graph replay). */
int qs_batch_create(int n_circuits, const qs_schedule *const *schedules, int dtype, void *stream,
                    qs_batch **out);
void qs_batch_free(qs_batch *b);
/* Launch configuration: CTAs per cluster in {1, 2, 4, 8}, threads in {128, 256, 512}. */
int qs_batch_set_config(qs_batch *b, int cluster_ctas, int threads);
int qs_batch_get_config(const qs_batch *b, int *cluster_ctas, int *threads);
/* One persistent launch of the whole batch on the batch's stream. */
int qs_batch_run(qs_batch *b);
/* The same launch, captured once into a CUDA graph (re-captured when the
 * configuration changes) and replayed. */
int qs_batch_run_graph(qs_batch *b);
/* Per circuit i: out[4i..4i+3] as qs_stats (FP64); synchronises the stream. */
int qs_batch_stats(qs_batch *b, double *out);
/* State i as complex128 in host memory (2^n_i amplitudes). */
int qs_batch_get_amplitudes(qs_batch *b, int i, double *host_c128);
/* Time all launch configurations; keep and report the fastest (ms per launch). */
int qs_batch_tune(qs_batch *b, int *cluster_ctas, int *threads, float *ms);
/* Autotuner of the batched path: for k_max in {3, 4, 5}, schedule every circuit
 * (qs_schedule_build, fused, phase merge), build the batch, tune its launch
 * configuration; report the fastest (k_max, cluster_ctas, threads, ms). */
int qs_batch_autotune(int n_circuits, const int *n_qubits, const qs_gate *const *gates, const int *n_gates,
                      int dtype, void *stream, int *k_max, int *cluster_ctas, int *threads, float *ms);

/* ------------------------------------------------------------------------
 * Cost models and planning (Sec. 3.3: the best cluster size depends on the
 * machine; Sec. 3.6: the scheduler packs gates into clusters of k <= k_max).
 * ---------------------------------------------------------------------- */
#define QS_NFEAT 12
/* Op features, in this order: n/32, dtype (1 = complex128), diagonal (phase)
 * op, k/5, tensor-core path, lowest target/n, highest target/n, targets below
 * bit 5 (/5), targets below bit 3 (/3), log2(state bytes)/40, phase CZ terms/n,
 * phase has odd (T-type) coefficients.  Predictions are times in ms. */
int qs_op_features(int n, int dtype, int kind, int k, const int *qubits, int path, int n_act, int odd,
                   double out[QS_NFEAT]);
/* max(2 bytes(state) / hbm_gbs, flops / peak) + 5 us, peaks FP32 70 TFLOP/s and
 * FP64 1.2 TFLOP/s for CUDA-core sweeps; tensor-core sweeps counted as HBM-bound. */
double qs_cost_analytic_ms(const double features[QS_NFEAT], double hbm_gbs);

/* Timing harness: `count` random ops (85% dense with k uniform in 1..5, targets
 * uniform, kernel path CUDA cores or tensor cores; 15% phase ops), n uniform in
 * [n_min, n_max] (5..33), each run once to upload and once timed with CUDA
 * events on a state the harness allocates; ops whose analytic estimate exceeds
 * max_ms are redrawn.  features: count x QS_NFEAT; ms: count. */
int qs_cost_sample(int n_min, int n_max, int dtype, int count, uint64_t seed, double max_ms, double *features,
                   double *ms);

/* The MLP: QS_NFEAT inputs, two tanh layers of 64, one linear output; FP64
 * parameters W1[F][64], b1[64], W2[64][64], b2[64], w3[64], b3 in one array,
 * trained on the GPU (forward, backward and Adam kernels of this library). */
typedef struct qs_mlp qs_mlp;
int qs_mlp_create(uint64_t seed, qs_mlp **out);       /* Glorot-uniform weights */
void qs_mlp_free(qs_mlp *m);
int qs_mlp_num_params(void);
int qs_mlp_get_params(const qs_mlp *m, double *out);
int qs_mlp_set_params(qs_mlp *m, const double *in);
/* X: B x QS_NFEAT (host), out: B */
int qs_mlp_forward(qs_mlp *m, const double *X, int B, double *out);
/* Gradient of mean (out - Y)^2 with respect to the parameters (host output). */
int qs_mlp_gradient(qs_mlp *m, const double *X, const double *Y, int B, double *grad, double *loss);
/* Full-batch Adam (beta 0.9 / 0.999), `epochs` steps at learning rate lr. */
int qs_mlp_train(qs_mlp *m, const double *X, const double *Y, int B, int epochs, double lr, double *loss);

enum { QS_COST_AUTO = 0, QS_COST_ANALYTIC = 1, QS_COST_MLP = 2 };
typedef struct qs_cost_model qs_cost_model;
int qs_cost_model_create(double hbm_gbs, qs_cost_model **out);   /* analytic until fitted */
void qs_cost_model_free(qs_cost_model *c);
/* Fit the MLP on log-time of the timings (features standardised; every fifth
 * sample by a seeded hash held out).  report: training loss, held-out median
 * |log error| of the MLP and of the analytic model, and whether the MLP will be
 * used (1: it beat the analytic model). */
int qs_cost_model_fit(qs_cost_model *c, const double *features, const double *ms, int count, int epochs,
                      uint64_t seed, double report[4]);
/* Predicted ms.  QS_COST_AUTO: the MLP where it was chosen by the fit and the
 * features lie inside the training range, the analytic model elsewhere. */
int qs_cost_model_predict(const qs_cost_model *c, const double *features, int count, int which, double *ms);
/* Plan a circuit started from |0...0>: for k_max in 2..5 build the schedule
 * with qs_schedule_build's default clustering search, choose each dense op's
 * kernel path (CUDA or tensor cores) by predicted time, and predict the
 * schedule as it is and with the exchanges of qs_schedule_choose_remap (Sec.
 * 3.6 bit-location mapping), keeping the faster; keep the k_max with the
 * smallest predicted total.  Tensor-core sweeps on the support after
 * |0...0> are predicted with the support's size as the state size; a phase
 * op right after a tensor-core sweep counts as folded.  The schedule records
 * the chosen paths and, when chosen, the exchanges (qs_schedule_get_remap).
 * The analytic model sees no difference between the two bit placements (it
 * counts bytes), so only a fitted network moves qubits. */
int qs_plan_circuit(int n, const qs_gate *gates, int n_gates, int dtype, const qs_cost_model *c, int which,
                    qs_schedule **out, int *k_max, double *predicted_ms);

#ifdef __cplusplus
}
#endif

#endif /* QS_H */

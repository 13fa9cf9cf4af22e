// Internal declarations shared by the translation units of libqs.
#pragma once

#include <cstdint>
#include <cstddef>
#include <array>
#include <vector>
#include <utility>
#include <new>
#include <exception>

#include "../../include/qs.h"

// Thread-local error message; returns `code` so callers can `return qs_fail(...)`.
int qs_fail(int code, const char *fmt, ...);

// Every C entry point runs its body through qs_guard, so that no C++ exception
// crosses the C boundary: a failed host allocation becomes QS_ENOMEM, any other
// exception QS_EINVAL with its message.
template <class F>
int qs_guard(F &&body) noexcept
{
    try {
        return body();
    } catch (const std::bad_alloc &) {
        return qs_fail(QS_ENOMEM, "host memory allocation failed");
    } catch (const std::exception &e) {
        return qs_fail(QS_EINVAL, "%s", e.what());
    } catch (...) {
        return qs_fail(QS_EINVAL, "unexpected exception");
    }
}

struct qs_state {
    int n = 0;
    int dtype = QS_C128;
    void *amp = nullptr;          // device, 2^n amplitudes
    bool owned = false;
    void *stream = nullptr;       // cudaStream_t
    int device = 0;
    // scratch, grown on demand and freed with the state
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    void *pinned = nullptr;       // small pinned host buffer for results
    size_t pinned_bytes = 0;
    int *status = nullptr;        // device word set by kernels whose bounded waits ran out
    void *side = nullptr;         // cudaStream_t: a second stream for work that overlaps the main one
    void *side_ev[2] = {nullptr, nullptr};   // cudaEvent_t: fork and join of that stream
    int path = 0;                 // QS_PATH_*
    bool fold_phase = true;       // qs_set_phase_fold
    bool pair_sweeps = false;     // qs_set_pair_sweeps
    // every amplitude equal (qs_init_uniform, nothing applied since): any
    // exchange of qubits leaves the state as it is
    bool perm_invariant = false;
    // Support: amplitudes may be nonzero only at indices i with
    // (i & ~sup_free) == sup_fix.  After qs_init_basis the support is one index
    // and memory outside the support is left unwritten; the tensor-core sweeps
    // work on the support only (their result is the same as on the
    // zero-filled state), and every other call first writes the zeros
    // (qs_materialize).  Full support: sup_free = ~0.
    uint64_t sup_free = ~0ULL;
    uint64_t sup_fix = 0;
    // Bit location of each qubit (the remapping of Sec. 3.6): index bit loc[q]
    // holds qubit q.  Always a set of disjoint exchanges (loc[loc[q]] == q);
    // the identity until a remapped schedule runs.  Calls that name qubits or
    // indices translate them; calls whose result depends on the index order
    // restore the identity first (one exchange sweep).
    int loc[64] = {0,  1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21,
                   22, 23, 24, 25, 26, 27, 28, 29, 30, 31, 32, 33, 34, 35, 36, 37, 38, 39, 40, 41, 42, 43,
                   44, 45, 46, 47, 48, 49, 50, 51, 52, 53, 54, 55, 56, 57, 58, 59, 60, 61, 62, 63};
};

inline void qs_loc_reset(qs_state *s)
{
    for (int q = 0; q < 64; q++) s->loc[q] = q;
}
// qubit q -> its index bit in state s
inline int qs_loc(const qs_state *s, int q) { return s->loc[q]; }
inline bool qs_loc_identity(const qs_state *s)
{
    for (int q = 0; q < s->n; q++)
        if (s->loc[q] != q) return false;
    return true;
}
// index in qubit order -> index in the state's bit order (and back: the same
// map, the locations being exchanges)
inline uint64_t qs_loc_index(const qs_state *s, uint64_t x)
{
    uint64_t r = 0;
    for (int q = 0; q < s->n; q++) r |= ((x >> q) & 1ULL) << s->loc[q];
    return r;
}
// Bring the qubits to the locations `want` (n entries, exchanges) or, for
// nullptr, to the identity: a relabelling when the state is the lazily
// written basis state, else exchange sweeps.
int qs_order_set(qs_state *s, const int *want);
// After qs_init_basis: move the one amplitude of the support to index x
// (nothing else written).
int qs_basis_move(qs_state *s, uint64_t x);

inline uint64_t qs_index_mask(int n) { return n >= 64 ? ~0ULL : ((1ULL << n) - 1); }
inline bool qs_support_full(const qs_state *s)
{
    const uint64_t a = qs_index_mask(s->n);
    return (s->sup_free & a) == a;
}
// Write zeros outside the support and make it full (no-op when full).
int qs_materialize(qs_state *s);

// One op of a schedule, host side.
struct qs_op_host {
    int kind = QS_OP_DENSE;
    int k = 0;
    int qubits[QS_MAX_DIAG_K] = {0};
    std::vector<int32_t> gates;          // circuit gate indices, in multiplication order
    std::vector<double> matrix;          // dense: 2^{2k} complex interleaved; diag: 2^k
    std::vector<int32_t> coeff;          // phase: n values mod 8
    std::vector<std::pair<int, int>> edges;   // phase: CZ pairs
    int path = 0;                        // dense: QS_PATH_* chosen by a planner (0: default policy)
};

// Device copy of a schedule's op data for one amplitude type.
struct qs_dev_sched {
    int device = -1;
    void *pool = nullptr;                // device
    size_t bytes = 0;
    std::vector<size_t> offset;          // byte offset of op i's data in pool
    std::vector<int> n_act;              // phase ops: number of CZ partner terms
    std::vector<size_t> tc_off;          // dense ops: offset of the tensor-core pack in op data (0: none)
    std::vector<std::array<int, 5>> tc_q;  // dense ops: the 5 qubits the tensor-core sweep uses
    // dense ops followed by a phase op that folds into their tensor-core sweep:
    // offsets in op data of the pack of the folded matrix and of its
    // qs_post_phase (0: no fold)
    std::vector<size_t> fold_off, post_off;
};

struct qs_schedule {
    int n = 0;
    std::vector<qs_op_host> ops;
    // qs_schedule_remap: the ops name index bits, qubit q at bit remap[q]
    // (exchanges); empty when the ops name the qubits themselves
    std::vector<int> remap;
    qs_dev_sched dev[2];                 // indexed by dtype
};

// Device layout of a phase op (see qs_apply.cu).
struct qs_phase_dev {
    uint64_t cmask[3];     // bit q of cmask[b] = bit b of coeff[q]
    int32_t n_act;         // qubits a with a non-empty partner mask
    int32_t pad;
    // followed by n_act entries of { uint64 partners; int32 a; int32 pad }
};
struct qs_phase_term {
    uint64_t partners;
    int32_t a;
    int32_t pad;
};

// A phase op folded into the tensor-core sweep of the dense op before it
// (device layout, in the schedule's op data).  For an index x = b + m spread
// over the sweep's five qubits (b: the group's base, those bits zero; m: the
// member, bit j on qubit j of the sweep), the phase factor not carried by the
// folded matrix is i^e(b) (-1)^popc(m & flip(b)) with
//   e(b) = popc(b & c1) + 2 popc(b & c2) + 2 sum_terms b_a popc(b & partners_a)  (mod 4)
//   bit j of flip(b) = popc(b & tp[j]) mod 2
// c1, c2: qubits off the sweep whose coefficient (mod 8) has bit 1 / bit 2 set
// (bit 0 is clear there, else there is no fold); tp[j]: CZ partners of the
// sweep's qubit j off the sweep; terms: CZ pairs with both ends off the sweep
// (qs_phase_term, partners above a, pairs counted mod 2).
struct qs_post_phase {
    uint64_t c1, c2;
    uint64_t tp[5];
    int32_t n_terms;
    int32_t pad;
    // followed by n_terms qs_phase_term
};
constexpr int QS_MAX_POST_TERMS = 64;

// Launchers (qs_apply.cu).  All validate nothing: callers check arguments.
// dev_tc: tensor-core operand pack of a 5-qubit cluster (qs_tc.cu) or null.
int qs_launch_dense(qs_state *s, const int *sorted_qubits, int k, const void *dev_matrix,
                    const void *dev_tc);
int qs_launch_diag(qs_state *s, const int *qubits, int k, const void *dev_table);
int qs_launch_phase(qs_state *s, const void *dev_phase, int n_act);
// Schedules of the clustering search's best `top` distinct runs (qs_schedule_build's
// ranking: lowest analytic cost, then fewer clusters), best first; the first is
// the schedule qs_schedule_build returns.  The caller frees them.
int qs_schedule_build_ranked(int n, const qs_gate *gates, int n_gates, const qs_sched_opts *opts, int top,
                             std::vector<qs_schedule *> &out);
// Exchange qubits a[j] <-> b[j] (j < m, validated by the caller) in one sweep.
int qs_launch_swap(qs_state *s, const int *a, const int *b, int m);
uint64_t qs_swap_index(uint64_t i, const int *a, const int *b, int m);

// Default kernel-path policy for a dense cluster (qs_apply.cu).
bool qs_tc_wanted(int dtype, int k, int n);

// Pack a phase op into its device layout (qs_circuit.cpp).
std::vector<uint8_t> qs_pack_phase(int n, const std::vector<int32_t> &coeff,
                                   const std::vector<std::pair<int, int>> &edges, int *n_act);

// Device scratch of at least `bytes` on the state (qs_api.cu).
int qs_state_scratch(qs_state *s, size_t bytes, void **out);
// Device status word of the state (allocated and zeroed on first use), and a
// check that returns QS_ETIMEOUT (and clears the word) if a kernel set it.
int qs_state_status(qs_state *s, int **out);
int qs_check_status(qs_state *s);

// Tensor-core 5-qubit sweep (qs_tc.cu).
std::vector<uint8_t> qs_pack_tc_c64(const std::vector<double> &sorted_matrix);
std::vector<uint8_t> qs_pack_tc_c128(const std::vector<double> &sorted_matrix);
size_t qs_tc_pack_bytes(int dtype);
// 5-qubit tensor-core sweep over the state's support; grow = the qubits that
// join the support (the cluster's own targets; an embedded cluster's padding
// qubits stay fixed).
// dev_post: a folded phase op (qs_post_phase, device) or null.
int qs_launch_dense5_tc(qs_state *s, const int *sorted_qubits, const void *dev_pack, uint64_t grow,
                        const void *dev_post = nullptr);
// Two consecutive 5-qubit clusters (sorted qubits q1, q2; complex64 tensor-core
// packs) in one sweep: complex64, full support, n >= 12, |q1 u q2| <= 10.
bool qs_pair_possible(const qs_state *s, const int *q1, const int *q2);
int qs_launch_pair5_tc(qs_state *s, const int *q1, const void *pack1, const int *q2, const void *pack2,
                       const void *dev_post = nullptr);
// One bounded mbarrier wait that cannot complete (qs_selftest_timeout).
int qs_launch_wait_selftest(qs_state *s, long polls);

// Host side of the hot path: supremacy-circuit generation (Fig. 1 caption),
// greedy gate clustering (Sec. 3.6, step 2), FP64 cluster unitaries in sorted
// qubit order (Sec. 3.2) and diagonal phase ops (Sec. 3.5).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <deque>
#include <limits>
#include <memory>
#include <new>
#include <set>
#include <thread>
#include <vector>

#include "qs_internal.h"

namespace {

// ----------------------------------------------------------------- gates (Sec. 2)
// 2x2 matrices, row-major (re, im) pairs.
constexpr double kR = 0.70710678118654752440;   // 1/sqrt(2), correctly rounded

void gate_matrix(int kind, double m[8])
{
    static const double H[8] = {kR, 0, kR, 0, kR, 0, -kR, 0};
    static const double T[8] = {1, 0, 0, 0, 0, 0, kR, kR};          // diag(1, e^{i pi/4})
    static const double TD[8] = {1, 0, 0, 0, 0, 0, kR, -kR};
    static const double SX[8] = {0.5, 0.5, 0.5, -0.5, 0.5, -0.5, 0.5, 0.5};
    static const double SY[8] = {0.5, 0.5, -0.5, -0.5, 0.5, 0.5, 0.5, 0.5};
    static const double X[8] = {0, 0, 1, 0, 1, 0, 0, 0};
    const double *src = H;
    switch (kind) {
    case QS_GATE_H: src = H; break;
    case QS_GATE_T: src = T; break;
    case QS_GATE_TDG: src = TD; break;
    case QS_GATE_SQRT_X: src = SX; break;
    case QS_GATE_SQRT_Y: src = SY; break;
    case QS_GATE_X: src = X; break;
    case QS_GATE_SQRT_XDG:    // adjoint: transpose and conjugate
    case QS_GATE_SQRT_YDG: {
        const double *b = kind == QS_GATE_SQRT_XDG ? SX : SY;
        const int tr[4] = {0, 2, 1, 3};
        for (int e = 0; e < 4; e++) { m[2 * e] = b[2 * tr[e]]; m[2 * e + 1] = -b[2 * tr[e] + 1]; }
        return;
    }
    default: break;
    }
    std::memcpy(m, src, sizeof(double) * 8);
}

bool is_diagonal(int kind) { return kind == QS_GATE_T || kind == QS_GATE_TDG || kind == QS_GATE_CZ; }

// ------------------------------------------------------- SplitMix64 (Steele et al.)
uint64_t splitmix64(uint64_t seed, uint64_t j)
{
    uint64_t z = seed + (j + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// -------------------------------------------------------------- clustering helpers
struct Clusterer {
    int n;
    const std::vector<qs_gate> &g;
    std::vector<std::vector<int>> queue;   // per qubit, gate indices in order
    std::vector<uint64_t> gmask;

    Clusterer(int n_, const std::vector<qs_gate> &gates) : n(n_), g(gates), queue(n_)
    {
        gmask.resize(g.size());
        for (size_t i = 0; i < g.size(); i++) {
            gmask[i] = 1ULL << g[i].q0;
            queue[g[i].q0].push_back((int)i);
            if (g[i].q1 >= 0) {
                gmask[i] |= 1ULL << g[i].q1;
                queue[g[i].q1].push_back((int)i);
            }
        }
    }

    bool ready(const std::vector<int> &pos, int gi) const
    {
        uint64_t m = gmask[gi];
        while (m) {
            int q = __builtin_ctzll(m);
            m &= m - 1;
            if (pos[q] >= (int)queue[q].size() || queue[q][pos[q]] != gi) return false;
        }
        return true;
    }

    void advance(std::vector<int> &pos, int gi) const
    {
        uint64_t m = gmask[gi];
        while (m) {
            int q = __builtin_ctzll(m);
            m &= m - 1;
            pos[q]++;
        }
    }

    std::vector<int> heads(const std::vector<int> &pos) const
    {
        std::vector<int> h;
        for (int q = 0; q < n; q++)
            if (pos[q] < (int)queue[q].size()) h.push_back(queue[q][pos[q]]);
        std::sort(h.begin(), h.end());
        h.erase(std::unique(h.begin(), h.end()), h.end());
        return h;
    }

    // Gates runnable on qubit set S: ascending-qubit sweeps taking ready heads
    // that act only inside S, repeated until a sweep takes nothing.
    void closure(uint64_t S, const std::vector<int> &pos0, std::vector<int> &members,
                 std::vector<int> &pos) const
    {
        pos = pos0;
        members.clear();
        bool changed = true;
        while (changed) {
            changed = false;
            for (int q = 0; q < n; q++) {
                if (!((S >> q) & 1)) continue;
                while (pos[q] < (int)queue[q].size()) {
                    int gi = queue[q][pos[q]];
                    if ((gmask[gi] & ~S) || !ready(pos, gi)) break;
                    members.push_back(gi);
                    advance(pos, gi);
                    changed = true;
                }
            }
        }
    }

    void grow(const std::vector<int> &pos, int seed, int k_max, std::vector<int> &members,
              uint64_t &S) const
    {
        S = gmask[seed];
        std::vector<int> after;
        closure(S, pos, members, after);
        std::vector<int> m2, a2, best_m, best_a;
        for (;;) {
            bool have = false;
            int best_len = 0, best_bits = 0, best_g = 0;
            uint64_t best_S = 0;
            for (int gi : heads(after)) {
                uint64_t qs = gmask[gi];
                if (!(qs & ~S)) continue;
                uint64_t S2 = S | qs;
                int bits = __builtin_popcountll(S2);
                if (bits > k_max) continue;
                closure(S2, pos, m2, a2);
                int len = (int)m2.size();
                // key (len, -bits, -g), larger wins
                bool better = !have || len > best_len ||
                              (len == best_len && (bits < best_bits ||
                                                   (bits == best_bits && gi < best_g)));
                if (better) {
                    have = true;
                    best_len = len; best_bits = bits; best_g = gi; best_S = S2;
                    best_m = m2; best_a = a2;
                }
            }
            if (!have || best_len <= (int)members.size()) break;
            S = best_S;
            members = best_m;
            after = best_a;
        }
    }

    std::vector<std::vector<int>> run(int k_max) const
    {
        std::vector<int> pos(n, 0);
        size_t remaining = g.size();
        std::vector<std::vector<int>> out;
        std::vector<int> members;
        while (remaining) {
            bool have = false;
            std::vector<int> best;
            int best_len = 0, best_bits = 0, best_s = 0;
            for (int s : heads(pos)) {
                if (!ready(pos, s)) continue;
                uint64_t S;
                grow(pos, s, k_max, members, S);
                int len = (int)members.size(), bits = __builtin_popcountll(S);
                bool better = !have || len > best_len ||
                              (len == best_len && (bits < best_bits ||
                                                   (bits == best_bits && s < best_s)));
                if (better) {
                    have = true;
                    best = members; best_len = len; best_bits = bits; best_s = s;
                }
            }
            for (int gi : best) advance(pos, gi);
            remaining -= best.size();
            out.push_back(best);
        }
        return out;
    }
};

// U <- G U for a 1-qubit gate on position j of a 2^k space (columns of U are
// updated pairwise, Sec. 2 Kronecker rule restricted to the cluster's qubits).
void left_apply_1q(std::vector<double> &U, int k, int j, const double m[8])
{
    const int d = 1 << k;
    for (int r0 = 0; r0 < d; r0++) {
        if ((r0 >> j) & 1) continue;
        int r1 = r0 | (1 << j);
        for (int c = 0; c < d; c++) {
            double ar = U[2 * (r0 * d + c)], ai = U[2 * (r0 * d + c) + 1];
            double br = U[2 * (r1 * d + c)], bi = U[2 * (r1 * d + c) + 1];
            U[2 * (r0 * d + c)] = (m[0] * ar - m[1] * ai) + (m[2] * br - m[3] * bi);
            U[2 * (r0 * d + c) + 1] = (m[0] * ai + m[1] * ar) + (m[2] * bi + m[3] * br);
            U[2 * (r1 * d + c)] = (m[4] * ar - m[5] * ai) + (m[6] * br - m[7] * bi);
            U[2 * (r1 * d + c) + 1] = (m[4] * ai + m[5] * ar) + (m[6] * bi + m[7] * br);
        }
    }
}

void left_apply_cz(std::vector<double> &U, int k, int ja, int jb)
{
    const int d = 1 << k;
    for (int r = 0; r < d; r++) {
        if (((r >> ja) & 1) && ((r >> jb) & 1)) {
            for (int c = 0; c < 2 * d; c++) U[2 * r * d + c] = -U[2 * r * d + c];
        }
    }
}

bool check_gate(int n, const qs_gate &g)
{
    if (g.kind < QS_GATE_H || g.kind > QS_GATE_SQRT_YDG) return false;
    if (g.q0 < 0 || g.q0 >= n) return false;
    if (g.kind == QS_GATE_CZ) return g.q1 >= 0 && g.q1 < n && g.q1 != g.q0;
    return g.q1 < 0;
}

void make_phase(int n, const std::vector<qs_gate> &g, const std::vector<int> &members,
                qs_op_host &op)
{
    op.kind = QS_OP_PHASE;
    op.gates.assign(members.begin(), members.end());
    op.coeff.assign(n, 0);
    op.edges.clear();
    uint64_t support = 0;
    for (int gi : members) {
        const qs_gate &x = g[gi];
        support |= 1ULL << x.q0;
        if (x.kind == QS_GATE_CZ) {
            support |= 1ULL << x.q1;
            op.edges.push_back({x.q0, x.q1});
        } else {
            op.coeff[x.q0] = (op.coeff[x.q0] + (x.kind == QS_GATE_T ? 1 : 7)) & 7;
        }
    }
    op.k = __builtin_popcountll(support);
    int j = 0;
    for (int q = 0; q < n && j < QS_MAX_K; q++)
        if ((support >> q) & 1) op.qubits[j++] = q;
}

uint64_t gmask_of(const qs_gate &x) { return (1ULL << x.q0) | (x.q1 >= 0 ? 1ULL << x.q1 : 0ULL); }

constexpr int kMaxSearchRuns = 64;
constexpr int kMaxSearchFirst = 16;
constexpr int kMaxSearchSlack0 = 64;
constexpr int kMaxSearchThreads = 32;
std::atomic<int> g_host_threads{0};   // qs_set_host_threads: 0 = every hardware thread

// Closures by qubit set: open addressing with linear probing over the 64-bit
// masks (a set is never empty, so 0 marks a free slot, and never holds all 64
// qubits, so ~0 marks a dropped one); the member lists live in a deque, so a
// reference stays valid while the table grows.  drop() marks the sets that
// meet a mask as dropped; the table is rebuilt when few free slots are left.
struct ClosureMemo {
    static constexpr uint64_t kDropped = ~0ULL;
    std::vector<uint64_t> key = std::vector<uint64_t>(1024, 0);
    std::vector<int> slot = std::vector<int>(1024, 0);
    std::deque<std::vector<int>> vals;
    std::vector<int> free_vals;
    size_t used = 0, dropped = 0;
    int shift = 64 - 10;

    size_t home(uint64_t k) const { return (size_t)((k * 0x9E3779B97F4A7C15ULL) >> shift); }

    const std::vector<int> *find(uint64_t k) const
    {
        const size_t mask = key.size() - 1;
        for (size_t i = home(k);; i = (i + 1) & mask) {
            if (key[i] == k) return &vals[slot[i]];
            if (key[i] == 0) return nullptr;
        }
    }

    void place(uint64_t k, int vi)
    {
        const size_t mask = key.size() - 1;
        size_t i = home(k);
        while (key[i] != 0 && key[i] != kDropped) i = (i + 1) & mask;
        if (key[i] == kDropped) dropped--;
        key[i] = k;
        slot[i] = vi;
    }

    // k is not in the table
    const std::vector<int> &insert(uint64_t k, std::vector<int> &&v)
    {
        if (2 * (used + dropped + 1) > key.size()) rehash(4 * (used + 1) > key.size() ? 2 * key.size() : key.size());
        int vi;
        if (!free_vals.empty()) {
            vi = free_vals.back();
            free_vals.pop_back();
            vals[vi] = std::move(v);
        } else {
            vi = (int)vals.size();
            vals.push_back(std::move(v));
        }
        place(k, vi);
        used++;
        return vals[vi];
    }

    void drop(uint64_t hit)
    {
        for (size_t i = 0; i < key.size(); i++) {
            if (key[i] == 0 || key[i] == kDropped || !(key[i] & hit)) continue;
            key[i] = kDropped;
            free_vals.push_back(slot[i]);
            used--;
            dropped++;
        }
    }

    void rehash(size_t cap)
    {
        std::vector<uint64_t> old_key(cap, 0);
        std::vector<int> old_slot(cap, 0);
        old_key.swap(key);
        old_slot.swap(slot);
        shift = 64 - __builtin_ctzll(cap);
        dropped = 0;
        for (size_t i = 0; i < old_key.size(); i++)
            if (old_key[i] != 0 && old_key[i] != kDropped) place(old_key[i], old_slot[i]);
    }
};

// The same greedy closure rule with diagonal gates free to pass one another:
// on a qubit, a gate may run before earlier unassigned gates of that qubit
// when it and all of them are diagonal (diagonal matrices commute, so the
// product is unchanged); a non-diagonal gate keeps its place.
//   available(g, q): every unassigned gate before g on q is diagonal, and so
//                    is g (or none precedes it);
//   ready(g):        available on each of its qubits;
//   closure(S):      sweeps over the qubits of S, ascending; on each, the
//                    unassigned gates in order: take a gate that acts only on
//                    S and is ready, pass over a diagonal gate that is not
//                    taken, stop at a non-diagonal one; repeat until a sweep
//                    takes nothing;
//   candidates:      per qubit, its first unassigned gate, if ready;
//   seeds, growth and ties as in Clusterer.
struct DiagClusterer {
    int n;
    const std::vector<qs_gate> &g;
    std::vector<std::vector<int>> queue;   // per qubit, gate indices in order
    std::vector<uint64_t> gmask;
    std::vector<char> diag, done;
    std::vector<int> first;                // per qubit: first gate of queue not done
    mutable std::vector<int> mark;         // gates taken by the closure being built
    mutable int stamp = 0;
    // closures by qubit set; a step drops those that read a queue it changed
    mutable ClosureMemo memo;
    mutable std::vector<int> cand;         // the last result of candidates()

    DiagClusterer(int n_, const std::vector<qs_gate> &gates)
        : n(n_), g(gates), queue(n_), gmask(gates.size()), diag(gates.size()), done(gates.size(), 0),
          first(n_, 0), mark(gates.size(), 0)
    {
        for (size_t i = 0; i < g.size(); i++) {
            gmask[i] = 1ULL << g[i].q0;
            queue[g[i].q0].push_back((int)i);
            if (g[i].q1 >= 0) {
                gmask[i] |= 1ULL << g[i].q1;
                queue[g[i].q1].push_back((int)i);
            }
            diag[i] = is_diagonal(g[i].kind);
        }
    }

    bool taken(int gi) const { return done[gi] || mark[gi] == stamp; }

    bool available(int q, int gi) const
    {
        for (size_t i = first[q]; i < queue[q].size(); i++) {
            const int h = queue[q][i];
            if (h == gi) return true;
            if (taken(h)) continue;
            if (!(diag[h] && diag[gi])) return false;
        }
        return false;
    }

    // the closure of S, held in the memo (the reference lasts until the step
    // drops entries)
    const std::vector<int> &closure(uint64_t S) const
    {
        if (const std::vector<int> *hit = memo.find(S)) return *hit;
        ++stamp;
        std::vector<int> members;
        members.reserve(32);
        bool changed = true;
        while (changed) {
            changed = false;
            for (uint64_t m = S; m; m &= m - 1) {
                const int q = __builtin_ctzll(m);
                // the scan stops at the first untaken non-diagonal gate, so
                // every untaken gate it has passed on q is diagonal: gi is
                // available on q when it is diagonal or none was passed, and
                // ready when also available on its other qubit
                bool passed = false;
                for (size_t i = first[q]; i < queue[q].size(); i++) {
                    const int gi = queue[q][i];
                    if (taken(gi)) continue;
                    if (gmask[gi] & ~S) {
                        if (!diag[gi]) break;
                        passed = true;
                        continue;
                    }
                    bool ok = !passed || diag[gi];
                    const uint64_t other = gmask[gi] & ~(1ULL << q);
                    if (ok && other) ok = available(__builtin_ctzll(other), gi);
                    if (ok) {
                        mark[gi] = stamp;
                        members.push_back(gi);
                        changed = true;
                    } else if (!diag[gi]) {
                        break;
                    } else {
                        passed = true;
                    }
                }
            }
        }
        return memo.insert(S, std::move(members));
    }

    // per qubit, its first gate not done and not in `members`, if ready (in
    // a buffer that the next call overwrites)
    const std::vector<int> &candidates(const std::vector<int> &members) const
    {
        ++stamp;
        for (int gi : members) mark[gi] = stamp;
        std::vector<int> &c = cand;
        c.clear();
        for (int q = 0; q < n; q++)
            for (size_t i = first[q]; i < queue[q].size(); i++) {
                const int gi = queue[q][i];
                if (taken(gi)) continue;
                // first untaken gate on q: available there; ready when also
                // available on its other qubit
                const uint64_t other = gmask[gi] & ~(1ULL << q);
                if (!other || available(__builtin_ctzll(other), gi)) c.push_back(gi);
                break;
            }
        std::sort(c.begin(), c.end());
        c.erase(std::unique(c.begin(), c.end()), c.end());
        return c;
    }

    void grow(int seed, int k_max, std::vector<int> &members, uint64_t &S) const
    {
        S = gmask[seed];
        const std::vector<int> *cur = &closure(S);
        for (;;) {
            const std::vector<int> *best_m = nullptr;
            int best_len = 0, best_bits = 0, best_g = 0;
            uint64_t best_S = 0;
            for (int gi : candidates(*cur)) {
                const uint64_t qs = gmask[gi];
                if (!(qs & ~S)) continue;
                const uint64_t S2 = S | qs;
                const int bits = __builtin_popcountll(S2);
                if (bits > k_max) continue;
                const std::vector<int> &m2 = closure(S2);
                const int len = (int)m2.size();
                const bool better = !best_m || len > best_len ||
                                    (len == best_len && (bits < best_bits || (bits == best_bits && gi < best_g)));
                if (better) {
                    best_len = len; best_bits = bits; best_g = gi; best_S = S2;
                    best_m = &m2;
                }
            }
            if (!best_m || best_len <= (int)cur->size()) break;
            S = best_S;
            cur = best_m;
        }
        members = *cur;
    }

    // The clusters grown from all seeds, ranked as the greedy rule ranks them
    // (more gates, then fewer qubits, then the lower seed), and one of them
    // taken: with slack < 0 the first; else, while the dense clusters taken so
    // far do not cover every qubit, the one within `slack` gates of the
    // largest that adds the fewest qubits to them (an all-diagonal one adds
    // none), then the first in rank; once they do, the first.  With
    // first_pick > 0 the first cluster of the run is instead the one of that
    // rank (the last one when there are fewer).
    std::vector<std::vector<int>> run(int k_max, int slack = -1, int first_pick = 0)
    {
        struct Opt {
            int len, bits, seed;
            uint64_t S;
            std::vector<int> members;
        };
        const uint64_t all = n >= 64 ? ~0ULL : ((1ULL << n) - 1);
        uint64_t sup = 0;
        size_t remaining = g.size();
        std::vector<std::vector<int>> out;
        std::vector<int> members;
        while (remaining) {
            std::vector<Opt> opts;
            const std::vector<int> seeds = candidates({});
            for (int sd : seeds) {
                uint64_t S;
                grow(sd, k_max, members, S);
                opts.push_back({(int)members.size(), __builtin_popcountll(S), sd, S, members});
            }
            std::sort(opts.begin(), opts.end(), [](const Opt &a, const Opt &b) {
                if (a.len != b.len) return a.len > b.len;
                if (a.bits != b.bits) return a.bits < b.bits;
                return a.seed < b.seed;
            });
            auto dense_opt = [&](const Opt &o) {
                for (int gi : o.members)
                    if (!diag[gi]) return true;
                return false;
            };
            size_t pick = 0;
            if (out.empty() && first_pick > 0) {
                pick = std::min((size_t)first_pick, opts.size() - 1);
            } else if (slack >= 0 && sup != all) {
                int best_new = 1 << 30;
                for (size_t i = 0; i < opts.size() && opts[i].len >= opts[0].len - slack; i++) {
                    const int added = dense_opt(opts[i]) ? __builtin_popcountll(opts[i].S & ~sup) : 0;
                    if (added < best_new) {
                        best_new = added;
                        pick = i;
                    }
                }
            }
            if (dense_opt(opts[pick])) sup |= opts[pick].S;
            const std::vector<int> &best = opts[pick].members;
            for (int gi : best) done[gi] = 1;
            // a closure on S reads only the queues of S's qubits: those that
            // miss the qubits of the cluster taken stay as they are
            memo.drop(opts[pick].S);
            for (int q = 0; q < n; q++)
                while (first[q] < (int)queue[q].size() && done[queue[q][first[q]]]) first[q]++;
            remaining -= best.size();
            out.push_back(best);
        }
        return out;
    }
};

void make_dense(const std::vector<qs_gate> &g, const std::vector<int> &members, qs_op_host &op)
{
    op.kind = QS_OP_DENSE;
    op.gates.assign(members.begin(), members.end());
    uint64_t support = 0;
    for (int gi : members) {
        support |= 1ULL << g[gi].q0;
        if (g[gi].q1 >= 0) support |= 1ULL << g[gi].q1;
    }
    int k = 0, where[64];
    for (int q = 0; q < 64; q++)
        if ((support >> q) & 1) { where[q] = k; op.qubits[k++] = q; }
    op.k = k;
    const int d = 1 << k;
    op.matrix.assign(2 * d * d, 0.0);
    for (int r = 0; r < d; r++) op.matrix[2 * (r * d + r)] = 1.0;
    for (int gi : members) {
        const qs_gate &x = g[gi];
        if (x.kind == QS_GATE_CZ) {
            left_apply_cz(op.matrix, k, where[x.q0], where[x.q1]);
        } else {
            double m[8];
            gate_matrix(x.kind, m);
            left_apply_1q(op.matrix, k, where[x.q0], m);
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ public API

static int supremacy_circuit_impl(int rows, int cols, const int *removed_rc, int n_removed, int cz_cycles,
                                  uint64_t seed, int *n_qubits, qs_gate *gates, int max_gates, int *n_gates)
{
    if (rows < 1 || cols < 1 || rows * cols > 4096 || cz_cycles < 0 || n_removed < 0 ||
        (n_removed > 0 && !removed_rc) || !n_qubits || !n_gates || max_gates < 0 ||
        (max_gates > 0 && !gates))
        return qs_fail(QS_EINVAL, "qs_supremacy_circuit: bad arguments");
    std::vector<int> id(rows * cols, 0);
    for (int i = 0; i < n_removed; i++) {
        int r = removed_rc[2 * i], c = removed_rc[2 * i + 1];
        if (r < 0 || r >= rows || c < 0 || c >= cols)
            return qs_fail(QS_EINVAL, "qs_supremacy_circuit: removed site out of the grid");
        id[r * cols + c] = -1;
    }
    int n = 0;
    for (int i = 0; i < rows * cols; i++)
        if (id[i] == 0) id[i] = n++; else id[i] = -1;
    if (n > QS_MAX_QUBITS || n < 1)
        return qs_fail(QS_EINVAL, "qs_supremacy_circuit: %d qubits out of range", n);
    *n_qubits = n;
    std::vector<qs_gate> out;
    for (int q = 0; q < n; q++) out.push_back({0, QS_GATE_H, q, -1});
    // layouts: {horizontal?, a, b}
    static const int L[8][3] = {{1, 1, 0}, {0, 0, 0}, {1, 0, 0}, {0, 1, 0},
                                {0, 0, 1}, {1, 1, 1}, {0, 1, 1}, {1, 0, 1}};
    std::vector<int> last(n, -1);          // previous single-qubit gate kind
    std::vector<char> prev_cz(n, 0), in_cz(n, 0);
    uint64_t draw = 0;
    for (int t = 1; t <= cz_cycles; t++) {
        const int *lay = L[(t - 1) % 8];
        std::vector<std::pair<int, int>> edges;
        for (int r = 0; r < rows; r++)
            for (int c = 0; c < cols; c++) {
                int a = id[r * cols + c];
                if (a < 0) continue;
                int r2 = r, c2 = c;
                if (lay[0]) { if (c % 2 != lay[1] || r % 2 != lay[2]) continue; c2 = c + 1; }
                else { if (r % 2 != lay[1] || c % 2 != lay[2]) continue; r2 = r + 1; }
                if (r2 >= rows || c2 >= cols) continue;
                int b = id[r2 * cols + c2];
                if (b < 0) continue;
                edges.push_back({std::min(a, b), std::max(a, b)});
            }
        std::sort(edges.begin(), edges.end());
        std::fill(in_cz.begin(), in_cz.end(), 0);
        for (auto &e : edges) in_cz[e.first] = in_cz[e.second] = 1;
        for (int q = 0; q < n; q++) {
            if (!prev_cz[q] || in_cz[q]) continue;
            int kind;
            if (last[q] < 0) {
                kind = QS_GATE_T;
            } else {
                int allowed[2], na = 0;
                const int order[3] = {QS_GATE_T, QS_GATE_SQRT_X, QS_GATE_SQRT_Y};
                for (int o = 0; o < 3; o++)
                    if (order[o] != last[q]) allowed[na++] = order[o];
                kind = allowed[splitmix64(seed, draw++) >> 63];
            }
            out.push_back({t, kind, q, -1});
            last[q] = kind;
        }
        for (auto &e : edges) out.push_back({t, QS_GATE_CZ, e.first, e.second});
        prev_cz = in_cz;
    }
    *n_gates = (int)out.size();
    if ((int)out.size() > max_gates)
        return qs_fail(QS_EINVAL, "qs_supremacy_circuit: need room for %d gates", (int)out.size());
    std::memcpy(gates, out.data(), sizeof(qs_gate) * out.size());
    return QS_OK;
}

static int schedule_from_groups(int n, const std::vector<qs_gate> &g, const std::vector<std::vector<int>> &groups,
                                const qs_sched_opts *opts, qs_schedule **out);

// ranked (nullable): also the best ranked_max distinct clusterings of the
// search, best first
static int schedule_build_impl(int n, const qs_gate *gates, int n_gates, const qs_sched_opts *opts,
                               qs_schedule **out, std::vector<std::vector<std::vector<int>>> *ranked = nullptr,
                               int ranked_max = 0)
{
    if (!out || n < 1 || n > QS_MAX_QUBITS || n_gates < 0 || (n_gates > 0 && !gates) || !opts)
        return qs_fail(QS_EINVAL, "qs_schedule_build: bad arguments");
    if (opts->fuse && (opts->k_max < 2 || opts->k_max > QS_MAX_K))
        return qs_fail(QS_EINVAL, "qs_schedule_build: k_max %d not in [2, %d]", opts->k_max, QS_MAX_K);
    if (opts->search_runs < 0 || opts->search_runs > kMaxSearchRuns)
        return qs_fail(QS_EINVAL, "qs_schedule_build: search_runs %d not in [0, %d]", opts->search_runs,
                       kMaxSearchRuns);
    if (opts->search_first < 0 || opts->search_first > kMaxSearchFirst)
        return qs_fail(QS_EINVAL, "qs_schedule_build: search_first %d not in [0, %d]", opts->search_first,
                       kMaxSearchFirst);
    if (opts->search_slack0 < 0 || opts->search_slack0 > kMaxSearchSlack0)
        return qs_fail(QS_EINVAL, "qs_schedule_build: search_slack0 %d not in [0, %d]", opts->search_slack0,
                       kMaxSearchSlack0);
    std::vector<qs_gate> g(gates, gates + n_gates);
    for (int i = 0; i < n_gates; i++)
        if (!check_gate(n, g[i])) return qs_fail(QS_EINVAL, "qs_schedule_build: bad gate %d", i);
    std::vector<std::vector<int>> groups;
    if (opts->fuse && opts->commute_diagonal) {
        // Run i = f * R + r: rule r (0: greedy; r >= 1: support-aware with
        // slack search_slack0 + r - 1) with its first cluster forced to rank f
        // (f = 0: the rule's own).  The runs are independent; a few host
        // threads take them in turn.
        const int R = std::max(1, (int)opts->search_runs);
        const int runs = R * std::max(1, (int)opts->search_first);
        std::vector<std::vector<std::vector<int>>> res(runs);
        std::vector<char> failed(runs, 0);
        std::atomic<int> next{0};
        auto worker = [&]() {
            for (int i = next++; i < runs; i = next++) {
                try {
                    DiagClusterer cl(n, g);
                    const int r = i % R;
                    res[i] = cl.run(opts->k_max, r == 0 ? -1 : opts->search_slack0 + r - 1, i / R);
                } catch (...) {
                    failed[i] = 1;             // out of host memory
                }
            }
        };
        int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        if (g_host_threads.load() > 0) hw = std::min(hw, g_host_threads.load());
        const int n_threads = std::min(runs, std::min(hw, kMaxSearchThreads));
        std::vector<std::thread> pool;
        for (int t = 1; t < n_threads; t++) {
            try {
                pool.emplace_back(worker);
            } catch (...) {
                break;                         // no thread to be had: fewer workers
            }
        }
        worker();
        for (auto &t : pool) t.join();
        for (int i = 0; i < runs; i++)
            if (failed[i]) return qs_fail(QS_ENOMEM, "qs_schedule_build: out of host memory");
        // sweeps cost time, phase ops little.  The cost of a run: its dense
        // clusters, each weighted by 2^(|support| - n) when the state starts as
        // a basis state (the support grows by each dense cluster's qubits),
        // else 1; the lowest cost wins, then fewer clusters, then the lower i.
        // (Sums of powers of two from 2^-n to 1: exact.)
        auto cost = [&](const std::vector<std::vector<int>> &cl) {
            double c = 0.0;
            uint64_t sup = 0;
            for (const auto &grp : cl) {
                bool diag = true;
                uint64_t qs = 0;
                for (int gi : grp) {
                    diag = diag && is_diagonal(g[gi].kind);
                    qs |= gmask_of(g[gi]);
                }
                if (diag) continue;
                sup |= qs;
                c += opts->search_from_basis ? std::ldexp(1.0, __builtin_popcountll(sup) - n) : 1.0;
            }
            return c;
        };
        // runs ranked: lowest cost, then fewer clusters, then the lower i
        std::vector<double> costs(runs);
        for (int i = 0; i < runs; i++) costs[i] = cost(res[i]);
        std::vector<int> rank(runs);
        for (int i = 0; i < runs; i++) rank[i] = i;
        std::stable_sort(rank.begin(), rank.end(), [&](int a, int b) {
            if (costs[a] != costs[b]) return costs[a] < costs[b];
            return res[a].size() < res[b].size();
        });
        if (ranked) {
            // distinct clusterings only, best first
            for (int i : rank) {
                bool dup = false;
                for (const auto &r : *ranked) dup = dup || r == res[i];
                if (!dup) ranked->push_back(res[i]);
                if ((int)ranked->size() >= ranked_max) break;
            }
        }
        groups = std::move(res[rank[0]]);
    } else if (opts->fuse) {
        Clusterer cl(n, g);
        groups = cl.run(opts->k_max);
    } else {
        for (int i = 0; i < n_gates; i++) groups.push_back({i});
    }
    if (ranked && ranked->empty()) ranked->push_back(groups);
    return schedule_from_groups(n, g, groups, opts, out);
}

// Ops of a schedule from its clusters (gate index lists, in order): all-diagonal
// clusters become phase ops (neighbours merged with merge_phase), the others
// dense ops with their FP64 unitaries.
static int schedule_from_groups(int n, const std::vector<qs_gate> &g, const std::vector<std::vector<int>> &groups,
                                const qs_sched_opts *opts, qs_schedule **out)
{
    std::unique_ptr<qs_schedule> sc(new (std::nothrow) qs_schedule());
    if (!sc) return qs_fail(QS_ENOMEM, "qs_schedule_build: out of host memory");
    sc->n = n;
    for (auto &members : groups) {
        bool diag = true;
        for (int gi : members) diag = diag && is_diagonal(g[gi].kind);
        qs_op_host op;
        if (diag) {
            if (opts->fuse && opts->merge_phase && !sc->ops.empty() &&
                sc->ops.back().kind == QS_OP_PHASE) {
                std::vector<int> all(sc->ops.back().gates.begin(), sc->ops.back().gates.end());
                all.insert(all.end(), members.begin(), members.end());
                sc->ops.pop_back();
                make_phase(n, g, all, op);
            } else {
                make_phase(n, g, members, op);
            }
        } else {
            make_dense(g, members, op);
        }
        sc->ops.push_back(std::move(op));
    }
    // trailing diagonal ops multiply every amplitude by a unit-modulus phase:
    // the output distribution does not see them (Sec. 3.6)
    if (opts->drop_final_diagonal)
        while (!sc->ops.empty() && sc->ops.back().kind == QS_OP_PHASE) sc->ops.pop_back();
    *out = sc.release();
    return QS_OK;
}

// A phase op from the pool (qs_schedule_from_ops): n coefficients, then
// n_pairs CZ pairs, integers stored as doubles.
static bool phase_from_pool(int n, int n_pairs, const double *pool, int64_t pool_len, int64_t at,
                            qs_op_host &op)
{
    if (n_pairs < 0 || at < 0 || at > pool_len || pool_len - at < n + 2 * (int64_t)n_pairs) return false;
    auto integer = [](double v, int lo, int hi, int &out) {
        if (!(v >= lo && v <= hi) || v != std::floor(v)) return false;
        out = (int)v;
        return true;
    };
    const double *src = pool + at;
    op.kind = QS_OP_PHASE;
    op.coeff.assign(n, 0);
    op.edges.clear();
    uint64_t support = 0;
    for (int q = 0; q < n; q++) {
        int c;
        if (!integer(src[q], -(1 << 30), 1 << 30, c)) return false;
        op.coeff[q] = ((c % 8) + 8) % 8;
        if (op.coeff[q]) support |= 1ULL << q;
    }
    for (int e = 0; e < n_pairs; e++) {
        int a, b;
        if (!integer(src[n + 2 * e], 0, n - 1, a) || !integer(src[n + 2 * e + 1], 0, n - 1, b) || a == b)
            return false;
        op.edges.push_back({a, b});
        support |= (1ULL << a) | (1ULL << b);
    }
    op.k = __builtin_popcountll(support);
    int j = 0;
    for (int q = 0; q < n && j < QS_MAX_K; q++)
        if ((support >> q) & 1) op.qubits[j++] = q;
    return true;
}

static int schedule_from_ops_impl(int n, int n_ops, const int *kinds, const int *ks, const int *qubits,
                                  const int64_t *offsets, const double *pool, int64_t pool_len,
                                  qs_schedule **out)
{
    if (!out || n < 1 || n > QS_MAX_QUBITS || n_ops < 0 ||
        (n_ops > 0 && (!kinds || !ks || !qubits || !offsets || !pool)))
        return qs_fail(QS_EINVAL, "qs_schedule_from_ops: bad arguments");
    std::unique_ptr<qs_schedule> sc(new (std::nothrow) qs_schedule());
    if (!sc) return qs_fail(QS_ENOMEM, "qs_schedule_from_ops: out of host memory");
    sc->n = n;
    for (int i = 0; i < n_ops; i++) {
        int k = ks[i];
        if (kinds[i] == QS_OP_PHASE) {
            qs_op_host op;
            if (!phase_from_pool(n, k, pool, pool_len, offsets[i], op)) {
                return qs_fail(QS_EINVAL, "qs_schedule_from_ops: bad phase op %d", i);
            }
            sc->ops.push_back(std::move(op));
            continue;
        }
        bool dense = kinds[i] == QS_OP_DENSE;
        // both kinds take at most QS_MAX_K qubits here (QS_MAX_K slots per op)
        if ((!dense && kinds[i] != QS_OP_DIAG) || k < 1 || k > QS_MAX_K || k > n) {
            return qs_fail(QS_EINVAL, "qs_schedule_from_ops: bad op %d", i);
        }
        // sort qubits ascending and permute the matrix accordingly (Sec. 3.2)
        int q[QS_MAX_K], perm[QS_MAX_K];
        uint64_t seen = 0;
        for (int j = 0; j < k; j++) {
            q[j] = qubits[QS_MAX_K * i + j];
            perm[j] = j;
            if (q[j] < 0 || q[j] >= n || ((seen >> q[j]) & 1)) {
                return qs_fail(QS_EINVAL, "qs_schedule_from_ops: bad qubits in op %d", i);
            }
            seen |= 1ULL << q[j];
        }
        for (int a = 1; a < k; a++)   // insertion sort of at most five positions
            for (int b = a; b > 0 && q[perm[b]] < q[perm[b - 1]]; b--) std::swap(perm[b], perm[b - 1]);
        const int d = 1 << k;
        int64_t need = dense ? 2LL * d * d : 2LL * d;
        if (offsets[i] < 0 || offsets[i] + need > pool_len) {
            return qs_fail(QS_EINVAL, "qs_schedule_from_ops: op %d reads past the pool", i);
        }
        qs_op_host op;
        op.kind = dense ? QS_OP_DENSE : QS_OP_DIAG;
        op.k = k;
        for (int j = 0; j < k; j++) op.qubits[j] = q[perm[j]];
        // new index bit j <-> old bit perm[j]
        auto remap = [&](int xn) {
            int xo = 0;
            for (int j = 0; j < k; j++) xo |= ((xn >> j) & 1) << perm[j];
            return xo;
        };
        const double *src = pool + offsets[i];
        if (dense) {
            op.matrix.resize(2 * d * d);
            for (int r = 0; r < d; r++)
                for (int c = 0; c < d; c++) {
                    int ro = remap(r), co = remap(c);
                    op.matrix[2 * (r * d + c)] = src[2 * (ro * d + co)];
                    op.matrix[2 * (r * d + c) + 1] = src[2 * (ro * d + co) + 1];
                }
        } else {
            op.matrix.resize(2 * d);
            for (int x = 0; x < d; x++) {
                op.matrix[2 * x] = src[2 * remap(x)];
                op.matrix[2 * x + 1] = src[2 * remap(x) + 1];
            }
        }
        sc->ops.push_back(std::move(op));
    }
    *out = sc.release();
    return QS_OK;
}

// The entry points of this file: host memory that runs out inside them (a
// standard container throwing) becomes QS_ENOMEM; no exception crosses the C
// boundary.
template <typename F>
static int guarded(const char *what, F &&f)
{
    try {
        return f();
    } catch (const std::bad_alloc &) {
        return qs_fail(QS_ENOMEM, "%s: out of host memory", what);
    } catch (...) {
        return qs_fail(QS_EINVAL, "%s: internal error", what);
    }
}

extern "C" int qs_supremacy_circuit(int rows, int cols, const int *removed_rc, int n_removed,
                                    int cz_cycles, uint64_t seed, int *n_qubits,
                                    qs_gate *gates, int max_gates, int *n_gates)
{
    return qs_guard([&]() -> int {
        return guarded("qs_supremacy_circuit", [&] {
            return supremacy_circuit_impl(rows, cols, removed_rc, n_removed, cz_cycles, seed, n_qubits, gates,
                                          max_gates, n_gates);
        });
    });
}

extern "C" int qs_schedule_build(int n, const qs_gate *gates, int n_gates,
                                 const qs_sched_opts *opts, qs_schedule **out)
{
    return qs_guard([&]() -> int {
        return guarded("qs_schedule_build", [&] { return schedule_build_impl(n, gates, n_gates, opts, out); });
    });
}

extern "C" int qs_schedule_from_ops(int n, int n_ops, const int *kinds, const int *ks,
                                    const int *qubits, const int64_t *offsets,
                                    const double *pool, int64_t pool_len, qs_schedule **out)
{
    return qs_guard([&]() -> int {
        return guarded("qs_schedule_from_ops", [&] {
            return schedule_from_ops_impl(n, n_ops, kinds, ks, qubits, offsets, pool, pool_len, out);
        });
    });
}

int qs_schedule_build_ranked(int n, const qs_gate *gates, int n_gates, const qs_sched_opts *opts, int top,
                             std::vector<qs_schedule *> &out)
{
    std::vector<std::vector<std::vector<int>>> ranked;
    qs_schedule *first = nullptr;
    int rc = schedule_build_impl(n, gates, n_gates, opts, &first, &ranked, std::max(1, top));
    if (rc) return rc;
    out.push_back(first);
    std::vector<qs_gate> g(gates, gates + n_gates);
    for (size_t i = 1; i < ranked.size(); i++) {
        qs_schedule *sc = nullptr;
        if ((rc = schedule_from_groups(n, g, ranked[i], opts, &sc))) return rc;
        out.push_back(sc);
    }
    return QS_OK;
}

// Stages for a state spread over 2^g parts (Sec. 3.4, Sec. 3.6 steps 1 and 3).
// The top g index bits of a stage hold its global qubits, on which no gate of
// the stage may act except diagonal ones (CZ, T: Sec. 3.5 applies them as
// conditional phases).  Greedy, in the gate list's order: a gate joins the
// present stage unless it is a non-diagonal gate on a global qubit or shares a
// qubit with a gate already left for later (so every qubit keeps its gate
// order).  The next stage's global qubits are the g whose next non-diagonal
// gate comes last (ties: the present global qubits, then the higher qubit),
// which keeps the number of global-to-local swaps small.
static int plan_stages_impl(int n, const qs_gate *gates, int n_gates, int g, const qs_sched_opts *opts,
                            qs_schedule **stages, int max_stages, int *n_stages, int *stage_of_gate)
{
    if (n < 2 || n > QS_MAX_QUBITS || g < 0 || g >= n || n_gates < 0 || (n_gates > 0 && !gates) || !opts ||
        !stages || max_stages < 1 || !n_stages)
        return qs_fail(QS_EINVAL, "qs_plan_stages: bad arguments");
    for (int i = 0; i < n_gates; i++)
        if (!check_gate(n, gates[i])) return qs_fail(QS_EINVAL, "qs_plan_stages: bad gate %d", i);
    std::vector<int> remaining(n_gates);
    for (int i = 0; i < n_gates; i++) remaining[i] = i;
    auto choose_global = [&](const std::vector<int> &rem, uint64_t current) {
        std::vector<long> next(n, std::numeric_limits<long>::max());
        for (size_t p = 0; p < rem.size(); p++) {
            const qs_gate &x = gates[rem[p]];
            if (is_diagonal(x.kind)) continue;
            if (next[x.q0] == std::numeric_limits<long>::max()) next[x.q0] = (long)p;
        }
        std::vector<int> order(n);
        for (int q = 0; q < n; q++) order[q] = q;
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            if (next[a] != next[b]) return next[a] > next[b];
            const bool ca = (current >> a) & 1, cb = (current >> b) & 1;
            if (ca != cb) return ca;
            return a > b;
        });
        uint64_t G = 0;
        for (int i = 0; i < g; i++) G |= 1ULL << order[i];
        return G;
    };
    int count = 0;
    uint64_t G = choose_global(remaining, 0);
    while (!remaining.empty()) {
        std::vector<int> take, rest;
        uint64_t blocked = 0;
        for (int gi : remaining) {
            const qs_gate &x = gates[gi];
            const uint64_t qm = gmask_of(x);
            if ((qm & blocked) || (!is_diagonal(x.kind) && (qm & G))) {
                rest.push_back(gi);
                blocked |= qm;
            } else {
                take.push_back(gi);
            }
        }
        if (take.empty()) {
            for (int i = 0; i < count; i++) qs_schedule_free(stages[i]);
            return qs_fail(QS_EINVAL, "qs_plan_stages: no gate can run with %d global qubits", g);
        }
        if (count >= max_stages) {
            for (int i = 0; i < count; i++) qs_schedule_free(stages[i]);
            return qs_fail(QS_EINVAL, "qs_plan_stages: more than %d stages", max_stages);
        }
        std::vector<qs_gate> sub(take.size());
        for (size_t i = 0; i < take.size(); i++) {
            sub[i] = gates[take[i]];
            if (stage_of_gate) stage_of_gate[take[i]] = count;
        }
        qs_schedule *sc = nullptr;
        int rc = schedule_build_impl(n, sub.data(), (int)sub.size(), opts, &sc);
        if (rc) {
            for (int i = 0; i < count; i++) qs_schedule_free(stages[i]);
            return rc;
        }
        // the stage's global qubits at the top g index bits: each one below
        // exchanged with a top bit whose own qubit is local
        int loc[64];
        for (int q = 0; q < n; q++) loc[q] = q;
        int t = n - 1;
        for (int q = 0; q < n - g; q++) {
            if (!((G >> q) & 1)) continue;
            while ((G >> t) & 1) t--;
            loc[q] = t;
            loc[t] = q;
            t--;
        }
        if ((rc = qs_schedule_remap(sc, loc))) {
            qs_schedule_free(sc);
            for (int i = 0; i < count; i++) qs_schedule_free(stages[i]);
            return rc;
        }
        stages[count++] = sc;
        remaining = std::move(rest);
        if (!remaining.empty()) G = choose_global(remaining, G);
    }
    *n_stages = count;
    return QS_OK;
}

extern "C" int qs_plan_stages(int n, const qs_gate *gates, int n_gates, int n_global, const qs_sched_opts *opts,
                              qs_schedule **stages, int max_stages, int *n_stages, int *stage_of_gate)
{
    return qs_guard([&]() -> int {
        return guarded("qs_plan_stages", [&] {
            return plan_stages_impl(n, gates, n_gates, n_global, opts, stages, max_stages, n_stages, stage_of_gate);
        });
    });
}

extern "C" int qs_set_host_threads(int n)
{
    if (n < 0) return qs_fail(QS_EINVAL, "qs_set_host_threads: %d < 0", n);
    g_host_threads.store(n);
    return QS_OK;
}

extern "C" int qs_schedule_num_qubits(const qs_schedule *sc) { return sc ? sc->n : 0; }
extern "C" int qs_schedule_num_ops(const qs_schedule *sc) { return sc ? (int)sc->ops.size() : 0; }

extern "C" int qs_schedule_op(const qs_schedule *sc, int i, qs_op_info *info, double *matrix,
                              int32_t *gate_idx, int32_t *coeff, int32_t *edges)
{
    return qs_guard([&]() -> int {
        if (!sc || i < 0 || i >= (int)sc->ops.size())
            return qs_fail(QS_EINVAL, "qs_schedule_op: bad schedule or index");
        const qs_op_host &op = sc->ops[i];
        if (info) {
            std::memset(info, 0, sizeof(*info));
            info->kind = op.kind;
            info->k = op.k;
            for (int j = 0; j < QS_MAX_K && j < op.k; j++) info->qubits[j] = op.qubits[j];
            info->n_gates = (int32_t)op.gates.size();
            info->n_edges = (int32_t)op.edges.size();
        }
        if (matrix && !op.matrix.empty())
            std::memcpy(matrix, op.matrix.data(), sizeof(double) * op.matrix.size());
        if (gate_idx && !op.gates.empty())
            std::memcpy(gate_idx, op.gates.data(), sizeof(int32_t) * op.gates.size());
        if (coeff && op.kind == QS_OP_PHASE)
            std::memcpy(coeff, op.coeff.data(), sizeof(int32_t) * op.coeff.size());
        if (edges && op.kind == QS_OP_PHASE)
            for (size_t e = 0; e < op.edges.size(); e++) {
                edges[2 * e] = op.edges[e].first;
                edges[2 * e + 1] = op.edges[e].second;
            }
        return QS_OK;
    });
}

// Phase op device layout: three coefficient bit-masks and, per qubit a with CZ
// partners b > a (pairs counted mod 2), the mask of those partners.
std::vector<uint8_t> qs_pack_phase(int n, const std::vector<int32_t> &coeff,
                                   const std::vector<std::pair<int, int>> &edges, int *n_act)
{
    qs_phase_dev hdr;
    std::memset(&hdr, 0, sizeof(hdr));
    for (int q = 0; q < n; q++) {
        int c = ((coeff[q] % 8) + 8) % 8;
        for (int b = 0; b < 3; b++)
            if ((c >> b) & 1) hdr.cmask[b] |= 1ULL << q;
    }
    std::vector<uint64_t> partners(n, 0);
    for (auto &e : edges) {
        int a = std::min(e.first, e.second), b = std::max(e.first, e.second);
        partners[a] ^= 1ULL << b;
    }
    std::vector<qs_phase_term> terms;
    for (int a = 0; a < n; a++)
        if (partners[a]) terms.push_back({partners[a], a, 0});
    hdr.n_act = (int32_t)terms.size();
    *n_act = hdr.n_act;
    std::vector<uint8_t> buf(sizeof(hdr) + terms.size() * sizeof(qs_phase_term));
    std::memcpy(buf.data(), &hdr, sizeof(hdr));
    if (!terms.empty())
        std::memcpy(buf.data() + sizeof(hdr), terms.data(), terms.size() * sizeof(qs_phase_term));
    return buf;
}

"""Gate clustering (Sec. 3.6, step 2) and cluster unitaries.  Oracle only.

Sec. 3.6 merges runs of 1- and 2-qubit gates into k-qubit clusters with
k <= k_max: it greedily tries to increase the number of qubits k of a cluster
while k <= k_max, and a small local search builds the largest cluster from the
gates not yet assigned before the rest are assigned to new clusters.  Gates on
different qubits commute and may be reordered; gates on the same qubit never
are.  The paper gives no more detail; this is the reading both implementations
follow:

  * every qubit keeps a queue of its unassigned gates in circuit order;
  * closure(S) for a qubit set S is the set of unassigned gates that can run
    using only the qubits in S: sweep the qubits of S in ascending order, and
    on each take gates off the head of its queue while the head gate acts only
    on S and heads the queue of each of its qubits; repeat sweeps until one
    takes nothing.  Gates are listed in the order they were taken;
  * growing from a seed gate s: S = qubits(s); then repeatedly, for every gate
    g at the head of some queue after closure(S) is taken (ascending index)
    with qubits(g) not inside S and |S u qubits(g)| <= k_max, evaluate
    closure(S u qubits(g)); keep the largest (ties: fewer qubits, then the
    lower g); stop when none is larger than closure(S);
  * one cluster is grown from every *ready* gate (one heading the queues of all
    its qubits); the largest wins (ties: fewer qubits, then the lower seed);
    its gates are removed from the queues; repeat until no gate is left.

With commute_diagonal the same rule runs on a relaxed order.  Diagonal gates
commute (their matrices are diagonal), so on a qubit a diagonal gate may run
before earlier unassigned gates of that qubit when all of them are diagonal; a
non-diagonal gate keeps its place:

  * available(g, q): every unassigned gate before g on q is diagonal and g is
    diagonal, or no unassigned gate precedes g on q; ready(g): available on
    each of its qubits;
  * closure(S): sweep the qubits of S in ascending order; on each, walk its
    unassigned gates in order: take a gate that acts only on S and is ready,
    pass over a diagonal gate that is not taken, stop at a non-diagonal one;
    repeat sweeps until one takes nothing;
  * growth candidates (and seeds): per qubit, its first unassigned gate (not
    yet in the cluster), if ready; the rest as above;
  * search (search_runs R > 1): run 0 is the rule above; run s >= 1 takes,
    while the dense clusters taken so far do not cover every qubit, among the
    clusters grown from all seeds (ranked as the rule ranks them: more gates,
    then fewer qubits, then the lower seed) within search_slack0 + s - 1
    gates of the largest the one adding the fewest qubits to them (an
    all-diagonal one adds none; ties: the first in rank), else the first; the run of lowest cost is kept
    (then the fewest clusters, then the lowest r), the cost being its number
    of dense clusters or, with from_basis, the sum over its dense clusters of
    2^(|support| - n), the support growing by each dense cluster's qubits from
    none (the sizes of the sweeps after a basis state);
  * where the support starts (search_first F > 1): each of the R runs is also
    made with its first cluster the one of rank f = 1..F-1 among those grown
    from all seeds (the last one when there are fewer); run f * R + r.

A cluster made only of diagonal gates (T, T^dagger, CZ) becomes a phase op;
neighbouring phase ops in the op list are merged (diagonal gates commute).
With fuse=False every gate is an op of its own (the plain gate-by-gate form).

The unitary of a dense cluster is the product of its gates, each embedded in
the 2^k space of the cluster's sorted qubits by the Kronecker rule of Sec. 2,
later gates on the left; qubit qubits[j] is bit j of the matrix index (Sec. 3.2
pre-permutes the matrix to sorted qubit order).
"""
import numpy as np

from . import gates as _gates
from . import sim as _sim

PHASE_COEFF = {"t": 1, "tdg": 7}


def _heads(n, queues, pos):
    return sorted(set(queues[q][pos[q]] for q in range(n) if pos[q] < len(queues[q])))


def _is_ready(queues, pos, qs, g):
    return all(pos[q] < len(queues[q]) and queues[q][pos[q]] == g for q in qs)


def _closure(gqs, queues, pos0, S):
    pos = dict(pos0)
    members = []
    changed = True
    while changed:
        changed = False
        for q in sorted(S):
            while pos[q] < len(queues[q]):
                g = queues[q][pos[q]]
                if not set(gqs[g]) <= S or not _is_ready(queues, pos, gqs[g], g):
                    break
                members.append(g)
                for p in gqs[g]:
                    pos[p] += 1
                changed = True
    return members, pos


def _grow(n, gqs, queues, pos, seed, k_max):
    S = set(gqs[seed])
    members, after = _closure(gqs, queues, pos, S)
    while True:
        best = None
        for g in _heads(n, queues, after):
            qs = set(gqs[g])
            if qs <= S or len(S | qs) > k_max:
                continue
            m2, a2 = _closure(gqs, queues, pos, S | qs)
            key = (len(m2), -len(S | qs), -g)
            if best is None or key > best[0]:
                best = (key, S | qs, m2, a2)
        if best is None or len(best[2]) <= len(members):
            break
        _, S, members, after = best
    return members, S


def clusters(n, gates, k_max):
    """Greedy clusters as lists of gate indices in a valid application order."""
    assert k_max >= 2
    gqs = [tuple(qs) for (_, _, qs) in gates]
    queues = [[] for _ in range(n)]
    for i, qs in enumerate(gqs):
        for q in qs:
            queues[q].append(i)
    pos = {q: 0 for q in range(n)}
    remaining = len(gates)
    out = []
    while remaining:
        ready = [g for g in _heads(n, queues, pos) if _is_ready(queues, pos, gqs[g], g)]
        best, best_key = None, None
        for s in ready:
            members, S = _grow(n, gqs, queues, pos, s, k_max)
            key = (len(members), -len(S), -s)
            if best_key is None or key > best_key:
                best, best_key = members, key
        for g in best:
            for q in gqs[g]:
                assert queues[q][pos[q]] == g
                pos[q] += 1
        remaining -= len(best)
        out.append(best)
    return out


def clusters_commuting(n, gates, k_max, search_runs=1, from_basis=True, search_first=1, search_slack0=0):
    """Clusters when diagonal gates may pass one another on a qubit: the best
    of search_runs x search_first runs (run 0 the greedy rule)."""
    def cost(cl):
        total, support = 0.0, set()
        for c in cl:
            if all(gates[g][1] in _gates.DIAGONAL for g in c):
                continue
            support |= set(q for g in c for q in gates[g][2])
            total += 2.0 ** (len(support) - n) if from_basis else 1.0
        return total, len(cl)

    R = max(1, search_runs)
    runs = [_commuting_run(n, gates, k_max, None if r == 0 else search_slack0 + r - 1, f)
            for f in range(max(1, search_first)) for r in range(R)]
    best = None
    for cl in runs:
        if best is None or cost(cl) < cost(best):
            best = cl
    return best


def _commuting_run(n, gates, k_max, support_slack, first_pick=0):
    assert k_max >= 2
    gqs = [tuple(qs) for (_, _, qs) in gates]
    diag = [name in _gates.DIAGONAL for (_, name, _) in gates]
    queues = [[] for _ in range(n)]
    for i, qs in enumerate(gqs):
        for q in qs:
            queues[q].append(i)
    done = set()

    def available(g, q, taken):
        for h in queues[q]:
            if h == g:
                return True
            if h in done or h in taken:
                continue
            if not (diag[h] and diag[g]):
                return False
        return False

    def ready(g, taken):
        return all(available(g, q, taken) for q in gqs[g])

    def closure(S):
        taken, order = set(), []
        changed = True
        while changed:
            changed = False
            for q in sorted(S):
                for g in queues[q]:
                    if g in done or g in taken:
                        continue
                    if not set(gqs[g]) <= S:
                        if not diag[g]:
                            break
                        continue
                    if ready(g, taken):
                        taken.add(g)
                        order.append(g)
                        changed = True
                    elif not diag[g]:
                        break
        return order

    def candidates(members):
        taken = set(members)
        out = set()
        for q in range(n):
            for g in queues[q]:
                if g in done or g in taken:
                    continue
                if ready(g, taken):
                    out.add(g)
                break
        return sorted(out)

    def grow(seed):
        S = set(gqs[seed])
        members = closure(S)
        while True:
            best = None
            for g in candidates(members):
                qs = set(gqs[g])
                if qs <= S or len(S | qs) > k_max:
                    continue
                m2 = closure(S | qs)
                key = (len(m2), -len(S | qs), -g)
                if best is None or key > best[0]:
                    best = (key, S | qs, m2)
            if best is None or len(best[2]) <= len(members):
                return members, S
            _, S, members = best

    out, support = [], set()
    while len(done) < len(gates):
        options = []
        for s in candidates([]):
            members, S = grow(s)
            options.append(((len(members), -len(S), -s), members, S))
        options.sort(key=lambda o: o[0], reverse=True)

        def dense(o):
            return not all(diag[g] for g in o[1])

        pick = 0
        if not out and first_pick > 0:
            pick = min(first_pick, len(options) - 1)
        elif support_slack is not None and len(support) < n:
            near = [i for i, o in enumerate(options) if o[0][0] >= options[0][0][0] - support_slack]
            pick = min(near, key=lambda i: (len(options[i][2] - support) if dense(options[i]) else 0, i))
        if dense(options[pick]):
            support |= options[pick][2]
        best = options[pick][1]
        done.update(best)
        out.append(best)
    return out


def cluster_unitary(gates, members, qubits):
    """Product of the member gates embedded in the 2^k space of `qubits`."""
    k = len(qubits)
    where = {q: j for j, q in enumerate(qubits)}
    U = np.eye(1 << k, dtype=np.complex128)
    for g in members:
        _, name, qs = gates[g]
        if name == "cz":
            E = _sim.kron_cz(k, where[qs[0]], where[qs[1]])
        else:
            E = _sim.kron_1q(k, where[qs[0]], _gates.matrix(name))
        U = E @ U
    return U


def _phase_op(n, gates, members):
    coeff = np.zeros(n, dtype=np.int64)
    edges = []
    for g in members:
        _, name, qs = gates[g]
        if name == "cz":
            edges.append((qs[0], qs[1]))
        else:
            coeff[qs[0]] += PHASE_COEFF[name]
    return {"kind": "phase", "gates": tuple(members),
            "qubits": tuple(sorted(set(q for g in members for q in gates[g][2]))),
            "coeff": coeff % 8, "edges": edges}


def schedule(n, gates, k_max=5, fuse=True, commute_diagonal=True, search_runs=1, search_from_basis=True,
             search_first=1, search_slack0=0):
    """Op list: dicts with kind 'dense' (qubits, gates, matrix) or 'phase'
    (qubits, gates, coeff, edges)."""
    if fuse:
        groups = (clusters_commuting(n, gates, k_max, search_runs, search_from_basis, search_first, search_slack0)
                  if commute_diagonal
                  else clusters(n, gates, k_max))
    else:
        groups = [[i] for i in range(len(gates))]
    ops = []
    for members in groups:
        if all(gates[g][1] in _gates.DIAGONAL for g in members):
            op = _phase_op(n, gates, members)
            if fuse and ops and ops[-1]["kind"] == "phase":
                prev = ops.pop()
                op = _phase_op(n, gates, list(prev["gates"]) + list(members))
            ops.append(op)
        else:
            qubits = tuple(sorted(set(q for g in members for q in gates[g][2])))
            ops.append({"kind": "dense", "gates": tuple(members), "qubits": qubits,
                        "matrix": cluster_unitary(gates, members, qubits)})
    return ops


def run_schedule(n, gates, ops, psi=None):
    """Apply an op list with the oracle's k-qubit / phase routines."""
    if psi is None:
        psi = _sim.basis_state(n, 0)
    for op in ops:
        if op["kind"] == "dense":
            _sim.apply_kq(psi, op["qubits"], op["matrix"])
        else:
            _sim.apply_phase(psi, op["coeff"], op["edges"])
    return psi

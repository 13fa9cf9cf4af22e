"""Phase ops folded into the tensor-core sweep before them, against the oracle.

A merged CZ / T phase (Sec. 2) right after a dense cluster runs inside that
cluster's sweep: the terms on the sweep's five qubits are multiplied into the
cluster matrix, and the rest -- CZ pairs with one or no end on those qubits and
the (even) coefficients off them, which act on each group as a conditional Z or
a phase of the group (Sec. 3.5) -- become a power of i per group and a sign per
member on the sweep's outputs.  Checked element by element against the oracle
(dense op, then the phase op, in complex128) and against the unfolded run, on
both amplitude types, for high, low (complex64: paired loads) and mixed
targets, for embedded clusters whose padding qubits carry phase terms, after
qs_init_basis (sweeps on part of the state), and for phase ops that must not
fold.
"""
import numpy as np
import pytest

import paper_1704_01127_gb300.qs as qs
from inputs import random_state, random_unitary, rng
from oracle import sim

pytestmark = pytest.mark.gpu

# one sweep of each kind: the folded phase adds at most one rounding per value
TOL = {qs.QS_C128: 1e-13, qs.QS_C64: 3e-6}
N = 12


def f32_round(psi):
    return psi.astype(np.complex64).astype(np.complex128)


def phase_case(n, sweep_qubits, seed, odd_off=False):
    """Coefficients: anything on the sweep's qubits, even off them (odd on one
    of them with odd_off); CZ pairs inside the sweep's qubits, from one of them
    to another qubit, and between two other qubits, one of them twice (the
    pair cancels)."""
    g = rng(seed)
    on = list(sweep_qubits)
    off = [q for q in range(n) if q not in on]
    coeff = np.zeros(n, dtype=np.int64)
    for q in on:
        coeff[q] = g.integers(0, 8)
    for q in off:
        coeff[q] = 2 * g.integers(0, 4)
    if odd_off:
        coeff[off[len(off) // 2]] = 1 + 2 * g.integers(0, 4)

    def two(pool):
        a, b = g.choice(pool, 2, replace=False)
        return int(a), int(b)

    pairs = [two(on) for _ in range(2)]
    pairs += [(int(g.choice(on)), int(g.choice(off))) for _ in range(4)]
    pairs += [two(off) for _ in range(4)]
    pairs.append(pairs[-1])
    return coeff, pairs


def oracle_run(psi, ops):
    out = psi.copy()
    for kind, a, b in ops:
        if kind == qs.QS_OP_DENSE:
            sim.apply_kq(out, list(a), b)
        else:
            sim.apply_phase(out, b, a)
    return out


def lib_run(n, dtype, ops, psi=None, basis=None, fold=True, path=qs.QS_PATH_AUTO):
    sc = qs.qs_schedule_from_ops(n, ops)
    try:
        h = qs.qs_alloc(n, dtype)
        try:
            qs.qs_set_path(h, path)
            qs.qs_set_phase_fold(h, fold)
            if basis is None:
                qs.qs_set_amplitudes(h, psi)
            else:
                qs.qs_init_basis(h, basis)
            ms = qs.qs_run_circuit_timed(h, sc)
            return qs.qs_get_amplitudes(h), ms
        finally:
            qs.qs_free(h)
    finally:
        qs.qs_schedule_free(sc)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("targets", [(1, 3, 4, 7, 9), (0, 1, 2, 3, 4), (7, 8, 9, 10, 11), (0, 5, 6, 10, 11)])
def test_fold_matches_oracle_and_unfolded(dtype, targets):
    seed = sum(targets) + 31 * dtype
    U = random_unitary(5, seed)
    coeff, pairs = phase_case(N, targets, seed)
    ops = [(qs.QS_OP_DENSE, targets, U), (qs.QS_OP_PHASE, pairs, coeff)]
    psi = random_state(N, seed + 1)
    if dtype == qs.QS_C64:
        psi = f32_round(psi)
    want = oracle_run(psi, ops)
    got, ms = lib_run(N, dtype, ops, psi=psi)
    assert ms[1] == -1 and ms[0] > 0                      # the phase op ran inside the sweep
    assert np.max(np.abs(got - want)) <= TOL[dtype]
    plain, ms_plain = lib_run(N, dtype, ops, psi=psi, fold=False)
    assert ms_plain[1] >= 0
    assert np.max(np.abs(got - plain)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_fold_off_the_sweep_is_bit_exact(dtype):
    """CZ pairs with at most one end on the sweep's qubits leave the matrix as it
    is: the folded run equals the unfolded one bit for bit (up to the sign of
    zeros).  (A pair inside is multiplied into the matrix, whose complex128
    digit planes then round differently at the level of the dropped planes.)"""
    targets = (2, 4, 5, 8, 9)
    U = random_unitary(5, 5)
    pairs = [(2, 3), (5, 6), (9, 10), (0, 1), (3, 11), (7, 8)]
    ops = [(qs.QS_OP_DENSE, targets, U), (qs.QS_OP_PHASE, pairs, np.zeros(N, dtype=np.int64))]
    psi = random_state(N, 6)
    got, ms = lib_run(N, dtype, ops, psi=psi)
    plain, _ = lib_run(N, dtype, ops, psi=psi, fold=False)
    assert ms[1] == -1
    assert np.array_equal(got, plain)


def test_fold_embedded_cluster_padding_qubits():
    """A 3-qubit complex128 cluster runs as U (x) 1 on five qubits, padded with
    the highest free ones (10, 11): phase terms there, odd coefficients
    included, fold into the 5-qubit matrix.  complex64 runs such a cluster on
    the CUDA cores, so its phase op runs on its own."""
    targets = (2, 5, 6)
    U = random_unitary(3, 8)
    coeff, pairs = phase_case(N, (2, 5, 6, 10, 11), 9)
    coeff[11] = 3
    pairs += [(10, 11), (11, 0), (10, 7)]
    ops = [(qs.QS_OP_DENSE, targets, U), (qs.QS_OP_PHASE, pairs, coeff)]
    psi = random_state(N, 10)
    want = oracle_run(psi, ops)
    got, ms = lib_run(N, qs.QS_C128, ops, psi=psi)
    assert ms[1] == -1
    assert np.max(np.abs(got - want)) <= TOL[qs.QS_C128]
    psi32 = f32_round(psi)
    got, ms = lib_run(N, qs.QS_C64, ops, psi=psi32)
    assert ms[1] >= 0
    assert np.max(np.abs(got - oracle_run(psi32, ops))) <= TOL[qs.QS_C64]


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_no_fold_for_odd_coefficient_off_the_sweep_or_cuda_cores(dtype):
    targets = (1, 3, 4, 7, 9)
    U = random_unitary(5, 12)
    psi = random_state(N, 13)
    if dtype == qs.QS_C64:
        psi = f32_round(psi)
    coeff, pairs = phase_case(N, targets, 14, odd_off=True)
    ops = [(qs.QS_OP_DENSE, targets, U), (qs.QS_OP_PHASE, pairs, coeff)]
    got, ms = lib_run(N, dtype, ops, psi=psi)
    assert ms[1] >= 0                                     # a T-type factor off the sweep: own sweep
    assert np.max(np.abs(got - oracle_run(psi, ops))) <= TOL[dtype]
    coeff, pairs = phase_case(N, targets, 15)
    ops = [(qs.QS_OP_DENSE, targets, U), (qs.QS_OP_PHASE, pairs, coeff)]
    got, ms = lib_run(N, dtype, ops, psi=psi, path=qs.QS_PATH_CUDA_CORES)
    assert ms[1] >= 0                                     # no tensor-core sweep to fold into
    assert np.max(np.abs(got - oracle_run(psi, ops))) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_fold_on_the_support_after_basis_state(dtype):
    """From |x>: the folded sweeps run on the support (part of the state) and
    widen it (all five qubits new, then two of five: 1 and 8 of each group's
    32 members read); a second phase op in a row runs on its own; bit for bit
    the result of the same ops on the zero-filled basis vector, and the
    oracle's."""
    n, x = 14, 0x1A6
    t1, t3, t2 = (0, 2, 3, 8, 9), (0, 1, 2, 3, 10), (4, 6, 11, 12, 13)
    c1, p1 = phase_case(n, t1, 20)
    c4, p4 = phase_case(n, t3, 25)
    c2, p2 = phase_case(n, t2, 21)
    c3, p3 = phase_case(n, t2, 22)
    ops = [(qs.QS_OP_DENSE, t1, random_unitary(5, 23)), (qs.QS_OP_PHASE, p1, c1),
           (qs.QS_OP_DENSE, t3, random_unitary(5, 26)), (qs.QS_OP_PHASE, p4, c4),
           (qs.QS_OP_DENSE, t2, random_unitary(5, 24)), (qs.QS_OP_PHASE, p2, c2), (qs.QS_OP_PHASE, p3, c3)]
    e = np.zeros(1 << n, dtype=np.complex128)
    e[x] = 1
    lazy, ms = lib_run(n, dtype, ops, basis=x)
    assert list(ms[[1, 3, 5]]) == [-1, -1, -1] and ms[6] >= 0
    full, _ = lib_run(n, dtype, ops, psi=e)
    assert np.array_equal(lazy, full)
    assert np.max(np.abs(lazy - oracle_run(e, ops))) <= 3 * TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_supremacy_circuit_final_layer_folds(dtype):
    """The trailing CZ layer of a supremacy circuit (Fig. 1) folds into the last
    cluster's sweep; the state is the oracle's."""
    n, g = qs.qs_supremacy_circuit(4, 5, 25, 4)
    sc = qs.qs_schedule_build(n, g, k_max=5)
    try:
        last = qs.qs_schedule_num_ops(sc) - 1
        assert qs.qs_schedule_op(sc, last)["kind"] == "phase"
        h = qs.qs_alloc(n, dtype)
        try:
            qs.qs_init_basis(h, 0)
            ms = qs.qs_run_circuit_timed(h, sc)
            got = qs.qs_get_amplitudes(h)
        finally:
            qs.qs_free(h)
    finally:
        qs.qs_schedule_free(sc)
    assert ms[last] == -1
    want = sim.run_circuit(n, qs.gates_to_tuples(g))
    assert np.max(np.abs(got - want)) <= (1e-12 if dtype == qs.QS_C128 else 2e-6)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_fold_of_the_identity_phase(dtype):
    """A phase op with no terms (all coefficients 0, no pairs) folds into the
    sweep and leaves the cluster's result bit for bit as it is."""
    targets = (3, 5, 6, 9, 11)
    U = random_unitary(5, 40)
    psi = random_state(N, 41)
    if dtype == qs.QS_C64:
        psi = f32_round(psi)
    ops = [(qs.QS_OP_DENSE, targets, U), (qs.QS_OP_PHASE, [], np.zeros(N, dtype=np.int64))]
    got, ms = lib_run(N, dtype, ops, psi=psi)
    alone, _ = lib_run(N, dtype, ops[:1], psi=psi)
    assert ms[1] == -1
    assert np.array_equal(got, alone)

"""Full-size checks in the launch configuration bench.py times (fused schedules
with the default clustering search, started with qs_init_basis so that the
first sweeps run on the reachable support, default kernel paths).

* 30 qubits (5x6 grid, 25 CZ cycles, seed 0) and 32 qubits (4x8, seed 1), in
  complex128 and complex64: the amplitudes at 2048 sampled indices (0, 2^n - 1
  and PCG64 draws) against the oracle's gate-by-gate complex128 state, stored
  in tests/golden/ by tests/golden/make_fullsize.py (absolute max |dpsi| within
  1e-12 for complex128 and 2e-6 for complex64; the relative figure is
  reported), and the output statistics against the oracle's.
* 30 qubits complex128: the circuit followed by its inverse returns |0...0>
  (|psi_0|^2 = 1 within 2e-12 and the norm within 1e-12, so every other
  amplitude is below 1e-6 in modulus and their squares sum below 2e-12).
* 33 qubits (3x11 grid, 25 CZ cycles), complex128 (128 GiB): norm, Porter-
  Thomas moment, circuit + inverse returns |0...0>.
* 34 qubits (5x7 minus a corner), complex64 only (128 GiB): norm drift and
  Porter-Thomas moments; circuit + inverse returns |0...0> within 1e-4.
* 32 qubits, complex64, uniform state (every p = 2^-32 exactly, so every CDF
  sum is exact and outcome j is floor(u_j 2^32), the rule the oracle is pinned
  to): 4096 samples bit for bit.  Above 30 qubits the super-block prefixes no
  longer fit the draw kernel's shared memory and are searched in device memory.
"""
import os

import numpy as np
import pytest

import paper_1704_01127_gb300.qs as qs
from oracle import circuit as ocircuit
from oracle import sim
from conftest import GOLDEN, read_golden

pytestmark = pytest.mark.gpu

TOL = {qs.QS_C128: 1e-12, qs.QS_C64: 2e-6}


def load_fullsize(name):
    """(rows, cols, cycles, seed, n), oracle statistics, indices, amplitudes."""
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip("%s not generated (tests/golden/make_fullsize.py)" % name)
    rows = read_golden(name)
    params = tuple(int(x) for x in rows[0][1:])
    stats = tuple(float(x) for x in rows[1][1:])
    idx = np.array([int(r[0]) for r in rows[2:]], dtype=np.uint64)
    amp = np.array([complex(float(r[1]), float(r[2])) for r in rows[2:]], dtype=np.complex128)
    return params, stats, idx, amp


def inverse_gates(gates):
    return qs.gates_from_tuples(ocircuit.inverse_circuit(qs.gates_to_tuples(gates)))


def run(h, n, gates, k_max=5):
    sc = qs.qs_schedule_build(n, gates, k_max=k_max)
    try:
        qs.qs_run_circuit(h, sc)
    finally:
        qs.qs_schedule_free(sc)


def test_30_qubits_c128_circuit_and_inverse():
    n, g = qs.qs_supremacy_circuit(5, 6, 25, 0)
    h = qs.qs_alloc(n, qs.QS_C128)
    try:
        qs.qs_init_basis(h, 0)
        run(h, n, g)
        st = qs.qs_stats(h)
        assert abs(st[0] - 1) < 1e-13
        assert 1.8 < st[3] < 3.0          # Porter-Thomas is 2; depth 25 is not fully converged
        run(h, n, inverse_gates(g))
        a0 = qs.qs_get_amplitudes_at(h, [0])[0]
        assert abs(abs(a0) ** 2 - 1) < 2e-12
        assert abs(qs.qs_norm(h) - 1) < 1e-12
    finally:
        qs.qs_free(h)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("name", ["fullsize_5x6_d25_s0.txt", "fullsize_4x8_d25_s1.txt"])
def test_fullsize_against_oracle(name, dtype):
    """Configs 2 and 3: the fused, support-started run of the library against
    the oracle's gate-by-gate state at sampled indices (Sec. 2 definitions)."""
    (rows, cols, cycles, seed, n), ostats, idx, want = load_fullsize(name)
    nq, g = qs.qs_supremacy_circuit(rows, cols, cycles, seed)
    assert nq == n
    assert qs.gates_to_tuples(g) == ocircuit.supremacy_circuit(rows, cols, cycles, seed)[1]
    h = qs.qs_alloc(n, dtype)
    try:
        qs.qs_init_basis(h, 0)
        run(h, n, g)
        got = qs.qs_get_amplitudes_at(h, idx)
        st = qs.qs_stats(h)
    finally:
        qs.qs_free(h)
    err = np.abs(got - want)
    rel = float(np.max(err) / np.max(np.abs(want)))
    print("%s dtype %d: max |dpsi| = %.3e (%.3e of the largest sampled |psi|), stats %s vs oracle %s"
          % (name, dtype, float(np.max(err)), rel, st, ostats))
    assert float(np.max(err)) <= TOL[dtype]
    # the oracle sums 2^n terms one after another in FP64 (its norm is off by
    # 1.8e-13 at 30 qubits and 3.5e-12 at 32); the library's float-float sums
    # are closer to exact, so the statistics agree to the oracle's rounding
    if dtype == qs.QS_C128:
        assert abs(st[0] - ostats[0]) < 1e-11
        assert abs(st[1] - ostats[1]) < 1e-10 * ostats[1]
        assert abs(st[3] - ostats[3]) < 1e-9 * ostats[3]
    else:
        assert abs(st[0] - ostats[0]) < 1e-5
        assert abs(st[1] - ostats[1]) < 1e-5 * ostats[1]
        assert abs(st[3] - ostats[3]) < 1e-3 * ostats[3]


def test_33_qubits_c128_norm_pt_and_inverse():
    n, g = qs.qs_supremacy_circuit(3, 11, 25, 3)
    assert n == 33
    h = qs.qs_alloc(n, qs.QS_C128)
    try:
        qs.qs_init_basis(h, 0)
        run(h, n, g)
        st = qs.qs_stats(h)
        assert abs(st[0] - 1) < 1e-13
        assert 1.8 < st[3] < 4.0          # 3x11 at depth 25 is further from Porter-Thomas
        run(h, n, inverse_gates(g))
        a0 = qs.qs_get_amplitudes_at(h, [0])[0]
        assert abs(abs(a0) ** 2 - 1) < 2e-12
        assert abs(qs.qs_norm(h) - 1) < 1e-12
    finally:
        qs.qs_free(h)


def test_34_qubits_c64_norm_pt_and_inverse():
    n, g = qs.qs_supremacy_circuit(5, 7, 25, 2, removed=[(4, 6)])
    assert n == 34
    h = qs.qs_alloc(n, qs.QS_C64)
    try:
        qs.qs_init_basis(h, 0)
        run(h, n, g)
        st = qs.qs_stats(h)
        assert abs(st[0] - 1) < 1e-5
        assert 1.8 < st[3] < 3.0
        run(h, n, inverse_gates(g))
        a0 = qs.qs_get_amplitudes_at(h, [0])[0]
        assert abs(abs(a0) ** 2 - 1) < 1e-4
    finally:
        qs.qs_free(h)


def test_sampling_32_qubits_uniform_c64():
    n, m, seed = 32, 4096, 2024
    h = qs.qs_alloc(n, qs.QS_C64)
    try:
        qs.qs_init_uniform(h)
        got = qs.qs_sample(h, seed, m)
    finally:
        qs.qs_free(h)
    want = np.array([(sim.splitmix64(seed, j) >> 11) >> (53 - n) for j in range(m)], dtype=np.uint64)
    assert np.array_equal(got, want)

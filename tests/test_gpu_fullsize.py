"""Full-size checks in the launch configuration bench.py times (fused schedules,
default kernel paths): properties that hold at any size, plus sampled
amplitudes compared between precisions.

* 30 qubits (5x6 grid, 25 CZ cycles), complex128: the circuit followed by its
  inverse returns |0...0> (|psi_0|^2 = 1 within 2e-12 and the norm within 1e-12,
  so every other amplitude is below 1e-6 in modulus and their squares sum
  below 2e-12); norm after the circuit within 1e-13.
* 32 qubits (4x8), complex64 against complex128 on 4096 sampled amplitudes
  (tolerance 2e-6); norm drift and Porter-Thomas moments of both.
* 34 qubits (5x7 minus a corner), complex64 only (128 GiB): norm drift and
  Porter-Thomas moments; circuit + inverse returns |0...0> within 1e-4.
* 32 qubits, complex64, uniform state (every p = 2^-32 exactly, so every CDF
  sum is exact and outcome j is floor(u_j 2^32), the rule the oracle is pinned
  to): 4096 samples bit for bit.  Above 30 qubits the super-block prefixes no
  longer fit the draw kernel's shared memory and are searched in device memory.
"""
import numpy as np
import pytest

import paper_1704_01127_gb300.qs as qs
from oracle import circuit as ocircuit
from oracle import sim

pytestmark = pytest.mark.gpu


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


def test_32_qubits_c64_against_c128_sampled():
    n, g = qs.qs_supremacy_circuit(4, 8, 25, 1)
    rng = np.random.Generator(np.random.PCG64(32))
    idx = np.concatenate([[0, (1 << n) - 1], rng.integers(0, 1 << n, 4094, dtype=np.uint64)])
    out = {}
    for dt in (qs.QS_C128, qs.QS_C64):
        h = qs.qs_alloc(n, dt)
        try:
            qs.qs_init_basis(h, 0)
            run(h, n, g)
            out[dt] = (qs.qs_get_amplitudes_at(h, idx), qs.qs_stats(h))
        finally:
            qs.qs_free(h)
    d = np.max(np.abs(out[qs.QS_C64][0] - out[qs.QS_C128][0]))
    assert d <= 2e-6
    assert abs(out[qs.QS_C128][1][0] - 1) < 1e-13 and abs(out[qs.QS_C64][1][0] - 1) < 1e-5
    for dt in out:
        assert 1.8 < out[dt][1][3] < 3.0


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

"""CUDA path against the oracle, element by element, through the C ABI.

Tolerances (absolute max |dpsi|): 1e-12 for complex128 and 2e-6 for complex64
(single sweeps are checked far tighter).  Integer outputs (samples) must match
bit for bit when both sides see the same amplitudes.
"""
import math

import numpy as np
import pytest

import paper_1704_01127_gb300.qs as qs
from inputs import random_state, random_unitary, random_diag, random_qubits, random_phase_poly
from oracle import sim, schedule, circuit

pytestmark = pytest.mark.gpu

TOL = {qs.QS_C128: 1e-12, qs.QS_C64: 2e-6}
SWEEP_TOL = {qs.QS_C128: 5e-14, qs.QS_C64: 3e-6}


def f32_round(psi):
    """The complex128 values a complex64 state holds after rounding."""
    return psi.astype(np.complex64).astype(np.complex128)


class State:
    def __init__(self, n, dtype):
        self.h = qs.qs_alloc(n, dtype)
        self.n, self.dtype = n, dtype

    def __enter__(self):
        return self

    def __exit__(self, *a):
        qs.qs_free(self.h)


def target_patterns(n, k):
    """Low, high, mixed and unsorted target sets for a k-qubit cluster."""
    pats = [list(range(k)), list(range(n - k, n)), list(reversed(range(k)))]
    if n >= k + 6:
        pats.append([0, 3, 5, n - 1, n - 2][:k])
        pats.append(random_qubits(n, k, 1000 + n * 7 + k))
        pats.append([5 + j for j in range(k)])
    return pats


@pytest.mark.parametrize("path", [qs.QS_PATH_AUTO, qs.QS_PATH_CUDA_CORES, qs.QS_PATH_TENSOR])
@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n", [5, 6, 9, 14, 17])
def test_apply_cluster(path, dtype, k, n):
    """Every kernel path (CUDA cores; tensor cores, smaller clusters embedded in
    5 qubits) on low, high, mixed and unsorted targets."""
    if k > n:
        pytest.skip("k > n")
    for t, qubits in enumerate(target_patterns(n, k)):
        U = random_unitary(k, 10 * n + k + t)
        psi = random_state(n, 7 * n + k + t)
        if dtype == qs.QS_C64:
            psi = f32_round(psi)
        ref = psi.copy()
        sim.apply_kq(ref, qubits, U)
        with State(n, dtype) as s:
            qs.qs_set_path(s.h, path)
            qs.qs_set_amplitudes(s.h, psi)
            qs.qs_apply_cluster(s.h, qubits, U)
            out = qs.qs_get_amplitudes(s.h)
        assert np.max(np.abs(out - ref)) < SWEEP_TOL[dtype], (qubits,)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_apply_cluster_n_equals_k(dtype):
    for k in range(1, 6):
        U = random_unitary(k, k)
        psi = f32_round(random_state(k, k + 50))
        ref = psi.copy()
        sim.apply_kq(ref, list(range(k))[::-1], U)
        with State(k, dtype) as s:
            qs.qs_set_amplitudes(s.h, psi)
            qs.qs_apply_cluster(s.h, list(range(k))[::-1], U)
            assert np.max(np.abs(qs.qs_get_amplitudes(s.h) - ref)) < SWEEP_TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("k", [1, 3, 7, 12])
def test_apply_diag(dtype, k):
    n = 14
    qubits = random_qubits(n, k, k)
    d = random_diag(k, k + 1)
    psi = f32_round(random_state(n, k + 2))
    ref = psi.copy()
    sim.apply_diag(ref, qubits, d)
    with State(n, dtype) as s:
        qs.qs_set_amplitudes(s.h, psi)
        qs.qs_apply_diag(s.h, qubits, d)
        assert np.max(np.abs(qs.qs_get_amplitudes(s.h) - ref)) < SWEEP_TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("n,n_edges", [(3, 2), (12, 0), (13, 9), (15, 20), (20, 60), (22, 100)])
def test_apply_phase(dtype, n, n_edges):
    coeff, edges = random_phase_poly(n, n_edges, n + n_edges)
    psi = f32_round(random_state(n, n))
    ref = psi.copy()
    sim.apply_phase(ref, coeff, edges)
    with State(n, dtype) as s:
        qs.qs_set_amplitudes(s.h, psi)
        qs.qs_apply_phase(s.h, coeff, edges)
        assert np.max(np.abs(qs.qs_get_amplitudes(s.h) - ref)) < SWEEP_TOL[dtype]


def run_lib(n, gates_arr, dtype, path=qs.QS_PATH_AUTO, **sched_kw):
    sc = qs.qs_schedule_build(n, gates_arr, **sched_kw)
    try:
        with State(n, dtype) as s:
            qs.qs_set_path(s.h, path)
            qs.qs_init_basis(s.h, 0)
            qs.qs_run_circuit(s.h, sc)
            return qs.qs_get_amplitudes(s.h), qs.qs_stats(s.h), qs.qs_probabilities(s.h)
    finally:
        qs.qs_schedule_free(sc)


def _run_from(n, g, dtype, x, lazy):
    """Run the fused schedule from |x>: lazily (qs_init_basis) or from the
    fully written basis vector (qs_set_amplitudes)."""
    sc = qs.qs_schedule_build(n, g, k_max=5)
    try:
        with State(n, dtype) as s:
            if lazy:
                qs.qs_init_basis(s.h, x)
            else:
                e = np.zeros(1 << n, dtype=np.complex128)
                e[x] = 1
                qs.qs_set_amplitudes(s.h, e)
            qs.qs_run_circuit(s.h, sc)
            return qs.qs_get_amplitudes(s.h)
    finally:
        qs.qs_schedule_free(sc)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("grid,x", [((4, 5), 0), ((4, 5), 0xB5A3), ((3, 7), 0x155555), ((4, 4), 7)])
def test_basis_start_on_the_support_is_bit_exact(dtype, grid, x):
    """Sweeps on the support after qs_init_basis give bit for bit the result of
    the same sweeps on the zero-filled basis vector, and match the oracle."""
    n, g = qs.qs_supremacy_circuit(grid[0], grid[1], 25, 2)
    x &= (1 << n) - 1
    lazy = _run_from(n, g, dtype, x, True)
    full = _run_from(n, g, dtype, x, False)
    assert np.array_equal(lazy, full)
    if dtype == qs.QS_C128:
        want = sim.run_circuit(n, qs.gates_to_tuples(g), psi=sim.basis_state(n, x))
        assert np.max(np.abs(lazy - want)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_basis_start_mixed_paths_match_oracle(dtype):
    """Tensor-core clusters on a growing support, then a CUDA-core cluster and a
    phase op (both write the zeros first), then tensor-core clusters again."""
    n = 14
    ops = [((0, 1, 2, 3, 4), qs.QS_PATH_TENSOR), ((7, 9, 10, 11, 13), qs.QS_PATH_TENSOR),
           ((3, 12), qs.QS_PATH_TENSOR), ((2, 5, 6), qs.QS_PATH_CUDA_CORES),
           ((0, 6, 8, 12, 13), qs.QS_PATH_TENSOR), ((1, 4, 5, 9), qs.QS_PATH_TENSOR)]
    x = 0x2A5
    ref = np.zeros(1 << n, dtype=np.complex128)
    ref[x] = 1
    with State(n, dtype) as s:
        qs.qs_init_basis(s.h, x)
        for j, (qq, path) in enumerate(ops):
            U = random_unitary(len(qq), 90 + j)
            qs.qs_set_path(s.h, path)
            qs.qs_apply_cluster(s.h, qq, U)
            sim.apply_kq(ref, qq, U)
            if j == 3:
                coeff, edges = random_phase_poly(n, 10, 77)
                qs.qs_apply_phase(s.h, coeff, edges)
                sim.apply_phase(ref, coeff, edges)
        got = qs.qs_get_amplitudes(s.h)
    assert np.max(np.abs(got - ref)) <= 4 * SWEEP_TOL[dtype]


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_basis_start_every_reader_sees_the_zeros(dtype):
    n, x = 16, 0x9C3
    N = 1 << n
    e = np.zeros(N, dtype=np.complex128)
    e[x] = 1
    with State(n, dtype) as s:
        qs.qs_init_basis(s.h, x)
        st = qs.qs_stats(s.h)
        # entropy -1 ln 1: the float-float logarithm leaves an error of ~1e-18
        assert st[0] == 1 and abs(st[1]) <= 1e-14 and st[3] == N
    with State(n, dtype) as s:
        qs.qs_init_basis(s.h, x)
        assert np.array_equal(qs.qs_probabilities(s.h), np.abs(e) ** 2)
    with State(n, dtype) as s:
        qs.qs_init_basis(s.h, x)
        assert np.all(qs.qs_sample(s.h, 5, 64) == x)
    with State(n, dtype) as s:
        qs.qs_init_basis(s.h, x)
        got = qs.qs_get_amplitudes_at(s.h, np.array([x, 0, N - 1], dtype=np.uint64))
        assert np.array_equal(got, np.array([1, 0, 0], dtype=np.complex128))
        assert np.array_equal(qs.qs_get_amplitudes(s.h), e)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_drop_final_diagonal_keeps_the_distribution(dtype):
    """Leaving out the trailing diagonal ops (Sec. 3.6) changes phases only:
    moduli, probabilities and statistics are the full circuit's (oracle)."""
    n, g = qs.qs_supremacy_circuit(4, 5, 25, 3)
    ref = sim.run_circuit(n, qs.gates_to_tuples(g))
    # the greedy clustering of this circuit ends with a phase op
    sc = qs.qs_schedule_build(n, g, k_max=5, search_runs=1, search_first=1)
    try:
        last = qs.qs_schedule_op(sc, qs.qs_schedule_num_ops(sc) - 1)["kind"]
    finally:
        qs.qs_schedule_free(sc)
    assert last == "phase"
    psi, st, p = run_lib(n, g, dtype, k_max=5, drop_final_diagonal=True, search_runs=1, search_first=1)
    assert np.max(np.abs(np.abs(psi) - np.abs(ref))) <= TOL[dtype]
    assert np.max(np.abs(psi - ref)) > 1e-3           # the phases did change
    np.testing.assert_allclose(p, sim.probabilities(ref), rtol=0, atol=1e-13 if dtype == qs.QS_C128 else 1e-7)
    want = sim.stats(ref)
    for a, b in zip(st, want):
        assert abs(a - b) <= (1e-10 if dtype == qs.QS_C128 else 1e-4) * max(1.0, abs(b))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_config_4x4_depth10_plain_c128(seed):
    """16 qubits, depth 10, complex128, gate by gate: full state and probabilities."""
    n, g = qs.qs_supremacy_circuit(4, 4, 10, seed)
    ref = sim.run_circuit(n, qs.gates_to_tuples(g))
    psi, st, p = run_lib(n, g, qs.QS_C128, fuse=False)
    assert np.max(np.abs(psi - ref)) <= 1e-12
    np.testing.assert_allclose(p, sim.probabilities(ref), rtol=0, atol=1e-13)
    assert abs(st[0] - 1) < 1e-13


@pytest.mark.parametrize("path", [qs.QS_PATH_AUTO, qs.QS_PATH_CUDA_CORES])
@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("grid,depth,k_max", [((4, 4), 10, 5), ((4, 5), 25, 4), ((4, 5), 25, 5),
                                              ((3, 6), 25, 3), ((2, 3), 12, 5)])
def test_fused_circuit_matches_oracle(path, dtype, grid, depth, k_max):
    n, g = qs.qs_supremacy_circuit(grid[0], grid[1], depth, 3)
    ref = sim.run_circuit(n, qs.gates_to_tuples(g))
    psi, st, p = run_lib(n, g, dtype, path=path, k_max=k_max)
    assert np.max(np.abs(psi - ref)) <= TOL[dtype]
    assert abs(st[0] - 1) < (1e-13 if dtype == qs.QS_C128 else 1e-5)


def test_stats_match_oracle():
    n, g = qs.qs_supremacy_circuit(4, 5, 25, 1)
    ref = sim.run_circuit(n, qs.gates_to_tuples(g))
    _, st, _ = run_lib(n, g, qs.QS_C128, k_max=5)
    want = sim.stats(ref)
    for a, b in zip(st, want):
        assert abs(a - b) <= 1e-10 * max(1.0, abs(b))


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("n", [2, 7, 10, 16, 21])
def test_sampling_bit_exact(dtype, n):
    """Same amplitudes on both sides -> the same outcomes, bit for bit."""
    psi = f32_round(random_state(n, 40 + n)) if dtype == qs.QS_C64 else random_state(n, 40 + n)
    m = 4096
    with State(n, dtype) as s:
        qs.qs_set_amplitudes(s.h, psi)
        got = qs.qs_sample(s.h, 12345 + n, m)
    want = sim.sample(psi, 12345 + n, m)
    assert np.array_equal(got, want)


def test_c64_probabilities_and_draws_over_every_exponent():
    """complex64 probabilities build each square from integers (exact, as the
    FP64 product of the float with itself) and add the two in FP64: bit for bit
    the FP64 result for floats of every exponent, signed zeros, the smallest
    and largest subnormals, the smallest normal and the largest finite float;
    draws from that state are the oracle's."""
    n = 12
    g = np.random.default_rng(77)
    bits = g.integers(0, 1 << 32, size=2 << n, dtype=np.uint64).astype(np.uint32)
    bits[(bits >> 23 & 0xFF) == 0xFF] &= 0x807FFFFF                 # no inf / nan: exponent 0 instead
    special = np.array([0.0, -0.0, 1e-45, -1e-45, 1.1754942e-38, 1.1754944e-38, 1.0, -1.0,
                        0.99999994, 3.4028235e38, -3.4028235e38, 2.0 ** -75, 0.5, 1e-20], dtype=np.float32)
    bits[:special.size] = special.view(np.uint32)
    f = bits.view(np.float32).astype(np.float64)
    psi = f[0::2] + 1j * f[1::2]
    want = f[0::2] * f[0::2] + f[1::2] * f[1::2]
    with State(n, qs.QS_C64) as s:
        qs.qs_set_amplitudes(s.h, psi)
        got = qs.qs_probabilities(s.h)
    assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
    # the same values normalised (in FP64, then rounded to complex64) for the draws
    psi = f32_round(psi / np.sqrt(np.sum(want)))
    with State(n, qs.QS_C64) as s:
        qs.qs_set_amplitudes(s.h, psi)
        got = qs.qs_sample(s.h, 99, 4096)
    assert np.array_equal(got, sim.sample(psi, 99, 4096))


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("n", [8, 12, 21])
def test_sample_stats_in_one_pass(dtype, n):
    """qs_sample_stats: the draws of qs_sample (and of the oracle) bit for bit;
    the statistics of qs_stats up to the order of the float-float sums, and the
    oracle's.  n = 8 has blocks shorter than 1024 (statistics in their own
    pass), n = 12 one block of 1024 per warp and a single thread block, n = 21
    many thread blocks."""
    psi = f32_round(random_state(n, 60 + n)) if dtype == qs.QS_C64 else random_state(n, 60 + n)
    m = 4096
    with State(n, dtype) as s:
        qs.qs_set_amplitudes(s.h, psi)
        draws, st = qs.qs_sample_stats(s.h, 555 + n, m)
        alone = qs.qs_sample(s.h, 555 + n, m)
        st_alone = qs.qs_stats(s.h)
        assert qs.qs_sample_stats(s.h, 1, 0)[0].size == 0
    assert np.array_equal(draws, alone)
    assert np.array_equal(draws, sim.sample(psi, 555 + n, m))
    # complex64 statistics form p, p^2 and p ln p in FP32 (relative 1e-7)
    tol_oracle = 1e-10 if dtype == qs.QS_C128 else 1e-6
    for a, b, c in zip(st, st_alone, sim.stats(psi)):
        assert abs(a - b) <= 1e-13 * max(1.0, abs(b))
        assert abs(a - c) <= tol_oracle * max(1.0, abs(c))


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_empty_inputs(dtype):
    """Degenerate calls: a schedule without ops leaves the state as it is (bit
    for bit), and zero draws return an empty array."""
    n = 9
    psi = f32_round(random_state(n, 3)) if dtype == qs.QS_C64 else random_state(n, 3)
    sc = qs.qs_schedule_from_ops(n, [])
    try:
        with State(n, dtype) as s:
            qs.qs_set_amplitudes(s.h, psi)
            qs.qs_run_circuit(s.h, sc)
            assert np.array_equal(qs.qs_get_amplitudes(s.h), psi)
            assert qs.qs_sample(s.h, 1, 0).size == 0
    finally:
        qs.qs_schedule_free(sc)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_bounded_wait_expiry_is_reported(dtype):
    """A bounded mbarrier wait that nothing completes reports QS_ETIMEOUT once;
    the word is cleared and the state keeps working (a cluster then matches
    the oracle).  No fault or hang is involved."""
    n = 10
    psi = f32_round(random_state(n, 8)) if dtype == qs.QS_C64 else random_state(n, 8)
    U = random_unitary(5, 9)
    ref = psi.copy()
    sim.apply_kq(ref, [1, 3, 4, 7, 9], U)
    with State(n, dtype) as s:
        assert qs.qs_selftest_timeout(s.h) == qs.QS_ETIMEOUT
        qs.qs_synchronize(s.h)                       # cleared: no error now
        qs.qs_set_amplitudes(s.h, psi)
        qs.qs_set_path(s.h, qs.QS_PATH_TENSOR)
        qs.qs_apply_cluster(s.h, [1, 3, 4, 7, 9], U)
        qs.qs_synchronize(s.h)
        got = qs.qs_get_amplitudes(s.h)
    assert np.max(np.abs(got - ref)) <= SWEEP_TOL[dtype]


def test_init_states():
    for n in (1, 7, 15):
        with State(n, qs.QS_C128) as s:
            qs.qs_init_uniform(s.h)
            psi = qs.qs_get_amplitudes(s.h)
            np.testing.assert_allclose(psi.real, 2.0 ** (-n / 2), rtol=1e-15)
            qs.qs_init_basis(s.h, (1 << n) - 1)
            psi = qs.qs_get_amplitudes(s.h)
            assert psi[-1] == 1 and np.count_nonzero(psi) == 1


SWAP_CASES = [
    (12, [(0, 5)]), (12, [(2, 9), (3, 10), (4, 11)]), (12, [(0, 1), (7, 3)]), (14, [(13, 0), (1, 12), (2, 4)]),
    (20, [(5, 19), (8, 12)]), (20, [(0, 19), (1, 18), (2, 17), (3, 16), (4, 15)]), (9, [(0, 8), (1, 7), (2, 6)]),
    (22, [(2, 21), (3, 20), (4, 19)]), (6, [(0, 5), (1, 4), (2, 3)]), (16, [(3, 4)]), (16, []),
]


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("n,pairs", SWAP_CASES)
def test_swap_qubits_bit_exact(dtype, n, pairs):
    """Qubit exchanges (the tiled kernel when a swapped qubit is below 3, the
    pairwise one otherwise) move amplitudes bit for bit as the oracle's
    permutation does."""
    psi = f32_round(random_state(n, 500 + n + len(pairs)))
    ref = psi.copy()
    a, b = [x for x, _ in pairs], [y for _, y in pairs]
    sim.apply_swap(ref, a, b)
    with State(n, dtype) as s:
        qs.qs_set_amplitudes(s.h, psi)
        qs.qs_swap_qubits(s.h, a, b)
        assert np.array_equal(qs.qs_get_amplitudes(s.h), ref)


def test_swap_qubits_after_basis_start_and_errors():
    """After qs_init_basis the zeros outside the support are written first; bad
    arguments are rejected."""
    with State(10, qs.QS_C128) as s:
        qs.qs_init_basis(s.h, 0b0000000101)
        qs.qs_swap_qubits(s.h, [0, 2], [9, 8])
        out = qs.qs_get_amplitudes(s.h)
        assert out[0b1100000000] == 1 and np.count_nonzero(out) == 1
        for a, b in (([0], [0]), ([0, 1], [2, 1]), ([10], [1]), ([-1], [2])):
            with pytest.raises(qs.QSError) as e:
                qs.qs_swap_qubits(s.h, a, b)
            assert e.value.code == qs.QS_EINVAL


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_schedule_uploaded_ahead_from_another_thread(dtype):
    """qs_schedule_upload in a second host thread while the first runs another
    circuit; the uploaded schedule then runs to the oracle's state."""
    import threading
    n, g = qs.qs_supremacy_circuit(4, 5, 20, 11)
    n2, g2 = qs.qs_supremacy_circuit(4, 5, 20, 12)
    ref = sim.run_circuit(n2, qs.gates_to_tuples(g2))
    sc1 = qs.qs_schedule_build(n, g, k_max=5)
    sc2 = qs.qs_schedule_build(n2, g2, k_max=5)
    try:
        with State(n, dtype) as s:
            qs.qs_init_basis(s.h, 0)
            err = []

            def up():
                try:
                    qs.qs_schedule_upload(sc2, dtype)
                    qs.qs_schedule_upload(sc2, dtype)      # a second call keeps the image
                except Exception as e:                     # reported below
                    err.append(e)
            th = threading.Thread(target=up)
            th.start()
            qs.qs_run_circuit(s.h, sc1)
            th.join()
            assert not err
            qs.qs_init_basis(s.h, 0)
            qs.qs_run_circuit(s.h, sc2)
            out = qs.qs_get_amplitudes(s.h)
        assert np.max(np.abs(out - ref)) <= TOL[dtype]
        with pytest.raises(qs.QSError) as e:
            qs.qs_schedule_upload(sc2, 5)
        assert e.value.code == qs.QS_EINVAL
    finally:
        qs.qs_schedule_free(sc1)
        qs.qs_schedule_free(sc2)


def test_errors_leave_gpu_usable():
    with State(8, qs.QS_C128) as s:
        for bad in ([0, 0], [8], [-1], list(range(6))):
            with pytest.raises(qs.QSError) as e:
                qs.qs_apply_cluster(s.h, bad, np.eye(1 << len(bad)))
            assert e.value.code == qs.QS_EINVAL
        with pytest.raises(qs.QSError):
            qs.qs_init_basis(s.h, 256)
        with pytest.raises(qs.QSError):
            qs.qs_apply_phase(s.h, np.zeros(8), [(3, 3)])
        qs.qs_init_basis(s.h, 3)
        assert abs(qs.qs_norm(s.h) - 1) == 0
    with pytest.raises(qs.QSError) as e:
        qs.qs_alloc(40, qs.QS_C128)
    assert e.value.code == qs.QS_EINVAL


def test_device_allocation_beyond_free_memory_is_enomem():
    """2^36 complex128 amplitudes (1 TiB) exceed the GPU's memory: QS_ENOMEM,
    and the device stays usable (a cluster sweep still matches the oracle)."""
    with pytest.raises(qs.QSError) as e:
        qs.qs_alloc(36, qs.QS_C128)
    assert e.value.code == qs.QS_ENOMEM
    U = random_unitary(3, 5)
    psi = random_state(12, 6)
    ref = psi.copy()
    sim.apply_kq(ref, [1, 7, 4], U)
    with State(12, qs.QS_C128) as s:
        qs.qs_set_amplitudes(s.h, psi)
        qs.qs_apply_cluster(s.h, [1, 7, 4], U)
        assert np.max(np.abs(qs.qs_get_amplitudes(s.h) - ref)) < SWEEP_TOL[qs.QS_C128]


@pytest.mark.parametrize("path", [qs.QS_PATH_CUDA_CORES, qs.QS_PATH_TENSOR])
def test_stream_switch_between_queued_sweeps(path):
    """Sweeps queued on one stream, then on another after qs_set_stream: the
    second stream starts after the first one's work, so the state equals the
    oracle's (without that ordering the two streams' sweeps and staged
    matrices would overlap)."""
    torch = pytest.importorskip("torch")
    n = 22
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    ops = [(random_qubits(n, 5, 300 + i), random_unitary(5, 400 + i)) for i in range(8)]
    psi = random_state(n, 17)
    ref = psi.copy()
    for q, U in ops:
        sim.apply_kq(ref, q, U)
    h = qs.qs_alloc(n, qs.QS_C128, s1)
    try:
        qs.qs_set_path(h, path)
        qs.qs_set_amplitudes(h, psi)
        for q, U in ops[:4]:
            qs.qs_apply_cluster(h, q, U)
        qs.qs_set_stream(h, s2)
        for q, U in ops[4:]:
            qs.qs_apply_cluster(h, q, U)
        out = qs.qs_get_amplitudes(h)
    finally:
        qs.qs_free(h)
    assert np.max(np.abs(out - ref)) < 1e-12


def test_wrapped_buffer_basis_start_is_written_in_full():
    """The caller can read a wrapped buffer directly, so qs_init_basis writes
    every amplitude of it at once (no deferred zeros)."""
    torch = pytest.importorskip("torch")
    n = 12
    buf = torch.ones(2 << n, dtype=torch.float64, device="cuda")
    h = qs.qs_wrap(buf, n, qs.QS_C128, torch.cuda.current_stream())
    try:
        qs.qs_init_basis(h, 37)
        qs.qs_synchronize(h)
        got = buf.cpu().numpy().view(np.complex128)
    finally:
        qs.qs_free(h)
    want = np.zeros(1 << n, dtype=np.complex128)
    want[37] = 1
    assert np.array_equal(got, want)


def test_wrap_torch_tensor():
    torch = pytest.importorskip("torch")
    n = 12
    buf = torch.zeros(2 << n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    h = qs.qs_wrap(buf, n, qs.QS_C128, stream)
    try:
        qs.qs_init_uniform(h)
        U = random_unitary(2, 3)
        qs.qs_apply_cluster(h, [0, 11], U)
        qs.qs_synchronize(h)
        got = buf.cpu().numpy().view(np.complex128)
    finally:
        qs.qs_free(h)
    ref = sim.uniform_state(n)
    sim.apply_kq(ref, [0, 11], U)
    assert np.max(np.abs(got - ref)) < 1e-15


def test_tc_c64_qubit0_paired():
    """complex64 tensor-core sweeps with qubit 0 as a target move amplitude
    pairs with 16-byte accesses (qs_wrap only adopts 16-byte aligned buffers):
    a 5-qubit and an embedded 4-qubit cluster on a wrapped buffer match the
    oracle, and a buffer 8 bytes off the boundary is refused."""
    torch = pytest.importorskip("torch")
    n = 13
    buf = torch.zeros((2 << n) + 2, dtype=torch.float32, device="cuda")
    psi0 = f32_round(random_state(n, 71))
    buf[: 2 << n] = torch.from_numpy(psi0.view(np.float64).astype(np.float32)).cuda()
    stream = torch.cuda.current_stream()
    with pytest.raises(qs.QSError) as e:
        qs.qs_wrap(buf.data_ptr() + 8, n, qs.QS_C64, stream)
    assert e.value.code == qs.QS_EINVAL
    h = qs.qs_wrap(buf.data_ptr(), n, qs.QS_C64, stream)
    ref = psi0.copy()
    try:
        qs.qs_set_path(h, qs.QS_PATH_TENSOR)
        for j, qq in enumerate([(0, 1, 2, 7, 11), (0, 4, 9, 12), (3, 0, 6, 10, 8)]):
            U = random_unitary(len(qq), 80 + j)
            qs.qs_apply_cluster(h, list(qq), U)
            sim.apply_kq(ref, list(qq), U)
        got = qs.qs_get_amplitudes(h)
    finally:
        qs.qs_free(h)
    assert np.max(np.abs(got - ref)) <= 3 * SWEEP_TOL[qs.QS_C64]


@pytest.mark.parametrize("targets", [(0, 1, 2, 8, 9), (2, 3, 4, 10, 11), (0, 1, 2, 3, 4), (1, 9, 10, 13, 15),
                                     (0, 5, 6, 10, 11), (3, 4, 5, 12, 13), (0, 4, 9, 12)])
def test_tc_c64_low_targets(targets):
    """complex64 tensor-core sweeps on low targets (a warp's rows far apart in
    memory, member pairs on qubit 0): on a dense state they match the oracle;
    from a basis state, the cluster on the one-amplitude support (layout with
    fixed bits) and on the zero-filled state (full layout) agree bit for bit."""
    n = 16
    U = random_unitary(len(targets), sum(targets))
    psi = f32_round(random_state(n, 5 + sum(targets)))
    ref = psi.copy()
    sim.apply_kq(ref, list(targets), U)
    with State(n, qs.QS_C64) as s:
        qs.qs_set_amplitudes(s.h, psi)
        qs.qs_apply_cluster(s.h, list(targets), U)
        got = qs.qs_get_amplitudes(s.h)
    assert np.max(np.abs(got - ref)) <= SWEEP_TOL[qs.QS_C64]
    x = 0x2D6B
    e = np.zeros(1 << n, dtype=np.complex128)
    e[x] = 1
    with State(n, qs.QS_C64) as s:
        qs.qs_init_basis(s.h, x)
        qs.qs_apply_cluster(s.h, list(targets), U)
        lazy = qs.qs_get_amplitudes(s.h)
    with State(n, qs.QS_C64) as s:
        qs.qs_set_amplitudes(s.h, e)
        qs.qs_apply_cluster(s.h, list(targets), U)
        full = qs.qs_get_amplitudes(s.h)
    assert np.array_equal(lazy, full)


# ------------------------------------------------ tensor-core 5-qubit sweep (c64)

@pytest.mark.parametrize("n", [5, 8, 11, 12, 13, 16, 19])
def test_tc_cluster_c64_matches_oracle(n):
    """Tensor-core path (tf32 head/tail split, FP32 accumulation) on every target
    pattern, from a single group (n = 5) through ragged and full 128-group tiles."""
    for t, qubits in enumerate(target_patterns(n, 5)):
        U = random_unitary(5, 300 + 10 * n + t)
        psi = f32_round(random_state(n, 400 + n + t))
        ref = psi.copy()
        sim.apply_kq(ref, qubits, U)
        out = {}
        for path in (qs.QS_PATH_TENSOR, qs.QS_PATH_CUDA_CORES):
            with State(n, qs.QS_C64) as s:
                qs.qs_set_path(s.h, path)
                qs.qs_set_amplitudes(s.h, psi)
                qs.qs_apply_cluster(s.h, qubits, U)
                out[path] = qs.qs_get_amplitudes(s.h)
        scale = np.max(np.abs(psi))
        assert np.max(np.abs(out[qs.QS_PATH_TENSOR] - ref)) < 2e-6 * max(scale, 1e-3) * 8, qubits
        assert np.max(np.abs(out[qs.QS_PATH_CUDA_CORES] - ref)) < SWEEP_TOL[qs.QS_C64]


def test_tc_fused_circuit_c64():
    n, g = qs.qs_supremacy_circuit(4, 5, 25, 7)
    ref = sim.run_circuit(n, qs.gates_to_tuples(g))
    sc = qs.qs_schedule_build(n, g, k_max=5)
    try:
        with State(n, qs.QS_C64) as s:
            qs.qs_set_path(s.h, qs.QS_PATH_TENSOR)
            qs.qs_init_basis(s.h, 0)
            qs.qs_run_circuit(s.h, sc)
            psi = qs.qs_get_amplitudes(s.h)
    finally:
        qs.qs_schedule_free(sc)
    assert np.max(np.abs(psi - ref)) <= 2e-6


@pytest.mark.parametrize("n", [5, 9, 12, 13, 17])
def test_tc_cluster_c128_matches_oracle(n):
    """complex128 on the tensor cores (exact integer digit planes): one sweep
    stays within 1e-14 of the FP64 oracle on every target pattern."""
    for t, qubits in enumerate(target_patterns(n, 5)):
        U = random_unitary(5, 500 + 10 * n + t)
        psi = random_state(n, 600 + n + t)
        ref = psi.copy()
        sim.apply_kq(ref, qubits, U)
        with State(n, qs.QS_C128) as s:
            qs.qs_set_path(s.h, qs.QS_PATH_TENSOR)
            qs.qs_set_amplitudes(s.h, psi)
            qs.qs_apply_cluster(s.h, qubits, U)
            out = qs.qs_get_amplitudes(s.h)
        assert np.max(np.abs(out - ref)) < SWEEP_TOL[qs.QS_C128], qubits


def test_tc_c128_zero_and_tiny_rows():
    """Rows of zeros and rows spanning many binades survive the digit split."""
    n = 12
    psi = random_state(n, 9)
    psi[: 1 << 9] = 0
    psi[1 << 10: 1 << 11] *= 1e-9
    U = random_unitary(5, 17)
    ref = psi.copy()
    sim.apply_kq(ref, [0, 1, 2, 3, 4], U)
    with State(n, qs.QS_C128) as s:
        qs.qs_set_path(s.h, qs.QS_PATH_TENSOR)
        qs.qs_set_amplitudes(s.h, psi)
        qs.qs_apply_cluster(s.h, [0, 1, 2, 3, 4], U)
        out = qs.qs_get_amplitudes(s.h)
    assert np.max(np.abs(out - ref)) < 1e-15
    assert np.all(out[: 1 << 9] == 0)


@pytest.mark.parametrize("targets", [[8, 9, 10, 11, 12], [0, 1, 2, 3, 4], [2, 5, 7, 10, 12]])
def test_tc_c128_fixed_point_paths(targets):
    """Members far below their row's largest value (the fixed point's general
    path, gaps past 2^25 and 2^60), exact rounding ties, zeros and subnormal
    inputs, and a state whose every row lies below 2^-998 (the general path
    for whole rows, results down in the subnormal range): one sweep against
    the FP64 oracle within 2^-44 of the largest input magnitude (the split
    keeps 47 bits below each row's top), or 2^-1000 for rows below ~2^-970,
    whose scale is raised so that no result leaves the normal double range."""
    n = 13
    g = np.random.Generator(np.random.PCG64(sum(targets)))
    u = g.integers(0, 71, 1 << n)
    psi = np.ldexp(1.0, -u) * np.exp(1j * g.uniform(0, 2 * np.pi, 1 << n))
    # rows led by 1.0 with ties of the 2^45 fixed point: (2k + 1) 2^-46
    lead = g.choice(1 << n, 64, replace=False)
    psi[lead] = 1.0
    ties = g.choice(1 << n, 512, replace=False)
    psi[ties] = (2 * g.integers(0, 8, 512) + 1) * 2.0 ** -46 * np.where(g.random(512) < 0.5, -1, 1)
    psi[g.choice(1 << n, 256, replace=False)] = 0
    psi[g.choice(1 << n, 64, replace=False)] = 1e-310
    U = random_unitary(5, 31 + targets[0])
    tiny = random_state(n, 41) * 1e-301
    for state in (psi, tiny):
        ref = state.copy()
        sim.apply_kq(ref, targets, U)
        with State(n, qs.QS_C128) as s:
            qs.qs_set_path(s.h, qs.QS_PATH_TENSOR)
            qs.qs_set_amplitudes(s.h, state)
            qs.qs_apply_cluster(s.h, targets, U)
            out = qs.qs_get_amplitudes(s.h)
        assert np.max(np.abs(out - ref)) <= max(2.0 ** -44 * np.max(np.abs(state)), 2.0 ** -1000), targets
        assert np.all(np.isfinite(out))


@pytest.mark.parametrize("x, clusters", [
    # the support after |x> grows by the qubits a cluster touches first: 5 new
    # (1 member of 32 in the support), then 1 (qubit 0, every other member),
    # 2, 3 (members scattered over the group), 4, and an embedded 3-qubit
    # cluster whose padding qubits lie outside the support
    (0x2D6B, [(3, 7, 9, 12, 14), (0, 3, 7, 9, 12), (1, 9, 12, 14, 15), (0, 2, 5, 6, 7),
              (4, 8, 10, 11, 15), (1, 13, 2), (13, 14, 15, 0, 1)]),
    (0, [(11, 12, 13, 14, 15), (6, 11, 12, 13, 14), (4, 5, 6, 7, 8), (0, 1, 2, 3, 4)]),
    (0xFFFF, [(0, 1, 2, 3, 4), (2, 3, 4, 5, 6), (5, 6, 7, 8, 9), (9, 10, 14), (11, 12, 13, 15, 0)]),
])
def test_tc_c128_support_growth_is_bit_exact(x, clusters):
    """complex128 sweeps that widen the support after qs_init_basis: only the
    members inside the support are split (compacted to the first K positions,
    the unitary's K positions permuted to match) and fewer K steps are
    issued.  Every accumulator sum is an exact integer, so the result equals
    bit for bit the same sweeps on the zero-filled basis vector (every member
    read); both match the oracle."""
    n = 16
    e = np.zeros(1 << n, dtype=np.complex128)
    e[x] = 1
    Us = [random_unitary(len(q), 70 + i) for i, q in enumerate(clusters)]
    ref = e.copy()
    for q, U in zip(clusters, Us):
        sim.apply_kq(ref, list(q), U)
    out = {}
    for lazy in (True, False):
        with State(n, qs.QS_C128) as s:
            qs.qs_set_path(s.h, qs.QS_PATH_TENSOR)
            if lazy:
                qs.qs_init_basis(s.h, x)
            else:
                qs.qs_set_amplitudes(s.h, e)
            for q, U in zip(clusters, Us):
                qs.qs_apply_cluster(s.h, list(q), U)
            out[lazy] = qs.qs_get_amplitudes(s.h)
    assert np.array_equal(out[True], out[False])
    assert np.max(np.abs(out[True] - ref)) < len(clusters) * SWEEP_TOL[qs.QS_C128]


def test_tc_c128_out_of_range_reported():
    """Amplitudes near 2^1016, whose results could pass the double range, are
    reported (QS_EINVAL at the next synchronising call, once) instead of
    returned as wrong numbers; the state then runs normal sweeps again."""
    n = 12
    U = random_unitary(5, 3)
    with State(n, qs.QS_C128) as s:
        qs.qs_set_path(s.h, qs.QS_PATH_TENSOR)
        qs.qs_set_amplitudes(s.h, random_state(n, 4) * 2.0 ** 1022)
        qs.qs_apply_cluster(s.h, [7, 8, 9, 10, 11], U)
        with pytest.raises(qs.QSError) as e:
            qs.qs_synchronize(s.h)
        assert e.value.code == qs.QS_EINVAL
        qs.qs_synchronize(s.h)
        psi = random_state(n, 5)
        ref = psi.copy()
        sim.apply_kq(ref, [7, 8, 9, 10, 11], U)
        qs.qs_set_amplitudes(s.h, psi)
        qs.qs_apply_cluster(s.h, [7, 8, 9, 10, 11], U)
        assert np.max(np.abs(qs.qs_get_amplitudes(s.h) - ref)) < SWEEP_TOL[qs.QS_C128]


def test_entropy_table_log_accuracy():
    """The table-driven logarithm of the entropy reduction against libm on
    probabilities spread over many binades (closed form: -sum p ln p)."""
    n = 14
    g = np.random.Generator(np.random.PCG64(5))
    mag = np.exp(g.uniform(-60, 0, 1 << n))
    psi = (mag * np.exp(1j * g.uniform(0, 6.3, 1 << n))).astype(np.complex128)
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2))
    p = np.abs(psi) ** 2
    want = -np.sum(p[p > 0] * np.log(p[p > 0]))
    with State(n, qs.QS_C128) as s:
        qs.qs_set_amplitudes(s.h, psi)
        got = qs.qs_stats(s.h)[1]
    assert abs(got - want) <= 1e-13 * max(1.0, abs(want))


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_remapped_schedule_against_oracle(dtype):
    """A schedule with its qubits moved to other index bits (Sec. 3.6): run from
    |0...0> (the basis amplitude is only relabelled), then read in every way.
    Indices and qubits given by the caller are translated; sampling, whole-state
    reads and probabilities first move the qubits back (one exchange sweep)."""
    n, g = qs.qs_supremacy_circuit(4, 5, 16, 21)
    ref = sim.run_circuit(n, qs.gates_to_tuples(g))
    sc = qs.qs_schedule_build(n, g, k_max=5)
    loc = np.arange(n)
    loc[[0, 17, 2, 12, 4, 19]] = [17, 0, 12, 2, 19, 4]
    qs.qs_schedule_remap(sc, loc)
    idx = np.array([0, 1, 5, 77, 1 << 17, (1 << n) - 1, 123457], dtype=np.uint64)
    try:
        with State(n, dtype) as s:
            qs.qs_init_basis(s.h, 0)
            qs.qs_run_circuit(s.h, sc)
            got = qs.qs_get_amplitudes_at(s.h, idx)
            assert np.max(np.abs(got - ref[idx.astype(np.int64)])) <= TOL[dtype]
            st = qs.qs_stats(s.h)
            assert abs(st[0] - 1) < (1e-13 if dtype == qs.QS_C128 else 1e-5)
            if dtype == qs.QS_C128:
                assert np.array_equal(qs.qs_sample(s.h, 99, 2000), sim.sample(ref, 99, 2000))
            out = qs.qs_get_amplitudes(s.h)
            assert np.max(np.abs(out - ref)) <= TOL[dtype]
            # a second run on a state that is not a basis state: exchange sweeps
            qs.qs_run_circuit(s.h, sc)
            ref2 = ref.copy()
            for (_, name, q) in qs.gates_to_tuples(g):
                sim.apply_gate(ref2, name, q)
            U = random_unitary(3, 8)
            qs.qs_apply_cluster(s.h, [0, 17, 6], U)        # qubits named as the caller knows them
            sim.apply_kq(ref2, [0, 17, 6], U)
            out = qs.qs_get_amplitudes(s.h)
            assert np.max(np.abs(out - ref2)) <= 2 * TOL[dtype]
    finally:
        qs.qs_schedule_free(sc)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_remapped_fullsize_against_oracle(dtype):
    """30 qubits with the library's choice of bit locations: the oracle's stored
    amplitudes through translated indices."""
    import os
    from conftest import GOLDEN, read_golden
    name = "fullsize_5x6_d25_s0.txt"
    if not os.path.exists(os.path.join(GOLDEN, name)):
        pytest.skip("golden file missing")
    rows = read_golden(name)
    idx = np.array([int(r[0]) for r in rows[2:]], dtype=np.uint64)
    want = np.array([complex(float(r[1]), float(r[2])) for r in rows[2:]])
    n, g = qs.qs_supremacy_circuit(5, 6, 25, 0)
    sc = qs.qs_schedule_build(n, g, k_max=5)
    try:
        loc = qs.qs_schedule_choose_remap(sc, dtype)
        assert not np.array_equal(loc, np.arange(n))
        qs.qs_schedule_remap(sc, loc)
        with State(n, dtype) as s:
            qs.qs_init_basis(s.h, 0)
            qs.qs_run_circuit(s.h, sc)
            got = qs.qs_get_amplitudes_at(s.h, idx)
    finally:
        qs.qs_schedule_free(sc)
    assert np.max(np.abs(got - want)) <= TOL[dtype]


PAIR_CASES = [
    (12, [0, 1, 2, 3, 4], [5, 6, 7, 8, 9]), (12, [7, 8, 9, 10, 11], [7, 8, 9, 10, 11]),
    (13, [0, 3, 6, 8, 9], [1, 2, 4, 5, 7]), (16, [2, 5, 9, 12, 13], [2, 5, 6, 7, 13]),
    (16, [11, 12, 13, 14, 15], [0, 1, 2, 12, 15]), (20, [15, 16, 17, 18, 19], [10, 11, 12, 18, 19]),
    (20, [0, 1, 2, 3, 19], [0, 4, 5, 6, 19]),
]


@pytest.mark.parametrize("n,q1,q2", PAIR_CASES)
def test_pair_sweep_matches_separate_sweeps_and_oracle(n, q1, q2):
    """Two consecutive 5-qubit complex64 clusters in one sweep (qs_pair.cu):
    bit for bit the two separate tensor-core sweeps, and within a sweep's
    rounding of the oracle; with a phase op after them folded into the pair."""
    U1, U2 = random_unitary(5, 600 + n), random_unitary(5, 700 + n)
    coeff, edges = random_phase_poly(n, 6, 800 + n)
    coeff = 2 * (np.asarray(coeff) // 2)            # even coefficients: the phase op folds
    psi = f32_round(random_state(n, 900 + n))
    for with_phase in (False, True):
        ops = [(qs.QS_OP_DENSE, q1, U1), (qs.QS_OP_DENSE, q2, U2)]
        if with_phase:
            ops.append((qs.QS_OP_PHASE, edges, coeff))
        sc = qs.qs_schedule_from_ops(n, ops)
        outs = []
        try:
            for pair in (True, False):
                with State(n, qs.QS_C64) as s:
                    qs.qs_set_pair_sweeps(s.h, pair)
                    qs.qs_set_amplitudes(s.h, psi)
                    ms = qs.qs_run_circuit_timed(s.h, sc)
                    outs.append(qs.qs_get_amplitudes(s.h))
                    if pair:
                        assert ms[0] > 0 and ms[1] == -1
        finally:
            qs.qs_schedule_free(sc)
        assert np.array_equal(outs[0], outs[1])
        ref = psi.copy()
        sim.apply_kq(ref, q1, U1)
        sim.apply_kq(ref, q2, U2)
        if with_phase:
            sim.apply_phase(ref, coeff, edges)
        assert np.max(np.abs(outs[0] - ref)) < 2 * SWEEP_TOL[qs.QS_C64]


def test_pair_sweeps_in_a_circuit_bit_exact():
    """A 24-qubit circuit (4x6 grid, 20 CZ cycles) with pair sweeps on and off: the same state bit for
    bit, within 2e-6 of the oracle."""
    n, g = qs.qs_supremacy_circuit(4, 6, 20, 5)
    ref = sim.run_circuit(n, qs.gates_to_tuples(g))
    sc = qs.qs_schedule_build(n, g, k_max=5)
    outs, paired = [], 0
    try:
        for pair in (True, False):
            with State(n, qs.QS_C64) as s:
                qs.qs_set_pair_sweeps(s.h, pair)
                qs.qs_init_basis(s.h, 0)
                ms = qs.qs_run_circuit_timed(s.h, sc)
                if pair:
                    paired = sum(1 for i in range(len(ms)) if ms[i] < 0 and qs.qs_schedule_op(sc, i)["kind"] == "dense")
                outs.append(qs.qs_get_amplitudes(s.h))
    finally:
        qs.qs_schedule_free(sc)
    assert paired >= 1
    assert np.array_equal(outs[0], outs[1])
    assert np.max(np.abs(outs[0] - ref)) <= 2e-6


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("g,uniform", [(3, False), (4, True)])
def test_staged_run_against_oracle(dtype, g, uniform):
    """Stages for a state held as 2^g parts (qs_plan_stages, Sec. 3.4/3.6) run
    in turn on one GPU: between stages the global and local qubits change
    places by exchange sweeps.  From |0...0> (the whole circuit) or from the
    uniform state (the circuit without its H layer, Sec. 3.6)."""
    n, gates = qs.qs_supremacy_circuit(4, 5, 20, 13)
    ref = sim.run_circuit(n, qs.gates_to_tuples(gates))
    body = gates[gates["cycle"] > 0] if uniform else gates
    stages, _ = qs.qs_plan_stages(n, body, g)
    try:
        assert len(stages) >= 2
        with State(n, dtype) as s:
            if uniform:
                qs.qs_init_uniform(s.h)
            else:
                qs.qs_init_basis(s.h, 0)
            for sc in stages:
                qs.qs_run_circuit(s.h, sc)
            out = qs.qs_get_amplitudes(s.h)
    finally:
        for sc in stages:
            qs.qs_schedule_free(sc)
    assert np.max(np.abs(out - ref)) <= TOL[dtype]


def test_staged_30_qubits_against_oracle():
    """30 qubits as 8 parts (3 global qubits), from the uniform state: the
    stored oracle amplitudes within 1e-12."""
    import os
    from conftest import GOLDEN, read_golden
    name = "fullsize_5x6_d25_s0.txt"
    if not os.path.exists(os.path.join(GOLDEN, name)):
        pytest.skip("golden file missing")
    rows = read_golden(name)
    idx = np.array([int(r[0]) for r in rows[2:]], dtype=np.uint64)
    want = np.array([complex(float(r[1]), float(r[2])) for r in rows[2:]])
    n, gates = qs.qs_supremacy_circuit(5, 6, 25, 0)
    stages, _ = qs.qs_plan_stages(n, gates[gates["cycle"] > 0], 3)
    try:
        with State(n, qs.QS_C128) as s:
            qs.qs_init_uniform(s.h)
            for sc in stages:
                qs.qs_run_circuit(s.h, sc)
            got = qs.qs_get_amplitudes_at(s.h, idx)
    finally:
        for sc in stages:
            qs.qs_schedule_free(sc)
    assert np.max(np.abs(got - want)) <= 1e-12

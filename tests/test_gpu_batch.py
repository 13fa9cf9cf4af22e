"""Batched persistent kernel: bit-exact against single-state CUDA-core runs of
the same schedules, within tolerance of the oracle, for every launch
configuration and through CUDA-graph replay."""
import numpy as np
import pytest

import paper_1704_01127_gb300.qs as qs
from oracle import sim

pytestmark = pytest.mark.gpu


def batch_circuits(seeds):
    out = []
    for s in seeds:
        r, c, d = qs.qs_batch_circuit_params(s)
        out.append(qs.qs_supremacy_circuit(r, c, d, s))
    return out


@pytest.fixture(scope="module")
def torch_stream():
    torch = pytest.importorskip("torch")
    return torch.cuda.Stream()


def single_run(n, sched, dtype):
    h = qs.qs_alloc(n, dtype)
    try:
        qs.qs_set_path(h, qs.QS_PATH_CUDA_CORES)
        qs.qs_init_basis(h, 0)
        qs.qs_run_circuit(h, sched)
        return qs.qs_get_amplitudes(h)
    finally:
        qs.qs_free(h)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("k_max", [3, 5])
def test_batch_bit_exact_vs_single_all_configs(dtype, k_max, torch_stream):
    circs = batch_circuits(range(6))
    scheds = [qs.qs_schedule_build(n, g, k_max=k_max) for (n, g) in circs]
    try:
        want = [single_run(n, sc, dtype) for (n, _), sc in zip(circs, scheds)]
        b = qs.qs_batch_create(scheds, dtype, torch_stream)
        try:
            for C in (1, 2, 4, 8):
                for T in (128, 256, 512):
                    qs.qs_batch_set_config(b, C, T)
                    qs.qs_batch_run(b)
                    for i, (n, _) in enumerate(circs):
                        got = qs.qs_batch_get_amplitudes(b, i, n)
                        assert np.array_equal(got, want[i]), (C, T, i)
        finally:
            qs.qs_batch_free(b)
    finally:
        for sc in scheds:
            qs.qs_schedule_free(sc)


def test_batch_graph_replay_and_stats(torch_stream):
    circs = batch_circuits(range(40, 56))
    scheds = [qs.qs_schedule_build(n, g, k_max=4) for (n, g) in circs]
    try:
        b = qs.qs_batch_create(scheds, qs.QS_C64, torch_stream)
        try:
            qs.qs_batch_set_config(b, 4, 256)
            qs.qs_batch_run(b)
            direct = [qs.qs_batch_get_amplitudes(b, i, n) for i, (n, _) in enumerate(circs)]
            for _ in range(3):
                qs.qs_batch_run_graph(b)
            st = qs.qs_batch_stats(b, len(circs))
            for i, (n, g) in enumerate(circs):
                got = qs.qs_batch_get_amplitudes(b, i, n)
                assert np.array_equal(got, direct[i])
                ref = sim.run_circuit(n, qs.gates_to_tuples(g))
                assert np.max(np.abs(got - ref)) <= 2e-6
                want = sim.stats(f32(got))
                assert abs(st[i][0] - want[0]) < 1e-12 and abs(st[i][3] - want[3]) < 1e-9 * want[3]
                assert abs(st[i][1] - want[1]) < 1e-10 * want[1]
        finally:
            qs.qs_batch_free(b)
    finally:
        for sc in scheds:
            qs.qs_schedule_free(sc)


def f32(psi):
    return psi.astype(np.complex64).astype(np.complex128)


def test_batch_tune_and_autotune(torch_stream):
    circs = batch_circuits(range(100, 132))
    scheds = [qs.qs_schedule_build(n, g, k_max=5) for (n, g) in circs]
    try:
        b = qs.qs_batch_create(scheds, qs.QS_C64, torch_stream)
        try:
            C, T, ms = qs.qs_batch_tune(b)
            assert C in (1, 2, 4, 8) and T in (128, 256, 512) and ms > 0
            assert qs.qs_batch_get_config(b) == (C, T)
        finally:
            qs.qs_batch_free(b)
    finally:
        for sc in scheds:
            qs.qs_schedule_free(sc)
    km, C, T, ms = qs.qs_batch_autotune(circs, qs.QS_C64, torch_stream)
    assert km in (3, 4, 5) and C in (1, 2, 4, 8) and T in (128, 256, 512) and ms > 0


def test_batch_rejects_bad_config(torch_stream):
    circs = batch_circuits([7])
    sc = qs.qs_schedule_build(circs[0][0], circs[0][1], k_max=5)
    try:
        b = qs.qs_batch_create([sc], qs.QS_C64, torch_stream)
        try:
            for C, T in ((3, 256), (2, 100), (16, 256)):
                with pytest.raises(qs.QSError):
                    qs.qs_batch_set_config(b, C, T)
        finally:
            qs.qs_batch_free(b)
    finally:
        qs.qs_schedule_free(sc)


def test_batch_512_circuits_autotuned_graph(torch_stream):
    """Config 4 at its stated size: all 512 circuits (seeds 0..511) in one
    persistent launch replayed from a CUDA graph with the autotuner's choice;
    every circuit's norm within 1e-5, and 23 circuits spread over the seeds
    (every grid) against the oracle within 2e-6."""
    circs = batch_circuits(range(512))
    km, C, T, _ = qs.qs_batch_autotune(circs, qs.QS_C64, torch_stream)
    scheds = [qs.qs_schedule_build(n, g, k_max=km, search_runs=1, search_first=1) for (n, g) in circs]
    try:
        b = qs.qs_batch_create(scheds, qs.QS_C64, torch_stream)
        try:
            qs.qs_batch_set_config(b, C, T)
            qs.qs_batch_run_graph(b)
            qs.qs_batch_run_graph(b)
            st = qs.qs_batch_stats(b, len(circs))
            assert np.max(np.abs(st[:, 0] - 1)) < 1e-5
            picked = list(range(0, 512, 23))
            assert {circs[i][0] for i in picked} == {16, 20, 21}
            for i in picked:
                n, g = circs[i]
                got = qs.qs_batch_get_amplitudes(b, i, n)
                ref = sim.run_circuit(n, qs.gates_to_tuples(g))
                assert np.max(np.abs(got - ref)) <= 2e-6, i
        finally:
            qs.qs_batch_free(b)
    finally:
        for sc in scheds:
            qs.qs_schedule_free(sc)

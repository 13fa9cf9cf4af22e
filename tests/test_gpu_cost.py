"""The learned cost model on the GPU: forward pass and gradients of the
library's FP64 MLP kernels against the CPU oracle, training, the timing
harness, the fitted model's fallback, and planned schedules against the
oracle."""
import numpy as np
import pytest

import paper_1704_01127_gb300.qs as qs
from oracle import mlp, sim

pytestmark = pytest.mark.gpu


@pytest.fixture
def net():
    h = qs.qs_mlp_create(11)
    yield h
    qs.qs_mlp_free(h)


def test_mlp_forward_and_gradient_match_oracle(net):
    g = np.random.Generator(np.random.PCG64(8))
    w = g.normal(0, 0.2, mlp.P)
    qs.qs_mlp_set_params(net, w)
    assert np.array_equal(qs.qs_mlp_get_params(net), w)
    X = g.normal(0, 1, (301, mlp.F))
    Y = g.normal(0, 1, 301)
    out = qs.qs_mlp_forward(net, X)
    want, _ = mlp.forward(w, X)
    np.testing.assert_allclose(out, want, rtol=1e-13, atol=1e-14)
    grad, loss = qs.qs_mlp_gradient(net, X, Y)
    ref = mlp.gradient(w, X, Y)
    assert abs(loss - mlp.loss(w, X, Y)) <= 1e-12 * mlp.loss(w, X, Y)
    np.testing.assert_allclose(grad, ref, rtol=1e-10, atol=1e-13)


def test_mlp_training_reduces_loss(net):
    g = np.random.Generator(np.random.PCG64(9))
    X = g.normal(0, 1, (2000, mlp.F))
    Y = np.sin(X[:, 0]) + 0.5 * X[:, 1] ** 2 - X[:, 2] * X[:, 3]
    w0 = qs.qs_mlp_get_params(net)
    before = mlp.loss(w0, X, Y)
    after = qs.qs_mlp_train(net, X, Y, epochs=800)
    assert after < 0.05 * before
    assert abs(after - mlp.loss(qs.qs_mlp_get_params(net), X, Y)) < 1e-9


def test_timing_harness_and_fit():
    feats, ms = qs.qs_cost_sample(10, 16, qs.QS_C64, 300, seed=1, max_ms=50)
    assert np.all(ms > 0) and feats.shape == (300, qs.QS_NFEAT)
    assert 0 < feats[:, 2].sum() < 150                      # some phase ops
    assert set(np.unique(feats[feats[:, 2] == 0, 4])) == {0.0, 1.0}   # both kernel paths timed
    cm = qs.qs_cost_model_create()
    try:
        rep = qs.qs_cost_model_fit(cm, feats, ms, epochs=400, seed=2)
        assert rep["mlp_holdout_median_abs_log_err"] > 0 and rep["analytic_holdout_median_abs_log_err"] > 0
        auto = qs.qs_cost_model_predict(cm, feats, qs.QS_COST_AUTO)
        an = qs.qs_cost_model_predict(cm, feats, qs.QS_COST_ANALYTIC)
        assert np.all(auto > 0) and np.all(an > 0)
        if not rep["use_mlp"]:
            assert np.array_equal(auto, an)
        # a feature vector outside the training range falls back to the analytic model
        far = qs.qs_op_features(30, qs.QS_C64, qs.QS_OP_DENSE, 5, (0, 1, 2, 3, 4), qs.QS_PATH_TENSOR)
        assert qs.qs_cost_model_predict(cm, far, qs.QS_COST_AUTO)[0] == qs.qs_cost_model_predict(
            cm, far, qs.QS_COST_ANALYTIC)[0]
    finally:
        qs.qs_cost_model_free(cm)


@pytest.fixture(scope="module")
def fitted():
    """A cost model fitted on 2400 measured timings of random ops on 20- to
    28-qubit states of both dtypes (the harness of config 5, smaller)."""
    F, T = [], []
    for dt in (qs.QS_C64, qs.QS_C128):
        f, t = qs.qs_cost_sample(20, 28, dt, 1200, seed=50 + dt, max_ms=100)
        F.append(f)
        T.append(t)
    F, T = np.concatenate(F), np.concatenate(T)
    cm = qs.qs_cost_model_create()
    rep = qs.qs_cost_model_fit(cm, F, T, epochs=1500, seed=3)
    yield cm, rep
    qs.qs_cost_model_free(cm)


def test_mlp_predicts_measured_times_better_than_analytic(fitted):
    """On held-out timings (every fifth, by a seeded hash) the fitted network's
    median |log error| is below the analytic bytes-over-bandwidth model's, so
    the fallback rule selects it."""
    cm, rep = fitted
    print("held-out median |log err|: mlp %.3f, analytic %.3f" % (
        rep["mlp_holdout_median_abs_log_err"], rep["analytic_holdout_median_abs_log_err"]))
    assert rep["mlp_holdout_median_abs_log_err"] < rep["analytic_holdout_median_abs_log_err"]
    assert rep["use_mlp"]


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_learned_plan_against_analytic_plan_measured(fitted, dtype):
    """What the trained network gains: one 28-qubit circuit (4x7 grid, 20 CZ
    cycles) planned with the learned model (auto fallback) and with the
    analytic model, both run and timed (CUDA events, best of 3).  The gain is
    printed; the plans' kernels are the same, so the bar is that the learned
    plan is no slower than the analytic one beyond 5% timing noise."""
    cm, _ = fitted
    n, g = qs.qs_supremacy_circuit(4, 7, 20, 0)
    h = qs.qs_alloc(n, dtype)
    res = {}
    try:
        for name, which in (("analytic", qs.QS_COST_ANALYTIC), ("learned", qs.QS_COST_AUTO)):
            sc, km, pred = qs.qs_plan_circuit(n, g, dtype, cm, which)
            try:
                best = None
                for _ in range(3):
                    qs.qs_init_basis(h, 0)
                    ms = qs.qs_run_circuit_timed(h, sc)
                    t = float(ms[ms >= 0].sum())
                    best = t if best is None else min(best, t)
                res[name] = (best, km, pred, qs.qs_schedule_num_ops(sc))
            finally:
                qs.qs_schedule_free(sc)
    finally:
        qs.qs_free(h)
    gain = res["analytic"][0] / res["learned"][0]
    print("dtype %d: analytic plan %.2f ms (k_max %d, %d ops), learned plan %.2f ms (k_max %d, %d ops): "
          "gain %.3fx" % (dtype, res["analytic"][0], res["analytic"][1], res["analytic"][3],
                          res["learned"][0], res["learned"][1], res["learned"][3], gain))
    assert gain > 1 / 1.05


@pytest.mark.parametrize("which", [qs.QS_COST_ANALYTIC, qs.QS_COST_AUTO])
@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_planned_schedule_matches_oracle(fitted, dtype, which):
    """Schedules planned with either model give the oracle's state (20 qubits)."""
    n, g = qs.qs_supremacy_circuit(4, 5, 25, 6)
    ref = sim.run_circuit(n, qs.gates_to_tuples(g))
    sc, km, t = qs.qs_plan_circuit(n, g, dtype, fitted[0], which)
    try:
        assert 2 <= km <= 5 and t > 0
        h = qs.qs_alloc(n, dtype)
        try:
            qs.qs_init_basis(h, 0)
            qs.qs_run_circuit(h, sc)
            psi = qs.qs_get_amplitudes(h)
        finally:
            qs.qs_free(h)
    finally:
        qs.qs_schedule_free(sc)
    assert np.max(np.abs(psi - ref)) <= (1e-12 if dtype == qs.QS_C128 else 2e-6)

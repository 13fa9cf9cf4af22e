"""Cost-model pieces that need no GPU: the MLP oracle against finite
differences, and the library's op features and analytic model against their
documented definitions."""
import math

import numpy as np
import pytest

import paper_1704_01127_gb300.qs as qs
from oracle import mlp


def test_mlp_oracle_gradient_matches_finite_differences():
    g = np.random.Generator(np.random.PCG64(3))
    w = g.normal(0, 0.3, mlp.P)
    X = g.normal(0, 1, (37, mlp.F))
    Y = g.normal(0, 1, 37)
    an = mlp.gradient(w, X, Y)
    idx = g.choice(mlp.P, 200, replace=False)
    for i in idx:
        h = 1e-6 * max(1.0, abs(w[i]))
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss(wp, X, Y) - mlp.loss(wm, X, Y)) / (2 * h)
        # central differences: truncation O(h^2), rounding ~1e-16 / h
        assert abs(fd - an[i]) <= 1e-7 * abs(an[i]) + 2e-9, i


def test_mlp_param_count():
    assert qs.qs_mlp_num_params() == mlp.P == 5057


def test_op_features_definition():
    f = qs.qs_op_features(30, qs.QS_C128, qs.QS_OP_DENSE, 3, (2, 9, 17), qs.QS_PATH_TENSOR)
    want = [30 / 32, 1, 0, 3 / 5, 1, 2 / 30, 17 / 30, 1 / 5, 1 / 3, (30 + 4) / 40, 0, 0]
    np.testing.assert_allclose(f, want, rtol=0, atol=1e-15)
    f = qs.qs_op_features(20, qs.QS_C64, qs.QS_OP_PHASE, n_act=7, odd=1)
    want = [20 / 32, 0, 1, 0, 0, 0, 0, 0, 0, (20 + 3) / 40, 7 / 20, 1]
    np.testing.assert_allclose(f, want, rtol=0, atol=1e-15)


def test_analytic_model_closed_forms():
    bw = 6696.8
    # complex64 sweep of 32 qubits on the tensor cores: 2 * 2^32 * 8 bytes / bw
    f = qs.qs_op_features(32, qs.QS_C64, qs.QS_OP_DENSE, 5, (0, 1, 2, 3, 4), qs.QS_PATH_TENSOR)
    assert abs(qs.qs_cost_analytic_ms(f, bw) - (2 * 2 ** 32 * 8 / (bw * 1e9) * 1e3 + 0.005)) < 1e-9
    # complex128 5-qubit sweep on FP64 CUDA cores: 2^30 (8*32 - 2) flops at 1.2 TFLOP/s
    f = qs.qs_op_features(30, qs.QS_C128, qs.QS_OP_DENSE, 5, (5, 6, 7, 8, 9), qs.QS_PATH_CUDA_CORES)
    assert abs(qs.qs_cost_analytic_ms(f, bw) - (2 ** 30 * 254 / 1.2e12 * 1e3 + 0.005)) < 1e-6

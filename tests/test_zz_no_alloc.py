"""The allocation-free statistics entry point, through the C ABI.

qs_stats_static serves callers that may not allocate device memory: it takes
amplitudes already on the device and keeps its partial sums in a fixed array
compiled into the library.  This file sorts last so that a run stopping at the
first failure has already run every other test; it also passes on its own in a
fresh process.
"""
import numpy as np
import pytest

import paper_1704_01127_gb300.qs as qs
from inputs import random_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,n", [(qs.QS_C128, 3), (qs.QS_C128, 20), (qs.QS_C64, 11), (qs.QS_C64, 23)])
def test_stats_static_matches_qs_stats_twice(dtype, n):
    h = qs.qs_alloc(n, dtype)
    try:
        qs.qs_set_amplitudes(h, random_state(n, 77 + n))
        want = qs.qs_stats(h)
        ptr = qs.qs_device_ptr(h)
        for _ in range(2):      # the shared array keeps the last call's contents
            got = qs.qs_stats_static(ptr, n, dtype)
            for a, b in zip(got, want):
                assert abs(a - b) <= 1e-12 * max(1.0, abs(b))
    finally:
        qs.qs_free(h)


def test_stats_static_rejects_bad_sizes():
    h = qs.qs_alloc(4, qs.QS_C128)
    try:
        ptr = qs.qs_device_ptr(h)
        for n in (0, 37, -3):
            with pytest.raises(qs.QSError) as e:
                qs.qs_stats_static(ptr, n, qs.QS_C128)
            assert e.value.code == qs.QS_EINVAL
        with pytest.raises(qs.QSError):
            qs.qs_stats_static(ptr, 4, 7)
    finally:
        qs.qs_free(h)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_stats_static_views_at_any_amplitude(dtype):
    """A view that starts at amplitude 1 of a state is accepted (aligned to one
    amplitude); a pointer half an amplitude in is rejected."""
    size = 16 if dtype == qs.QS_C128 else 8
    h = qs.qs_alloc(5, dtype)
    ref = qs.qs_alloc(4, dtype)
    try:
        psi = random_state(5, 91)
        qs.qs_set_amplitudes(h, psi)
        qs.qs_set_amplitudes(ref, psi[1:17])
        want = qs.qs_stats(ref)
        ptr = qs.qs_device_ptr(h)
        got = qs.qs_stats_static(ptr + size, 4, dtype)
        for a, b in zip(got, want):
            assert abs(a - b) <= 1e-12 * max(1.0, abs(b))
        with pytest.raises(qs.QSError) as e:
            qs.qs_stats_static(ptr + size // 2, 4, dtype)
        assert e.value.code == qs.QS_EINVAL
    finally:
        qs.qs_free(h)
        qs.qs_free(ref)

"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Holds no arithmetic of the method: only random states, unitaries and diagonal
phases drawn from numpy's PCG64 with a fixed seed.
"""
import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def random_state(n, seed):
    """Normalised complex128 vector of 2^n Gaussian amplitudes."""
    g = rng(seed)
    v = g.standard_normal(1 << n) + 1j * g.standard_normal(1 << n)
    v /= np.sqrt(np.vdot(v, v).real)
    return v.astype(np.complex128)


def random_unitary(k, seed):
    """Haar-like 2^k x 2^k unitary: QR of a complex Gaussian matrix."""
    g = rng(seed)
    d = 1 << k
    z = (g.standard_normal((d, d)) + 1j * g.standard_normal((d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return (q * ph).astype(np.complex128)


def random_diag(k, seed):
    g = rng(seed)
    return np.exp(1j * g.uniform(0, 2 * np.pi, 1 << k)).astype(np.complex128)


def random_qubits(n, k, seed):
    g = rng(seed)
    return [int(x) for x in g.permutation(n)[:k]]


def random_phase_poly(n, n_edges, seed):
    g = rng(seed)
    coeff = g.integers(0, 8, n)
    edges = []
    for _ in range(n_edges):
        a, b = g.permutation(n)[:2]
        edges.append((int(min(a, b)), int(max(a, b))))
    return coeff, edges

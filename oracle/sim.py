"""Gate-by-gate complex128 simulator (Sec. 2, Sec. 3.2).  Oracle only.

The arithmetic lives in statevec.c (plain loops, compiled with gcc); this module
marshals numpy arrays into it, runs circuits gate by gate in their listed order,
and provides the dense Kronecker-product form of Sec. 2 for n <= 10.
"""
import ctypes
import numpy as np

from . import build as _build
from . import gates as _gates

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.or_apply_1q.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
        L.or_apply_cz.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.or_apply_kq.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, dp]
        L.or_apply_kq.restype = ctypes.c_int
        L.or_apply_diag.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, dp]
        L.or_apply_diag.restype = ctypes.c_int
        L.or_apply_phase.argtypes = [dp, ctypes.c_int, ip, ctypes.c_int, ip]
        L.or_apply_phase.restype = ctypes.c_int
        L.or_probabilities.argtypes = [dp, ctypes.c_int, dp]
        L.or_norm.argtypes = [dp, ctypes.c_int]
        L.or_norm.restype = ctypes.c_double
        L.or_stats.argtypes = [dp, ctypes.c_int, dp]
        L.or_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.or_splitmix64.restype = ctypes.c_uint64
        L.or_sample.argtypes = [dp, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, u64p]
        L.or_sample.restype = ctypes.c_int
        L.or_apply_swap.argtypes = [dp, ctypes.c_int, ip, ip, ctypes.c_int]
        L.or_apply_swap.restype = ctypes.c_int
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def set_threads(t):
    """Host threads for the element-wise loops (gates, phases, probabilities)."""
    lib().or_set_threads(int(t))


def max_threads():
    return int(lib().or_max_threads())


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _check_state(psi):
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    n = int(psi.size).bit_length() - 1
    assert psi.size == 1 << n
    return n


def basis_state(n, x=0):
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    return psi


def uniform_state(n):
    """(2^{-n/2}, ..., 2^{-n/2}): the state after the cycle-0 H layer (Sec. 3.6)."""
    return np.full(1 << n, 2.0 ** (-n / 2.0), dtype=np.complex128)


def apply_1q(psi, q, u):
    n = _check_state(psi)
    uu = _gates.interleaved(u)
    lib().or_apply_1q(_dp(psi.view(np.float64)), n, int(q), _dp(uu))


def apply_cz(psi, a, b):
    n = _check_state(psi)
    lib().or_apply_cz(_dp(psi.view(np.float64)), n, int(a), int(b))


def apply_kq(psi, qubits, U):
    """Sec. 3.2 gather / mat-vec / scatter; qubits[j] <-> bit j of U's index."""
    n = _check_state(psi)
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    uu = _gates.interleaved(U)
    rc = lib().or_apply_kq(_dp(psi.view(np.float64)), n, _ip(q), len(q), _dp(uu))
    assert rc == 0, rc


def apply_diag(psi, qubits, d):
    n = _check_state(psi)
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    dd = np.ascontiguousarray(d, dtype=np.complex128).view(np.float64)
    rc = lib().or_apply_diag(_dp(psi.view(np.float64)), n, _ip(q), len(q), _dp(dd))
    assert rc == 0, rc


def apply_swap(psi, a, b):
    """Exchange qubit a[j] with qubit b[j] for every j (index permutation)."""
    n = _check_state(psi)
    aa = np.ascontiguousarray(a, dtype=np.int32)
    bb = np.ascontiguousarray(b, dtype=np.int32)
    rc = lib().or_apply_swap(_dp(psi.view(np.float64)), n, _ip(aa), _ip(bb), int(aa.size))
    assert rc == 0, rc


def apply_phase(psi, coeff, edges):
    """psi_i *= exp(i pi m(i)/4), m(i) = sum_q coeff[q] i_q + 4 sum_(a,b) i_a i_b."""
    n = _check_state(psi)
    c = np.ascontiguousarray(coeff, dtype=np.int32)
    assert c.size == n
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    rc = lib().or_apply_phase(_dp(psi.view(np.float64)), n, _ip(c), e.size // 2,
                              _ip(e) if e.size else None)
    assert rc == 0, rc


def apply_gate(psi, name, qubits):
    if name == "cz":
        apply_cz(psi, qubits[0], qubits[1])
    else:
        apply_1q(psi, qubits[0], _gates.matrix(name))


def run_circuit(n, gates, psi=None):
    """Apply the gates one by one, in list order, to |0...0> (or to psi)."""
    if psi is None:
        psi = basis_state(n, 0)
    for (_, name, qs) in gates:
        apply_gate(psi, name, qs)
    return psi


def probabilities(psi):
    n = _check_state(psi)
    p = np.empty(1 << n, dtype=np.float64)
    lib().or_probabilities(_dp(psi.view(np.float64)), n, _dp(p))
    return p


def norm(psi):
    n = _check_state(psi)
    return lib().or_norm(_dp(psi.view(np.float64)), n)


def stats(psi):
    """(sum p, entropy -sum p ln p, mean N p, mean (N p)^2)."""
    n = _check_state(psi)
    out = np.zeros(4, dtype=np.float64)
    lib().or_stats(_dp(psi.view(np.float64)), n, _dp(out))
    return tuple(float(x) for x in out)


def sample(psi, seed, m):
    n = _check_state(psi)
    out = np.zeros(int(m), dtype=np.uint64)
    rc = lib().or_sample(_dp(psi.view(np.float64)), n, ctypes.c_uint64(seed), int(m),
                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    assert rc == 0, rc
    return out


def splitmix64(seed, j):
    return int(lib().or_splitmix64(ctypes.c_uint64(seed), ctypes.c_uint64(j)))


# --------------------------------------------------------------------------
# Dense Kronecker form (Sec. 2), n <= 10.
# --------------------------------------------------------------------------

def kron_1q(n, q, u):
    """1 (x) ... (x) U (x) ... (x) 1 with n-q-1 identities left of U and q right."""
    I2 = np.eye(2, dtype=np.complex128)
    m = np.ones((1, 1), dtype=np.complex128)
    for pos in range(n - 1, -1, -1):
        m = np.kron(m, u if pos == q else I2)
    return m


def kron_cz(n, a, b):
    idx = np.arange(1 << n)
    d = np.where(((idx >> a) & 1) & ((idx >> b) & 1), -1.0, 1.0).astype(np.complex128)
    return np.diag(d)


def dense_unitary(n, gates):
    """Product of the 2^n x 2^n gate matrices, last gate leftmost."""
    assert n <= 10
    U = np.eye(1 << n, dtype=np.complex128)
    for (_, name, qs) in gates:
        G = kron_cz(n, *qs) if name == "cz" else kron_1q(n, qs[0], _gates.matrix(name))
        U = G @ U
    return U

"""Python binding of the qs C ABI (include/qs.h): argument marshalling only.

Every computation runs in libqs.so (host C++ for circuit generation and
scheduling, CUDA kernels for every state sweep and reduction).  Importing this
module fails loudly if the library has not been built; there is no fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqs.so")

QS_OK, QS_EINVAL, QS_ENOMEM, QS_ECUDA, QS_ETIMEOUT, QS_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
QS_C64, QS_C128 = 0, 1
QS_MAX_K = 5
QS_OP_DENSE, QS_OP_PHASE, QS_OP_DIAG = 0, 1, 2
QS_PATH_AUTO, QS_PATH_CUDA_CORES, QS_PATH_TENSOR = 0, 1, 2
GATE_KIND = {"h": 0, "t": 1, "x_1_2": 2, "y_1_2": 3, "cz": 4, "x": 5, "tdg": 6,
             "x_1_2dg": 7, "y_1_2dg": 8}
GATE_NAME = {v: k for k, v in GATE_KIND.items()}

GATE_DTYPE = np.dtype([("cycle", np.int32), ("kind", np.int32), ("q0", np.int32), ("q1", np.int32)])


class QSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("qs error %d: %s" % (code, msg))
        self.code = code


class _SchedOpts(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int32), ("fuse", ctypes.c_int32),
                ("merge_phase", ctypes.c_int32), ("drop_final_diagonal", ctypes.c_int32),
                ("commute_diagonal", ctypes.c_int32), ("search_runs", ctypes.c_int32),
                ("search_from_basis", ctypes.c_int32), ("search_first", ctypes.c_int32),
                ("search_slack0", ctypes.c_int32)]


class _OpInfo(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32),
                ("qubits", ctypes.c_int32 * QS_MAX_K), ("n_gates", ctypes.c_int32),
                ("n_edges", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None
_VP, _DP, _IP = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
_U64P, _I64P, _I32P = (ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int64),
                       ctypes.POINTER(ctypes.c_int32))

_SIGS = {
    "qs_last_error": ([], ctypes.c_char_p),
    "qs_alloc": ([ctypes.c_int, ctypes.c_int, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "qs_wrap": ([_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "qs_free": ([_VP], None),
    "qs_num_qubits": ([_VP], ctypes.c_int),
    "qs_dtype": ([_VP], ctypes.c_int),
    "qs_device_ptr": ([_VP], _VP),
    "qs_set_stream": ([_VP, _VP], ctypes.c_int),
    "qs_init_basis": ([_VP, ctypes.c_uint64], ctypes.c_int),
    "qs_init_uniform": ([_VP], ctypes.c_int),
    "qs_set_amplitudes": ([_VP, _DP], ctypes.c_int),
    "qs_get_amplitudes": ([_VP, _DP], ctypes.c_int),
    "qs_get_amplitudes_at": ([_VP, _U64P, ctypes.c_int64, _DP], ctypes.c_int),
    "qs_apply_cluster": ([_VP, _IP, ctypes.c_int, _DP], ctypes.c_int),
    "qs_apply_diag": ([_VP, _IP, ctypes.c_int, _DP], ctypes.c_int),
    "qs_apply_phase": ([_VP, _IP, ctypes.c_int, _IP], ctypes.c_int),
    "qs_norm": ([_VP, _DP], ctypes.c_int),
    "qs_probabilities": ([_VP, _DP, ctypes.c_int], ctypes.c_int),
    "qs_stats": ([_VP, _DP], ctypes.c_int),
    "qs_sample": ([_VP, ctypes.c_uint64, ctypes.c_int64, _U64P], ctypes.c_int),
    "qs_sample_stats": ([_VP, ctypes.c_uint64, ctypes.c_int64, _U64P, _DP], ctypes.c_int),
    "qs_synchronize": ([_VP], ctypes.c_int),
    "qs_supremacy_circuit": ([ctypes.c_int, ctypes.c_int, _IP, ctypes.c_int, ctypes.c_int,
                              ctypes.c_uint64, _IP, _VP, ctypes.c_int, _IP], ctypes.c_int),
    "qs_schedule_build": ([ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(_SchedOpts),
                           ctypes.POINTER(_VP)], ctypes.c_int),
    "qs_schedule_from_ops": ([ctypes.c_int, ctypes.c_int, _IP, _IP, _IP, _I64P, _DP,
                              ctypes.c_int64, ctypes.POINTER(_VP)], ctypes.c_int),
    "qs_schedule_free": ([_VP], None),
    "qs_schedule_num_qubits": ([_VP], ctypes.c_int),
    "qs_schedule_num_ops": ([_VP], ctypes.c_int),
    "qs_schedule_op": ([_VP, ctypes.c_int, ctypes.POINTER(_OpInfo), _DP, _I32P, _I32P, _I32P],
                       ctypes.c_int),
    "qs_run_circuit": ([_VP, _VP], ctypes.c_int),
    "qs_run_circuit_timed": ([_VP, _VP, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "qs_set_device": ([ctypes.c_int], ctypes.c_int),
    "qs_set_path": ([_VP, ctypes.c_int], ctypes.c_int),
    "qs_schedule_upload": ([_VP, ctypes.c_int], ctypes.c_int),
    "qs_set_pair_sweeps": ([_VP, ctypes.c_int], ctypes.c_int),
    "qs_schedule_remap": ([_VP, _IP], ctypes.c_int),
    "qs_schedule_get_remap": ([_VP, _IP], ctypes.c_int),
    "qs_plan_stages": ([ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.POINTER(_VP), ctypes.c_int, _IP,
                        _IP], ctypes.c_int),
    "qs_schedule_choose_remap": ([_VP, ctypes.c_int, _IP], ctypes.c_int),
    "qs_set_host_threads": ([ctypes.c_int], ctypes.c_int),
    "qs_swap_qubits": ([_VP, _IP, _IP, ctypes.c_int], ctypes.c_int),
    "qs_set_phase_fold": ([_VP, ctypes.c_int], ctypes.c_int),
    "qs_selftest_timeout": ([_VP], ctypes.c_int),
    "qs_stats_static": ([_VP, ctypes.c_int, ctypes.c_int, _VP, _DP], ctypes.c_int),
    "qs_batch_circuit_params": ([ctypes.c_uint64, _IP, _IP, _IP], ctypes.c_int),
    "qs_op_features": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP, ctypes.c_int, ctypes.c_int,
                        ctypes.c_int, _DP], ctypes.c_int),
    "qs_cost_analytic_ms": ([_DP, ctypes.c_double], ctypes.c_double),
    "qs_cost_sample": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_double,
                        _DP, _DP], ctypes.c_int),
    "qs_mlp_create": ([ctypes.c_uint64, ctypes.POINTER(_VP)], ctypes.c_int),
    "qs_mlp_free": ([_VP], None),
    "qs_mlp_num_params": ([], ctypes.c_int),
    "qs_mlp_get_params": ([_VP, _DP], ctypes.c_int),
    "qs_mlp_set_params": ([_VP, _DP], ctypes.c_int),
    "qs_mlp_forward": ([_VP, _DP, ctypes.c_int, _DP], ctypes.c_int),
    "qs_mlp_gradient": ([_VP, _DP, _DP, ctypes.c_int, _DP, _DP], ctypes.c_int),
    "qs_mlp_train": ([_VP, _DP, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_double, _DP], ctypes.c_int),
    "qs_cost_model_create": ([ctypes.c_double, ctypes.POINTER(_VP)], ctypes.c_int),
    "qs_cost_model_free": ([_VP], None),
    "qs_cost_model_fit": ([_VP, _DP, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _DP], ctypes.c_int),
    "qs_cost_model_predict": ([_VP, _DP, ctypes.c_int, ctypes.c_int, _DP], ctypes.c_int),
    "qs_plan_circuit": ([ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, ctypes.POINTER(_VP), _IP,
                         _DP], ctypes.c_int),
    "qs_batch_create": ([ctypes.c_int, ctypes.POINTER(_VP), ctypes.c_int, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "qs_batch_free": ([_VP], None),
    "qs_batch_set_config": ([_VP, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "qs_batch_get_config": ([_VP, _IP, _IP], ctypes.c_int),
    "qs_batch_run": ([_VP], ctypes.c_int),
    "qs_batch_run_graph": ([_VP], ctypes.c_int),
    "qs_batch_stats": ([_VP, _DP], ctypes.c_int),
    "qs_batch_get_amplitudes": ([_VP, ctypes.c_int, _DP], ctypes.c_int),
    "qs_batch_tune": ([_VP, _IP, _IP, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "qs_batch_autotune": ([ctypes.c_int, _IP, ctypes.POINTER(_VP), _IP, ctypes.c_int, _VP, _IP, _IP, _IP,
                           ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "qs_schedule_upload_bytes": ([_VP, ctypes.c_int], ctypes.c_int64),
}


def lib():
    """The loaded libqs.so; raises ImportError if it was never built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libqs.so is not built (run paper_1704_01127_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _check(rc):
    if rc != QS_OK:
        raise QSError(rc, lib().qs_last_error().decode())
    return rc


def _dp(a):
    return a.ctypes.data_as(_DP)


def _ip(a):
    return a.ctypes.data_as(_IP)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream   # torch.cuda.Stream


# ----------------------------------------------------------------- state API

def qs_alloc(n, dtype=QS_C128, stream=None):
    h = _VP()
    _check(lib().qs_alloc(int(n), int(dtype), _stream_ptr(stream), ctypes.byref(h)))
    return h


def qs_wrap(dev_ptr, n, dtype=QS_C128, stream=None):
    """Adopt a device buffer (int pointer or a CUDA torch tensor); not freed by qs_free."""
    if hasattr(dev_ptr, "data_ptr"):
        dev_ptr = dev_ptr.data_ptr()
    h = _VP()
    _check(lib().qs_wrap(_VP(dev_ptr), int(n), int(dtype), _stream_ptr(stream), ctypes.byref(h)))
    return h


def qs_free(h):
    lib().qs_free(h)


def qs_num_qubits(h):
    return lib().qs_num_qubits(h)


def qs_dtype(h):
    return lib().qs_dtype(h)


def qs_device_ptr(h):
    return lib().qs_device_ptr(h)


def qs_set_stream(h, stream):
    _check(lib().qs_set_stream(h, _stream_ptr(stream)))


def qs_init_basis(h, x=0):
    _check(lib().qs_init_basis(h, ctypes.c_uint64(int(x))))


def qs_init_uniform(h):
    _check(lib().qs_init_uniform(h))


def qs_set_amplitudes(h, psi):
    a = _c128(psi)
    assert a.size == 1 << qs_num_qubits(h)
    _check(lib().qs_set_amplitudes(h, _dp(a.view(np.float64))))


def qs_get_amplitudes(h):
    out = np.empty(1 << qs_num_qubits(h), dtype=np.complex128)
    _check(lib().qs_get_amplitudes(h, _dp(out.view(np.float64))))
    return out


def qs_get_amplitudes_at(h, indices):
    idx = np.ascontiguousarray(indices, dtype=np.uint64)
    out = np.empty(idx.size, dtype=np.complex128)
    _check(lib().qs_get_amplitudes_at(h, idx.ctypes.data_as(_U64P), int(idx.size), _dp(out.view(np.float64))))
    return out


def qs_apply_cluster(h, qubits, U):
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    u = _c128(U)
    d = 1 << q.size
    assert u.shape == (d, d)
    _check(lib().qs_apply_cluster(h, _ip(q), int(q.size), _dp(u.reshape(-1).view(np.float64))))


def qs_apply_diag(h, qubits, d):
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    dd = _c128(d)
    assert dd.size == 1 << q.size
    _check(lib().qs_apply_diag(h, _ip(q), int(q.size), _dp(dd.view(np.float64))))


def qs_swap_qubits(h, a, b):
    """Exchange qubit a[j] with qubit b[j] for every j (one sweep)."""
    aa = np.ascontiguousarray(a, dtype=np.int32)
    bb = np.ascontiguousarray(b, dtype=np.int32)
    assert aa.size == bb.size
    _check(lib().qs_swap_qubits(h, _ip(aa), _ip(bb), int(aa.size)))


def qs_apply_phase(h, coeff, edges):
    c = np.ascontiguousarray(coeff, dtype=np.int32)
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1))
    _check(lib().qs_apply_phase(h, _ip(c), int(e.size // 2), _ip(e) if e.size else None))


def qs_norm(h):
    out = ctypes.c_double()
    _check(lib().qs_norm(h, ctypes.byref(out)))
    return out.value


def qs_stats(h):
    out = np.zeros(4, dtype=np.float64)
    _check(lib().qs_stats(h, _dp(out)))
    return tuple(float(x) for x in out)


def qs_probabilities(h, out=None, out_on_device=False):
    """FP64 probabilities: into a new host array, a given host array, or (with
    out_on_device) a device pointer / CUDA tensor."""
    if out_on_device:
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else int(out)
        _check(lib().qs_probabilities(h, ctypes.cast(ptr, _DP), 1))
        return out
    if out is None:
        out = np.empty(1 << qs_num_qubits(h), dtype=np.float64)
    _check(lib().qs_probabilities(h, _dp(out), 0))
    return out


def qs_sample(h, seed, m):
    out = np.zeros(int(m), dtype=np.uint64)
    _check(lib().qs_sample(h, ctypes.c_uint64(int(seed)), int(m), out.ctypes.data_as(_U64P)))
    return out


def qs_sample_stats(h, seed, m):
    """(draws as qs_sample, statistics as qs_stats) from one pass."""
    out = np.zeros(int(m), dtype=np.uint64)
    st = np.zeros(4, dtype=np.float64)
    _check(lib().qs_sample_stats(h, ctypes.c_uint64(int(seed)), int(m), out.ctypes.data_as(_U64P), _dp(st)))
    return out, tuple(float(x) for x in st)


def qs_synchronize(h):
    _check(lib().qs_synchronize(h))


def qs_selftest_timeout(h):
    """Status code of one bounded wait that runs out (QS_ETIMEOUT expected)."""
    return lib().qs_selftest_timeout(h)


# --------------------------------------------------------------- circuit API

def qs_supremacy_circuit(rows, cols, cz_cycles, seed, removed=()):
    """(n, gates) with gates a structured array of (cycle, kind, q0, q1)."""
    rem = np.ascontiguousarray(np.asarray(removed, dtype=np.int32).reshape(-1))
    n = ctypes.c_int()
    cnt = ctypes.c_int()
    cap = 64 + 2 * rows * cols * (cz_cycles + 1)
    gates = np.zeros(cap, dtype=GATE_DTYPE)
    _check(lib().qs_supremacy_circuit(int(rows), int(cols), _ip(rem) if rem.size else None,
                                      int(rem.size // 2), int(cz_cycles), ctypes.c_uint64(int(seed)),
                                      ctypes.byref(n), gates.ctypes.data_as(_VP), cap, ctypes.byref(cnt)))
    return n.value, gates[:cnt.value].copy()


def gates_from_tuples(gates):
    """Structured gate array from (cycle, name, qubits) tuples."""
    out = np.zeros(len(gates), dtype=GATE_DTYPE)
    for i, (cyc, name, qs) in enumerate(gates):
        out[i] = (cyc, GATE_KIND[name], qs[0], qs[1] if len(qs) > 1 else -1)
    return out


def gates_to_tuples(gates):
    return [(int(g["cycle"]), GATE_NAME[int(g["kind"])],
             (int(g["q0"]),) if int(g["q1"]) < 0 else (int(g["q0"]), int(g["q1"])))
            for g in gates]


def qs_schedule_build(n, gates, k_max=5, fuse=True, merge_phase=True, drop_final_diagonal=False,
                      commute_diagonal=True, search_runs=13, search_from_basis=True, search_first=16,
                      search_slack0=5):
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    opts = _SchedOpts(int(k_max), int(bool(fuse)), int(bool(merge_phase)), int(bool(drop_final_diagonal)),
                      int(bool(commute_diagonal)), int(search_runs), int(bool(search_from_basis)),
                      int(search_first), int(search_slack0))
    h = _VP()
    _check(lib().qs_schedule_build(int(n), g.ctypes.data_as(_VP), int(g.size), ctypes.byref(opts),
                                   ctypes.byref(h)))
    return h


def qs_plan_stages(n, gates, n_global, k_max=5, max_stages=64, **kw):
    """(list of stage schedules, stage of every gate); see qs_schedule_build
    for the clustering options."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    d = dict(fuse=True, merge_phase=True, drop_final_diagonal=False, commute_diagonal=True, search_runs=13,
             search_from_basis=True, search_first=16, search_slack0=5)
    d.update(kw)
    opts = _SchedOpts(int(k_max), int(d["fuse"]), int(d["merge_phase"]), int(d["drop_final_diagonal"]),
                      int(d["commute_diagonal"]), int(d["search_runs"]), int(d["search_from_basis"]),
                      int(d["search_first"]), int(d["search_slack0"]))
    arr = (_VP * max_stages)()
    cnt = ctypes.c_int()
    of = np.zeros(max(g.size, 1), dtype=np.int32)
    _check(lib().qs_plan_stages(int(n), g.ctypes.data_as(_VP), int(g.size), int(n_global), ctypes.byref(opts), arr,
                                int(max_stages), ctypes.byref(cnt), _ip(of)))
    return [arr[i] for i in range(cnt.value)], of[:g.size]


def qs_schedule_from_ops(n, ops):
    """ops: list of (kind, qubits, complex matrix or diagonal), or for a phase
    op (QS_OP_PHASE, CZ pairs, n coefficients)."""
    kinds, ks, qubits, offsets, pool = [], [], [], [], []
    at = 0
    for kind, qs, m in ops:
        kinds.append(kind)
        ks.append(len(qs))
        if kind == QS_OP_PHASE:
            qubits.extend([0] * QS_MAX_K)
            flat = np.concatenate([np.asarray(m, dtype=np.float64).reshape(-1),
                                   np.asarray(qs, dtype=np.float64).reshape(-1)])
            offsets.append(at)
            pool.append(flat)
            at += flat.size
            continue
        qubits.extend(list(qs) + [0] * (QS_MAX_K - len(qs)))
        flat = _c128(m).reshape(-1).view(np.float64)
        offsets.append(at)
        pool.append(flat)
        at += flat.size
    pool = np.ascontiguousarray(np.concatenate(pool) if pool else np.zeros(1))
    kinds, ks, qubits = (np.ascontiguousarray(x, dtype=np.int32) for x in (kinds, ks, qubits))
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    h = _VP()
    _check(lib().qs_schedule_from_ops(int(n), int(kinds.size), _ip(kinds), _ip(ks), _ip(qubits),
                                      offsets.ctypes.data_as(_I64P), _dp(pool), int(pool.size),
                                      ctypes.byref(h)))
    return h


def qs_schedule_free(h):
    lib().qs_schedule_free(h)


def qs_schedule_num_ops(h):
    return lib().qs_schedule_num_ops(h)


def qs_schedule_op(h, i):
    """Op i as a dict: kind, qubits, gates, and matrix (dense/diag) or coeff/edges (phase)."""
    info = _OpInfo()
    _check(lib().qs_schedule_op(h, int(i), ctypes.byref(info), None, None, None, None))
    k, kind = info.k, info.kind
    gidx = np.zeros(max(info.n_gates, 1), dtype=np.int32)
    out = {"kind": {QS_OP_DENSE: "dense", QS_OP_PHASE: "phase", QS_OP_DIAG: "diag"}[kind]}
    n = lib().qs_schedule_num_qubits(h)
    if kind == QS_OP_PHASE:
        coeff = np.zeros(n, dtype=np.int32)
        edges = np.zeros(max(2 * info.n_edges, 1), dtype=np.int32)
        _check(lib().qs_schedule_op(h, int(i), None, None, gidx.ctypes.data_as(_I32P),
                                    coeff.ctypes.data_as(_I32P), edges.ctypes.data_as(_I32P)))
        out["coeff"] = coeff
        out["edges"] = [(int(edges[2 * e]), int(edges[2 * e + 1])) for e in range(info.n_edges)]
        out["support"] = k
    else:
        d = 1 << k
        m = np.zeros(d * d if kind == QS_OP_DENSE else d, dtype=np.complex128)
        _check(lib().qs_schedule_op(h, int(i), None, _dp(m.view(np.float64)),
                                    gidx.ctypes.data_as(_I32P), None, None))
        out["qubits"] = tuple(int(x) for x in info.qubits[:k])
        out["matrix"] = m.reshape(d, d) if kind == QS_OP_DENSE else m
    out["gates"] = tuple(int(x) for x in gidx[:info.n_gates])
    return out


def qs_run_circuit(h, sched):
    _check(lib().qs_run_circuit(h, sched))


def qs_run_circuit_timed(h, sched):
    """Run a schedule; returns the device time of every op in milliseconds
    (-1 for a phase op that ran inside the sweep before it)."""
    out = np.zeros(max(qs_schedule_num_ops(sched), 1), dtype=np.float32)
    _check(lib().qs_run_circuit_timed(h, sched, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out[:qs_schedule_num_ops(sched)]


def qs_set_device(device):
    _check(lib().qs_set_device(int(device)))


def qs_schedule_upload_bytes(sched, dtype):
    v = lib().qs_schedule_upload_bytes(sched, int(dtype))
    if v < 0:
        _check(v)
    return int(v)


def qs_schedule_upload(sched, dtype):
    """Build and copy the schedule's device image for dtype now (current device)."""
    _check(lib().qs_schedule_upload(sched, int(dtype)))


def qs_schedule_remap(sched, loc):
    """Relabel the schedule's ops: qubit q to index bit loc[q] (exchanges)."""
    l = np.ascontiguousarray(loc, dtype=np.int32)
    _check(lib().qs_schedule_remap(sched, _ip(l)))


def qs_schedule_get_remap(sched):
    n = lib().qs_schedule_num_qubits(sched)
    l = np.zeros(n, dtype=np.int32)
    _check(lib().qs_schedule_get_remap(sched, _ip(l)))
    return l


def qs_schedule_choose_remap(sched, dtype):
    """The library's pick of loc for a schedule started from |0...0>."""
    n = lib().qs_schedule_num_qubits(sched)
    l = np.zeros(n, dtype=np.int32)
    _check(lib().qs_schedule_choose_remap(sched, int(dtype), _ip(l)))
    return l


def qs_set_host_threads(n):
    _check(lib().qs_set_host_threads(int(n)))


def qs_stats_static(dev_ptr, n, dtype, stream=None):
    """Allocation-free statistics of 2^n amplitudes already in device memory
    (int pointer or CUDA tensor): (sum p, entropy, mean N p, mean (N p)^2)."""
    if hasattr(dev_ptr, "data_ptr"):
        dev_ptr = dev_ptr.data_ptr()
    out = np.zeros(4, dtype=np.float64)
    _check(lib().qs_stats_static(_VP(dev_ptr), int(n), int(dtype), _stream_ptr(stream), _dp(out)))
    return tuple(float(x) for x in out)


def qs_set_path(h, path):
    _check(lib().qs_set_path(h, int(path)))


def qs_set_pair_sweeps(h, on):
    _check(lib().qs_set_pair_sweeps(h, 1 if on else 0))


def qs_set_phase_fold(h, on):
    _check(lib().qs_set_phase_fold(h, 1 if on else 0))


# ------------------------------------------------------------------- batches

def qs_batch_circuit_params(seed):
    r, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().qs_batch_circuit_params(ctypes.c_uint64(int(seed)), ctypes.byref(r), ctypes.byref(c),
                                         ctypes.byref(d)))
    return r.value, c.value, d.value


def qs_batch_create(schedules, dtype=QS_C64, stream=None):
    arr = (_VP * len(schedules))(*[s.value if isinstance(s, _VP) else s for s in schedules])
    h = _VP()
    _check(lib().qs_batch_create(len(schedules), arr, int(dtype), _stream_ptr(stream), ctypes.byref(h)))
    return h


def qs_batch_free(b):
    lib().qs_batch_free(b)


def qs_batch_set_config(b, cluster_ctas, threads):
    _check(lib().qs_batch_set_config(b, int(cluster_ctas), int(threads)))


def qs_batch_get_config(b):
    c, t = ctypes.c_int(), ctypes.c_int()
    _check(lib().qs_batch_get_config(b, ctypes.byref(c), ctypes.byref(t)))
    return c.value, t.value


def qs_batch_run(b):
    _check(lib().qs_batch_run(b))


def qs_batch_run_graph(b):
    _check(lib().qs_batch_run_graph(b))


def qs_batch_stats(b, n_circuits):
    out = np.zeros(4 * n_circuits, dtype=np.float64)
    _check(lib().qs_batch_stats(b, _dp(out)))
    return out.reshape(n_circuits, 4)


def qs_batch_get_amplitudes(b, i, n):
    out = np.empty(1 << n, dtype=np.complex128)
    _check(lib().qs_batch_get_amplitudes(b, int(i), _dp(out.view(np.float64))))
    return out


def qs_batch_tune(b):
    c, t, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(lib().qs_batch_tune(b, ctypes.byref(c), ctypes.byref(t), ctypes.byref(ms)))
    return c.value, t.value, ms.value


def qs_batch_autotune(circuits, dtype=QS_C64, stream=None):
    """circuits: list of (n, gates) -> (k_max, cluster_ctas, threads, ms)."""
    gates = [np.ascontiguousarray(g, dtype=GATE_DTYPE) for (_, g) in circuits]
    nq = np.ascontiguousarray([n for (n, _) in circuits], dtype=np.int32)
    ng = np.ascontiguousarray([g.size for g in gates], dtype=np.int32)
    ptrs = (_VP * len(gates))(*[g.ctypes.data for g in gates])
    km, c, t, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    _check(lib().qs_batch_autotune(len(gates), _ip(nq), ptrs, _ip(ng), int(dtype), _stream_ptr(stream),
                                   ctypes.byref(km), ctypes.byref(c), ctypes.byref(t), ctypes.byref(ms)))
    return km.value, c.value, t.value, ms.value


# ---------------------------------------------------------------- cost models

QS_NFEAT = 12
QS_COST_AUTO, QS_COST_ANALYTIC, QS_COST_MLP = 0, 1, 2


def qs_op_features(n, dtype, kind, k=0, qubits=(), path=0, n_act=0, odd=0):
    q = np.zeros(5, dtype=np.int32)
    q[:len(qubits)] = qubits
    out = np.zeros(QS_NFEAT, dtype=np.float64)
    _check(lib().qs_op_features(int(n), int(dtype), int(kind), int(k), _ip(q), int(path), int(n_act), int(odd),
                                _dp(out)))
    return out


def qs_cost_analytic_ms(features, hbm_gbs=6696.8):
    f = np.ascontiguousarray(features, dtype=np.float64)
    return float(lib().qs_cost_analytic_ms(_dp(f), float(hbm_gbs)))


def qs_cost_sample(n_min, n_max, dtype, count, seed, max_ms=200.0):
    feats = np.zeros((int(count), QS_NFEAT), dtype=np.float64)
    ms = np.zeros(int(count), dtype=np.float64)
    _check(lib().qs_cost_sample(int(n_min), int(n_max), int(dtype), int(count), ctypes.c_uint64(int(seed)),
                                float(max_ms), _dp(feats), _dp(ms)))
    return feats, ms


def qs_mlp_create(seed=0):
    h = _VP()
    _check(lib().qs_mlp_create(ctypes.c_uint64(int(seed)), ctypes.byref(h)))
    return h


def qs_mlp_free(h):
    lib().qs_mlp_free(h)


def qs_mlp_num_params():
    return int(lib().qs_mlp_num_params())


def qs_mlp_get_params(h):
    out = np.zeros(qs_mlp_num_params(), dtype=np.float64)
    _check(lib().qs_mlp_get_params(h, _dp(out)))
    return out


def qs_mlp_set_params(h, w):
    w = np.ascontiguousarray(w, dtype=np.float64)
    assert w.size == qs_mlp_num_params()
    _check(lib().qs_mlp_set_params(h, _dp(w)))


def qs_mlp_forward(h, X):
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(X.shape[0], dtype=np.float64)
    _check(lib().qs_mlp_forward(h, _dp(X), int(X.shape[0]), _dp(out)))
    return out


def qs_mlp_gradient(h, X, Y):
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    g = np.zeros(qs_mlp_num_params(), dtype=np.float64)
    loss = ctypes.c_double()
    _check(lib().qs_mlp_gradient(h, _dp(X), _dp(Y), int(X.shape[0]), _dp(g), ctypes.byref(loss)))
    return g, loss.value


def qs_mlp_train(h, X, Y, epochs, lr=3e-3):
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    loss = ctypes.c_double()
    _check(lib().qs_mlp_train(h, _dp(X), _dp(Y), int(X.shape[0]), int(epochs), float(lr), ctypes.byref(loss)))
    return loss.value


def qs_cost_model_create(hbm_gbs=6696.8):
    h = _VP()
    _check(lib().qs_cost_model_create(float(hbm_gbs), ctypes.byref(h)))
    return h


def qs_cost_model_free(h):
    lib().qs_cost_model_free(h)


def qs_cost_model_fit(h, features, ms, epochs=1500, seed=0):
    f = np.ascontiguousarray(features, dtype=np.float64)
    t = np.ascontiguousarray(ms, dtype=np.float64)
    rep = np.zeros(4, dtype=np.float64)
    _check(lib().qs_cost_model_fit(h, _dp(f), _dp(t), int(t.size), int(epochs), ctypes.c_uint64(int(seed)),
                                   _dp(rep)))
    return {"train_loss": rep[0], "mlp_holdout_median_abs_log_err": rep[1],
            "analytic_holdout_median_abs_log_err": rep[2], "use_mlp": bool(rep[3])}


def qs_cost_model_predict(h, features, which=QS_COST_AUTO):
    f = np.ascontiguousarray(features, dtype=np.float64).reshape(-1, QS_NFEAT)
    out = np.zeros(f.shape[0], dtype=np.float64)
    _check(lib().qs_cost_model_predict(h, _dp(f), int(f.shape[0]), int(which), _dp(out)))
    return out


def qs_plan_circuit(n, gates, dtype, model, which=QS_COST_AUTO):
    """(schedule, k_max, predicted_ms)."""
    g = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    h = _VP()
    km = ctypes.c_int()
    t = ctypes.c_double()
    _check(lib().qs_plan_circuit(int(n), g.ctypes.data_as(_VP), int(g.size), int(dtype), model, int(which),
                                 ctypes.byref(h), ctypes.byref(km), ctypes.byref(t)))
    return h, km.value, t.value

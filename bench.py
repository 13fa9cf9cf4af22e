"""Benchmark: one supremacy circuit per step through the whole hot path.

A step = generate the circuit (host), schedule it into clusters and build the
FP64 cluster unitaries (host), prepare |0...0>, apply every op (one HBM sweep
each), and reduce the output distribution (norm, entropy, Porter-Thomas moments).
The default workload is the 30-qubit 5x6-grid circuit with 25 CZ cycles in
complex128, fused into clusters of k <= 5 plus merged CZ/T phase diagonals.

Prints one JSON line.  `value` is the job's wall time per circuit (device-timed,
max over ranks, divided by the circuits all ranks simulated).
With --gpus N > 1 (under torchrun) every rank simulates its own circuits
(replicas; no data exchange between GPUs).
"""
import argparse
import concurrent.futures
import inspect
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "circuit wall time and effective HBM GB/s per cluster sweep (fraction of roofline) vs plain"

WORKLOADS = {
    # name: (rows, cols, removed, cz_cycles, dtype, k_max)
    "5x6_d25_c128": (5, 6, (), 25, "c128", 5),
    "5x6_d25_c64": (5, 6, (), 25, "c64", 5),
    "4x8_d25_c64": (4, 8, (), 25, "c64", 5),
    "4x4_d10_c128": (4, 4, (), 10, "c128", 5),
    # small cases (256 MB states, still larger than L2) for profiler captures
    "4x6_d25_c128": (4, 6, (), 25, "c128", 5),
    "5x5_d25_c64": (5, 5, (), 25, "c64", 5),
}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def measured_traffic(kernel, n):
    """DRAM bytes (read + write) per launch from the committed ncu record of
    `kernel`, scaled from the captured state size to 2^n amplitudes; None when
    there is no record or the kernel's source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
        if f.get("kernel") != kernel:
            continue
        src = os.path.join(ROOT, f["source"])
        if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != f["sha256"]:
            return None
        return int(f["dram_bytes"]) * 2 ** (n - int(f["n"]))
    return None


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args=None, backend=None):
    """Rank / world from the torchrun environment; a process group (NCCL on GPU
    boxes, gloo otherwise) when more than one rank runs.  Ranks are replicas:
    each simulates its own circuits, and the group only carries the timing."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x):
    """The largest x over all ranks (the job's elapsed time)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_seconds_per_circuit(elapsed_max, circuits_per_rank, world):
    """Whole-job wall time divided by the circuits all ranks simulated."""
    return elapsed_max / (circuits_per_rank * world)


# ------------------------------------------------------------------ our arm

def classify_sweeps(qs, sc, op_ms, n, dtype):
    """Split a run started with qs_init_basis into full-state sweeps and sweeps
    on the support after |0...0> (the library's rule: tensor-core sweeps cover
    the qubits touched so far; any other op first writes the zeros).
    Returns ({(kind, k): [ms]}, [partial ms], partial bytes, ops run, fills)."""
    amp = 16 if dtype == qs.QS_C128 else 8
    full, free, fills, ran = (1 << n) - 1, 0, 0, 0
    kernel_ms, partial_ms, partial_bytes = {}, [], 0
    nops = qs.qs_schedule_num_ops(sc)
    ops = [qs.qs_schedule_op(sc, i) for i in range(nops)]
    for i in range(nops):
        if op_ms[i] < 0:     # ran inside the sweep before it (folded phase op, second cluster of a pair)
            continue
        ran += 1
        op = ops[i]
        k = len(op.get("qubits", ())) if op["kind"] == "dense" else 0
        paired = (op["kind"] == "dense" and i + 1 < nops and op_ms[i + 1] < 0 and ops[i + 1]["kind"] == "dense")
        if paired:           # two clusters in one sweep (full support only)
            for q in op["qubits"] + ops[i + 1]["qubits"]:
                free |= 1 << q
            kernel_ms.setdefault(("pair", 5), []).append(float(op_ms[i]))
            continue
        was_full = free == full
        before = bin(free).count("1")
        touched = 0
        if op["kind"] == "dense" and n >= 5 and (
                (dtype == qs.QS_C64 and k >= 4) or (dtype == qs.QS_C128 and k >= 2)):
            for q in op["qubits"]:
                free |= 1 << q
            # reads the support before the sweep, writes it after
            touched = (1 << before) + (1 << bin(free).count("1"))
        elif free != full:
            # zeros written outside the support, then a full sweep
            free, fills = full, fills + 1
            touched = 3 << n
        if was_full:
            kernel_ms.setdefault((op["kind"], k), []).append(float(op_ms[i]))
        else:
            partial_ms.append(float(op_ms[i]))
            partial_bytes += touched * amp
    return kernel_ms, partial_ms, partial_bytes, ran, fills


def run_ours(args):
    import numpy as np
    import torch
    from paper_1704_01127_gb300 import build as _build
    _build.build()
    import paper_1704_01127_gb300.qs as qs

    world, rank, local, dist = dist_setup(args)
    qs.qs_set_device(local)
    torch.cuda.set_device(local)
    rows, cols, removed, cycles, dt, k_max = WORKLOADS[args.workload]
    dtype = qs.QS_C128 if dt == "c128" else qs.QS_C64
    amp_bytes = 16 if dtype == qs.QS_C128 else 8
    hbm_gbs, sm_max_mhz, peak_src = load_peaks()

    stream = torch.cuda.Stream()
    n, _ = qs.qs_supremacy_circuit(rows, cols, cycles, 0, removed=removed)
    h = qs.qs_alloc(n, dtype, stream)
    qs.qs_set_phase_fold(h, not args.no_fold)
    state_bytes = amp_bytes << n

    kernel_ms = {}      # (kind, k) -> per-launch ms of full-state sweeps in the timed region
    partial_ms = []     # sweeps that ran on part of the state (the support after |0...0>)
    partial_bytes = [0]  # amplitudes they read and wrote (support before + after), in bytes
    launches = [0]

    # a1-a3 run on the host; the next step's are prepared in a second thread
    # while the GPU runs this one (ctypes releases the GIL in library calls)
    prep_pool = concurrent.futures.ThreadPoolExecutor(max_workers=1)

    # the clustering search leaves cores to the thread that launches kernels
    qs.qs_set_host_threads(args.search_threads)

    def prepare(seed):
        qs.qs_set_device(local)
        nq, gates = qs.qs_supremacy_circuit(rows, cols, cycles, seed, removed=removed)       # a1
        sc = qs.qs_schedule_build(nq, gates, k_max=k_max, fuse=not args.plain)                # a2, a3
        if args.remap:                            # qubits to index bits (Sec. 3.6)
            qs.qs_schedule_remap(sc, qs.qs_schedule_choose_remap(sc, dtype))
        qs.qs_schedule_upload(sc, dtype)          # operands packed and copied ahead of the run
        return sc

    def one_step(prepared, next_seed, record):
        """Runs the prepared schedule; returns (stats, ops, next prepared)."""
        sc = prepared.result()
        nxt = prep_pool.submit(prepare, next_seed)
        try:
            qs.qs_init_basis(h, 0)
            op_ms = qs.qs_run_circuit_timed(h, sc)                                            # a4-a6
            st = qs.qs_stats(h)                                                               # a7
            if record:
                km, pm, pb, ran, fills = classify_sweeps(qs, sc, op_ms, n, dtype)
                for kk, v in km.items():
                    kernel_ms.setdefault(kk, []).extend(v)
                partial_ms.extend(pm)
                partial_bytes[0] += pb
                launches[0] += ran + 1 + 2 + fills
            return st, len(op_ms), nxt
        finally:
            qs.qs_schedule_free(sc)

    # one seed more than steps: the last timed step prepares one more schedule,
    # so the timed region holds as many preparations as steps
    seeds = [rank * 1000 + s for s in range(args.warmup + args.steps + 1)]
    prepared = prep_pool.submit(prepare, seeds[0])
    for i in range(args.warmup):
        _, _, prepared = one_step(prepared, seeds[i + 1], False)
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        t0 = time.perf_counter()
        stats = None
        for i in range(args.warmup, args.warmup + args.steps):
            stats, nops, prepared = one_step(prepared, seeds[i + 1], True)
        qs.qs_schedule_free(prepared.result())
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    prep_pool.shutdown()
    barrier(dist)
    dev_s = ev0.elapsed_time(ev1) / 1e3
    elapsed = max_over_ranks(dist, max(dev_s, wall))
    per_circuit = job_seconds_per_circuit(elapsed, args.steps, world)

    # dominant kernel: the (kind, k) class with the most device time over
    # full-state sweeps (each reads and writes the whole state once)
    dom_key = max(kernel_ms, key=lambda kk: sum(kernel_ms[kk]))
    dom_ms = statistics.mean(kernel_ms[dom_key])
    sweep_bytes = 2 * state_bytes
    achieved_gbs = sweep_bytes / (dom_ms * 1e-3) / 1e9
    kind, k = dom_key
    flops = (1 << n) * (8 * (1 << k) - 2) if kind == "dense" else 0
    # kernel path of the default policy: tensor cores for complex64 5-qubit and
    # complex128 2..5-qubit clusters, CUDA cores otherwise
    tensor = kind == "dense" and n >= 5 and ((dtype == qs.QS_C64 and k >= 4) or (dtype == qs.QS_C128 and k >= 2))
    if kind == "dense" and dtype == qs.QS_C128 and not tensor:
        # native FP64: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock
        fp64_peak = 152 * 2 * 2 * sm_max_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops / (dom_ms * 1e-3) / 1e12, "peak": fp64_peak,
                "unit": "TFLOP/s", "peak_source": "derived FP64 (152 SM x 2 FMA/clk x 2 x %.0f MHz)" % sm_max_mhz}
        kname = "k_dense<double,%d>" % k
    else:
        roof = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_gbs, "unit": "GB/s",
                "peak_source": peak_src}
        kname = ("k_dense5_tc_c128_pipe<false>" if dtype == qs.QS_C128 else "k_dense5_tc_c64<false>") if tensor else (
            "k_pair5_tc_c64<false>" if kind == "pair" else
            "k_dense<%s,%d>" % ("double" if dtype == qs.QS_C128 else "float", k) if kind == "dense"
            else "k_phase<%s>" % ("double" if dtype == qs.QS_C128 else "float"))
        if kind == "pair":
            roof["note"] = "two clusters per launch: per-cluster effective rate = 2 x achieved"
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = measured_traffic(kname, n)
    roof["kernel"] = kname
    roof["kernel_ms"] = dom_ms
    roof["algorithmic_bytes"] = sweep_bytes
    roof["effective_hbm_gbs"] = achieved_gbs
    roof["hbm_frac"] = achieved_gbs / hbm_gbs

    sweeps = {("%s_k%d" % kk if kk[0] == "dense" else "dense_pair" if kk[0] == "pair" else kk[0]): {
        "launches": len(v), "mean_ms": statistics.mean(v),
        "gbs": sweep_bytes / (statistics.mean(v) * 1e-3) / 1e9,
        **({"clusters_per_launch": 2} if kk[0] == "pair" else {}),
        "hbm_frac": sweep_bytes / (statistics.mean(v) * 1e-3) / 1e9 / hbm_gbs}
        for kk, v in sorted(kernel_ms.items())}
    sweeps["partial_support"] = {
        "launches": len(partial_ms), "total_ms": sum(partial_ms), "bytes": partial_bytes[0],
        "gbs": partial_bytes[0] / (sum(partial_ms) * 1e-3) / 1e9 if partial_ms else None,
        "hbm_frac": partial_bytes[0] / (sum(partial_ms) * 1e-3) / 1e9 / hbm_gbs if partial_ms else None,
        "what": "sweeps before the reachable indices cover the state: each reads the support before it and "
                "writes the support after it (2^|support| amplitudes each); bytes = those amplitudes, GB/s over "
                "their summed device time"}

    # plain gate-by-gate form of the same circuit (the comparison of the metric)
    plain = None
    if not args.plain and not args.no_plain and rank == 0:
        nq, gates = qs.qs_supremacy_circuit(rows, cols, cycles, seeds[args.warmup + args.steps - 1], removed=removed)
        sc = qs.qs_schedule_build(nq, gates, fuse=False)
        try:
            qs.qs_init_basis(h, 0)
            qs.qs_run_circuit(h, sc)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            qs.qs_init_basis(h, 0)
            e0.record(stream)
            qs.qs_run_circuit(h, sc)
            e1.record(stream)
            torch.cuda.synchronize()
            plain = {"s_per_circuit": e0.elapsed_time(e1) / 1e3, "ops": qs.qs_schedule_num_ops(sc),
                     "dtype": dt}
        finally:
            qs.qs_schedule_free(sc)

    # end to end through the public API with host buffers
    e2e = None
    if rank == 0 and not args.no_e2e:
        # 8 circuits in a row (seeds rank*1000 + 0..7): as in the timed steps,
        # the next circuit's host part (a1-a3) runs in a second thread while
        # this one runs, reports and samples; the first preparation (pipeline
        # fill) and one extra at the end are inside the timed region
        m, n_e2e = 1 << 20, 8
        e2e_seeds = [rank * 1000 + s for s in range(n_e2e + 1)]
        e2e_pool = concurrent.futures.ThreadPoolExecutor(max_workers=1)
        t0 = time.perf_counter()
        nxt = e2e_pool.submit(prepare, e2e_seeds[0])
        for i in range(n_e2e):
            sc = nxt.result()
            nxt = e2e_pool.submit(prepare, e2e_seeds[i + 1])
            try:
                qs.qs_init_basis(h, 0)
                qs.qs_run_circuit(h, sc)              # uploads the schedule's matrices
                qs.qs_sample_stats(h, e2e_seeds[i], m)  # statistics and draws, one pass
            finally:
                qs.qs_schedule_free(sc)
        qs.qs_schedule_free(nxt.result())
        e2e_s = (time.perf_counter() - t0) / n_e2e
        # bytes the uploads moved (counted outside the timed loop)
        h2d = 0
        for i in range(n_e2e):
            sc = prepare(e2e_seeds[i])
            h2d += qs.qs_schedule_upload_bytes(sc, dtype)
            qs.qs_schedule_free(sc)
        e2e_pool.shutdown()
        e2e = {"value": e2e_s, "unit": "s/circuit", "h2d_bytes_per_step": h2d // n_e2e,
               "d2h_bytes_per_step": 4 * 8 + 8 * m,
               "circuits": n_e2e,
               "what": "host gate list -> schedule -> matrices to device -> run -> stats and 2^20 samples to host "
                       "(next circuit's schedule built while this one runs)"}

    qs.qs_free(h)
    extras = rank == 0 and args.workload == "5x6_d25_c128" and not args.plain
    # the spec form (learned schedule, complex64) on the 30- and 32-qubit
    # circuits, against the plain complex128 form and the oracle's amplitudes
    target = target_form(qs, stream, hbm_gbs) if extras and not args.no_target else None
    # the batched workload: 512 circuits in one graph-replayed persistent launch
    batch = batch_section(qs, stream, 5, 3)[0] if extras and not args.no_batch else None
    if rank != 0:
        return None
    # the first step touches the freshly allocated 16 GiB array (page faults):
    # it warms up, the second is reported
    cpu = None if args.no_cpu_baseline else cpu_baseline(args)
    line = {
        "metric": METRIC, "value": per_circuit, "unit": "s/circuit", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if dtype == qs.QS_C128 else "f32", "data": "synthetic",
        "config": {"workload": "%dx%d grid, %d qubits, %d CZ cycles, %s, %s" % (
            rows, cols, n, cycles, dt, "gate by gate" if args.plain else "fused k<=%d + phase diagonals" % k_max),
            "seeds": "rank*1000 + step", "l2": "state %.1f GiB > L2 129 MB (no flush needed)" % (state_bytes / 2**30),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "phase_fold": not args.no_fold, "search_threads": args.search_threads, "remap": args.remap,
            "schedule_upload": "in the preparation thread, ahead of the run",
            "cluster_search": _search_config(qs, args.plain)},
        "roofline": roof, "sweeps": sweeps, "plain": plain,
        "speedup_vs_plain": (plain["s_per_circuit"] / per_circuit) if plain else None,
        "porter_thomas": {"sum_p": stats[0], "entropy": stats[1], "m2": stats[3]},
        "e2e": e2e, "gpu_launches": launches[0], "clocks": clk.summary(), "cpu_baseline": cpu,
        "target_form": target, "batch512": batch,
    }
    return line


# ------------------------------------------------------- batched workload

def batch_section(qs, stream, steps, warmup, clock_index=None):
    """512 independent circuits (seeds 0..511; grids 4x4 / 4x5 / 3x7, depths
    8..40), complex64, one persistent launch replayed from a CUDA graph, against
    a loop of single-circuit launches of the same schedules.  Returns the
    measured figures and the per-launch device time."""
    import torch
    n_circ = 512
    circs = []
    for s_ in range(n_circ):
        r, c, d = qs.qs_batch_circuit_params(s_)
        circs.append(qs.qs_supremacy_circuit(r, c, d, s_))
    t0 = time.perf_counter()
    k_max, C, T, tune_ms = qs.qs_batch_autotune(circs, qs.QS_C64, stream)
    tune_s = time.perf_counter() - t0
    # the greedy clustering rule, as the autotuner's schedules (the 208-run
    # search would spend ~10 s of host time on 512 small circuits)
    scheds = [qs.qs_schedule_build(n, g, k_max=k_max, search_runs=1, search_first=1) for (n, g) in circs]
    b = qs.qs_batch_create(scheds, qs.QS_C64, stream)
    qs.qs_batch_set_config(b, C, T)
    for _ in range(warmup):
        qs.qs_batch_run_graph(b)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(clock_index) if clock_index is not None else None
    if clk:
        clk.__enter__()
    e0.record(stream)
    for _ in range(steps):
        qs.qs_batch_run_graph(b)
    e1.record(stream)
    torch.cuda.synchronize()
    if clk:
        clk.__exit__(None, None, None)
    elapsed = e0.elapsed_time(e1) / 1e3
    st = qs.qs_batch_stats(b, n_circ)
    qs.qs_batch_free(b)
    # loop of single-circuit launches (default kernel paths), same schedules
    states = {}
    for (n, _) in circs:
        if n not in states:
            states[n] = qs.qs_alloc(n, qs.QS_C64, stream)

    def loop():
        for (n, _), sc in zip(circs, scheds):
            qs.qs_init_basis(states[n], 0)
            qs.qs_run_circuit(states[n], sc)
    loop()
    torch.cuda.synchronize()
    e0.record(stream)
    loop()
    e1.record(stream)
    torch.cuda.synchronize()
    loop_s = e0.elapsed_time(e1) / 1e3
    for h in states.values():
        qs.qs_free(h)
    for sc in scheds:
        qs.qs_schedule_free(sc)
    per_launch = elapsed / steps
    out = {"workload": "512 circuits (seeds 0..511), grids 4x4/4x5/3x7, 8..40 CZ cycles, c64, one persistent "
                       "launch per step replayed from a CUDA graph",
           "autotuned": {"k_max": k_max, "cluster_ctas": C, "threads": T, "tune_ms": tune_ms,
                         "tune_wall_s": tune_s},
           "l2": "states total %.0f MB; inputs re-initialised every launch" % (
               sum(8 << n for (n, _) in circs) / 1e6),
           "launches": steps, "s_per_launch": per_launch,
           "circuits_per_s": n_circ / per_launch, "loop_circuits_per_s": n_circ / loop_s,
           "speedup_vs_loop": loop_s / per_launch,
           "mean_m2": float(st[:, 3].mean()), "max_norm_drift": float(abs(st[:, 0] - 1).max())}
    return out, elapsed, (clk.summary() if clk else None)


def run_batch(args):
    """The batched workload on its own (config 4)."""
    import torch
    from paper_1704_01127_gb300 import build as _build
    _build.build()
    import paper_1704_01127_gb300.qs as qs
    world, rank, local, dist = dist_setup(args)
    qs.qs_set_device(local)
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    barrier(dist)
    out, elapsed, clocks = batch_section(qs, stream, args.steps, args.warmup, local)
    elapsed = max_over_ranks(dist, elapsed)
    if rank != 0:
        return None
    per_launch = elapsed / args.steps
    return {
        "metric": METRIC, "value": per_launch / 512, "unit": "s/circuit", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_launch * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {k: out[k] for k in ("workload", "autotuned", "l2")},
        "circuits_per_s": out["circuits_per_s"], "loop_circuits_per_s": out["loop_circuits_per_s"],
        "speedup_vs_loop": out["speedup_vs_loop"], "mean_m2": out["mean_m2"],
        "max_norm_drift": out["max_norm_drift"], "gpu_launches": args.steps, "clocks": clocks,
    }


def load_golden_amplitudes(name):
    """Oracle amplitudes at sampled indices, stored by tests/golden/make_fullsize.py
    (params, indices, complex values); None if the file is absent."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", name)
    if not os.path.exists(path):
        return None
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    params = tuple(int(x) for x in rows[0][1:])
    idx = np.array([int(r[0]) for r in rows[2:]], dtype=np.uint64)
    amp = np.array([complex(float(r[1]), float(r[2])) for r in rows[2:]], dtype=np.complex128)
    return params, idx, amp


def target_form(qs, stream, hbm_gbs, harness_count=1500):
    """The learned-schedule complex64 form on the 30-qubit (5x6, seed 0) and
    32-qubit (4x8, seed 1) circuits with 25 CZ cycles: a cost model fitted on
    GPU timings of random complex64 ops (26-32 qubits), circuits planned with it
    (auto fallback) and with the analytic model, each run a4-a7 (|0...0>,
    sweeps, statistics) and timed with CUDA events (best of 3 after a warm
    run), amplitudes at the stored oracle indices compared with the oracle, and
    the plain gate-by-gate complex128 form of the same circuit timed once."""
    import numpy as np
    import torch
    t0 = time.perf_counter()
    F, T = qs.qs_cost_sample(26, 32, qs.QS_C64, harness_count, seed=64, max_ms=100.0)
    harness_s = time.perf_counter() - t0
    cm = qs.qs_cost_model_create(hbm_gbs)
    t1 = time.perf_counter()
    rep = qs.qs_cost_model_fit(cm, F, T, epochs=1500, seed=7)
    fit_s = time.perf_counter() - t1
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(h, sc, reps):
        best = None
        for _ in range(reps):
            e0.record(stream)
            qs.qs_init_basis(h, 0)
            qs.qs_run_circuit(h, sc)
            st = qs.qs_stats(h)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            best = t if best is None else min(best, t)
        return best, st

    circuits = []
    for name in ("fullsize_5x6_d25_s0.txt", "fullsize_4x8_d25_s1.txt"):
        gold = load_golden_amplitudes(name)
        if gold is None:
            continue
        (rows, cols, cycles, seed, n), idx, want = gold
        nq, g = qs.qs_supremacy_circuit(rows, cols, cycles, seed)
        res = {"grid": "%dx%d" % (rows, cols), "qubits": nq, "cz_cycles": cycles, "seed": seed, "dtype": "c64"}
        h = qs.qs_alloc(nq, qs.QS_C64, stream)
        try:
            for label, which in (("learned", qs.QS_COST_AUTO), ("analytic", qs.QS_COST_ANALYTIC)):
                sc, km, pred = qs.qs_plan_circuit(nq, g, qs.QS_C64, cm, which)
                try:
                    timed(h, sc, 1)                              # uploads the schedule
                    best, st = timed(h, sc, 3)
                    got = qs.qs_get_amplitudes_at(h, idx)
                    qs.qs_init_basis(h, 0)
                    op_ms = qs.qs_run_circuit_timed(h, sc)
                    kms, pms, pbytes, _, _ = classify_sweeps(qs, sc, op_ms, nq, qs.QS_C64)
                    err = float(np.max(np.abs(got - want)))
                    sweep_bytes = 2 * (8 << nq)
                    dom = max(kms, key=lambda kk: sum(kms[kk])) if kms else None
                    roof = None
                    if dom is not None:
                        dms = statistics.mean(kms[dom])
                        roof = {"kernel": "%s_k%d" % dom if dom[0] == "dense" else dom[0],
                                "launches": len(kms[dom]), "kernel_ms": dms,
                                "achieved_gbs": sweep_bytes / (dms * 1e-3) / 1e9,
                                "frac": sweep_bytes / (dms * 1e-3) / 1e9 / hbm_gbs}
                    moved = int(np.sum(qs.qs_schedule_get_remap(sc) != np.arange(nq)))
                    res[label] = {"k_max": km, "ops": qs.qs_schedule_num_ops(sc), "predicted_s": pred / 1e3,
                                  "qubits_moved": moved,
                                  "s_per_circuit": best, "max_abs_dpsi_vs_oracle": err,
                                  "rel_dpsi": err / float(np.max(np.abs(want))),
                                  "norm": st[0], "m2": st[3], "full_sweep_roofline": roof,
                                  "partial_support": {"launches": len(pms), "total_ms": sum(pms),
                                                      "gbs": pbytes / (sum(pms) * 1e-3) / 1e9 if pms else None}}
                finally:
                    qs.qs_schedule_free(sc)
        finally:
            qs.qs_free(h)
        res["gain_learned_vs_analytic"] = res["analytic"]["s_per_circuit"] / res["learned"]["s_per_circuit"]
        # plain gate-by-gate complex128 form of the same circuit
        hp = qs.qs_alloc(nq, qs.QS_C128, stream)
        try:
            scp = qs.qs_schedule_build(nq, g, fuse=False)
            try:
                best, _ = timed(hp, scp, 1)
            finally:
                qs.qs_schedule_free(scp)
        finally:
            qs.qs_free(hp)
        res["plain_c128_s_per_circuit"] = best
        res["speedup_vs_plain_c128"] = best / res["learned"]["s_per_circuit"]
        res["within_tolerance"] = res["learned"]["max_abs_dpsi_vs_oracle"] <= 2e-6
        circuits.append(res)
    qs.qs_cost_model_free(cm)
    return {"what": "learned-schedule (MLP cost model, auto fallback) complex64 form against the analytic-model "
                    "plan and the plain gate-by-gate complex128 form; a4-a7 per circuit, CUDA events, best of 3",
            "cost_model": {"harness_timings": int(T.size), "harness_s": harness_s, "fit_s": fit_s,
                           "mlp_holdout_median_abs_log_err": rep["mlp_holdout_median_abs_log_err"],
                           "analytic_holdout_median_abs_log_err": rep["analytic_holdout_median_abs_log_err"],
                           "uses_mlp": rep["use_mlp"]},
            "circuits": circuits}


# ------------------------------------------------------- learned scheduling

def run_learned(args):
    """Harness timings of random clusters -> MLP fitted on the GPU -> circuits
    planned with the analytic model and with the learned model (auto fallback),
    both measured; grids 4x7 / 5x6 / 3x11, 30 CZ cycles, complex64 and complex128."""
    import numpy as np
    import torch
    from paper_1704_01127_gb300 import build as _build
    _build.build()
    import paper_1704_01127_gb300.qs as qs
    world, rank, local, dist = dist_setup(args)
    qs.qs_set_device(local)
    torch.cuda.set_device(local)
    hbm_gbs, _, _ = load_peaks()
    t0 = time.perf_counter()
    F, T = [], []
    # (n range, samples, ms cap): cheap sizes in bulk, large ones sparsely
    plan = [((18, 26), 7500, 400.0), ((27, 30), 2000, 400.0), ((31, 33), 500, 400.0)]
    for dt in (qs.QS_C64, qs.QS_C128):
        for (lo, hi), cnt, cap in plan:
            f, t = qs.qs_cost_sample(lo, hi, dt, cnt, seed=1000 * dt + lo, max_ms=cap)
            F.append(f)
            T.append(t)
    F, T = np.concatenate(F), np.concatenate(T)
    harness_s = time.perf_counter() - t0
    cm = qs.qs_cost_model_create(hbm_gbs)
    t1 = time.perf_counter()
    rep = qs.qs_cost_model_fit(cm, F, T, epochs=2000, seed=7)
    fit_s = time.perf_counter() - t1
    rows = []
    for (r, c) in ((4, 7), (5, 6), (3, 11)):
        for dt in (qs.QS_C64, qs.QS_C128):
            n, g = qs.qs_supremacy_circuit(r, c, 30, 0)
            h = qs.qs_alloc(n, dt)
            res = {"grid": "%dx%d" % (r, c), "qubits": n, "dtype": "c128" if dt else "c64"}
            for name, which in (("analytic", qs.QS_COST_ANALYTIC), ("learned", qs.QS_COST_AUTO)):
                sc, km, pred = qs.qs_plan_circuit(n, g, dt, cm, which)
                times = []
                for rep_i in range(2):
                    qs.qs_init_basis(h, 0)
                    ms = qs.qs_run_circuit_timed(h, sc)
                    times.append(float(ms[ms >= 0].sum()))   # -1: a phase op run inside the sweep before it
                paths = [qs.qs_schedule_op(sc, i) for i in range(qs.qs_schedule_num_ops(sc))]
                res[name] = {"k_max": km, "predicted_s": pred / 1e3, "measured_s": min(times) / 1e3,
                             "ops": len(paths),
                             "qubits_moved": int(np.sum(qs.qs_schedule_get_remap(sc) != np.arange(n)))}
                qs.qs_schedule_free(sc)
            res["gain"] = res["analytic"]["measured_s"] / res["learned"]["measured_s"]
            qs.qs_free(h)
            rows.append(res)
    qs.qs_cost_model_free(cm)
    if rank != 0:
        return None
    geo = float(np.exp(np.mean([np.log(r["gain"]) for r in rows])))
    return {"metric": METRIC, "value": sum(r["learned"]["measured_s"] for r in rows) / len(rows), "unit": "s/circuit",
            "n_gpus": world, "steps": 1, "warmup": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "mixed", "data": "synthetic",
            "config": {"workload": "learned scheduling: 4x7, 5x6, 3x11 grids, 30 CZ cycles, c64 and c128"},
            "harness": {"timings": int(T.size), "seconds": harness_s}, "fit": dict(rep, seconds=fit_s),
            "circuits": rows, "geomean_gain_learned_vs_analytic": geo}


def _search_config(qs, plain):
    """The clustering search the schedules were built with (the binding's
    defaults), as reported in the JSON line."""
    if plain:
        return None
    p = inspect.signature(qs.qs_schedule_build).parameters
    R, F, s0 = (p[k].default for k in ("search_runs", "search_first", "search_slack0"))
    return {"runs": R * F, "first_clusters": F,
            "rules": "greedy + support-aware slack %d..%d" % (s0, s0 + R - 2),
            "cost": "sum over dense sweeps of 2^(|support| - n) from |0...0>"}


# ------------------------------------------------------- single-kernel timing

def run_kernel(args):
    """One kernel at a time on a full synthetic state (the per-kernel roofline
    table and the small cases ncu captures): --kernel dense|diag|phase|stats|
    sample|fill|mlp, --n qubits, --dtype c64|c128, --k cluster size, --targets
    (comma list; default the k highest qubits), --path auto|cuda|tensor, --reps
    launches.  Every launch is timed with CUDA events on the state's stream; the
    JSON line gives the mean time, the algorithmic bytes of one launch and
    their rate against the measured HBM copy bandwidth."""
    import numpy as np
    import torch
    from paper_1704_01127_gb300 import build as _build
    _build.build()
    import paper_1704_01127_gb300.qs as qs
    torch.cuda.set_device(0)
    hbm_gbs, _, peak_src = load_peaks()
    stream = torch.cuda.Stream()
    n, k = args.n, args.k
    dtype = qs.QS_C128 if args.dtype == "c128" else qs.QS_C64
    amp = 16 if dtype == qs.QS_C128 else 8
    g = np.random.Generator(np.random.PCG64(12345 + n + 31 * k))
    targets = [int(x) for x in args.targets.split(",")] if args.targets else list(range(n - k, n))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    times = []

    def timed(fn):
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    if args.kernel == "mlp":
        net = qs.qs_mlp_create(1)
        X = g.standard_normal((args.batch, qs.QS_NFEAT))
        Y = g.standard_normal(args.batch)
        qs.qs_mlp_train(net, X, Y, 5)
        t = time.perf_counter()
        qs.qs_mlp_train(net, X, Y, args.reps)
        per = (time.perf_counter() - t) / args.reps * 1e3
        qs.qs_mlp_free(net)
        print(json.dumps({"kernel": "mlp training epoch (k_mlp_fwd, k_mlp_delta, k_mlp_grad, k_adam)",
                          "batch": args.batch, "epochs": args.reps, "ms_per_epoch": per}))
        return None
    h = qs.qs_alloc(n, dtype, stream)
    path = {"auto": qs.QS_PATH_AUTO, "cuda": qs.QS_PATH_CUDA_CORES, "tensor": qs.QS_PATH_TENSOR}[args.path]
    qs.qs_set_path(h, path)
    qs.qs_init_uniform(h)
    full = amp << n
    if args.kernel == "pair":
        # two 5-qubit clusters in a row, as one pair sweep (qs_set_pair_sweeps) or two
        t2 = [int(x) for x in args.targets2.split(",")] if args.targets2 else list(range(n - 10, n - 5))
        ops = []
        for tg in (targets, t2):
            z = g.standard_normal((32, 32)) + 1j * g.standard_normal((32, 32))
            ops.append((qs.QS_OP_DENSE, tg, np.linalg.qr(z)[0]))
        sc = qs.qs_schedule_from_ops(n, ops)
        qs.qs_set_pair_sweeps(h, not args.no_pair)
        fn = lambda: qs.qs_run_circuit(h, sc)
        what, bytes_ = ("two clusters on %s then %s, %s" % (targets, t2, "separate sweeps" if args.no_pair
                                                             else "one pair sweep")), 2 * full
    elif args.kernel == "dense":
        z = g.standard_normal((1 << k, 1 << k)) + 1j * g.standard_normal((1 << k, 1 << k))
        U, _ = np.linalg.qr(z)
        fn, what, bytes_ = (lambda: qs.qs_apply_cluster(h, targets, U)), "dense k=%d on %s" % (k, targets), 2 * full
    elif args.kernel == "swap":
        # exchange qubits targets[j] <-> targets2[j] (qs_swap_qubits)
        a = [int(x) for x in args.targets.split(",")] if args.targets else [2, 3, 4]
        b = [int(x) for x in args.targets2.split(",")] if args.targets2 else list(range(n - 1, n - 1 - len(a), -1))
        fn, what, bytes_ = (lambda: qs.qs_swap_qubits(h, a, b)), "exchange of %s with %s" % (a, b), 2 * full
    elif args.kernel == "diag":
        d = np.exp(1j * g.uniform(0, 2 * np.pi, 1 << k))
        fn, what, bytes_ = (lambda: qs.qs_apply_diag(h, targets, d)), "diag k=%d on %s" % (k, targets), 2 * full
    elif args.kernel == "phase":
        coeff = g.integers(0, 8, n)
        edges = [tuple(sorted(int(x) for x in g.permutation(n)[:2])) for _ in range(n)]
        fn, what, bytes_ = (lambda: qs.qs_apply_phase(h, coeff, edges)), "phase, %d CZ terms" % n, 2 * full
    elif args.kernel == "stats":
        fn, what, bytes_ = (lambda: qs.qs_stats(h)), "statistics pass", full
    elif args.kernel == "sample":
        fn, what, bytes_ = ((lambda: qs.qs_sample(h, 7, args.m)),
                            "%d draws (bytes: the block sums read the state once)" % args.m, full)
    elif args.kernel == "fill":
        def fn():
            qs.qs_init_basis(h, 0)
            qs.qs_device_ptr(h)          # writes the zeros outside the support
        what, bytes_ = "basis state written in full", full
    else:
        raise SystemExit("unknown kernel %s" % args.kernel)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    for _ in range(args.reps):
        times.append(timed(fn))
    qs.qs_free(h)
    ms = statistics.mean(times)
    print(json.dumps({"kernel": args.kernel, "what": what, "n": n, "dtype": args.dtype, "path": args.path,
                      "reps": args.reps, "mean_ms": ms, "min_ms": min(times),
                      "algorithmic_bytes": bytes_, "gbs": bytes_ / (ms * 1e-3) / 1e9,
                      "hbm_frac": bytes_ / (ms * 1e-3) / 1e9 / hbm_gbs, "peak_gbs": hbm_gbs,
                      "peak_source": peak_src}))
    return None


# ------------------------------------------------------------ oracle (CPU) leg

def host_cpu():
    """CPU model and core count of this host, for the baseline's record."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return {"model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def _oracle_chunks(args):
    """The workload's circuit from the oracle's generator and a fresh |0...0>."""
    from oracle import circuit as ocircuit
    from oracle import sim as osim
    rows, cols, removed, cycles, dt, k_max = WORKLOADS[args.workload]
    n, gates = ocircuit.supremacy_circuit(rows, cols, cycles, 0, removed=removed)
    return (rows, cols, cycles), n, gates, osim


def _time_gates(osim, psi, gates):
    t0 = time.perf_counter()
    for g in gates:
        osim.apply_gate(psi, g[1], g[2])
    return time.perf_counter() - t0


def cpu_baseline(args):
    """The oracle, as it stands, on a bounded sample of the workload: a
    contiguous run of the circuit's gates applied gate by gate to the full state
    on the host (all cores, median of three runs), scaled to the whole circuit
    by its gate count; and the same on one core with a shorter run."""
    (rows, cols, cycles), n, gates, osim = _oracle_chunks(args)
    psi = osim.basis_state(n, 0)
    G = len(gates)
    cores = os.cpu_count() or 1
    osim.set_threads(cores)
    _time_gates(osim, psi, gates[:2])               # first touch of the array
    used = osim.max_threads()
    # runs start a quarter, half and three quarters into the circuit, so that
    # they hold its mix of single-qubit gates and CZs (the first 2^n gates are
    # all Hadamards)
    span, runs = 16, []
    for r in range(3):
        lo = (r + 1) * G // 4
        runs.append(_time_gates(osim, psi, gates[lo:lo + span]) * G / span)
    osim.set_threads(1)
    span1, runs1 = 2, []
    for r in range(3):
        lo = (r + 1) * G // 5
        runs1.append(_time_gates(osim, psi, gates[lo:lo + span1]) * G / span1)
    osim.set_threads(cores)
    del psi
    cpu = host_cpu()
    what = ("contiguous runs of %d gates (starting 1/4, 1/2, 3/4 into the circuit for all cores, 1/5, "
            "2/5, 3/5 for one core) of the %dx%d, %d-cycle circuit (%d gates) applied gate by gate to the "
            "full 2^%d-amplitude complex128 state by the oracle, after a 2-gate warm-up that first touches "
            "the array; median of 3 runs, scaled to the whole circuit by its gate count")
    return {"value": statistics.median(runs), "unit": "s/circuit", "cores": used, "kind": "oracle",
            "sample": what % (span, rows, cols, cycles, G, n), "cpu": cpu["model"], "nproc": cpu["nproc"],
            "runs": runs,
            "single_core": {"value": statistics.median(runs1), "unit": "s/circuit", "cores": 1,
                            "sample": what % (span1, rows, cols, cycles, G, n), "runs": runs1}}


def run_reference(args):
    """The oracle as the reference arm.  The K timed steps split the workload's
    circuit into K contiguous runs of gates (ceil(G/K) each; the last may be
    shorter), applied gate by gate to the full state on all host cores, so the
    K steps together apply the whole circuit once: `value` is that measured
    circuit time, `ms_per_step` the mean time of a step.  Each warm-up step
    applies one gate (the first touches the array)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    (rows, cols, cycles), n, gates, osim = _oracle_chunks(args)
    G = len(gates)
    cores = os.cpu_count() or 1
    osim.set_threads(cores)
    used = osim.max_threads()
    psi = osim.basis_state(n, 0)
    for w in range(args.warmup):
        _time_gates(osim, psi, gates[w % G:w % G + 1])
    psi[:] = 0
    psi[0] = 1
    c = -(-G // args.steps)
    times, done = [], 0
    for j in range(args.steps):
        chunk = gates[j * c:(j + 1) * c]
        times.append(_time_gates(osim, psi, chunk))
        done += len(chunk)
    del psi
    total = sum(times)
    v = total if done >= G else total * G / max(done, 1)
    cpu = host_cpu()
    sample = ("the %dx%d, %d-cycle circuit (%d gates) applied gate by gate to |0...0> (2^%d complex128 "
              "amplitudes) by the oracle on %d host threads, split into %d steps of up to %d contiguous "
              "gates; %s" % (rows, cols, cycles, G, n, used, args.steps, c,
                             "value = the measured time of the whole circuit" if done >= G else
                             "value scaled from %d of its gates" % done))
    cb = {"value": v, "unit": "s/circuit", "cores": used, "kind": "oracle", "sample": sample,
          "cpu": cpu["model"], "nproc": cpu["nproc"], "gates_timed": done, "circuit_gates": G}
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "s/circuit", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "%dx%d grid, %d CZ cycles, gate-by-gate complex128 oracle on the host" % (
                rows, cols, cycles)},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "s/circuit", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch512_c64", "learned"], default="5x6_d25_c128")
    ap.add_argument("--plain", action="store_true", help="gate-by-gate form instead of fused")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fold", action="store_true",
                    help="run every phase op as its own sweep (no folding into the tensor-core sweep before it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-target", action="store_true",
                    help="skip the learned-schedule complex64 runs of the 30- and 32-qubit circuits")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-circuit batched run")
    ap.add_argument("--search-threads", type=int, default=max(1, (os.cpu_count() or 1) - 2),
                    help="host threads of the clustering search (the launching thread keeps the rest)")
    ap.add_argument("--remap", action="store_true",
                    help="move each schedule's qubits to the index bits the library picks (Sec. 3.6)")
    ap.add_argument("--kernel", choices=["dense", "pair", "swap", "diag", "phase", "stats", "sample", "fill", "mlp"],
                    help="time one kernel on a full synthetic state instead of circuits")
    ap.add_argument("--n", type=int, default=28)
    ap.add_argument("--k", type=int, default=5)
    ap.add_argument("--dtype", choices=["c64", "c128"], default="c128")
    ap.add_argument("--targets", default="")
    ap.add_argument("--targets2", default="", help="--kernel pair: the second cluster's targets")
    ap.add_argument("--no-pair", action="store_true", help="--kernel pair: two separate sweeps")
    ap.add_argument("--path", choices=["auto", "cuda", "tensor"], default="auto")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--m", type=int, default=1 << 20)
    ap.add_argument("--batch", type=int, default=4096)
    args = ap.parse_args()
    if args.warmup < 3:
        print("note: warmup raised to 3", file=sys.stderr)
        args.warmup = 3
    if args.kernel:
        line = run_kernel(args)
    elif args.impl == "reference":
        line = run_reference(args)
    elif args.workload == "batch512_c64":
        line = run_batch(args)
    elif args.workload == "learned":
        line = run_learned(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()

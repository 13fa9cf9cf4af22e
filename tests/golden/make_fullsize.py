"""Write the oracle's amplitudes of a full-size supremacy circuit at sampled indices.

Calls only ``oracle/`` (and the seeded index generator of ``tests/inputs.py``):
the circuit comes from the oracle's generator (Fig. 1 rules), the state from its
gate-by-gate complex128 simulator (Sec. 2), the statistics from its serial
reductions.  Nothing here touches the CUDA library.

    python tests/golden/make_fullsize.py 5 6 25 0      # 30 qubits, 16 GiB of host memory
    python tests/golden/make_fullsize.py 4 8 25 1      # 32 qubits, 64 GiB of host memory

Output: tests/golden/fullsize_<R>x<C>_d<D>_s<seed>.txt with the circuit's
parameters, the oracle's (sum p, entropy, mean N p, mean (N p)^2), and one line
"index re im" per sampled index (indices 0 and 2^n - 1 first, then M - 2
indices drawn by PCG64 from the seed 7 * 2^20 + n, in draw order), values
written with 17 significant digits so that they read back exactly.
"""
import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

from oracle import circuit, sim  # noqa: E402
from inputs import rng  # noqa: E402


def sample_indices(n, m):
    g = rng(7 * (1 << 20) + n)
    rest = g.integers(0, 1 << n, m - 2, dtype=np.uint64)
    return np.concatenate([np.array([0, (1 << n) - 1], dtype=np.uint64), rest])


def golden_name(rows, cols, cycles, seed):
    return "fullsize_%dx%d_d%d_s%d.txt" % (rows, cols, cycles, seed)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("rows", type=int)
    ap.add_argument("cols", type=int)
    ap.add_argument("cycles", type=int)
    ap.add_argument("seed", type=int)
    ap.add_argument("--m", type=int, default=2048, help="sampled indices")
    ap.add_argument("--threads", type=int, default=0, help="host threads (0: all)")
    ap.add_argument("--out", default=HERE)
    a = ap.parse_args()
    if a.threads:
        sim.set_threads(a.threads)
    n, gates = circuit.supremacy_circuit(a.rows, a.cols, a.cycles, a.seed)
    t0 = time.time()
    psi = sim.run_circuit(n, gates)
    t_run = time.time() - t0
    st = sim.stats(psi)
    idx = sample_indices(n, a.m)
    amp = psi[idx.astype(np.int64)]
    path = os.path.join(a.out, golden_name(a.rows, a.cols, a.cycles, a.seed))
    with open(path, "w") as f:
        f.write("# Oracle amplitudes of the %dx%d-grid supremacy circuit (Fig. 1 rules), %d CZ cycles,\n"
                % (a.rows, a.cols, a.cycles))
        f.write("# seed %d, n = %d qubits, %d gates, applied gate by gate to |0...0> in complex128\n"
                % (a.seed, n, len(gates)))
        f.write("# (Sec. 2).  Written by tests/golden/make_fullsize.py %d %d %d %d --m %d,\n"
                % (a.rows, a.cols, a.cycles, a.seed, a.m))
        f.write("# which calls only oracle/ (%d host threads, %.0f s for the circuit).\n"
                % (sim.max_threads(), t_run))
        f.write("params %d %d %d %d %d\n" % (a.rows, a.cols, a.cycles, a.seed, n))
        f.write("stats %.17g %.17g %.17g %.17g\n" % st)
        for i, z in zip(idx, amp):
            f.write("%d %.17g %.17g\n" % (int(i), z.real, z.imag))
    print("%s: n=%d, %d gates, %.1f s, stats %s" % (path, n, len(gates), t_run, st))


if __name__ == "__main__":
    main()

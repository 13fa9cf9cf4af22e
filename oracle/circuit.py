"""Supremacy-circuit generator (Fig. 1 caption, Sec. 3.6).  Oracle only.

Rules, as the Fig. 1 caption states them:
  * cycle 0: a Hadamard on every qubit;
  * cycles t >= 1: one of eight staggered nearest-neighbour CZ layouts, repeated
    every 8 cycles so that every coupling of the 2-D grid is used once per 8;
  * in cycle t a qubit gets a single-qubit gate iff it was in a CZ in cycle t-1
    but is not in one in cycle t;
  * its first such gate is T; later ones are drawn uniformly from
    {T, X^{1/2}, Y^{1/2}} minus the previous single-qubit gate on that qubit.

Readings where the paper is silent (the layout figure is missing):
  * qubit q = r*C + c on an R x C grid (row-major, removed sites skipped);
  * H(a,b) = edges (r,c)-(r,c+1) with c%2 == a and r%2 == b,
    V(a,b) = edges (r,c)-(r+1,c) with r%2 == a and c%2 == b,
    cycle t uses [H(1,0), V(0,0), H(0,0), V(1,0), V(0,1), H(1,1), V(1,1),
    H(0,1)][(t-1) % 8];
  * the random choice: draw r = (SplitMix64 output j) >> 63 for the j-th
    non-first single-qubit gate (cycles ascending, qubits ascending) and take
    the r-th of the two allowed gates in the order T < X^{1/2} < Y^{1/2};
  * within a cycle the single-qubit gates (ascending qubit) come before the CZs
    (ascending (a, b), a < b); they act on disjoint qubits and commute.
"""

MASK64 = (1 << 64) - 1

LAYOUTS = (("H", 1, 0), ("V", 0, 0), ("H", 0, 0), ("V", 1, 0),
           ("V", 0, 1), ("H", 1, 1), ("V", 1, 1), ("H", 0, 1))

ONE_QUBIT_CHOICES = ("t", "x_1_2", "y_1_2")


def splitmix64(seed, j):
    """Output j (j >= 0) of SplitMix64 (Steele, Lea, Flood 2014) seeded with seed."""
    z = (seed + (j + 1) * 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def grid_sites(rows, cols, removed=()):
    """Row-major list of the grid sites that hold a qubit."""
    removed = set(tuple(s) for s in removed)
    return [(r, c) for r in range(rows) for c in range(cols) if (r, c) not in removed]


def layout_edges(rows, cols, t, removed=()):
    """CZ pairs (a, b), a < b, of cycle t >= 1, sorted."""
    sites = grid_sites(rows, cols, removed)
    index = {s: i for i, s in enumerate(sites)}
    kind, a, b = LAYOUTS[(t - 1) % 8]
    edges = []
    for (r, c) in sites:
        if kind == "H":
            if c % 2 == a and r % 2 == b and (r, c + 1) in index:
                edges.append((index[(r, c)], index[(r, c + 1)]))
        else:
            if r % 2 == a and c % 2 == b and (r + 1, c) in index:
                edges.append((index[(r, c)], index[(r + 1, c)]))
    return sorted((min(e), max(e)) for e in edges)


def supremacy_circuit(rows, cols, cz_cycles, seed, removed=()):
    """Return (n, gates) with gates a list of (cycle, name, qubits) tuples."""
    sites = grid_sites(rows, cols, removed)
    n = len(sites)
    gates = [(0, "h", (q,)) for q in range(n)]
    prev_cz = set()
    last = {}
    draw = 0
    for t in range(1, cz_cycles + 1):
        edges = layout_edges(rows, cols, t, removed)
        in_cz = set(q for e in edges for q in e)
        for q in range(n):
            if q in prev_cz and q not in in_cz:
                if q not in last:
                    g = "t"
                else:
                    allowed = [x for x in ONE_QUBIT_CHOICES if x != last[q]]
                    g = allowed[splitmix64(seed, draw) >> 63]
                    draw += 1
                gates.append((t, g, (q,)))
                last[q] = g
        for (a, b) in edges:
            gates.append((t, "cz", (a, b)))
        prev_cz = in_cz
    return n, gates


def inverse_circuit(gates):
    """Gates of C^dagger: reversed order, each gate replaced by its adjoint."""
    from .gates import INVERSE_NAME
    return [(cyc, INVERSE_NAME[name], qs) for (cyc, name, qs) in reversed(gates)]


def to_text(n, gates):
    """Circuit text format: first line the qubit count, then 'cycle name q [q]'."""
    lines = ["%d" % n]
    for (cyc, name, qs) in gates:
        lines.append("%d %s %s" % (cyc, name, " ".join(str(q) for q in qs)))
    return "\n".join(lines) + "\n"


def from_text(text):
    rows = [ln.split() for ln in text.strip().splitlines() if ln.strip()]
    n = int(rows[0][0])
    gates = [(int(r[0]), r[1], tuple(int(x) for x in r[2:])) for r in rows[1:]]
    return n, gates


BATCH_GRIDS = ((4, 4), (4, 5), (3, 7))


def batch_circuit_params(seed):
    """Grid and CZ-cycle count of circuit `seed` of the batched workload (grids
    uniform over 4x4, 4x5, 3x7; depths uniform over 8..40).  Reading: r is output
    0 of SplitMix64 seeded with seed XOR 0x6A09E667F3BCC909; the grid is r mod 3
    in the order above and the depth 8 + ((r >> 32) mod 33)."""
    r = splitmix64(seed ^ 0x6A09E667F3BCC909, 0)
    rows, cols = BATCH_GRIDS[r % 3]
    return rows, cols, 8 + ((r >> 32) % 33)

"""Oracle -- test infrastructure only.

A plain, slow, obviously correct CPU restatement of what the simulator computes,
written from Haener & Steiger, "0.5 Petabyte Simulation of a 45-Qubit Quantum
Circuit" (Sec. 2, Sec. 3.2, Sec. 3.6, Fig. 1).  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference legs of
``bench.py`` may import it.  It shares no code, header, constant or helper with
the CUDA library in ``paper_1704_01127_gb300`` and never imports it.

Modules
  gates     exact gate matrices of Sec. 2
  circuit   supremacy-circuit generator (Fig. 1 caption, Sec. 3.6)
  sim       gate-by-gate complex128 simulator (C core in statevec.c) + dense
            Kronecker mode for n <= 10 (Sec. 2)
  schedule  greedy k-qubit clustering (Sec. 3.6, step 2) and cluster unitaries
  build     compiles statevec.c with gcc

Parity status: the final-state amplitudes of the generated supremacy circuits
are pinned only through the properties the definitions fix (H layer, norm,
Kronecker product, inverse circuit, Porter-Thomas moments); the paper prints no
amplitudes.  The cluster counts of Table 1 pin the scheduler only loosely
(the CZ layouts are this project's reading).
"""

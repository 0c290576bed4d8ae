"""CPU oracle for the iFCI increment CI solve — TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 implementation of what the GPU library computes, written
from the paper's Methods section ("Incremental Full Configuration Interaction",
Eqs. 1-5) and from the textbook Slater–Condon rules.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
It shares no code with the CUDA path (no kernels, headers, tables or helpers);
the only common module is ``synth`` (seeded input draws).

Modules
-------
``sc_fci.c``   Slater–Condon elements on spin-orbital bit strings, dense H,
               matrix-free matvec, brute-force 1-/2-RDMs and <S-S+>.
``fci.py``     Frozen-body subsystems, determinant lists, dense/Lanczos lowest
               singlet, E_0, increments (Eqs. 2-5), RDM gradient.
``build.py``   Compiles ``sc_fci.c`` with gcc into ``oracle/_build``.

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test against closed forms, brute force,
invariants or the paper's Table 1 counts.
"""

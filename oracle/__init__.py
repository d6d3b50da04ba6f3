"""Plain FP64 CPU oracle for the entropic lattice-BGK step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this package.  The product library never does, and the two share no code.

Parity status of each part is listed in the docstrings of ``oracle.core`` and
``oracle.analysis``.
"""

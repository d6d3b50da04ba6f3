"""GB300 (sm_103a) lattice-BGK library with the entropic equilibrium (arXiv 2303.08163).

The compute path is the C-ABI shared library built from ``csrc/``; this package holds the
thin ctypes binding (``paper_2303_08163_gb300.lbm``), seeded input generators
(``inputs``) and host-side fits of probe series (``fits``).
"""

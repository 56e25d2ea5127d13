"""FP64 CPU oracle of the KBC lattice Boltzmann FSI method -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.
"""

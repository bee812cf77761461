"""CPU FP64 oracle of the lattice Boltzmann hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this package.  The product path never does.
"""

"""GB300-native lattice Boltzmann hot path (stream-collide, adjoint, batches).

The compute path is the C-ABI library ``libxlb.so`` (CUDA for sm_103a) declared
in ``include/xlb.h``; ``paper_2311_16080_gb300.xlb`` is its thin binding.
Importing this package loads nothing; the library is loaded on first use and a
missing library raises instead of falling back to any CPU code.
"""

"""GB300-native partial-assembly finite element operators (H1 diffusion and mass on hexahedra).

The compute path lives in the CUDA library ``libfe.so`` (C ABI declared in ``include/fe.h``);
``paper_2603_09038_gb300.fe`` is its thin ctypes binding.  Importing this package loads nothing;
``fe.load()`` loads the library and raises if it is missing.
"""

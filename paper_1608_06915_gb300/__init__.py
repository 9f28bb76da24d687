"""Grid-refined entropic lattice Boltzmann (KBC, D3Q27) on GB300.

The compute path is the CUDA library ``liblbm.so`` (C ABI, ``include/lbm.h``);
``paper_1608_06915_gb300.lbm`` is its thin ctypes binding and
``paper_1608_06915_gb300.inputs`` builds seeded synthetic workloads.
"""

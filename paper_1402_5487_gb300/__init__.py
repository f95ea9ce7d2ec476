"""GB300 (sm_103a) parametric lattice Boltzmann method (arXiv:1402.5487).

The compute path is libplbm.so: hand-written CUDA kernels behind the C ABI of
``include/plbm.h``.  ``plbm`` is its thin ctypes binding; ``inputs`` holds the
seeded synthetic workloads; ``build`` compiles the library in-tree with nvcc.
Importing this package loads nothing heavy; the shared library is loaded on
first use and a missing library raises instead of falling back to the CPU.
"""

__all__ = ["plbm", "inputs", "build"]

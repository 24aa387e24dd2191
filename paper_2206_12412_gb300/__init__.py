"""GB300 (sm_103a) lattice Boltzmann method for antiplane shear with dynamic
mode III crack propagation (arXiv 2206.12412).

The compute path is the CUDA library ``liblbm.so`` behind the C ABI in
``include/lbm.h``; ``lbm`` is its Python binding and ``workloads`` builds the
seeded synthetic problems.  Importing this package loads nothing; the library
is loaded (and built in-tree if needed) on first use.
"""
__all__ = ["lbm", "workloads", "build"]

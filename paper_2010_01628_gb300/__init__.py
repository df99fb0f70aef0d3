"""GB300 (sm_103a) D3Q19 central-moment lattice Boltzmann library.

The compute path is ``csrc/`` (CUDA kernels behind the C ABI of
``include/lbm.h``), built into ``liblbm.so`` by ``build.py``; ``binding`` is
the ctypes layer with the same entry-point names.  Importing this package
loads nothing; ``from paper_2010_01628_gb300 import binding`` loads the
library and fails loudly if it has not been built.
"""
__all__ = ["binding", "build", "inputs"]

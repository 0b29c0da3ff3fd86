"""GB300-native (sm_103a) lattice Boltzmann hot path of arXiv:2009.04604.

Fused BGK/TRT stream-collide on D2Q9, D3Q19 and D3Q27 with the paper's
single-node curved-wall boundary rules (ELIBB-F, -FQ, -U, -UQ) and the BFL
comparison rule in the same pass, behind the
C ABI of ``include/lbm.h`` (``liblbm.so``). ``lbm`` is the ctypes binding,
``build`` compiles the library, ``workloads`` holds the seeded input generators.
"""
__all__ = ["lbm", "build", "workloads"]

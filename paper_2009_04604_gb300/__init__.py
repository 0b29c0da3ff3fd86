"""GB300-native (sm_103a) lattice Boltzmann hot path of arXiv:2009.04604.

Fused BGK stream-collide on D2Q9/D3Q19 with the paper's single-node curved-wall
boundary rule (ELIBB) and the BFL comparison rule in the same pass, behind the
C ABI of ``include/lbm.h`` (``liblbm.so``). ``lbm`` is the ctypes binding,
``build`` compiles the library, ``workloads`` holds the seeded input generators.
"""
__all__ = ["lbm", "build", "workloads"]

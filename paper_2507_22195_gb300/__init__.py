"""GB300-native hot path of the entropy-variable macro-element HDG method
(arXiv 2507.22195): residual, local Jacobian, static condensation with a
batched dense LU, and recovery, behind the C-ABI of include/mehdg.h.

Submodules: ``mehdg`` (ctypes binding of libmehdg.so), ``build`` (nvcc build
of the library), ``inputs`` (seeded synthetic meshes and states).
"""
__all__ = ["mehdg", "build", "inputs"]

"""GB300-native matrix-free FMG Stokes solver (P1-P1 PSPG and P2-P1 Taylor-Hood
on hierarchical hybrid grids of Kuhn-box macro meshes).

The compute path lives in libhhg.so (CUDA, sm_103a) behind the C ABI of
include/hhg.h; ``paper_2010_13513_gb300.hhg`` is its ctypes binding and
``paper_2010_13513_gb300.build`` compiles it.
"""
__all__ = ["hhg", "build"]

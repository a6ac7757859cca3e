"""GB300-native advection step of the modified method of characteristics
(Kohl, Mohr, Eibl, Ruede, arXiv 2103.02388): CUDA kernels for sm_103a behind
the C ABI of include/elm.h, with a thin Python binding (``elm.Mesh``).

Submodules are imported on demand: ``inputs`` (seeded synthetic workloads)
needs neither torch's CUDA nor the library.
"""
__all__ = ["elm", "inputs", "build"]

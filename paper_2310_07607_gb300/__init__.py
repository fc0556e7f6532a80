"""GB300-native explicit local space-time adaptive monodomain stepping (SIPG-DG + S-LTS + AMR).

The numerical path lives in libmdl.so (CUDA for sm_103a behind the C ABI of
include/mdl.h); this package holds its build script and a thin ctypes binding.
"""
from .mdl import Batch, Sim, MdlError, load, to_c, integral_noalloc, LIB_PATH  # noqa: F401

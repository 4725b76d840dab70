"""GB300 (sm_103a) solver library for the CN-FV tau-preconditioned Krylov method.

The compute path is the CUDA shared library libtfde.so (C ABI in
include/tfde.h); `paper_2511_21198_gb300.tfde` is its thin ctypes binding.
"""
__all__ = ["tfde"]

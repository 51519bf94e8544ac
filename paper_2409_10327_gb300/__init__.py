"""GB300 hash-grid secondary-ray renderer (arXiv 2409.10327, the hash renderer of Sec. 3).

The compute lives in ``librt_gb300.so`` (hand-written sm_103a CUDA behind the
C ABI of ``include/rt.h``); :mod:`.binding` is its thin ctypes binding.
Importing :mod:`.binding` fails loudly when the library has not been built.
"""
__all__ = ["binding", "build"]

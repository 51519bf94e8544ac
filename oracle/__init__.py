"""FP64 CPU oracle for the hash-grid secondary-ray renderer (TEST INFRASTRUCTURE).

This package is a plain, slow, obviously-correct restatement of the five
stages of the paper's hash renderer (Sec. 3.1-3.2, Eq. 1, Eq. 2) in float64
PyTorch CPU ops.  It exists only to check the CUDA library:

  * only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
    ``--impl reference`` legs of ``bench.py`` may import it;
  * it shares no code, header, table or constant with the CUDA path, and it
    never imports ``paper_2409_10327_gb300``;
  * the product path never calls it, and fails loudly when the CUDA
    library is missing instead of falling back to it.

Modules, in the order of the paper's pipeline (Fig. 1 / Sec. 3.2 overview):

  hashgrid  stage (a): f = H(x), multi-resolution hash encoding
  mlp       stage (b): a, r, n = B(f);  stage (c): v, t = I(f, w)
  sampling  direction sampling (SplitMix64 counters, cosine-weighted lobe)
  shading   env-map lookup, simplified-Disney BRDF, Eq. 1 / Eq. 2 sums
  render    the full path including the bounce x' = x + t w (stage (d)),
            and its FP64 gradient for the distillation loss

Parity status of each function is stated in its module header.
"""
from . import hashgrid, mlp, sampling, shading, render  # noqa: F401

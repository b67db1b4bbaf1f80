"""GB300-native annealed, vortex-preserved stout smoothing of Z(3) centre-vortex fields.

Implements the smoothing path of Virgili, Kamleh & Leinweber,
"Smoothing algorithms for projected center-vortex gauge fields"
(arXiv:2203.09764) as hand-written sm_103a CUDA behind a C ABI
(include/vs.h, libvs.so); ``paper_2203_09764_gb300.vs`` is the Python binding.
"""

__all__ = ["vs", "build"]

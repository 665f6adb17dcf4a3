"""GB300-native Gaussian-process likelihood and kriging (Franey, Ranjan &
Chipman): power-exponential correlation assembly, blocked Cholesky, profile
-2 log-likelihood over theta batches, and kriging prediction, as hand-written
sm_103a CUDA kernels behind the C ABI declared in ``include/gp.h``.

The CUDA library is loaded on first use by ``paper_1203_1269_gb300.gp``;
importing this package alone does not touch the GPU.
"""
__all__ = ["gp", "inputs"]

"""SCALE local-energy path on GB300 (sm_103a): C-ABI CUDA library + thin Python binding.

The library (csrc/, include/scale.h) evaluates log psi, amplitude ratios, local energies
(low-rank and full-recompute paths), Woodbury commits with FP64 refresh, and per-sample
log-psi gradients of the SCALE convolutional-backflow ansatz (arXiv 2604.25775, Sec. II).
Importing the package loads nothing; the library is loaded on first use.
"""
__all__ = ["inputs", "binding", "build", "autograd"]

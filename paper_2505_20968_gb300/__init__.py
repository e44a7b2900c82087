"""GB300 (sm_103a) library for the matrix-free AD-PRD operator of polarised
non-LTE radiative transfer (arXiv 2505.20968).

The C ABI is include/prd.h; `binding.PRD` wraps it for PyTorch device
tensors; `inputs` builds the seeded synthetic workloads.  Import of the
binding is lazy so that the input generator works without a GPU.
"""
__all__ = ["inputs", "binding"]

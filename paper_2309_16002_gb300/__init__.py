"""RBRP (robust blockwise random pivoting) interpolative decomposition on GB300.

The compute path is the CUDA library built from csrc/ (sm_103a) behind the C ABI
declared in include/rbrp.h; `paper_2309_16002_gb300.rbrp` is its thin ctypes
binding.  Importing the package itself loads nothing, so the input generators in
`workloads` can be used on machines without a GPU.
"""

__all__ = ["workloads"]

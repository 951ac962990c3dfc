"""GB300 (sm_103a) implementation of the training-step hot path of LiteGS
(arXiv 2503.01199): Morton re-sort, Cluster-Cull-Compact, EWA preprocess,
tile binning, differentiable tile rasterisation with per-Gaussian gradient
reduction and opacity-gradient moments, and sparse Adam.

The kernels live in csrc/ and are exposed through the C ABI of
include/lgs.h (liblgs.so, built in-tree by build.py). ``binding`` wraps that
ABI for torch tensors; ``pipeline`` strings the calls into a training step.
Submodules are imported on demand so that importing the package does not
load CUDA.
"""

__all__ = ["binding", "pipeline", "scenegen", "build"]

"""libgfopt: GB300-native hot path of the Green's-function pixel-by-pixel optimizer
(Wang et al., arXiv:2202.05388, Sec. II-III).

The package is deliberately light at import time: ``workloads`` holds only the
synthetic input recipes, ``gfopt`` loads the compiled CUDA library on first use
and fails loudly when it is missing.
"""

__all__ = ["workloads"]

"""GlassNet per-pixel forward pass (arXiv 2405.19056) on sm_103a.

The compute path is the CUDA library built from ``csrc/`` (see
``include/glassnet.h``); ``glassnet`` is its Python binding.
"""
from . import glassnet  # noqa: F401

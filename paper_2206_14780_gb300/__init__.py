"""GB300-native semi-implicit SPH viscous solve (arXiv 2206.14780): C-ABI library + thin binding.

The compute path lives in ``csrc/`` (CUDA for sm_103a) behind ``include/sphvisc.h``;
``binding`` marshals torch device tensors into those calls; ``build`` compiles it.
"""
from . import binding  # noqa: F401

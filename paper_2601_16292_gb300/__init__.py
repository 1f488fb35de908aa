"""GB300-native columnar agent-step engine (AMBER's per-step population update).

The compute path is libamb.so (CUDA, sm_103a) behind the C ABI in
include/amb.h; ``amb`` is its ctypes binding.
"""
from . import amb  # noqa: F401
from .amb import Population, AmbError  # noqa: F401

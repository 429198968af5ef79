"""GB300-native multilevel spectral domain decomposition (hot path).

The CUDA library (csrc/, built into lib/libmsdd.so by build.py) implements
the set-up and the preconditioned CG solve behind the C ABI of
include/msdd.h; msdd.py is the ctypes binding.
"""
from . import msdd  # noqa: F401
from .msdd import Hierarchy, BandBatch, MsddError, assemble_rhs, num_unknowns  # noqa: F401
from .msdd import WarmStartNet, fine_layout, nn_patches, nn_start_vectors  # noqa: F401
from .msdd import batch_plan, batch_run  # noqa: F401

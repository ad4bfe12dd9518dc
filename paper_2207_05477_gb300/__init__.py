"""GB300 (sm_103a) Evoformer block: C-ABI CUDA library (libevo.so) and its Python binding."""
from . import synth  # noqa: F401

__all__ = ["synth", "evo", "build"]

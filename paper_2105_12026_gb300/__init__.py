"""GB300-native exemplar-based clustering (EBC) summarisation hot path.

The compute lives in a CUDA library (csrc/, built for sm_103a) behind the C
ABI of include/ebc.h; ``ebc`` is its Python binding.  ``synth`` generates
seeded synthetic inputs.
"""
__all__ = ["ebc", "synth", "build"]

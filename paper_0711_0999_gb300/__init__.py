"""GB300-native nonequilibrium-DMFT lattice step (Falicov-Kimball model in a field).

The compute path is the CUDA library ``libnedmft.so`` (C ABI in
``include/nedmft.h``); ``paper_0711_0999_gb300.api`` is its Python binding.
Importing the package does not load the library; the first API call does,
and raises if it has not been built.
"""

__all__ = ["api", "synth", "build"]

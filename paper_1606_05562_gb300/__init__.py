"""GB300-native implementation of the orthogonal 16-point approximate DCT of
arXiv 1606.05562 (da Silveira et al.).

The compute path is the CUDA library ``libatdct16.so`` built from ``csrc/``
(C ABI in ``include/atdct16.h``); ``atdct16`` is its thin Python binding and
``synth`` draws seeded synthetic inputs.  Importing the package loads nothing;
the library is loaded on first use.
"""

__all__ = ["atdct16", "synth", "build"]

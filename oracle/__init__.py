"""CPU oracle for the orthogonal 16-point approximate DCT (da Silveira, Bayer,
Cintra, Kulasekera, Madanayake, Kozakevicius, arXiv 1606.05562).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, links or executes anything in this package.  Only
the test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.

The oracle is deliberately plain: direct 16x16 matrix products (never the fast
factorisation it is used to check), exact integer / rational arithmetic where
the method's result has an exact definition, FP64 elsewhere.
"""

from .atdct16_oracle import *  # noqa: F401,F403

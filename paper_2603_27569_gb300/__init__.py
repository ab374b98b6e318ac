"""GB300-native batched complex-to-complex FFT (Stockham, radix-8/4/2, four-step).

The compute path is the C-ABI library ``libfftgb.so`` built from ``csrc/``;
this package is its thin Python binding.  Importing the package does not load
the library; the first call that needs it does, and raises if it is missing.
"""
from ._binding import *  # noqa: F401,F403

"""GB300-native Shouji pre-alignment filter (arXiv 1809.07858) -- Python binding.

The compute path is the C-ABI library ``libshouji.so`` (hand-written sm_103a
CUDA, declared in ``include/shouji.h``); this package only marshals
arguments.  Importing it does not load the library; the first call does, and
fails loudly when the library has not been built.
"""
from .binding import *  # noqa: F401,F403
from .binding import __all__  # noqa: F401

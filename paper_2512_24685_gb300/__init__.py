"""GB300-native second-order stabilizer Renyi entropy (XOR-FWHT) library.

Python binding of ``libsre`` (see ``include/sre.h``).  Importing the package
does not load the CUDA library; the first call that needs it does, and fails
loudly if the library is missing or no CUDA device is present.
"""
from .binding import *  # noqa: F401,F403
from .binding import __all__  # noqa: F401

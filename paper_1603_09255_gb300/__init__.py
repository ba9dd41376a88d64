"""GB300 (sm_103a) engine for the per-generation update of sPEGG-style
forward-time population-genetics simulation.  The compute path is the CUDA
library libspegg_gb300.so behind the C ABI in include/spegg.h; this package is
its ctypes binding (``spegg``) and its build script (``build``)."""
from . import spegg  # noqa: F401
from .spegg import Population, SpeggError, summarize  # noqa: F401

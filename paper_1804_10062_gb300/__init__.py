"""GB300-native QuickMergesort (Edelkamp & Weiss, arXiv 1804.10062).

The compute path is the CUDA library ``libqms.so`` (hand-written kernels for
sm_103a behind the C ABI of ``include/qms.h``); ``qms`` is its thin ctypes
binding.  There is no CPU fallback: if the library cannot be loaded the
binding raises.
"""
from .qms import *  # noqa: F401,F403

"""GB300-native worldline Wilson loops (Mazur & Heyl, arXiv:1407.7486).

The compute path is ``libwln.so`` (hand-written sm_103a CUDA kernels behind a
C ABI, declared in ``include/wln.h``); ``wln`` is its ctypes binding and
``inputs`` builds the seeded synthetic workloads.
"""
from .inputs import Profile, PROFILE_CONST_B, PROFILE_FLUX_TUBE  # noqa: F401
from .wln import Context, Ensemble, WlnError, load  # noqa: F401

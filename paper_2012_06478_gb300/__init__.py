"""GB300 engine for the random-walker step of the Realistic Microstructure
Simulator (Lee, Fieremans & Novikov, arXiv 2012.06478): Monte Carlo diffusion
in voxelised cell-label volumes, hand-written sm_103a CUDA kernels behind a
C ABI (include/rms.h), with this package as a thin Python binding."""
from .api import *  # noqa: F401,F403
from .api import __all__  # noqa: F401

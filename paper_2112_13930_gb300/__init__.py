"""GB300 (sm_103a) lattice kinetic scheme for MHD with Shercliff thin-conducting-wall closures
(Yahia & Premnath, arXiv 2112.13930): C-ABI CUDA library plus a thin Python binding."""
from . import build  # noqa: F401
from .lks import (BF16_DEV, F16_DEV, F32, F64, LINK, MOMENT, MOMENTS_NODES, MOMENTS_PROFILES,  # noqa: F401
                  Lattice, LksError, footprint_bytes, load)

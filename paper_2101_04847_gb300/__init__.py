"""GB300 (sm_103a) two-component D2Q9 Shan-Chen lattice Boltzmann solver for
2D Rayleigh-Taylor turbulence (arXiv 2101.04847), behind the C ABI of
include/lbm.h.  ``lbm`` is the ctypes binding; ``build`` compiles the library.
"""
from . import lbm  # noqa: F401
from .lbm import Solver, default_params, load_library  # noqa: F401

"""GB300 (sm_103a) implementation of the thermal LBM-PIBM-DEM lattice step of
Zhang et al., "Particulate immersed boundary method for complex
fluid-particle interaction problems with heat transfer" (arXiv 1502.01159).

The compute path is the C-ABI CUDA library ``libpibm.so`` (include/pibm.h);
this package holds its sources (csrc/), its build (build.py) and the ctypes
binding (_native.py).  There is no CPU fallback: without the library every
call raises."""
from ._native import (ADIABATIC, FIELDS, Ensemble, HERTZ_MD, HERTZ_MD_HIST, ISOTHERMAL, PERIODIC, SPRING_DASHPOT, STORE_BF16, STORE_F16,
                      STORE_F32, STORE_F64, TUNE_DEM_PARTICLES_PER_CTA, TUNE_LATTICE_THREADS, TUNE_LATTICE_ROW_TILES, TUNE_TC_WAIT_POLLS, TUNE_WIDE_INDEX, TUNE_COUPLING_THREADS, TUNE_COUPLING_ORDER, TUNE_LATTICE_PAIRS, WALL, PibmError,
                      Simulation, load)

__all__ = ["Simulation", "Ensemble", "PibmError", "load", "FIELDS", "PERIODIC", "WALL", "ADIABATIC", "ISOTHERMAL",
           "SPRING_DASHPOT", "HERTZ_MD", "HERTZ_MD_HIST", "STORE_F32", "STORE_F64", "STORE_F16", "STORE_BF16",
           "TUNE_DEM_PARTICLES_PER_CTA", "TUNE_LATTICE_ROW_TILES", "TUNE_LATTICE_THREADS", "TUNE_WIDE_INDEX", "TUNE_TC_WAIT_POLLS",
           "TUNE_COUPLING_THREADS", "TUNE_COUPLING_ORDER", "TUNE_LATTICE_PAIRS"]

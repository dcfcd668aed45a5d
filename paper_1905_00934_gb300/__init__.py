"""GB300-native (sm_103a) library for one ADMM iteration of UDM(m)-PCG(n) statistical
dual-energy CT reconstruction (Li et al., Sec. 3), with a C ABI (include/dect.h)
and this thin ctypes binding (`dect`)."""
from . import dect  # noqa: F401
from .solver import Geometry, Spectra, Solver, cdm_fbp  # noqa: F401

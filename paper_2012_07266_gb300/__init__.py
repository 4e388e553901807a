"""GB300-native particle-mesh weak-lensing forward model (MADLens method,
arXiv:2012.07266): FastPM kick-drift-kick steps, Born lightcone projection with
sub-evolution and PGD sharpening, and hand-written adjoints, as a C-ABI CUDA
library (include/pm.h) with a thin Python binding."""
from . import lib  # noqa: F401

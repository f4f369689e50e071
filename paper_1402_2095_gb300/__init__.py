"""GB300-native f-thermostat (FTH): elements of f(M) for SPD M from colored-noise
GLE dynamics (Nava, Ceriotti, Dryzun, Parrinello).  The compute path is libfth.so
(hand-written sm_103a CUDA behind the C ABI of include/fth.h); this package holds
its build script, the ctypes binding and the host-side GLE fitter."""
from .binding import FTH, FthError, Pool, Server, gle_propagator, load  # noqa: F401

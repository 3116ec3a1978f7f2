"""GB300-native multigrid solver for linear magnetohydrostatic equilibria
(MacTaggart, Elsheikh, McLaughlin & Simitev, "Non-symmetric
magnetohydrostatic equilibria: a multigrid approach").

The solver is the C-ABI library libmhs.so (CUDA kernels for sm_103a, header
include/mhs.h).  ``from paper_1307_6720_gb300 import mhs`` loads it through
its ctypes binding and raises ImportError when the library is not built
(``paper_1307_6720_gb300.build.build()`` compiles it).
"""

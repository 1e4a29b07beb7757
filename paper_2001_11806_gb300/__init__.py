"""GB300-native lattice Boltzmann stream-collide library (CUDA, sm_103a).

The compute path is ``liblbm.so`` (C ABI declared in include/lbm.h); this
package is a thin ctypes binding over it plus seeded input generators.
Importing the package does not load the library; ``lib()`` does, and fails
loudly if it has not been built.
"""
from ._lib import lib, LbmError  # noqa: F401

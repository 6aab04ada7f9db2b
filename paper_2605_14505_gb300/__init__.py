"""GB300-native (sm_103a) DDF lattice Boltzmann stream-and-collide for the
Boussinesq stratified Taylor-Green vortex.

The compute path is ``liblbm.so`` (CUDA, built in-tree by ``build.py``) behind
the C ABI of ``include/lbm.h``; ``lbm`` is its ctypes binding.
"""
from . import lbm  # noqa: F401
from .lbm import Simulation, LbmError  # noqa: F401

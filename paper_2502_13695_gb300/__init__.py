"""GB300-native particle-in-cell library for few-cycle laser pulses driving
dielectrics (Keldysh photoionisation, Lorentz dielectric, Boris/Esirkepov).

The compute path is the CUDA library built from ``csrc/`` (see ``build``);
``pic`` is its ctypes binding and ``workloads`` the seeded synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "pic", "build"]

"""GB300 (sm_103a) solver for the phase-field lattice Boltzmann method of
two-phase EHD flow with Onsager-Wien dissociation (arXiv 2501.04920).

The solver is the C-ABI library ``libehdlb.so`` (include/ehdlb.h) built from
``csrc/``; ``ehdlb`` is its ctypes binding and ``workloads`` holds the lattice
parameters of the standard droplet cases.
"""
from . import ehdlb, workloads  # noqa: F401
from .ehdlb import FIELDS, FP32, FP64, Lattice  # noqa: F401

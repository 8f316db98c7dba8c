"""GB300-native (sm_103a) SSP2(222) / SSP3(332) IMEX step for resistive and two-fluid
special-relativistic MHD (after Wright & Hawke, arXiv:1808.09721).

The compute path is the CUDA library librmhd.so (C ABI in include/rmhd.h);
this package only builds it, marshals arguments (`_lib`, `sim.Sim`) and
provides seeded synthetic workloads (`workloads`).
"""
from ._lib import (DEVICE, FLOATFLOAT, FP64, HOST, MIXED, OUTFLOW, PERIODIC, RESISTIVE, SSP2, SSP3, TWO_FLUID,  # noqa: F401
                   RmhdError)


def __getattr__(name):
    if name == "Sim":
        from .sim import Sim
        return Sim
    raise AttributeError(name)

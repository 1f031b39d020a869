"""GB300 (sm_103a) kernel-independent FMM for long-range forces in DEM.

The compute path is the C-ABI library lib/libkifmm.so (CUDA kernels); the
Python layer (kifmm.py) only marshals arguments.
"""
from .kifmm import (Plan, KifmmError, KifmmPotential, KifmmEnergy, energy, far_image_operator, field,  # noqa: F401
                    load, lr_stride, potential, PRECISIONS)

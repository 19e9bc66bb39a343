"""GB300-native full-sky Taylor lensing (Naess & Louis 2013, arXiv:1307.0719).

The computation runs in the CUDA library libtaylens.so (C ABI in include/taylens.h);
this package only marshals arguments. PyTorch provides device memory and streams.
"""
from .api import Plan, LensFunction, lens, synth_derivs, deflection, FP64, MIXED_FP32, MIXED_TF32, MIXED_TF32x3  # noqa: F401

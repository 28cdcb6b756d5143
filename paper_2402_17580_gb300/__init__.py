"""GB300 (sm_103a) point solver for the Ti-6Al-4V phase model of
Proell et al., arXiv 2402.17580.

The compute path is the CUDA library ``_build/libms_gb300.so`` behind the C ABI
of ``include/ms.h``; this package only builds it and marshals arguments
(see ``_binding``).  PyTorch is not needed; where a caller uses it, it only
provides device memory and streams.
"""
from ._binding import (MS_EXPLICIT, MS_F32, MS_F64, MS_F64ACC, MS_IMPLICIT, MS_KAHAN,
                       MS_PTR_DEVICE, Context, MSError, Surrogate, Thermal, default_params,
                       library_path, load, thermal_params)
from .build import build

__all__ = ["Context", "Surrogate", "Thermal", "thermal_params", "MSError", "default_params", "load", "build", "library_path",
           "MS_F32", "MS_F64ACC", "MS_KAHAN", "MS_F64", "MS_PTR_DEVICE", "MS_EXPLICIT",
           "MS_IMPLICIT"]

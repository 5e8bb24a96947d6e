"""GB300-native FastDOG dual hot path (Abbas & Swoboda, CVPR 2022).

The compute path is the C-ABI library ``_build/libfastdog.so`` (hand-written
sm_103a CUDA).  ``capi`` binds it with ctypes under the same names as
``include/fastdog.h``; ``Instance`` is a thin convenience wrapper over those
calls.  There is no CPU fallback: using the binding without the compiled
library raises.
"""
from .capi import (  # noqa: F401
    FDOG_ECUDA, FDOG_EINFEASIBLE, FDOG_EINVAL, FDOG_ENOCONVERGE, FDOG_ENOMEM, FDOG_EQ, FDOG_ESTATE, FDOG_ETIMEOUT,
    FDOG_EUNSUPPORTED, FDOG_GE, FDOG_LE, FDOG_OK, Batch, FdogError, Instance, Params, Server, host_cache_release, lib,
    library_path,
)

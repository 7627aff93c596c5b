"""B300-native batched mixed-state multislice ptychography (arXiv 2505.14372).

The forward model and its adjoint run in hand-written sm_103a CUDA kernels
behind the C-ABI of libptycho (include/ptycho.h); this package is the thin
Python binding (torch tensors for device memory and streams).
"""
from .api import (AdamState, Context, Geometry, adam_opt, fft2, kernels_launched,  # noqa: F401
                  make_groups, scratch_bytes, version, Server)
from .autograd import PtychoFn, simulate  # noqa: F401
from ._lib import PtychoError  # noqa: F401

"""GB300-native NUFFT and NUFFT-Jacobian products (Wang & Fessler, arXiv 2111.02912).

The compute lives in libnufftjac.so (hand-written sm_103a CUDA kernels behind a
C ABI, include/nufftjac.h).  This package only marshals torch tensors into that
ABI: ``_abi`` mirrors the C entry points one to one, ``Plan`` wraps a plan
handle for device tensors.
"""
from ._abi import (NufftError, nufft_adjoint, nufft_default_opts, nufft_destroy, nufft_forward,  # noqa: F401
                   nufft_get_info, nufft_jvp_omega, nufft_launch_count, nufft_plan, nufft_profile_enable,
                   nufft_profile_read, nufft_set_points, nufft_vjp_omega_x, nufft_workspace_bytes)
from .plan import Plan  # noqa: F401

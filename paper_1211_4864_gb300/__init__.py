"""GB300-native short-range particle-particle force path of HACC (arXiv:1211.4864).

Chaining-mesh binning (or the paper's RCB fat-leaf tree) -> per-cell (per-leaf)
neighbour lists -> pair force
f_SR(s) = (s + eps)^-3/2 - poly[5](s) -> kick, plus the adjoint, as
hand-written CUDA for sm_103a behind the C ABI of ``include/hacc_sr.h``.
PyTorch supplies device memory, streams and autograd.  There is no CPU
fallback: without the CUDA library every call raises.
"""

from ._lib import HaccError, library_path, load  # noqa: F401
from .sr import (Launch, ShortRange, SRParams, hacc_bin, hacc_bin_noalloc, hacc_build_lists, hacc_count_pairs,  # noqa: F401
                 hacc_drift_offsets, hacc_get_status, hacc_kick,
                 hacc_kernel_launches, hacc_mesh_plan, hacc_moments, hacc_rcb_build, hacc_rcb_lists,
                 hacc_sr_force, hacc_sr_force_adjoint, hacc_sr_force_adjoint_symmetric, hacc_sr_force_symmetric,
                 hacc_sr_potential, hacc_version,
                 kick_drift_autograd, sr_force_autograd, trajectory_autograd)

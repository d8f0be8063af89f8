"""GB300 (sm_103a) hash-based multi-phase SpGEMM.

C = A*B on CSR matrices through the C ABI of libspgemm.so (include/spgemm.h):
intermediate-product counting, row grouping, the allocation (symbolic) phase,
row pointers and the accumulation (numeric) phase with sorted output, all as
hand-written CUDA kernels. Python only marshals arguments; PyTorch provides
device memory and streams.
"""
from .api import DeviceCSR, Plan, default_opts, split_rows  # noqa: F401
from ._lib import SpgemmError  # noqa: F401

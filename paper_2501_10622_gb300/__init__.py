"""GB300-native (sm_103a) single-scale hot path of CWTHF, the continuous
wavelet transform halo finder of arXiv:2501.10622.

The compute lives in libcwthf.so (CUDA kernels behind the C ABI of
include/cwthf.h); this package holds its ctypes binding, the seeded input
generators and the build script.
"""
from ._lib import (HALO_DTYPE, MS_HALO_DTYPE, Context, CwthfError, Params, catalogue_to_numpy, check_ng,
                   default_params, error_string, header_symbols, lib, ms_catalogue_to_numpy, paper_scales,
                   supported_sizes, workspace_bytes)

__all__ = ["HALO_DTYPE", "MS_HALO_DTYPE", "Context", "CwthfError", "Params", "catalogue_to_numpy", "check_ng",
           "default_params", "error_string", "header_symbols", "lib", "ms_catalogue_to_numpy", "paper_scales",
           "supported_sizes", "workspace_bytes"]

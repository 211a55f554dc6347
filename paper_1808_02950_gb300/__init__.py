"""GB300 library for the 8x8 approximate-DCT block codec of arXiv 1808.02950.

The compute path is the CUDA library ``libtdct.so`` (C ABI in
``include/tdct.h``); this package builds it in-tree and binds it with
ctypes (``_lib``).  ``synth`` holds the seeded synthetic input generators.
Importing the package does not load the library; the first call does, and a
missing or unloadable library raises instead of falling back to anything.
"""
from ._lib import (  # noqa: F401
    N1, T1, TDCT_BF16, TDCT_BF16X3, TDCT_FP32, TDCT_I16, TDCT_LOAD_BULK, TDCT_LOAD_PLAIN, TDCT_LOAD_STAGED, TDCT_PATH_AUTO, TDCT_PATH_BUTTERFLY, TDCT_PATH_TENSOR, TDCT_PATH_TENSOR_PIPELINED,
    TDCT_U8, TdctError, TdctPlan, load, make_planes, make_planes_raw, tdct_codec_error,
    tdct_codec_error_batched, tdct_codec_error_batched_noalloc, tdct_codec_error_batched_host, tdct_ssim_batched, tdct_search, tdct_codec_error_jam, tdct_dct_codec_error, tdct_forward, tdct_debug_inject_wait_timeout, tdct_debug_search_hit_cap, tdct_plan_create,
    tdct_shutdown, tdct_sweep_batched, tdct_dct_sweep_batched, tdct_sync_status, tdct_version, tdct_zonal_inverse,
)

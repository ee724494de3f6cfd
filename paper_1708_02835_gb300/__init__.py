"""GB300-native exact Gaussian log-likelihood with a Matern covariance.

Python binding of libegs.so (C ABI in include/egs.h).  Every function here
only marshals arguments: the covariance generation, tile Cholesky, solve and
reductions all run in the library's sm_103a CUDA kernels.  There is no CPU
fallback: if the library is missing, importing the binding raises.

Method: Abdulah et al., "ExaGeoStat: A High Performance Unified Software for
Geostatistics on Manycore Systems", arXiv:1708.02835 -- Eq. 1 (Gaussian
log-likelihood), Eq. 2 (Matern covariance), Algorithm 2 (evaluation).
"""
from .binding import (  # noqa: F401
    EGS_OK, EGS_ERR_ARG, EGS_ERR_NOT_PD, EGS_ERR_OOM, EGS_ERR_CUDA, EGS_ERR_TIMEOUT, EGS_ERR_BUSY,
    EGS_ERR_UNIMPLEMENTED, EGS_FP64, EGS_MIX_FP32, EGS_MIX_TF32, EGS_MIX_BF16, PRECISIONS,
    EgsError, NotPositiveDefinite, MixedInaccurate, egs_info, egs_opts, load_library, library_path,
    egs_last_error, egs_version, egs_default_tile, egs_tiles_bytes, egs_loglik_workspace_bytes,
    egs_matern_tiles, egs_potrf_tiles, egs_trsv_tiles, egs_loglik, egs_loglik_ex, egs_loglik_ind, egs_predict, egs_tc_gemm_test, egs_tc_gemm_test_withhold, egs_ozaki_gemm_test,
    egs_batch, egs_batch_autotune, egs_batch_tuned_tile, egs_loglik_batched, egs_server, egs_trsv_tiles_noalloc, egs_simulate, egs_trace_last, TRACE_CLASSES,
    egs_set_allocator, use_torch_allocator,
)

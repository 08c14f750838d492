"""GB300-native space-time reduced-order model (Choi et al., space-time ROM for
linear dynamical systems).  The compute path is the CUDA library libst_rom.so
(C ABI: include/st_rom.h); this package is its ctypes binding."""
from .binding import (  # noqa: F401
    LIB_PATH,
    Model,
    StError,
    ST_DGEMM_OZAKI,
    ST_DGEMM_SIMT,
    ST_ERR_ARG,
    ST_ERR_BREAKDOWN,
    ST_ERR_NONFINITE,
    ST_ERR_NOT_CONVERGED,
    ST_ERR_SINGULAR,
    ST_ERR_STATE,
    ST_ERR_TIMEOUT,
    ST_FP32_ASSEMBLY,
    ST_FP32_LU,
    ST_FP64,
    ST_OK,
    check,
    last_error,
    lib,
    options,
    ptr,
    st_model_file_info,
    st_probe_fp64_fma,
)

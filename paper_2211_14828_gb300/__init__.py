"""GB300-native rBKI-TK / rBKI-TK-TR (arXiv 2211.14828): CUDA kernels for sm_103a behind the
C ABI in include/rbki.h, with a thin ctypes binding."""
from ._binding import (  # noqa: F401
    LIB_PATH, RbkiError, lib, rbki_kernel_launches, rbki_krylov_product, rbki_krylov_product_noalloc, rbki_mode_basis,
    rbki_diag_krylov_stall, rbki_diag_batched_stall,
    rbki_syev, rbki_tucker, rbki_htr, RbkiServer, rbki_tucker_workspace, rbki_profile_enable, rbki_profile_reset,
    rbki_profile_read, PROF_KRYLOV, PROF_SKETCH, PROF_GRAM, PROF_TTM, PROF_STAGE, PROF_SAMPLE,
    rbki_sample_units, rbki_split_mode, rbki_tucker_batch, rbki_tucker_batched, rbki_tucker_batched_workspace,
    rbki_divide_and_conquer, rbki_wave_autotune, rbki_wave_tune_table, rbki_wave_tune_save, rbki_wave_tune_load,
    rbki_wave_tune_reset, BatchedPlan,
    F64, F32, BF16, F16, PREC_FP64, PREC_BF16, PREC_FP16, FLAG_HOST_IO, FLAG_SPLIT,
    FLAG_SERIAL_MODES, FLAG_SEQUENTIAL, FLAG_POWER, FLAG_ADAPTIVE_Q, FLAG_TR_SVD, FLAG_ASYNC, FLAG_REFINE_FP32,
)

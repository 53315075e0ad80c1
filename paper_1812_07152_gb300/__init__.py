"""GB300-native evaluation of HMatrix-matrix products Y = K~ W (MatRox, arXiv 1812.07152).

The compute path is libhmat.so (hand-written sm_103a CUDA behind a C ABI, see
include/hmat.h); this package only builds it and marshals arguments to it.
"""
from .hmat import (  # noqa: F401
    HmatError, HMAT_OK, HMAT_EINVAL, HMAT_ENOMEM, HMAT_ECUDA, HMAT_ETIMEOUT, HMAT_EUNSUPPORTED,
    HMAT_EDEVICE, HMAT_EBUSY, HMAT_MODE_FP64, HMAT_MODE_MIXED, HMAT_LOAD_MIXED, HMAT_LOAD_MIXED_ONLY,
    HMAT_DTYPE_F64, HMAT_DTYPE_F32, HMAT_BUILD_ID_GPU, HMAT_BUILD_NEAR_OTF, hmat_eval_typed, hmat_eval_host_typed,
    hmat_batch_eval_typed, hmat_server_matrix_stats, hmat_batch_info, hmat_batch_autotune, hmat_batch_schedule,
    DeviceHMatrix, hmat_load, hmat_build, hmat_structure, hmat_eval, hmat_reserve,
    hmat_status_poll, hmat_info, hmat_free, hmat_strerror, library, exported_symbols, hmat_eval_host,
    hmat_profile, hmat_phase_times, hmat_measure_fp64_peak, PHASES, hmat_batch_create, hmat_batch_eval,
    hmat_batch_free, hmat_server_create, hmat_server_submit, hmat_server_wait, hmat_server_stats,
    hmat_server_free, hmat_autotune, hmat_tune_apply, hmat_selftest_timeout, hmat_selftest_chain_timeout, hmat_selftest_row_id, hmat_selftest_device_check,
    hmat_selftest_conversions, hmat_plan_create, hmat_plan_build, hmat_plan_free,
)

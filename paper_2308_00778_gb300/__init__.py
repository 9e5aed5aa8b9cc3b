"""GB300-native LSQR hot path of the Gaia AVU-GSR solver (arXiv 2308.00778).

Python face of ``libgsr.so`` (C ABI declared in ``include/gsr.h``). The
binding only marshals arguments: every step of the path runs in the library's
CUDA kernels. PyTorch tensors may be passed wherever the ABI takes a device
pointer; their ``data_ptr()`` is forwarded unchanged.
"""
import os as _os

from .gsr import (  # noqa: F401
    GSR_AOS, GSR_DEVICE, GSR_FP32, GSR_FP64, GSR_HOST, GSR_MIXED, GSR_PLAIN, GSR_SOA, GSR_WARM_JACOBI,
    GSR_WARM_LEARNED, GSR_WARM_NONE, GsrError, SolveInfo, SolveParams, Status, gsr_aprod1, gsr_aprod1_f32,
    gsr_aprod2, gsr_aprod2_f32, gsr_aprod2_plan, gsr_residual, gsr_residual_static, gsr_create, gsr_create_sections, gsr_sections,
    gsr_default_params, gsr_destroy, gsr_dims, gsr_last_error, gsr_lsqr_solve, gsr_set_rhs, gsr_set_rows,
    gsr_set_system, lib, library_path, Context, Net, gsr_net_create, gsr_net_destroy, gsr_net_forward,
    gsr_net_gradients, gsr_net_get_params, gsr_net_last_error, gsr_net_load, gsr_net_num_params, gsr_net_save,
    gsr_net_set_params, gsr_net_train_step, gsr_warm_features, gsr_warm_start, gsr_net_layer_forward,
    gsr_net_layer_backward, gsr_net_apply_gradients, gsr_fp64_fma_rate, dfma_probe_tflops, gsr_aprod12_f32,
    gsr_tc_wait_check, tc_wait_check,
)

#: trained warm-start network shipped with the package (``python -m paper_2308_00778_gb300.train``
#: wrote it; the .json beside it records the training run and its held-out evaluation)
WARM_WEIGHTS = _os.path.join(_os.path.dirname(_os.path.abspath(__file__)), "weights", "warmstart.bin")

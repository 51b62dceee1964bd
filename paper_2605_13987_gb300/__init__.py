"""GB300-native weighting-field solver for 3D diamond sensors (arXiv 2605.13987).

The computation lives in libwt.so (CUDA, sm_103a) behind the C ABI of
include/wt.h; this package only marshals arguments to it (``_binding``) and
offers a small object wrapper (``Sensor``) and a torch.autograd.Function
over the library's derivative (``autograd.Eq1Loss``).  Importing the package does not
load the library; the first call does, and fails if it was not built.
"""
from ._binding import (  # noqa: F401
    WTError, load_library, LIB_PATH,
    WT_FP32, WT_FP64,
    wt_create, wt_add_columns, wt_fit, wt_relax, wt_extend, wt_sample_H, wt_eq1, wt_eq1_noalloc, wt_eq1_direct,
    wt_eq1_loss, wt_eq1_loss_grad, wt_batch_run, wt_get_tuning,
    wt_set_resistivity_profile, wt_eq1_loss_grad_profile, wt_shape, wt_static_field, wt_drift, wt_sync,
    wt_eq1_tangents, wt_features, WT_N_FEATURES, FEATURE_NAMES,
    wt_get_charges, wt_get_capacitance, wt_get_modes, wt_get_info, wt_set_timing, wt_get_timing,
    wt_destroy,
)
from .sensor import Sensor, extend_batch  # noqa: F401

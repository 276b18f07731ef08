"""GB300-native reference-less transmission-matrix retrieval with FFT-structured
probing (arXiv 2302.13524).

The computation runs in libtmr.so (hand-written sm_103a CUDA kernels behind the
C ABI of include/tmr.h); this package is its thin ctypes binding with the same
function names.  Importing it fails when the library has not been built.
"""
from ._lib import (  # noqa: F401
    DEFOCUS_ANGULAR_2X, DEFOCUS_SAME_GRID, TMR_COST_AMPLITUDE, TMR_COST_INTENSITY, INIT, MLP, TMR_INIT_LEARNED, TMR_LOSS_MSE, TMR_LOSS_PHASE, TMR_ERR_CUDA, TMR_ERR_INVALID_ARG, TMR_ERR_NUMERIC, TMR_ERR_OOM, TMR_ERR_TIMEOUT,
    TMR_ERR_UNSUPPORTED, TMR_INIT_BP, TMR_INIT_RANDOM, TMR_INIT_SPECTRAL, TMR_OK,
    TMR_PIX_F32, TMR_PIX_U16, TMR_PREC_FP32, TMR_PREC_MIXED, TMR_ROW_CONVERGED, TMR_ROW_MAXITER, TMR_ROW_NUMERIC, TMR_ROW_ZERO, Handle,
    LIB_PATH, TMRError, header_symbols, lib, tmr_create, tmr_default_options, tmr_defocus_fit,
    tmr_defocus_forward, tmr_destroy, tmr_forward, tmr_grad, tmr_last_error, tmr_retrieve,
    tmr_learned_rows, tmr_mlp_create, tmr_mlp_destroy, tmr_mlp_forward, tmr_mlp_get_params,
    tmr_gemm_bf16, tmr_mlp_grad, tmr_mlp_set_loss, tmr_mlp_set_params, tmr_mlp_train_step, tmr_retrieve_from, tmr_retrieve_rows_static,
    tmr_autotune_report, tmr_phase_fit_report, tmr_schedule, tmr_set_init_model, tmr_sync, tmr_workspace_bytes, half_grid, tmr_half_sample,
    tmr_preprocess, tmr_preprocess_workspace_bytes)
from .retriever import Retriever, preprocess  # noqa: F401,E402

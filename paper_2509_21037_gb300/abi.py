"""ctypes mirror of include/sc.h, include/sc_implicit.h, include/sc_probe.h, include/sc_pipeline.h and
include/sc_dense.h (argument marshalling only)."""
from __future__ import annotations

import ctypes

c_i8p = ctypes.c_void_p
c_vp = ctypes.c_void_p
c_i32 = ctypes.c_int32
c_i64 = ctypes.c_int64
c_sz = ctypes.c_size_t
c_int = ctypes.c_int

STATUS = {0: "SC_OK", 1: "SC_ERR_INVALID_ARG", 2: "SC_ERR_NOT_SPD", 3: "SC_ERR_CUDA", 4: "SC_ERR_OOM",
          5: "SC_ERR_TIMEOUT", 6: "SC_ERR_INTERNAL", 7: "SC_ERR_STATE"}
SC_OK, SC_ERR_INVALID_ARG, SC_ERR_NOT_SPD, SC_ERR_CUDA, SC_ERR_OOM, SC_ERR_TIMEOUT, SC_ERR_INTERNAL, SC_ERR_STATE = range(8)


class SubdomainDesc(ctypes.Structure):
    _fields_ = [("n", c_i32), ("m", c_i32), ("L_colptr", c_vp), ("L_rowind", c_vp),
                ("Bt_colptr", c_vp), ("Bt_rowind", c_vp), ("Bt_sign", c_vp), ("lambda_map", c_vp), ("Bt_val", c_vp)]


SC_FP64, SC_SPLIT_BF16 = 0, 1


SC_TILE_32, SC_TILE_TC128 = 0, 1


class Options(ctypes.Structure):
    _fields_ = [("precision", c_i32), ("n_slices", c_i32), ("sub_slices", c_vp), ("ws_limit", c_i64),
                ("persistent", c_i32), ("tile", c_i32), ("sub_tile", c_vp), ("poll_limit", c_i64)]


class Sizes(ctypes.Structure):
    _fields_ = [("plan_bytes", c_sz), ("ws_bytes", c_sz), ("F_doubles", c_i64), ("L_values", c_i64),
                ("nsub", c_i32), ("max_m", c_i32)]


class Stats(ctypes.Structure):
    _fields_ = [("flops_trsm", ctypes.c_double), ("flops_syrk", ctypes.c_double),
                ("flops_trsm_exec", ctypes.c_double), ("flops_syrk_exec", ctypes.c_double),
                ("flops_dense", ctypes.c_double), ("bytes_assembly", ctypes.c_double),
                ("bytes_apply", ctypes.c_double), ("n_supernodes", c_i64), ("n_trsm_tasks", c_i64),
                ("n_syrk_tasks", c_i64), ("n_apply_tasks", c_i64), ("y_doubles", c_i64),
                ("max_supernode", c_i64), ("n_waves", c_i64)]


SC_NUM_FEATURES = 10


class Selector(ctypes.Structure):
    _fields_ = [("n_variants", c_i32), ("slices", c_vp), ("tiles", c_vp), ("n_hidden", c_i32),
                ("params_dev", c_vp), ("x_shift", c_vp), ("x_scale", c_vp), ("y_shift", c_vp), ("y_scale", c_vp)]


# every symbol include/sc.h declares, with (argtypes, restype)
SC_SYMBOLS = {
    "sc_plan": ([ctypes.POINTER(c_vp), c_i32, ctypes.POINTER(SubdomainDesc), c_i64, ctypes.POINTER(Options)], c_int),
    "sc_get_sizes": ([c_vp, ctypes.POINTER(Sizes)], c_int),
    "sc_get_stats": ([c_vp, ctypes.POINTER(Stats)], c_int),
    "sc_get_offsets": ([c_vp, c_vp, c_vp], c_int),
    "sc_upload_plan": ([c_vp, c_vp, c_sz, c_vp], c_int),
    "sc_assemble_batch": ([c_vp, c_vp, c_vp, c_vp, c_sz, c_vp], c_int),
    "sc_device_status": ([c_vp, c_vp, c_vp], c_int),
    "sc_assemble_batch_static": ([c_vp, c_vp, c_vp, c_vp], c_int),
    "sc_apply": ([c_vp, c_vp, c_vp, c_vp, c_vp], c_int),
    "sc_apply_fixed": ([c_vp, c_vp, c_vp, c_vp, c_vp], c_int),
    "sc_apply_mixed": ([c_vp, c_vp, c_vp, c_vp, c_i32, c_vp], c_int),
    "sc_apply_digits_size": ([c_vp, ctypes.POINTER(ctypes.c_int64)], c_int),
    "sc_apply_digits_prepare": ([c_vp, c_vp, c_vp, c_vp], c_int),
    "sc_apply_digits": ([c_vp, c_vp, c_vp, c_vp, c_vp], c_int),
    "sc_apply_digits_status": ([c_vp, c_vp, c_vp], c_int),
    "sc_export_F": ([c_vp, c_vp, c_i32, c_vp, c_i32, c_vp], c_int),
    "sc_enable_stage_timing": ([c_vp, c_i32], c_int),
    "sc_stage_times": ([c_vp, ctypes.POINTER(ctypes.c_float), c_i32], c_int),
    "sc_export_plan": ([c_vp, c_vp, c_sz], c_int),
    "sc_workspace_layout": ([c_vp, c_vp, c_vp, c_vp], c_int),
    "sc_subdomain_features": ([c_vp, c_vp, c_vp], c_int),
    "sc_select_workspace": ([c_vp, ctypes.POINTER(Selector), ctypes.POINTER(c_sz)], c_int),
    "sc_select": ([c_vp, ctypes.POINTER(Selector), c_vp, ctypes.c_double, ctypes.c_double, c_vp, c_sz, c_vp, c_vp,
                   c_vp], c_int),
    "sc_last_error": ([c_vp], ctypes.c_char_p),
    "sc_destroy": ([c_vp], None),
}

class ImplicitSizes(ctypes.Structure):
    _fields_ = [("plan_bytes", c_sz), ("ws_bytes", c_sz), ("L_values", c_i64), ("n_supernodes", c_i64),
                ("nnz_visited", c_i64), ("max_levels", c_i64), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double), ("n_cluster_subdomains", c_i64)]


class ImplicitOptions(ctypes.Structure):
    _fields_ = [("cluster_min_work", c_i64), ("pairs", c_i32), ("reserved", c_i32)]


# every symbol include/sc_implicit.h declares
IMPLICIT_SYMBOLS = {
    "sci_plan": ([ctypes.POINTER(c_vp), c_i32, ctypes.POINTER(SubdomainDesc), c_i64,
                  ctypes.POINTER(ImplicitOptions)], c_int),
    "sci_get_sizes": ([c_vp, ctypes.POINTER(ImplicitSizes)], c_int),
    "sci_upload_plan": ([c_vp, c_vp, c_sz, c_vp], c_int),
    "sci_apply": ([c_vp, c_vp, c_vp, c_vp, c_vp, c_sz, c_vp], c_int),
    "sci_device_status": ([c_vp, c_vp, c_vp], c_int),
    "sci_export_plan": ([c_vp, c_vp, c_sz], c_int),
    "sci_last_error": ([c_vp], ctypes.c_char_p),
    "sci_destroy": ([c_vp], None),
}

class PipeSubdomain(ctypes.Structure):
    _fields_ = [("n", c_i32), ("K_colptr", c_vp), ("K_rowind", c_vp), ("K_val", c_vp), ("nfixed", c_i32),
                ("fixed", c_vp), ("perm", c_vp)]


class PipeChunk(ctypes.Structure):
    _fields_ = [("lo", c_i32), ("hi", c_i32), ("plan", c_vp), ("L_dev", c_vp), ("F_dev", c_vp),
                ("ws_dev", c_vp), ("ws_bytes", c_sz)]


class PipeTimes(ctypes.Structure):
    _fields_ = [("wall_ms", ctypes.c_double), ("factor_ms", ctypes.c_double), ("h2d_ms", ctypes.c_double),
                ("assembly_ms", ctypes.c_double), ("serial_ms", ctypes.c_double), ("h2d_bytes", c_i64)]


# every symbol include/sc_pipeline.h declares
PIPELINE_SYMBOLS = {
    "scp_create": ([ctypes.POINTER(c_vp), c_i32, ctypes.POINTER(PipeSubdomain), c_i32, ctypes.POINTER(PipeChunk),
                    c_i32], c_int),
    "scp_run": ([c_vp, c_vp, ctypes.POINTER(PipeTimes)], c_int),
    "scp_last_error": ([c_vp], ctypes.c_char_p),
    "scp_destroy": ([c_vp], None),
}

# every symbol include/sc_probe.h declares
PROBE_SYMBOLS = {
    "sc_probe_fp64_fma": ([c_i32, c_i32, c_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(c_i64), c_vp],
                          c_int),
}

DENSE_SYMBOLS = {
    "scd_create": ([ctypes.POINTER(c_vp), c_i32], c_int),
    "scd_trsm_syrk": ([c_vp, c_i32, c_i32, c_vp, c_vp, c_vp, c_vp], c_int),
    "scd_destroy": ([c_vp], None),
}


def _declare(lib, table):
    for name, (args, res) in table.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res


def declare(lib):
    _declare(lib, SC_SYMBOLS)
    _declare(lib, IMPLICIT_SYMBOLS)
    _declare(lib, PROBE_SYMBOLS)


def declare_pipeline(lib):
    _declare(lib, PIPELINE_SYMBOLS)


def declare_dense(lib):
    _declare(lib, DENSE_SYMBOLS)

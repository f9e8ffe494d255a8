"""ctypes declarations of the C ABI in include/elm.h.  Loading fails loudly
when libelm.so has not been built: there is no fallback implementation."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libelm.so")

i32, i64, dbl, vp = C.c_int32, C.c_int64, C.c_double, C.c_void_p


class elm_problem(C.Structure):
    _fields_ = [("X", vp), ("x_dtype", i32), ("act", i32), ("N", i64), ("n", i64),
                ("ldx", i64), ("W", vp), ("ldw", i64), ("b", vp), ("a", vp), ("L", i64),
                ("T", vp), ("m", i64), ("ldt", i64), ("beta", vp), ("ldb", i64)]


class elm_train_opts(C.Structure):
    _fields_ = [("precision", i32), ("max_refine", i32), ("tol_rank", dbl),
                ("refine_tol", dbl), ("flags", i32), ("wait_limit_ns", i32),
                ("block_split", i32), ("lanes", i32)]


class elm_tune_choice(C.Structure):
    _fields_ = [("panel_cluster", i32), ("panel_width", i32), ("hidden_stages", i32),
                ("gram_stages", i32), ("lanes", i32), ("reserved", i32), ("best_ms", dbl)]


class elm_result(C.Structure):
    _fields_ = [("rank", i64), ("refine_iters", i32), ("status", i32), ("rel_update", dbl),
                ("form", i32), ("reserved", i32)]


# (name, restype, argtypes) for every entry point declared in include/elm.h
SIGNATURES = [
    ("elm_create", C.c_int, [C.POINTER(vp), C.c_int, vp]),
    ("elm_destroy", C.c_int, [vp]),
    ("elm_set_stream", C.c_int, [vp, vp]),
    ("elm_status_string", C.c_char_p, [C.c_int]),
    ("elm_last_error", C.c_char_p, [vp]),
    ("elm_hidden", C.c_int, [vp, vp, C.c_int, i64, i64, i64, vp, i64, vp, vp, i64, C.c_int,
                             C.c_int, vp, i64]),
    ("elm_pinv_rank", C.c_int, [vp, vp, i64, i64, i64, dbl, C.POINTER(i64), vp, vp, i64]),
    ("elm_train", C.c_int, [vp, C.POINTER(elm_problem), i64, C.POINTER(elm_train_opts),
                            C.POINTER(elm_result)]),
    ("elm_predict", C.c_int, [vp, vp, C.c_int, i64, i64, i64, vp, i64, vp, vp, i64, C.c_int,
                              vp, i64, i64, vp, i64]),
    ("elm_phase_times", C.c_int, [vp, C.POINTER(dbl), C.c_int]),
    ("elm_phase_name", C.c_char_p, [C.c_int]),
    ("elm_launch_counter", i64, []),
    ("elm_hidden_noalloc", C.c_int, [vp, C.c_int, i64, i64, i64, vp, i64, vp, vp, i64, C.c_int,
                                     vp, i64, vp]),
    ("elm_hidden_noalloc_bytes", C.c_int, [i64, i64, i64, C.POINTER(i64)]),
    ("elm_rows_create", C.c_int, [vp, vp, C.c_int, i64, i64, i64, vp, i64, vp, vp, i64, C.c_int,
                                  vp, i64, i64, C.c_int, C.POINTER(vp)]),
    ("elm_rows_gram", C.c_int, [vp, vp, i64, vp, i64]),
    ("elm_rows_residual", C.c_int, [vp, vp, i64, vp, i64]),
    ("elm_rows_destroy", C.c_int, [vp]),
    ("elm_factor_gram", C.c_int, [vp, vp, i64, i64, i64, C.c_int, dbl, C.POINTER(vp),
                                  C.POINTER(i64)]),
    ("elm_factor_solve", C.c_int, [vp, vp, i64, i64, vp, i64]),
    ("elm_factor_destroy", C.c_int, [vp]),
    ("elm_autotune", C.c_int, [vp, C.POINTER(elm_problem), i64, C.POINTER(elm_train_opts),
                               C.c_char_p, C.POINTER(elm_tune_choice)]),
    ("elm_autotune_load", C.c_int, [vp, C.c_char_p]),
]

_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libelm.so is not built (run __graft_entry__.build() or "
                              "python -m paper_2011_02436_gb300.build)")
        lib = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib

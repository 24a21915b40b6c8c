"""ctypes binding of libtdbem.so (include/tdbem.h): argument marshalling only.

Every computation runs inside the CUDA library; this module converts numpy
arrays and torch CUDA tensors to pointers and sizes and checks status codes.
It raises if the library or a CUDA device is missing: there is no CPU path.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdbem.so")

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_CAPACITY = -1, -2, -3, -4, -5
SLP, DLP, ADLP = 0, 1, 2
P0, P1 = 0, 1
FP64, MIXED = 0, 1
EULER, RADAU2 = 0, 1


class TdbemError(RuntimeError):
    pass


class Op(C.Structure):
    _fields_ = [("op", C.c_int32), ("prec", C.c_int32), ("c", C.c_double), ("ng", C.c_int32),
                ("reserved", C.c_int32)]


class AcaCfg(C.Structure):
    _fields_ = [("eps", C.c_double), ("eps_aca", C.c_double), ("max_face_rank", C.c_int32),
                ("flags", C.c_int32), ("model", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("nblocks", "nnear", "nfar", "sum_rank", "max_rank", "sum_face_rank",
                                         "stored_complex", "dense_complex", "entries_regular", "entries_tube",
                                         "pairs_singular")] + \
               [(n, C.c_double) for n in ("ms_plan", "ms_singular", "ms_near", "ms_far", "ms_total")] + \
               [("pool_growths", C.c_int64), ("launches", C.c_int64), ("aca_tests", C.c_int64),
                ("pool_first", C.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None

EXPORTS = {
    "tdbem_ctx_create": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "tdbem_ctx_destroy": (C.c_int, [C.c_void_p]),
    "tdbem_last_error": (C.c_char_p, [C.c_void_p]),
    "tdbem_ctx_sync": (C.c_int, [C.c_void_p]),
    "tdbem_ctx_set_near_batch": (C.c_int, [C.c_void_p, C.c_int64]),
    "tdbem_ctx_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "tdbem_ctx_set_pool_scale": (C.c_int, [C.c_void_p, C.c_double]),
    "tdbem_measure_peak": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "tdbem_mesh_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                    C.POINTER(C.c_void_p)]),
    "tdbem_mesh_destroy": (C.c_int, [C.c_void_p]),
    "tdbem_mesh_ndof": (C.c_int64, [C.c_void_p, C.c_int32]),
    "tdbem_freqs_cq_bdf2": (C.c_int, [C.c_void_p, C.c_int32, C.c_double, C.c_double, C.POINTER(C.c_void_p)]),
    "tdbem_freqs_gcq": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                  C.POINTER(C.c_void_p)]),
    "tdbem_freqs_steps": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "tdbem_tensor_recompress": (C.c_int, [C.c_void_p, C.c_double]),
    "tdbem_lowrank_recompress": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                           C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    "tdbem_freqs_points": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]),
    "tdbem_march_step_points": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_int32)]),
    "tdbem_march_create": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                     C.c_int32, C.c_int32, C.POINTER(C.c_void_p)]),
    "tdbem_march_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32,
                                   C.POINTER(C.c_int32)]),
    "tdbem_march_destroy": (C.c_int, [C.c_void_p]),
    "tdbem_freqs_get": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32), C.c_void_p]),
    "tdbem_freqs_destroy": (C.c_int, [C.c_void_p]),
    "tdbem_tree_build": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                   C.POINTER(C.c_void_p)]),
    "tdbem_tree_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    "tdbem_tree_destroy": (C.c_int, [C.c_void_p]),
    "tdbem_entries": (C.c_int, [C.c_void_p, C.POINTER(Op), C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                C.c_int64, C.c_void_p, C.c_int64, C.c_void_p]),
    "tdbem_entries_path": (C.c_int, [C.c_void_p, C.POINTER(Op), C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                     C.c_int64, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]),
    "tdbem_entries_noalloc": (C.c_int, [C.c_void_p, C.POINTER(Op), C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                        C.c_int64, C.c_void_p, C.c_int64, C.c_void_p]),
    "tdbem_compress": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Op), C.c_void_p, C.c_void_p,
                                 C.POINTER(AcaCfg), C.POINTER(C.c_void_p)]),
    "tdbem_tensor_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "tdbem_tensor_entries": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "tdbem_tensor_blocks": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tdbem_tensor_partition": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tdbem_tensor_destroy": (C.c_int, [C.c_void_p]),
    "tdbem_apply_weighted": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "tdbem_apply_freq": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]),
    "tdbem_apply_weighted_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "tdbem_zgemm": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p,
                              C.c_int64, C.c_void_p, C.c_int64]),
    "tdbem_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_int32,
                              C.c_int32, C.POINTER(C.c_int32), C.c_void_p]),
    "tdbem_tensor_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "tdbem_tensor_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "tdbem_tensor_load": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_void_p)]),
    "tdbem_model_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "tdbem_model_load": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_void_p)]),
    "tdbem_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Op), C.c_void_p, C.c_void_p, C.POINTER(AcaCfg),
                                 C.c_void_p]),
    "tdbem_rank_bin": (C.c_int, [C.c_int32]),
    "tdbem_model_create": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_void_p)]),
    "tdbem_model_destroy": (C.c_int, [C.c_void_p]),
    "tdbem_model_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tdbem_model_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tdbem_model_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "tdbem_model_adam_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int32]),
    "tdbem_model_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_int32,
                                    C.c_double, C.c_uint64, C.POINTER(C.c_double)]),
    "tdbem_model_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "tdbem_harvest": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Op), C.c_void_p, C.c_void_p, C.POINTER(AcaCfg),
                                C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]),
}


def load(path=None, build=True):
    """Load libtdbem.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if build:
        from . import build as _b
        _b.build()
    if not os.path.exists(path):
        raise TdbemError("libtdbem.so not found at %s (run paper_2505_00715_gb300/build.py)" % path)
    L = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(rc, ctx=None, what=""):
    if rc != OK:
        msg = _lib.tdbem_last_error(ctx).decode() if ctx else ""
        raise TdbemError("%s failed with status %d: %s" % (what, rc, msg))

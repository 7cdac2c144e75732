"""ctypes binding of libpicpml (include/picpml.h): argument marshalling only.

Every step of the PIC path runs in the CUDA kernels of libpicpml.so; this
module converts Python arguments into the C structs and raises on a non-zero
status.  There is no CPU fallback: if the library cannot be loaded, importing
the binding's users fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpicpml.so")

PIC_FP32, PIC_FP64, PIC_FP32_FIXED64 = 0, 1, 2
PREC = {"fp32": PIC_FP32, "fp64": PIC_FP64, "fixed64": PIC_FP32_FIXED64}
ALPHA = {"zero": 0, "one": 1, "damped": 2, "weight": 3}
TUNING_TILE = 2   # PIC_TUNING_TILE: the tile-resident particle kernel
SOLVER = {"yee": 0, "ck": 1}
STATUS = {0: "PIC_OK", -1: "PIC_EINVAL", -2: "PIC_ENOMEM", -3: "PIC_ECUDA", -4: "PIC_ECFL",
          -5: "PIC_EOVERFLOW", -6: "PIC_ETIMEOUT", -7: "PIC_ENOTIMPL", -8: "PIC_ESTATE",
          -9: "PIC_EPARTICLE"}


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class GridDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("d", C.c_double * 3), ("dt", C.c_double),
                ("cfl", C.c_double), ("shape_order", C.c_int), ("prec", C.c_int),
                ("sort_every", C.c_int), ("split_fp64", C.c_int), ("filter_passes", C.c_int),
                ("solver", C.c_int)]


class PmlDesc(C.Structure):
    _fields_ = [("ncell", C.c_int * 6), ("sigma_max_coef", C.c_double), ("delta_cells", C.c_double),
                ("exponent", C.c_double), ("alpha_mode", C.c_int), ("v_assumed", C.c_double),
                ("face_alpha_set", C.c_int), ("face_alpha", C.c_int * 6)]


class SpeciesDesc(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("mom", C.c_void_p), ("n", C.c_longlong),
                ("capacity", C.c_longlong), ("q", C.c_double), ("m", C.c_double),
                ("immobile", C.c_int)]


class BatchDesc(C.Structure):
    _fields_ = [("nruns", C.c_int), ("nx", C.POINTER(C.c_int)), ("nz", C.POINTER(C.c_int)),
                ("npml", C.POINTER(C.c_int)), ("d", C.c_double * 2), ("dt", C.c_double),
                ("cfl", C.c_double), ("shape_order", C.c_int), ("prec", C.c_int), ("pml", PmlDesc),
                ("q", C.c_double), ("m", C.c_double), ("pos", C.c_void_p), ("mom", C.c_void_p)]


# every symbol include/picpml.h declares, with its ctypes signature
VP = C.c_void_p
SIGNATURES = {
    "pic_init": (C.c_int, [C.POINTER(VP), C.POINTER(GridDesc), VP]),
    "pml_init": (C.c_int, [VP, C.POINTER(PmlDesc)]),
    "pic_add_species": (C.c_int, [VP, C.POINTER(SpeciesDesc), C.POINTER(C.c_int)]),
    "push": (C.c_int, [VP]),
    "deposit": (C.c_int, [VP]),
    "field_step": (C.c_int, [VP]),
    "step_n": (C.c_int, [VP, C.c_int]),
    "push_deposit": (C.c_int, [VP]),
    "pic_launch_count": (C.c_int, [VP, C.POINTER(C.c_longlong)]),
    "pic_particle_steps": (C.c_int, [VP, C.POINTER(C.c_longlong)]),
    "pic_autotune": (C.c_int, [VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pic_set_tuning": (C.c_int, [VP, C.c_int, C.c_int]),
    "pic_sort": (C.c_int, [VP]),
    "pic_grid_info": (C.c_int, [VP, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "pic_get_field": (C.c_int, [VP, C.c_int, VP, C.c_int]),
    "pic_set_field": (C.c_int, [VP, C.c_int, VP, C.c_int]),
    "pic_set_prescribed": (C.c_int, [VP, C.c_int]),
    "pic_set_conductor": (C.c_int, [VP, VP]),
    "pic_set_old_positions": (C.c_int, [VP, C.c_int, VP]),
    "pic_get_current_fixed": (C.c_int, [VP, C.c_int, VP]),
    "pic_num_particles": (C.c_int, [VP, C.c_int, C.POINTER(C.c_longlong)]),
    "pic_inject": (C.c_int, [VP, C.c_int, VP, VP, C.c_longlong]),
    "pic_diag": (C.c_int, [VP, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pic_diag_static": (C.c_int, [VP, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pic_sync": (C.c_int, [VP]),
    "pic_state_size": (C.c_int, [VP, C.POINTER(C.c_longlong)]),
    "pic_get_state": (C.c_int, [VP, VP]),
    "pic_set_state": (C.c_int, [VP, VP]),
    "pic_batch_init": (C.c_int, [C.POINTER(VP), C.POINTER(BatchDesc), VP]),
    "pic_batch_step": (C.c_int, [VP, C.c_int]),
    "pic_batch_get_field": (C.c_int, [VP, C.c_int, C.c_int, VP, C.c_int]),
    "pic_batch_set_prescribed": (C.c_int, [VP, C.c_int]),
    "pic_batch_particle_steps": (C.c_int, [VP, C.POINTER(C.c_longlong)]),
    "pic_batch_info": (C.c_int, [VP, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "pic_batch_tuning": (C.c_int, [VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float), C.c_int]),
    "pic_batch_sync": (C.c_int, [VP]),
    "pic_batch_last_error": (C.c_char_p, [VP]),
    "pic_batch_destroy": (None, [VP]),
    "pic_last_error": (C.c_char_p, [VP]),
    "pic_destroy": (None, [VP]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads libpicpml.so (built by paper_2201_09084_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"libpicpml.so not built ({path}); run "
                                  "python -c 'import __graft_entry__ as g; g.build()'")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(code, ctx=None):
    if code != 0:
        msg = load().pic_last_error(ctx)
        raise PicError(code, msg.decode() if msg else "")

"""ctypes binding of libocg.so (argument marshalling only; every step runs in the library).

Names follow the C ABI in include/ocg.h.  Device vectors are passed as torch CUDA tensors
(only their data pointers cross the boundary)."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libocg.so")

OCG_OK, OCG_EINVAL, OCG_ENOMEM, OCG_ECUDA, OCG_ENOTCONV, OCG_ENAN, OCG_ESTATE = 0, -1, -2, -3, -4, -5, -6
OCG_F64, OCG_F32 = 0, 1
OCG_PREC_FP64, OCG_PREC_FP32, OCG_PREC_MIXED = 0, 1, 2
OCG_HIST = 128
OCG_NOALLOC_MAX_CELLS = 1 << 20


class OctreeDesc(C.Structure):
    _fields_ = [("n0", C.c_int32), ("max_depth", C.c_int32), ("refine", C.c_int32),
                ("n_spheres", C.c_int32), ("n_boxes", C.c_int32), ("tile_log2", C.c_int32),
                ("band", C.c_double), ("spheres", (C.c_double * 4) * 4),
                ("boxes", (C.c_double * 6) * 4), ("n_sines", C.c_int32), ("reserved2", C.c_int32),
                ("sines", (C.c_double * 5) * 8)]


OCG_SWEEP_AUTO, OCG_SWEEP_OCTET, OCG_SWEEP_CELL, OCG_SWEEP_QUAD, OCG_SWEEP_TILE = -1, 0, 1, 2, 3


class MGParams(C.Structure):
    _fields_ = [("mu", C.c_int32), ("nu_pre", C.c_int32), ("nu_post", C.c_int32),
                ("nu_coarsest", C.c_int32), ("beta_restrict", C.c_double), ("alpha", C.c_double),
                ("coef_dtype", C.c_int32), ("bf16_coarse", C.c_int32), ("sweep_form", C.c_int32),
                ("mu_min_cells", C.c_int32), ("coarsening", C.c_int32), ("reserved", C.c_int32)]


OCG_COARSEN_ALGEBRAIC = 0
OCG_COARSEN_GEOMETRIC = 1


OCG_SOLVE_EAGER = 1
OCG_SOLVE_TRANSPOSE = 2
OCG_SOLVE_UNROLLED = 4
OCG_SOLVE_BICGSTAB = 8
OCG_SOLVE_WARM = 16


class SolveParams(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int32), ("precision", C.c_int32),
                ("nullspace", C.c_int32), ("flags", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("rel_res", C.c_double),
                ("true_rel_res", C.c_double), ("kernels", C.c_int64), ("hist", C.c_double * OCG_HIST)]


class OcgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libocg error %d: %s" % (code, msg))
        self.code = code


_lib = None

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

# (name, restype, argtypes)
_SIGS = [
    ("ocg_last_error", C.c_char_p, []),
    ("ocg_octree_build", C.c_int, [C.POINTER(OctreeDesc), C.POINTER(C.c_void_p)]),
    ("ocg_octree_rebuild", C.c_int, [C.c_void_p, C.POINTER(OctreeDesc), C.POINTER(C.c_double),
                                     C.POINTER(C.c_void_p)]),
    ("ocg_octree_destroy", None, [C.c_void_p]),
    ("ocg_octree_counts", C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    ("ocg_octree_export_leaves", C.c_int, [C.c_void_p] + [C.c_void_p] * 4),
    ("ocg_octree_export_neighbours", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ocg_octree_export_faces", C.c_int, [C.c_void_p] + [C.c_void_p] * 7),
    ("ocg_octree_export_faces_range", C.c_int, [C.c_void_p, C.c_int64, C.c_int64] + [C.c_void_p] * 7),
    ("ocg_octree_export_level", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)] + [C.c_void_p] * 4),
    ("ocg_setup_hierarchy", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.POINTER(MGParams),
                                      C.c_void_p, C.POINTER(C.c_void_p)]),
    ("ocg_hier_destroy", None, [C.c_void_p]),
    ("ocg_hier_update_beta", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ocg_hier_export_coefs", C.c_int, [C.c_void_p, C.c_int32] + [C.c_void_p] * 4),
    ("ocg_hier_tuning", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("ocg_apply_A", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    ("ocg_face_grad", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ocg_vcycle", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ocg_vcycle_transpose", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ocg_pcg_solve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveParams),
                                C.POINTER(SolveStats), C.c_void_p]),
    ("ocg_apply_A_f32_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("ocg_probe_set", C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    ("ocg_probe_read", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                 C.POINTER(C.c_int64)]),
    ("ocg_launch_count", C.c_int, [C.POINTER(C.c_int64)]),
    ("ocg_set_allocator", C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
    ("ocg_batch_create", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("ocg_batch_destroy", None, [C.c_void_p]),
    ("ocg_batch_info", C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("ocg_pcg_solve_batched", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveParams),
                                        C.c_void_p, C.c_void_p]),
]

OCG_PROBE_OFF, OCG_PROBE_SWEEP, OCG_PROBE_RESTRICT, OCG_PROBE_PROLONG, OCG_PROBE_APPLY = 0, 1, 2, 3, 4
OCG_PROBE_TAIL = 5

EXPORTED = [n for n, _, _ in _SIGS]


def lib():
    """Load libocg.so (built in-tree); raises if it is missing — there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libocg.so is not built (run paper_2604_18886_b300/build.py)")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != OCG_OK:
        msg = lib().ocg_last_error().decode(errors="replace")
        raise OcgError(code, msg)
    return code


def ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())

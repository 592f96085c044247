"""ctypes binding of libatlasgb.so: the C ABI of include/atlas_gb.h under the
same names, argument marshalling only.

Every ``atlas_*`` function here takes plain integers (handles, device
pointers, sizes, stream) exactly like its C counterpart and raises
``AtlasError`` when the call returns a negative code.  The library is loaded
from the package directory; if it has not been built the import fails
loudly -- there is no CPU fallback.  With the environment variable
ATLASGB_BOUNDSCHECK=1 the bounds-checked build of the same library is loaded
instead (kernels that check every table index; see build.py).
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
BOUNDSCHECK = os.environ.get("ATLASGB_BOUNDSCHECK", "") == "1"
LIB_PATH = os.path.join(_PKG, "libatlasgb_boundscheck.so" if BOUNDSCHECK else "libatlasgb.so")

ATLAS_F32, ATLAS_F64, ATLAS_BF16 = 0, 1, 2
ATLAS_OP_GRADIENT, ATLAS_OP_DIVERGENCE, ATLAS_OP_GRADIENT_ADJOINT = 0, 1, 2
ATLAS_OP_DIVERGENCE_ADJOINT, ATLAS_OP_LAPLACIAN = 3, 4
ATLAS_OP_CURL, ATLAS_OP_VECTOR_GRADIENT, ATLAS_OP_CURL_ADJOINT = 5, 6, 7
ATLAS_PROJ_ROTATED_LONLAT, ATLAS_PROJ_MERCATOR, ATLAS_PROJ_LAMBERT_CONFORMAL = 0, 1, 2
ATLAS_PROJ_POLAR_STEREOGRAPHIC = 3
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EALIGN", -5: "EDTYPE", -6: "ESTATE", -7: "EBOUNDS"}


class AtlasError(RuntimeError):
    def __init__(self, code: int, func: str, msg: str):
        self.code = code
        super().__init__("%s failed: %s (%d): %s" % (func, ERRORS.get(code, "?"), code, msg))


class atlas_batch_desc(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("fvm", ctypes.c_void_p), ("in0", ctypes.c_void_p),
                ("in1", ctypes.c_void_p), ("out0", ctypes.c_void_p), ("out1", ctypes.c_void_p),
                ("nlev", ctypes.c_int), ("ld", ctypes.c_int64)]


class atlas_batch_tune(ctypes.Structure):
    _fields_ = [("vec", ctypes.c_int), ("tile_items", ctypes.c_int), ("threads", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("plain_waves", ctypes.c_int)]


P = ctypes.c_void_p
PP = ctypes.POINTER(ctypes.c_void_p)
I32 = ctypes.c_int
I64 = ctypes.c_int64
SZ = ctypes.c_size_t

# name: (restype, argtypes, checked)
_SIGS = {
    "atlas_init": (I32, [], True),
    "atlas_finalize": (I32, [], True),
    "atlas_version": (ctypes.c_char_p, [], False),
    "atlas_info": (ctypes.c_char_p, [], False),
    "atlas_last_error": (ctypes.c_char_p, [], False),
    "atlas_grid_octahedral": (I32, [I32, PP], True),
    "atlas_grid_info": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I32), PP, PP, PP], True),
    "atlas_grid_destroy": (None, [P], False),
    "atlas_mesh_build": (I32, [P, PP], True),
    "atlas_mesh_info": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64), PP, PP, PP, PP, PP, PP], True),
    "atlas_mesh_destroy": (None, [P], False),
    "atlas_fvm_build_dual": (I32, [P, ctypes.c_double, PP], True),
    "atlas_fvm_info": (I32, [P, PP, PP, PP, PP], True),
    "atlas_fvm_prepare": (I32, [P, ctypes.c_uint, ctypes.c_uint], True),
    "atlas_fvm_set_launch": (I32, [P, I32, I32, I32, I32, I32, I32, I32], True),
    "atlas_fvm_set_group": (I32, [P, I32, I32, I32, I32, I32, I32, I32], True),
    "atlas_kernel_status": (I32, [ctypes.POINTER(ctypes.c_uint), I32], True),
    "atlas_fp64_fma_rate_kernel": (I32, [P, I32, I32, I64, P], True),
    "atlas_fvm_tile_info": (I32, [P, I32, I32, I32, I64, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                  ctypes.POINTER(I64), ctypes.POINTER(I64)], True),
    "atlas_debug_tile_hang": (I32, [I32], True),
    "atlas_debug_tile_wait_hint": (I32, [ctypes.c_uint], True),
    "atlas_debug_tile_unions": (I32, [I32], True),
    "atlas_fvm_tile_union_groups": (I32, [P, I32, I32, ctypes.POINTER(I64)], True),
    "atlas_fvm_group_table": (I32, [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64), P, P, P], True),
    "atlas_fvm_tile_table": (I32, [P, I32, I32, I32, I32, ctypes.POINTER(I64), ctypes.POINTER(I64), P, P,
                                   ctypes.POINTER(I64), P, P], True),
    "atlas_fvm_stencil_table": (I32, [P, I32, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I32),
                                      P, P, P, P], True),
    "atlas_fvm_destroy": (None, [P], False),
    "atlas_nabla_gradient": (I32, [P, P, P, P, I32, I64, I32, P], True),
    "atlas_nabla_divergence": (I32, [P, P, P, P, I32, I64, I32, P], True),
    "atlas_nabla_laplacian": (I32, [P, P, P, I32, I64, I32, P], True),
    "atlas_nabla_gradient_adjoint": (I32, [P, P, P, P, I32, I64, I32, P], True),
    "atlas_nabla_divergence_adjoint": (I32, [P, P, P, P, I32, I64, I32, P], True),
    "atlas_nabla_curl": (I32, [P, P, P, P, I32, I64, I32, P], True),
    "atlas_nabla_curl_adjoint": (I32, [P, P, P, P, I32, I64, I32, P], True),
    "atlas_grid_regular_gaussian": (I32, [I32, P], True),
    "atlas_grid_regional": (I32, [I32, I32, I32, P, PP], True),
    "atlas_grid_regional_info": (I32, [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(I32), PP, PP],
                                 True),
    "atlas_fvm_regional_info": (I32, [P, PP, PP], True),
    "atlas_fvm_integral_workspace_bytes": (SZ, [P, I32], False),
    "atlas_fvm_check": (I32, [P, ctypes.POINTER(ctypes.c_double)], True),
    "atlas_part_interior": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)], True),
    "atlas_part_apply_nodes": (I32, [P, I32, P, P, P, P, I64, I64, I32, I64, I32, P], True),
    "atlas_debug_fail_allocations": (I32, [I32], True),
    "atlas_fvm_save": (I32, [P, ctypes.c_char_p], True),
    "atlas_fvm_radius": (I32, [P, ctypes.POINTER(ctypes.c_double)], True),
    "atlas_fvm_load": (I32, [ctypes.c_char_p, PP, PP, PP], True),
    "atlas_fvm_integral": (I32, [P, P, I64, I64, I32, I64, I32, P, P, SZ, P], True),
    "atlas_remap_create": (I32, [P, P, P], True),
    "atlas_remap_info": (I32, [P, P, P, P], True),
    "atlas_remap_apply": (I32, [P, P, P, I32, I64, I64, I32, P], True),
    "atlas_remap_destroy": (None, [P], False),
    "atlas_part_create": (I32, [P, I32, I32, I32, P], True),
    "atlas_part_info": (I32, [P, P, P, P, P], True),
    "atlas_part_neighbour": (I32, [P, I32, P, P, P, P, P], True),
    "atlas_part_apply": (I32, [P, I32, P, P, P, P, I32, I64, I32, P], True),
    "atlas_part_destroy": (None, [P], False),
    "atlas_nabla_vector_gradient": (I32, [P, P, P, P, P, P, P, I32, I64, I32, P], True),
    "atlas_nabla_workspace_bytes": (SZ, [P, I32, I32, I64, I32], False),
    "atlas_nabla_gradient_edges": (I32, [P, P, P, P, P, SZ, I32, I64, I32, P], True),
    "atlas_nabla_gradient_edges_averaged": (I32, [P, P, P, P, P, SZ, I32, I64, I32, P], True),
    "atlas_nabla_divergence_edges": (I32, [P, P, P, P, P, SZ, I32, I64, I32, P], True),
    "atlas_nabla_laplacian_edges": (I32, [P, P, P, P, SZ, I32, I64, I32, P], True),
    "atlas_nabla_laplacian_edges_noalloc": (I32, [P, P, P, I32, I64, I32, P], True),
    "atlas_batch_create": (I32, [ctypes.POINTER(atlas_batch_desc), I32, I32, ctypes.POINTER(atlas_batch_tune), PP], True),
    "atlas_batch_launch": (I32, [P, P], True),
    "atlas_batch_info": (I32, [P, ctypes.POINTER(I64), ctypes.POINTER(I64)], True),
    "atlas_batch_destroy": (None, [P], False),
    "atlas_field_sync": (I32, [P, P, SZ, I32, P], True),
}

if not os.path.exists(LIB_PATH):
    raise ImportError("libatlasgb.so is not built (%s); run `python -c \"import __graft_entry__ as g; g.build()\"` "
                      "or `python paper_1908_07038_gb300/build.py`" % LIB_PATH)

lib = ctypes.CDLL(LIB_PATH)


def _wrap(name, restype, argtypes, checked):
    fn = getattr(lib, name)
    fn.restype = restype
    fn.argtypes = argtypes
    if not checked:
        return fn

    def call(*args):
        rc = fn(*args)
        if rc != 0:
            raise AtlasError(rc, name, (lib.atlas_last_error() or b"").decode())
        return rc

    call.__name__ = name
    call.raw = fn
    return call


lib.atlas_last_error.restype = ctypes.c_char_p
lib.atlas_last_error.argtypes = []
for _n, (_r, _a, _c) in _SIGS.items():
    globals()[_n] = _wrap(_n, _r, _a, _c)

EXPORTED = tuple(_SIGS)

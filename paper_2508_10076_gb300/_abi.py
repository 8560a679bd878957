"""ctypes declarations of the libtk C ABI (include/tk.h).  Argument marshalling only.

Loading fails loudly if the shared library is missing: there is no fallback path.
"""

import ctypes as C
import os

from .build import LIB

c_i32p = C.POINTER(C.c_int32)
c_i64p = C.POINTER(C.c_int64)
c_intp = C.POINTER(C.c_int)
c_dblp = C.POINTER(C.c_double)
c_vp = C.c_void_p
c_szp = C.POINTER(C.c_size_t)

# allocator hooks of tk_ctx_create (tk_alloc_fn, tk_free_fn)
ALLOC_FN = C.CFUNCTYPE(c_vp, C.c_size_t, c_vp)
FREE_FN = C.CFUNCTYPE(None, c_vp, C.c_size_t, c_vp)

# name: (restype, argtypes)
SIGNATURES = {
    "tk_version": (C.c_int, []),
    "tk_status_string": (C.c_char_p, [C.c_int]),
    "tk_ctx_create": (C.c_int, [C.c_int, c_vp, ALLOC_FN, FREE_FN, c_vp, C.POINTER(c_vp)]),
    "tk_ctx_set_budget": (C.c_int, [c_vp, C.c_size_t]),
    "tk_ctx_reserve": (C.c_int, [c_vp, C.c_size_t]),
    "tk_ctx_release": (C.c_int, [c_vp, C.c_size_t]),
    "tk_ctx_memory": (C.c_int, [c_vp, c_szp, c_szp, c_szp, c_i64p]),
    "tk_ctx_alloc": (C.c_int, [c_vp, C.c_size_t, C.POINTER(c_vp)]),
    "tk_ctx_free": (C.c_int, [c_vp, c_vp]),
    "tk_ctx_destroy": (None, [c_vp]),
    "tk_ctx_last_error": (C.c_char_p, [c_vp]),
    "tk_ctx_sync": (C.c_int, [c_vp, c_vp]),
    "tk_ctx_launch_count": (C.c_int64, [c_vp]),
    "tk_ctx_selftest_timeout": (C.c_int, [c_vp, c_vp]),
    "tk_ctx_profile": (C.c_int, [c_vp, C.c_int]),
    "tk_ctx_profile_read": (C.c_int, [c_vp, C.c_int, C.c_char_p, c_i64p, c_dblp, c_intp]),
    "tk_space_create": (C.c_int, [c_vp, C.c_int, C.c_int, c_i32p, c_i64p, C.c_int, C.POINTER(c_vp)]),
    "tk_space_dual": (C.c_int, [c_vp, c_vp, C.POINTER(c_vp)]),
    "tk_space_destroy": (None, [c_vp]),
    "tk_space_dim": (C.c_int64, [c_vp]),
    "tk_space_reduced_dim": (C.c_int64, [c_vp]),
    "tk_tmap_create": (C.c_int, [c_vp, C.c_int, C.POINTER(c_vp), C.c_int, C.POINTER(c_vp), C.POINTER(c_vp)]),
    "tk_tmap_destroy": (None, [c_vp]),
    "tk_tmap_numel": (C.c_int64, [c_vp]),
    "tk_tmap_nlegs": (C.c_int, [c_vp, c_intp, c_intp]),
    "tk_tmap_leg": (C.c_int, [c_vp, c_vp, C.c_int, C.POINTER(c_vp)]),
    "tk_tmap_hash": (C.c_uint64, [c_vp]),
    "tk_tmap_nblocks": (C.c_int, [c_vp]),
    "tk_tmap_block": (C.c_int, [c_vp, C.c_int, c_i32p, c_i64p, c_i64p, c_i64p]),
    "tk_tmap_ntreepairs": (C.c_int64, [c_vp]),
    "tk_tmap_treepair": (C.c_int, [c_vp, C.c_int64, c_i32p, c_i64p, c_i64p, c_i64p]),
    "tk_tmap_upload": (C.c_int, [c_vp, c_vp, C.c_int, c_vp, C.c_size_t, c_vp, c_vp]),
    "tk_tmap_download": (C.c_int, [c_vp, c_vp, C.c_int, c_vp, c_vp, C.c_size_t, c_vp]),
    "tk_tmap_alloc": (C.c_int, [c_vp, c_vp, C.c_int, C.POINTER(c_vp)]),
    "tk_permute_plan": (C.c_int, [c_vp, c_vp, C.c_int, c_intp, C.c_int, c_intp, C.c_int, C.POINTER(c_vp)]),
    "tk_adjoint_plan": (C.c_int, [c_vp, c_vp, C.c_int, C.POINTER(c_vp)]),
    "tk_contract_plan": (C.c_int, [c_vp, c_vp, C.c_int, c_intp, C.c_int, c_intp, c_vp, C.c_int, c_intp,
                                   C.c_int, c_intp, C.c_int, c_intp, C.c_int, c_intp, C.c_int, C.c_int,
                                   C.c_int, C.POINTER(c_vp)]),
    "tk_compose_plan": (C.c_int, [c_vp, c_vp, c_vp, C.c_int, C.c_int, C.c_int, C.POINTER(c_vp)]),
    "tk_plan_destroy": (None, [c_vp]),
    "tk_plan_output": (C.c_int, [c_vp, c_vp, C.POINTER(c_vp)]),
    "tk_plan_workspace_bytes": (C.c_size_t, [c_vp]),
    "tk_plan_flops": (C.c_double, [c_vp]),
    "tk_plan_tensor_flops": (C.c_double, [c_vp]),
    "tk_plan_permute_stats": (C.c_int, [c_vp, C.c_int, c_vp]),
    "tk_plan_permute_bytes": (C.c_double, [c_vp]),
    "tk_plan_ntransform": (C.c_int64, [c_vp, C.c_int]),
    "tk_plan_transform": (C.c_int, [c_vp, C.c_int, C.c_int64, c_i64p, c_i64p, c_dblp]),
    "tk_permute": (C.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp]),
    "tk_contract": (C.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, C.c_size_t, c_vp]),
    "tk_contract_noalloc": (C.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "tk_noalloc_scratch_bytes": (C.c_size_t, []),
    "tk_contract_batch": (C.c_int, [c_vp, C.c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "tk_svd_plan": (C.c_int, [c_vp, c_vp, C.c_int, C.POINTER(c_vp)]),
    "tk_svd_outputs": (C.c_int, [c_vp, c_vp, C.POINTER(c_vp), C.POINTER(c_vp), C.POINTER(C.c_int64)]),
    "tk_svd_nblocks": (C.c_int64, [c_vp]),
    "tk_svd_block": (C.c_int, [c_vp, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                               C.POINTER(C.c_int64)]),
    "tk_svd": (C.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, C.c_size_t, c_vp]),
    "tk_svd_truncate": (C.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "tk_plan_autotune": (C.c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, C.c_size_t, c_vp, c_vp]),
    "tk_plan_set_choice": (C.c_int, [c_vp, c_vp, C.c_int]),
    "tk_copy_h2d": (C.c_int, [c_vp, c_vp, c_vp, C.c_size_t, c_vp]),
    "tk_copy_d2h": (C.c_int, [c_vp, c_vp, c_vp, C.c_size_t, c_vp]),
    "tk_probe_fp64_peak": (C.c_int, [c_vp, C.c_double, c_dblp, c_dblp, c_vp]),
    "tk_fsymbol": (C.c_double, [C.c_int, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "tk_rsymbol": (C.c_double, [C.c_int, C.c_int32, C.c_int32, C.c_int32]),
}

_LIB = None


def load(path: str = LIB):
    """Load libtk.so (build it first with paper_2508_10076_gb300.build.build_library())."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libtk.so not found at {path}; run paper_2508_10076_gb300.build.build_library()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib

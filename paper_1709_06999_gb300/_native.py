"""ctypes declarations of the C ABI in include/galario_gb300.h.

Loading fails loudly when the shared library is missing: there is no CPU
fallback anywhere in the package.
"""
from __future__ import annotations

import ctypes as ct
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgalario_gb300.so")

P = ct.c_void_p
I32 = ct.c_int
I64 = ct.c_int64
D = ct.c_double

_SIGNATURES = {
    "gal_create": (I32, [ct.POINTER(P), I32]),
    "gal_destroy": (None, [P]),
    "gal_reserve": (I32, [P, I32, I32]),
    "gal_strerror": (ct.c_char_p, [I32]),
    "gal_last_cuda_error": (ct.c_char_p, [P]),
    "gal_check": (I32, [P]),
    "gal_launch_count": (ct.c_uint64, [P]),
    "gal_set_stage_timing": (I32, [P, I32]),
    "gal_stage_times": (I32, [P, ct.POINTER(D), ct.POINTER(I64)]),
    "gal_data_destroy": (None, [P]),
}
for _p in ("f32", "f64"):
    _SIGNATURES.update({
        f"gal_data_create_{_p}": (I32, [P, P, P, P, P, P, I64, P, ct.POINTER(P)]),
        f"gal_data_create_freq_{_p}": (I32, [P, P, P, P, P, P, P, I64, P, ct.POINTER(P)]),
        f"gal_data_create_sorted_{_p}": (I32, [P, P, P, P, P, P, I64, P, ct.POINTER(P)]),
        f"gal_z_order_{_p}": (I32, [P, P, I64, P]),
        f"gal_sweep_{_p}": (I32, [P, P, I32, D, D, I32, D, D, P, P]),
        f"gal_sample_image_{_p}": (I32, [P, P, I32, D, D, D, D, I64, P, P, P, P]),
        f"gal_sample_profile_{_p}": (I32, [P, P, I32, D, D, I32, D, D, D, D, D, I64, P, P, P, P]),
        f"gal_chi2_image_{_p}": (I32, [P, P, I32, D, D, D, D, P, P, P]),
        f"gal_chi2_profile_{_p}": (I32, [P, P, I32, D, D, I32, D, D, D, D, D, P, P, P]),
        f"gal_chi2_image_host_{_p}": (I32, [P, P, I32, D, D, D, D, P, P, P]),
        f"gal_chi2_image_host_async_{_p}": (I32, [P, P, I32, D, D, D, D, P, P, P]),
        f"gal_get_image_size_{_p}": (I32, [P, P, P, I64, D, D, D, ct.POINTER(I64),
                                            ct.POINTER(D), P]),
        f"gal_sample_image_multi_{_p}": (I32, [P, P, I32, D, D, I32, P, P, P, I64, P, P, P, P]),
        f"gal_chi2_image_multi_{_p}": (I32, [P, P, I32, D, D, I32, P, P, P, P, P, P]),
        f"gal_chi2_profile_multi_{_p}": (I32, [P, P, I32, D, D, I32, D, D, D, I32, P, P, P, P, P,
                                               P]),
    })

_SIGNATURES["gal_chi2_image_noalloc_f32"] = (I32, [P, I32, D, D, D, D, P, P, P, P, P, I64, P, P])


class GalRequest(ct.Structure):
    """struct gal_request of include/galario_gb300.h."""
    _fields_ = [("image", P), ("intensity", P), ("nr", I32), ("Rmin", D), ("dR", D),
                ("inc", D), ("nxy", I32), ("dxy", D), ("dRA", D), ("dDec", D), ("PA", D),
                ("data", P), ("pb_fwhm", D), ("full_plane", I32)]


class GalOpts(ct.Structure):
    """struct gal_opts of include/galario_gb300.h."""
    _fields_ = [("pb_fwhm", D), ("full_plane", I32)]


_OPTS = ct.POINTER(GalOpts)
for _p in ("f32", "f64"):
    _SIGNATURES.update({
        f"gal_sample_image_ex_{_p}": (I32, [P, P, I32, D, D, D, D, _OPTS, I64, P, P, P, P]),
        f"gal_sample_profile_ex_{_p}": (I32, [P, P, I32, D, D, I32, D, D, D, D, D, _OPTS, I64, P,
                                              P, P, P]),
        f"gal_chi2_image_ex_{_p}": (I32, [P, P, I32, D, D, D, D, _OPTS, P, P, P]),
        f"gal_chi2_profile_ex_{_p}": (I32, [P, P, I32, D, D, I32, D, D, D, D, D, _OPTS, P, P, P]),
    })


class GalServerStats(ct.Structure):
    """struct gal_server_stats of include/galario_gb300.h."""
    _fields_ = [("submitted", ct.c_uint64), ("completed", ct.c_uint64),
                ("launches", ct.c_uint64), ("max_inflight", ct.c_uint64),
                ("data_bytes", ct.c_size_t), ("workspace_bytes", ct.c_size_t),
                ("peak_bytes", ct.c_size_t)]


_SIGNATURES.update({
    "gal_workspace_bytes": (ct.c_size_t, [P]),
    "gal_set_hbm_budget": (I32, [P, ct.c_size_t]),
    "gal_device": (I32, [P]),
    "gal_data_info": (I32, [P, ct.POINTER(I64), ct.POINTER(I32)]),
    "gal_server_create": (I32, [I32, ct.c_size_t, I32, I32, ct.POINTER(P)]),
    "gal_server_add_data_f32": (I32, [P, P, P, P, P, P, I64, ct.POINTER(P)]),
    "gal_server_add_data_f64": (I32, [P, P, P, P, P, P, I64, ct.POINTER(P)]),
    "gal_server_add_data_sorted_f32": (I32, [P, P, P, P, P, P, I64, ct.POINTER(P)]),
    "gal_server_add_data_sorted_f64": (I32, [P, P, P, P, P, P, I64, ct.POINTER(P)]),
    "gal_server_submit": (I32, [P, ct.POINTER(GalRequest), ct.POINTER(ct.c_uint64)]),
    "gal_server_submit_many": (I32, [P, ct.POINTER(GalRequest), I32, ct.POINTER(ct.c_uint64)]),
    "gal_server_wait": (I32, [P, ct.c_uint64, I32, ct.POINTER(D), ct.POINTER(D)]),
    "gal_server_get_stats": (I32, [P, ct.POINTER(GalServerStats)]),
    "gal_server_destroy": (None, [P]),
    "gal_chi2_batch": (I32, [P, ct.POINTER(GalRequest), I32, P, P]),
    "gal_set_batch_tuning": (I32, [P, I32]),
    "gal_set_batch_shape": (I32, [P, I32, I32, I32, I32, I32, I32]),
    "gal_get_batch_shape": (I32, [P, I32, I32, I32, ct.POINTER(I32), ct.POINTER(I32)]),
    "gal_set_fft_radix": (I32, [I32, I32, I32, I32, I32]),
    "gal_get_fft_radix": (I32, [I32, I32, I32, ct.POINTER(I32), ct.POINTER(I32)]),
    "gal_chi2_batch_capture": (I32, [P, ct.POINTER(GalRequest), I32, P, P, ct.POINTER(P)]),
    "gal_graph_update": (I32, [P, ct.POINTER(GalRequest), I32, P]),
    "gal_graph_launch": (I32, [P, P]),
    "gal_graph_destroy": (None, [P]),
})

EXPORTED = sorted(_SIGNATURES)

_lib = None


def load(path: str = LIB_PATH) -> ct.CDLL:
    """Load the library (once) and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library not built: {path} is missing. Build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc).")
    lib = ct.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib

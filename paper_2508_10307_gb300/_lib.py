"""ctypes declarations of the C ABI in include/htsvd.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libhtsvd.so")

HTSVD_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "CUDA", 4: "OOM", 5: "TIMEOUT", 6: "DEGENERATE_BASIS"}
HTSVD_ERR_DEGENERATE_BASIS = 6

EXPORTED = ["htsvd_denoise", "htsvd_denoise_f32", "htsvd_estimate_sigma", "htsvd_denoise_batch",
            "htsvd_denoise_vjp", "htsvd_num_groups", "htsvd_status_string", "htsvd_release_workspace",
            "htsvd_profile_enable", "htsvd_profile_collect", "htsvd_denoise_noalloc", "htsvd_denoise_adaptive",
            "htsvd_denoise_video", "htsvd_denoise_tau_sweep", "htsvd_sure", "htsvd_denoise_cube",
            "htsvd_sure_weights", "htsvd_tune_weights", "htsvd_project_patches", "htsvd_denoise_volume",
            "htsvd_denoise_volume_adaptive"]


class CParams(ctypes.Structure):
    _fields_ = [
        ("ps", ctypes.c_int32),
        ("stride", ctypes.c_int32),
        ("window", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("tau_mult", ctypes.c_double),
        ("match_mode", ctypes.c_int32),
        ("gcp_gamma", ctypes.c_double),
        ("agg_mode", ctypes.c_int32),
        ("adapt", ctypes.c_int32),
        ("beta", ctypes.c_double),
        ("rank_gamma", ctypes.c_int32),
        ("tile", ctypes.c_int32),
        ("h_sigma_out", ctypes.POINTER(ctypes.c_double)),
        ("d_mask_out", ctypes.c_void_p),
        ("d_weights_out", ctypes.c_void_p),
        ("d_basis_out", ctypes.c_void_p),
        ("d_coef_out", ctypes.c_void_p),
        ("strict_basis", ctypes.c_int32),
        ("h_basis_gap_out", ctypes.POINTER(ctypes.c_double)),
    ]


class CImage(ctypes.Structure):
    _fields_ = [
        ("d_in", ctypes.c_void_p),
        ("H", ctypes.c_int32),
        ("W", ctypes.c_int32),
        ("C", ctypes.c_int32),
        ("sigma", ctypes.c_double),
        ("d_out", ctypes.c_void_p),
        ("d_idx_out", ctypes.c_void_p),
    ]


_lib = None


class HtsvdError(RuntimeError):
    pass


class DegenerateBasisError(HtsvdError):
    """A global-basis slice has coinciding eigenvalues (strict mode)."""


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libhtsvd.so; raises if it is missing (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise HtsvdError(f"{path} is missing: build it with `python -m paper_2508_10307_gb300.build`")
    lib = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    P = ctypes.POINTER(CParams)
    lib.htsvd_denoise.argtypes = [vp, i32, i32, i32, dbl, P, vp, vp, vp]
    lib.htsvd_denoise_f32.argtypes = [vp, i32, i32, i32, dbl, P, vp, vp, vp, vp]
    lib.htsvd_estimate_sigma.argtypes = [vp, i32, i32, i32, P, ctypes.POINTER(ctypes.c_double), vp]
    lib.htsvd_denoise_batch.argtypes = [ctypes.POINTER(CImage), i32, P, vp]
    lib.htsvd_denoise_vjp.argtypes = [vp, i32, i32, i32, dbl, P, vp, vp, vp, vp, vp, vp, vp]
    lib.htsvd_denoise_noalloc.argtypes = [vp, i32, i32, i32, dbl, P, vp, vp]
    lib.htsvd_denoise_cube.argtypes = [vp, i32, i32, i32, dbl, P, vp, vp, vp]
    lib.htsvd_denoise_adaptive.argtypes = [vp, i32, i32, i32, i32, i32, P, vp, ctypes.POINTER(ctypes.c_double), vp]
    lib.htsvd_denoise_video.argtypes = [vp, i32, i32, i32, i32, i32, dbl, P, vp, vp, ctypes.POINTER(ctypes.c_double),
                                        vp]
    lib.htsvd_denoise_tau_sweep.argtypes = [vp, i32, i32, i32, dbl, ctypes.POINTER(ctypes.c_double), i32, P, vp,
                                            ctypes.POINTER(ctypes.c_double), vp]
    lib.htsvd_sure.argtypes = [vp, i32, i32, i32, dbl, ctypes.POINTER(ctypes.c_double), i32, vp, dbl, P,
                               ctypes.POINTER(ctypes.c_double), vp]
    lib.htsvd_sure_weights.argtypes = [vp, i32, i32, i32, dbl, vp, vp, dbl, P, ctypes.POINTER(ctypes.c_double), vp, vp]
    lib.htsvd_tune_weights.argtypes = [vp, i32, i32, i32, dbl, vp, dbl, i32, dbl, P, vp,
                                       ctypes.POINTER(ctypes.c_double), vp]
    lib.htsvd_denoise_volume.argtypes = [vp, i32, i32, i32, dbl, P, vp, vp, vp]
    lib.htsvd_denoise_volume_adaptive.argtypes = [vp, i32, i32, i32, i32, i32, i32, P, vp,
                                                  ctypes.POINTER(ctypes.c_double), vp]
    lib.htsvd_project_patches.argtypes = [vp, i32, i32, i32, vp, ctypes.c_int64, vp, vp, vp, vp]
    lib.htsvd_internal_project_simt.argtypes = [vp, i32, i32, i32, vp, ctypes.c_int64, vp, vp, vp]
    lib.htsvd_internal_volume_bases.argtypes = [vp, vp]
    lib.htsvd_internal_volume_bases.restype = ctypes.c_double
    lib.htsvd_internal_alu_probe.argtypes = [i32, i32]
    lib.htsvd_internal_alu_probe.restype = ctypes.c_double
    lib.htsvd_internal_filter_tile.argtypes = [i32, i32, i32, P]
    lib.htsvd_internal_filter_tile.restype = i32
    lib.htsvd_internal_noalloc_bytes.argtypes = [i32, i32, i32, P]
    lib.htsvd_internal_noalloc_bytes.restype = ctypes.c_int64
    lib.htsvd_num_groups.argtypes = [i32, i32, P]
    lib.htsvd_num_groups.restype = ctypes.c_int64
    lib.htsvd_status_string.argtypes = [ctypes.c_int]
    lib.htsvd_status_string.restype = ctypes.c_char_p
    lib.htsvd_release_workspace.argtypes = []
    lib.htsvd_profile_enable.argtypes = [i32]
    lib.htsvd_profile_enable.restype = ctypes.c_int
    lib.htsvd_profile_collect.argtypes = [i32, ctypes.c_char_p, i32, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_double)]
    lib.htsvd_profile_collect.restype = i32
    for name in ["htsvd_denoise", "htsvd_denoise_f32", "htsvd_estimate_sigma", "htsvd_denoise_batch",
                 "htsvd_denoise_vjp", "htsvd_release_workspace", "htsvd_denoise_noalloc", "htsvd_denoise_adaptive",
                 "htsvd_denoise_video", "htsvd_denoise_tau_sweep", "htsvd_sure", "htsvd_denoise_cube",
                 "htsvd_sure_weights", "htsvd_tune_weights", "htsvd_project_patches",
                 "htsvd_internal_project_simt", "htsvd_denoise_volume", "htsvd_denoise_volume_adaptive"]:
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def check(status: int, what: str) -> None:
    if status != HTSVD_OK:
        msg = _lib.htsvd_status_string(status).decode() if _lib is not None else ""
        cls = DegenerateBasisError if status == HTSVD_ERR_DEGENERATE_BASIS else HtsvdError
        raise cls(f"{what} failed: {STATUS_NAMES.get(status, status)} ({msg})")


def profile_enable(on: bool) -> None:
    check(load().htsvd_profile_enable(1 if on else 0), "htsvd_profile_enable")


def profile_collect(max_kernels: int = 32) -> dict:
    """{kernel name: (launches, total device ms)} since the last collect."""
    lib = load()
    nl = 48
    names = ctypes.create_string_buffer(max_kernels * nl)
    cnt = (ctypes.c_int64 * max_kernels)()
    ms = (ctypes.c_double * max_kernels)()
    n = lib.htsvd_profile_collect(max_kernels, names, nl, cnt, ms)
    if n < 0:
        raise HtsvdError("htsvd_profile_collect failed")
    raw = names.raw
    out = {}
    for i in range(n):
        nm = raw[i * nl:(i + 1) * nl].split(b"\0", 1)[0].decode()
        out[nm] = (int(cnt[i]), float(ms[i]))
    return out

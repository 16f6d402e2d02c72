"""The C-ABI library loads and exports every symbol include/htsvd.h declares (CPU only);
argument errors are reported before any device work."""
import ctypes
import os
import re

import pytest

import paper_2508_10307_gb300 as H
from paper_2508_10307_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(headers=("htsvd.h",)):
    names = set()
    for h in headers:
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(htsvd_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ["htsvd_denoise", "htsvd_denoise_f32", "htsvd_estimate_sigma", "htsvd_denoise_batch",
              "htsvd_denoise_vjp", "htsvd_num_groups", "htsvd_status_string", "htsvd_release_workspace"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    lib = H.load_library()
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    for n in _declared(headers):
        assert hasattr(lib, n), n
    assert set(_lib.EXPORTED) == set(_declared())


def test_num_groups_matches_reference_grid():
    assert H.num_groups(128, 128, dict(stride=3)) == 41 * 41
    assert H.num_groups(512, 512, dict(stride=2)) == 253 * 253
    assert H.num_groups(2160, 3840, dict(stride=3)) == 719 * 1279
    assert H.num_groups(7, 100, None) == -1


def test_status_strings():
    lib = H.load_library()
    assert lib.htsvd_status_string(0) == b"ok"
    assert lib.htsvd_status_string(1) == b"invalid argument"
    assert b"degenerate" in lib.htsvd_status_string(6)
    assert _lib.STATUS_NAMES[6] == "DEGENERATE_BASIS"


def test_params_struct_matches_the_header():
    # the ctypes mirror lists the header's fields in order (a mismatch would shift every later field)
    src = open(os.path.join(ROOT, "include", "htsvd.h")).read()
    body = re.sub(r"/\*.*?\*/", "", src[src.index("typedef struct htsvd_params {"):src.index("} htsvd_params;")],
                  flags=re.S)
    fields = re.findall(r"\b(\w+)\s*;", body)
    assert fields == [f for f, _ in _lib.CParams._fields_]


def test_noalloc_rejects_bad_arguments_on_the_host():
    lib = H.load_library()
    cp = H.HtsvdParams.of(dict(K=12)).c()
    one = ctypes.c_void_p(1)
    assert lib.htsvd_denoise_noalloc(one, 40, 40, 3, 10.0, ctypes.byref(cp), one, None) == 1
    cp = H.HtsvdParams.of(None).c()
    assert lib.htsvd_denoise_noalloc(one, 40, 40, 3, -1.0, ctypes.byref(cp), one, None) == 1   # sigma must be given
    assert lib.htsvd_denoise_noalloc(one, 40, 40, 2, 10.0, ctypes.byref(cp), one, None) == 1
    assert lib.htsvd_denoise_noalloc(None, 40, 40, 3, 10.0, ctypes.byref(cp), one, None) == 1
    assert lib.htsvd_internal_noalloc_bytes(40, 40, 2, ctypes.byref(cp)) == -1


def _call_denoise(H_, W_, C, params, ptr=1):
    lib = H.load_library()
    cp = H.HtsvdParams.of(params).c()
    return lib.htsvd_denoise(ctypes.c_void_p(ptr), H_, W_, C, 10.0, ctypes.byref(cp), ctypes.c_void_p(ptr), None,
                             None)


@pytest.mark.parametrize("shape,params,code", [
    ((7, 40, 3), dict(), 1),                   # smaller than a patch
    ((40, 40, 2), dict(), 1),                  # C not 1 or 3
    ((40, 40, 3), dict(K=12), 1),              # K not a power of two
    ((40, 40, 3), dict(ps=4), 2),              # only ps = 8 is built
    ((40, 40, 3), dict(K=64), 2),              # K > 32 not built
    ((40, 40, 3), dict(window=65), 2),         # window > 64 not built
    ((9, 9, 1), dict(K=8, window=3), 1),       # fewer than K candidates in the window
    ((40, 40, 3), dict(tile=17), 1),           # filter tile edge out of range
    ((40, 40, 3), dict(tile=-1), 1),
])
def test_invalid_arguments_are_rejected_on_the_host(shape, params, code):
    assert _call_denoise(*shape, params) == code


def test_null_pointers_rejected():
    assert _call_denoise(40, 40, 3, dict(), ptr=0) == 1


def test_adaptive_rejects_bad_subimage_sizes_on_the_host():
    lib = H.load_library()
    cp = H.HtsvdParams().c()
    for sub_h, sub_w in ((0, 16), (16, 0), (-3, 16)):
        assert lib.htsvd_denoise_adaptive(ctypes.c_void_p(1), 64, 64, 3, sub_h, sub_w, ctypes.byref(cp),
                                          ctypes.c_void_p(1), None, None) == 1
    assert lib.htsvd_denoise_adaptive(None, 64, 64, 3, 32, 32, ctypes.byref(cp), ctypes.c_void_p(1), None,
                                      None) == 1


@pytest.mark.parametrize("n,sub", [(512, 256), (100, 30), (50, 64), (129, 8), (2160, 256)])
def test_subimage_bounds_match_the_oracle_reading(n, sub):
    from oracle import htsvd_oracle as O
    assert H.subimage_bounds(n, sub) == O.subimage_bounds(n, sub)


def test_video_rejects_bad_arguments_on_the_host():
    lib = H.load_library()
    cp = H.HtsvdParams().c()
    dp = ctypes.c_void_p(1)
    call = lambda vid, F, T: lib.htsvd_denoise_video(vid, F, 64, 64, 3, T, 10.0, ctypes.byref(cp), dp, None, None,
                                                     None)
    assert call(dp, 0, 1) == 1                 # no frames
    assert call(dp, 3, -1) == 1                # negative temporal radius
    assert call(None, 3, 1) == 1               # null clip
    assert lib.htsvd_denoise_video(dp, 3, 64, 64, 2, 1, 10.0, ctypes.byref(cp), dp, None, None, None) == 1


def test_tau_sweep_rejects_bad_arguments_on_the_host():
    lib = H.load_library()
    dp = ctypes.c_void_p(1)
    ok = (ctypes.c_double * 2)(1.0, 2.0)
    bad = (ctypes.c_double * 2)(1.0, -2.0)

    def call(mults, n, params=None):
        cp = H.HtsvdParams.of(params).c()
        return lib.htsvd_denoise_tau_sweep(dp, 64, 64, 3, 10.0, mults, n, ctypes.byref(cp), dp, None, None)

    assert call(ok, 0) == 1                    # no thresholds
    assert call(bad, 2) == 1                   # negative multiplier
    assert call(None, 2) == 1                  # null list
    assert call(ok, 2, dict(K=4)) == 2         # cached coefficients need K >= 8


def test_sure_rejects_bad_arguments_on_the_host():
    lib = H.load_library()
    dp = ctypes.c_void_p(1)
    cp = H.HtsvdParams().c()
    res = (ctypes.c_double * 2)()
    ok = (ctypes.c_double * 2)(1.0, 2.0)
    zero = (ctypes.c_double * 2)(1.0, 0.0)
    call = lambda sigma, m, n, probe=dp, eps=1.0: lib.htsvd_sure(dp, 64, 64, 3, sigma, m, n, probe, eps,
                                                                  ctypes.byref(cp), res, None)
    assert call(10.0, ok, 0) == 1              # no thresholds
    assert call(10.0, ok, 2, eps=-1.0) == 1    # negative step
    assert call(10.0, ok, 2, eps=1e300) == 1   # step not finite in float32
    assert call(10.0, ok, 2, eps=1e-60) == 1   # step vanishing in float32
    assert call(0.0, ok, 2) == 1               # sigma must be positive
    assert call(10.0, zero, 2) == 1            # multipliers must be positive
    assert call(10.0, ok, 2, None) == 1        # no probe



def test_binding_checks_buffers_before_they_reach_the_library():
    """The C ABI takes bare pointers; the binding checks shape, dtype, layout and device of every
    buffer the kernels index, so a wrong buffer raises instead of being read out of bounds."""
    torch = pytest.importorskip("torch")
    from paper_2508_10307_gb300 import _need
    t = torch.zeros((4, 5, 3), dtype=torch.float32)
    with pytest.raises(ValueError, match="probe: expected shape"):
        _need(t, "probe", (4, 5, 1), torch.float32)
    with pytest.raises(TypeError, match="w: expected"):
        _need(t, "w", (4, 5, 3), torch.int32)
    with pytest.raises(ValueError, match="contiguous"):
        _need(t.transpose(0, 1), "out", (5, 4, 3), torch.float32)
    with pytest.raises(ValueError, match="CUDA"):
        _need(t, "grad_out", (4, 5, 3), torch.float32)     # a host tensor never reaches the library


def test_volume_adaptive_rejects_bad_arguments_on_the_host():
    lib = H.load_library()
    cp = H.HtsvdParams.of(None).c()
    one = ctypes.c_void_p(1)
    sig = (ctypes.c_double * 8)()
    f = lib.htsvd_denoise_volume_adaptive
    assert f(None, 32, 32, 32, 16, 16, 16, ctypes.byref(cp), one, sig, None) == 1          # no input
    assert f(one, 32, 32, 32, 16, 16, 16, ctypes.byref(cp), None, sig, None) == 1          # no output
    assert f(one, 32, 32, 32, 0, 16, 16, ctypes.byref(cp), one, sig, None) == 1            # part size 0
    assert f(one, 0, 32, 32, 16, 16, 16, ctypes.byref(cp), one, sig, None) == 1            # empty volume
    assert f(one, 2048, 1024, 1024, 512, 512, 512, ctypes.byref(cp), one, sig, None) == 2  # 2^31 voxels
    # every part is checked before any device work (no GPU is touched here)
    vp = H.HtsvdParams.of(dict(H.VOLUME_DEFAULTS)).c()
    assert f(one, 16, 16, 16, 2, 16, 16, ctypes.byref(vp), one, sig, None) == 1            # parts 2 deep
    assert f(one, 16, 16, 16, 16, 16, 3, ctypes.byref(vp), one, sig, None) == 1            # parts 3 wide
    small = H.HtsvdParams.of(dict(H.VOLUME_DEFAULTS, window=1, K=4)).c()
    assert f(one, 16, 16, 16, 8, 8, 8, ctypes.byref(small), one, sig, None) == 1           # 1 cube per window < K
    for bad in (dict(K=12), dict(window=9), dict(match_mode="gcp")):
        c = H.HtsvdParams.of(dict(H.VOLUME_DEFAULTS, **bad)).c()
        assert f(one, 16, 16, 16, 8, 8, 8, ctypes.byref(c), one, sig, None) == 1
    c = H.HtsvdParams.of(dict(H.VOLUME_DEFAULTS, ps=8)).c()
    assert f(one, 16, 16, 16, 8, 8, 8, ctypes.byref(c), one, sig, None) == 2


def test_volume_rejects_bad_arguments_on_the_host():
    lib = H.load_library()
    one, four = ctypes.c_void_p(1), ctypes.c_void_p(4)
    f = lambda vol, D, Hh, Wd, sigma, prm, out=four: lib.htsvd_denoise_volume(
        vol, D, Hh, Wd, sigma, ctypes.byref(H.HtsvdParams.of(dict(H.VOLUME_DEFAULTS, **prm)).c()), out, None, None)
    assert f(None, 16, 16, 16, 10.0, {}) == 1                  # no volume
    assert f(four, 16, 16, 16, 10.0, {}, None) == 1            # no output
    assert f(one, 16, 16, 16, 10.0, {}) == 1                   # volume not 4-byte aligned
    assert f(four, 16, 16, 16, float("nan"), {}) == 1          # sigma not a number
    assert f(four, 16, 16, 16, float("inf"), {}) == 1
    assert f(four, 3, 16, 16, 10.0, {}) == 1                   # thinner than a cube
    assert f(four, 16, 16, 16, 10.0, dict(ps=8)) == 2          # only 4 x 4 x 4 cubes are built
    assert f(four, 16, 16, 16, 10.0, dict(K=12)) == 1          # K not a power of two
    assert f(four, 16, 16, 16, 10.0, dict(K=64)) == 1          # K above 32
    assert f(four, 16, 16, 16, 10.0, dict(window=9)) == 1      # window above 8
    assert f(four, 16, 16, 16, 10.0, dict(match_mode="gcp")) == 1
    assert f(four, 16, 16, 16, 10.0, dict(window=1, K=4)) == 1  # one cube per window, fewer than K
    assert f(four, 2048, 1024, 1024, 10.0, {}) == 2            # 2^31 voxels


def test_cube_rejects_bad_arguments_on_the_host():
    lib = H.load_library()
    one = ctypes.c_void_p(1)
    f = lambda cube, Hh, Wd, N, sigma, prm, out=one: lib.htsvd_denoise_cube(
        cube, Hh, Wd, N, sigma, ctypes.byref(H.HtsvdParams.of(prm).c()), out, None, None)
    assert f(None, 64, 64, 31, 10.0, {}) == 1                  # no cube
    assert f(one, 64, 64, 31, 10.0, {}, None) == 1             # no output
    assert f(one, 64, 64, 31, -1.0, {}) == 1                   # sigma must be given
    assert f(one, 64, 64, 31, float("inf"), {}) == 1
    assert f(one, 64, 64, 1, 10.0, {}) == 1                    # N below 2
    assert f(one, 64, 64, 65, 10.0, {}) == 1                   # N above 64
    assert f(one, 64, 64, 31, 10.0, dict(match_mode="gcp")) == 1
    assert f(one, 7, 64, 31, 10.0, {}) == 1                    # smaller than a patch
    assert f(one, 9, 9, 31, 10.0, dict(K=8, window=3)) == 1    # fewer than K candidates
    assert f(one, 8192, 8192, 64, 10.0, {}) == 2               # H W N reaches 2^31


def test_projection_rejects_bad_arguments_on_the_host():
    lib = H.load_library()
    four, sixteen = ctypes.c_void_p(4), ctypes.c_void_p(16)
    f = lambda img, Hh, Wd, C, pos, n, basis=sixteen, coef=sixteen: lib.htsvd_project_patches(
        img, Hh, Wd, C, pos, n, basis, coef, None, None)
    assert f(four, 24, 24, 2, four, 4) == 1                    # C not 1 or 3
    assert f(four, 7, 24, 3, four, 4) == 1                     # smaller than a patch
    assert f(four, 24, 24, 3, four, -1) == 1                   # negative count
    assert f(four, 24, 24, 3, four, 0) == 0                    # nothing to do: no device work
    assert f(None, 24, 24, 3, four, 4) == 1                    # no image
    assert f(four, 24, 24, 3, four, 4, None) == 1              # no bases
    assert f(four, 24, 24, 3, None, 4) == 1                    # no positions, and not every corner
    assert f(ctypes.c_void_p(5), 24, 24, 3, four, 4) == 1      # image not 4-byte aligned
    assert f(four, 24, 24, 3, four, 4, coef=ctypes.c_void_p(20)) == 1    # coefficients not 16-byte aligned


def test_estimate_sigma_f32_and_vjp_refuse_bad_arguments_on_the_host():
    lib = H.load_library()
    one = ctypes.c_void_p(1)
    cp = H.HtsvdParams().c()
    s = ctypes.c_double()
    assert lib.htsvd_estimate_sigma(None, 64, 64, 3, ctypes.byref(cp), ctypes.byref(s), None) == 1
    assert lib.htsvd_estimate_sigma(one, 64, 64, 3, ctypes.byref(cp), None, None) == 1
    assert lib.htsvd_estimate_sigma(one, 64, 64, 2, ctypes.byref(cp), ctypes.byref(s), None) == 1
    assert lib.htsvd_estimate_sigma(one, 7, 64, 3, ctypes.byref(cp), ctypes.byref(s), None) == 1
    f32 = lambda x, Hh, C, prm=None, out=one: lib.htsvd_denoise_f32(
        x, Hh, 64, C, 10.0, ctypes.byref(H.HtsvdParams.of(prm).c()), None, out, None, None)
    assert f32(None, 64, 3) == 1
    assert f32(one, 64, 3, out=None) == 1
    assert f32(one, 64, 2) == 1
    assert f32(one, 64, 3, dict(K=12)) == 1
    assert f32(one, 64, 3, dict(ps=4)) == 2
    vjp = lambda sigma, x=one, idx=one, out=one, g=one, gx=one, C=3: lib.htsvd_denoise_vjp(
        x, 64, 64, C, sigma, ctypes.byref(cp), idx, None, out, g, gx, None, None)
    assert vjp(10.0, x=None) == 1
    assert vjp(10.0, idx=None) == 1
    assert vjp(10.0, out=None) == 1
    assert vjp(10.0, g=None) == 1
    assert vjp(10.0, gx=None) == 1
    assert vjp(-1.0) == 1                       # the forward's sigma must be passed
    assert vjp(10.0, C=2) == 1


def test_parameters_refuse_unknown_names():
    """A misspelt parameter raises instead of silently taking its default."""
    with pytest.raises(ValueError, match="unknown parameters"):
        H.HtsvdParams.of(dict(windw=5))
    assert H.HtsvdParams.of(dict(window=5, K=8, tile=4, strict_basis=True)).window == 5
    assert H.HtsvdParams.of(dict(H.VOLUME_DEFAULTS)).ps == 4
    for bad in (dict(match_mode="nonsense"), dict(agg_mode="median")):
        with pytest.raises(ValueError, match="match_mode must be one of"):
            H.HtsvdParams.of(bad).c()

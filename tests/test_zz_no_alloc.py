"""The allocation-free entry point (htsvd_denoise_noalloc) against htsvd_denoise.

Callers that cannot let a library allocate device memory (their own pool owns it, or
cudaFree's device-wide synchronisation is not acceptable in their loop) use the
allocation-free call, which keeps its temporaries in one fixed array in device memory.
It must give the same image as the ordinary entry point, call after call, although the
array keeps whatever the previous call left in it. This file is collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402
from paper_2508_10307_gb300 import synth  # noqa: E402

PIX_TOL = 1e-3


def _noalloc(x, sigma, prm):
    lib = H.load_library()
    Hh, Ww, C = x.shape
    out = torch.empty((Hh, Ww, C), dtype=torch.float32, device=x.device)
    cp = H.HtsvdParams.of(prm).c()
    st = lib.htsvd_denoise_noalloc(ctypes.c_void_p(x.data_ptr()), Hh, Ww, C, float(sigma), ctypes.byref(cp),
                                   ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


@pytest.mark.parametrize("C", [3, 1])
def test_noalloc_matches_denoise_on_two_calls_in_a_row(C):
    prm = dict(ps=8, stride=3, window=21, K=16 if C == 1 else 32)
    imgs = []
    for seed, (h, w, sig) in ((31, (96, 120, 20.0)), (32, (80, 64, 35.0))):
        clean = synth.clean_image(h, w, C, seed)
        imgs.append((torch.from_numpy(synth.add_gaussian(clean, sig, seed)).cuda(), sig))
    for x, sig in imgs:                       # two calls in a row, different sizes and noise levels
        st, out = _noalloc(x, sig, prm)
        assert st == 0
        ref = H.denoise(x, sig, prm)
        torch.cuda.synchronize()
        err = float((out - ref).abs().max())
        assert err <= PIX_TOL, err


def test_noalloc_rejects_images_beyond_its_array():
    x = torch.zeros((1024, 1024, 3), dtype=torch.uint8, device="cuda")
    st, _ = _noalloc(x, 10.0, dict(ps=8, stride=3, window=18, K=32))
    assert st == 1                            # HTSVD_ERR_INVALID_ARG, nothing launched

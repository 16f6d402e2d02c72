"""The allocation-free entry point (htsvd_denoise_noalloc) against htsvd_denoise and the FP64 oracle.

Callers that cannot let a library allocate device memory (their own pool owns it, or
cudaFree's device-wide synchronisation is not acceptable in their loop) use the
allocation-free call, which keeps its temporaries in one fixed array in device memory.
It must give the image of the ordinary entry point (bit for bit where it takes the same
tiles), call after call, although the array keeps whatever the previous call left in it,
and it must not allocate: free device memory and the torch allocator's counters stay put
across its calls. This file is collected last.
"""
import ctypes
import os
import re

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402
from oracle import htsvd_oracle as O  # noqa: E402
from paper_2508_10307_gb300 import synth  # noqa: E402

PIX_TOL = 1e-3
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_constant(name):
    src = open(os.path.join(ROOT, "include", "htsvd.h")).read()
    return int(re.search(r"#define\s+" + name + r"\s+(\d+)", src).group(1))


def _noalloc(x, sigma, prm, out=None, cp=None):
    lib = H.load_library()
    Hh, Ww, C = x.shape
    if out is None:
        out = torch.empty((Hh, Ww, C), dtype=torch.float32, device=x.device)
    if cp is None:
        cp = H.HtsvdParams.of(prm).c()
    st = lib.htsvd_denoise_noalloc(ctypes.c_void_p(x.data_ptr()), Hh, Ww, C, float(sigma), ctypes.byref(cp),
                                   ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out


def _need_bytes(h, w, C, prm):
    cp = H.HtsvdParams.of(prm).c()
    return int(H.load_library().htsvd_internal_noalloc_bytes(h, w, C, ctypes.byref(cp)))


CASES = {3: [(31, 96, 120, 20.0), (32, 80, 64, 35.0)], 1: [(33, 72, 88, 25.0), (34, 64, 56, 15.0)]}


@pytest.mark.parametrize("C", [3, 1])
def test_noalloc_matches_denoise_and_oracle_on_two_calls_in_a_row(C):
    prm = dict(ps=8, stride=3, window=21, K=16 if C == 1 else 32)
    for seed, h, w, sig in CASES[C]:          # two calls in a row, different sizes and noise levels
        clean = synth.clean_image(h, w, C, seed)
        noisy = synth.add_gaussian(clean, sig, seed)
        x = torch.from_numpy(noisy).cuda()
        st, out = _noalloc(x, sig, prm)
        assert st == 0
        ref = H.denoise(x, sig, prm)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)          # same kernels, same tiles: the same bits
        r = O.denoise(noisy, sig, prm)
        err = float(np.abs(out.cpu().numpy() - r.out).max())
        assert err <= PIX_TOL, err


def test_noalloc_allocates_no_device_memory():
    lib = H.load_library()
    prm = dict(ps=8, stride=3, window=21, K=32)
    imgs, outs = [], []
    for seed, h, w, sig in CASES[3]:
        x = torch.from_numpy(synth.add_gaussian(synth.clean_image(h, w, 3, seed), sig, seed)).cuda()
        H.denoise(x, sig, prm)                 # loads every kernel the call launches
        imgs.append((x, sig))
        outs.append(torch.empty((h, w, 3), dtype=torch.float32, device="cuda"))
    _noalloc(imgs[0][0], imgs[0][1], prm, outs[0])  # resolves the scratch array's address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        for (x, sig), o in zip(imgs, outs):
            st, _ = _noalloc(x, sig, prm, o)
            assert st == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == stats0
    assert lib.htsvd_release_workspace() == 0


def test_noalloc_honours_the_optional_outputs():
    prm = dict(ps=8, stride=3, window=15, K=16, agg_mode="sparsity", tile=3)
    noisy = synth.add_gaussian(synth.clean_image(56, 64, 3, 35), 20.0, 35)
    x = torch.from_numpy(noisy).cuda()
    ref, info = H.denoise(x, 20.0, prm, return_info=True, masks=True, weights=True, basis=True, coeffs=True)
    n = info["weights"].shape[0]
    p = H.HtsvdParams.of(prm)
    cp = p.c()
    masks = torch.empty_like(info["masks"])
    weights = torch.empty_like(info["weights"])
    basis = torch.empty_like(info["basis"])
    coeffs = torch.empty_like(info["coeffs"])
    sig_out, gap_out = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
    cp.d_mask_out, cp.d_weights_out = masks.data_ptr(), weights.data_ptr()
    cp.d_basis_out, cp.d_coef_out = basis.data_ptr(), coeffs.data_ptr()
    cp.h_sigma_out, cp.h_basis_gap_out = ctypes.pointer(sig_out), ctypes.pointer(gap_out)
    st, out = _noalloc(x, 20.0, prm, cp=cp)
    torch.cuda.synchronize()
    assert st == 0 and n > 0
    assert torch.equal(out, ref)
    assert torch.equal(masks, info["masks"]) and torch.equal(weights, info["weights"])
    assert torch.equal(basis, info["basis"]) and torch.equal(coeffs, info["coeffs"])
    assert sig_out.value == 20.0
    r = O.denoise(noisy, 20.0, {k: v for k, v in prm.items() if k != "tile"})
    assert abs(gap_out.value - r.extra["basis_gap"]) <= 1e-6 * r.extra["basis_gap"]


def test_noalloc_strict_basis_rejects_a_constant_image():
    x = torch.full((40, 48, 3), 77, dtype=torch.uint8, device="cuda")
    st, _ = _noalloc(x, 25.0, dict(ps=8, stride=3, window=9, K=8, strict_basis=True))
    assert st == 6                            # HTSVD_ERR_DEGENERATE_BASIS


def test_noalloc_size_limits_match_the_header():
    if torch.cuda.get_device_properties(0).multi_processor_count != 152:
        pytest.skip("the header states the limits for a 152-SM GB300 (the filter tiles follow the SM count)")
    prm = dict(ps=8, stride=3, window=18, K=32)
    cap = 32 << 20                            # HTSVD_NOALLOC_SCRATCH_BYTES
    same, top = _header_constant("HTSVD_NOALLOC_SAME_TILES_RGB_EDGE"), _header_constant("HTSVD_NOALLOC_MAX_RGB_EDGE")
    assert _need_bytes(top, top, 3, prm) <= cap < _need_bytes(top + 1, top + 1, 3, prm)
    for e, exact in ((same, True), (top, False)):
        noisy = synth.add_gaussian(synth.clean_image(e, e, 3, 36), 25.0, 36)
        x = torch.from_numpy(noisy).cuda()
        st, out = _noalloc(x, 25.0, prm)
        ref = H.denoise(x, 25.0, prm)
        torch.cuda.synchronize()
        assert st == 0
        if exact:
            assert torch.equal(out, ref)
        else:
            assert float((out - ref).abs().max()) <= PIX_TOL
    x = torch.zeros((top + 1, top + 1, 3), dtype=torch.uint8, device="cuda")
    st, _ = _noalloc(x, 25.0, prm)
    assert st == 1                            # HTSVD_ERR_INVALID_ARG, nothing launched

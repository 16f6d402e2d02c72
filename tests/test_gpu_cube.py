"""Hyperspectral cubes (Alg. 1 with C = N bands, reading R18) on the GPU against the FP64 oracle.

Bar as for images: match indices bit-exact, threshold masks bit-exact (except coefficients the
oracle itself finds within 1e-9 of tau), pixels within 1e-3, PSNR within 0.01 dB, bases within 1e-9.
"""
import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth
from tests._common import PIX_TOL, PSNR_TOL, max_abs, pack_masks, psnr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402


def _case(Hh, Ww, N, sigma, seed):
    clean = synth.clean_cube(Hh, Ww, N, seed)
    return synth.quantize(clean), synth.add_gaussian(clean, sigma, seed)


@pytest.mark.parametrize("shape,prm,sigma", [
    ((64, 64, 31), dict(ps=8, stride=3, window=15, K=16), 12.0),     # the 31-band cubes of the ICVL size class
    ((48, 56, 34), dict(ps=8, stride=3, window=11, K=8), 15.0),      # 34 bands (Real-HSI): a real middle slice
    ((40, 45, 5), dict(ps=8, stride=2, window=9, K=4, agg_mode="sparsity"), 20.0),
    ((56, 60, 34), dict(ps=8, stride=3, window=18, K=32), 12.0),     # the benchmarked cube geometry
    ((30, 33, 7), dict(ps=8, stride=2, window=9, K=2), 15.0),
])
def test_cube_parity(shape, prm, sigma):
    Hh, Ww, N = shape
    clean, noisy = _case(Hh, Ww, N, sigma, 60 + N)
    r = O.denoise(noisy, sigma, prm, keep_masks=True)
    x = torch.from_numpy(noisy).cuda()
    out, info = H.denoise_cube(x, sigma, prm, return_info=True, masks=True, weights=True, basis=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(info["idx"].cpu().numpy().astype(np.int64), r.idx)
    b = info["basis"].cpu().numpy()
    z = b[..., 0] + 1j * b[..., 1]
    # slices of high band frequency carry little energy, so eigen-gaps can be small: an eigenvector
    # moves by about (rounding of the scatter matrix) / (relative gap), hence the looser bound there
    tol = max(1e-9, 1e-13 / r.extra["basis_gap"])
    assert np.abs(z[0] - r.U).max() < tol and np.abs(z[1] - r.V).max() < tol
    om = pack_masks(r.masks)
    gm = info["masks"].cpu().numpy().view(np.uint32)[:, :om.shape[1]]
    amb = {(int(g), int(i)) for g, i in r.ambiguous}
    bad = 0
    for g, wd in zip(*np.nonzero(om != gm)):
        d = int(om[g, wd]) ^ int(gm[g, wd])
        bad += sum(1 for bit in range(32) if (d >> bit) & 1 and (int(g), int(wd) * 32 + bit) not in amb)
    assert bad == 0, f"{bad} mask bits differ"
    o = out.cpu().numpy()
    assert max_abs(o, r.out) <= PIX_TOL
    assert abs(psnr(o, clean) - psnr(r.out, clean)) <= PSNR_TOL
    if prm.get("agg_mode") == "sparsity":
        np.testing.assert_array_equal(np.rint(1.0 / info["weights"].cpu().numpy()), np.rint(1.0 / r.weights))


def test_cube_zero_threshold_is_the_identity_and_rgb_modes_are_refused():
    _, noisy = _case(32, 40, 7, 12.0, 71)
    x = torch.from_numpy(noisy).cuda()
    out = H.denoise_cube(x, 12.0, dict(ps=8, stride=3, window=9, K=8, tau_mult=1e-12))
    assert max_abs(out.cpu().numpy(), noisy) <= 2e-3
    from paper_2508_10307_gb300 import _lib
    for mode in ("gcp", "green"):
        with pytest.raises(_lib.HtsvdError):
            H.denoise_cube(x, 12.0, dict(ps=8, stride=3, window=9, K=8, match_mode=mode))


def test_cube_equal_bands_give_the_gray_result():
    """N equal bands: every band of the cube result equals the gray denoiser's result (pinned on the
    oracle by test_hsi_identical_bands_reduce_to_the_gray_denoiser), here through the two CUDA paths."""
    clean = synth.clean_image(40, 48, 1, 73)
    g = synth.add_gaussian(clean, 12.0, 73)
    prm = dict(ps=8, stride=3, window=9, K=8, tau_mult=2.7)
    gray = H.denoise(torch.from_numpy(g).cuda(), 12.0, prm).cpu().numpy()
    cube = H.denoise_cube(torch.from_numpy(np.repeat(g, 6, axis=2)).cuda(), 12.0, prm).cpu().numpy()
    assert max_abs(cube, np.repeat(gray, 6, axis=2)) <= PIX_TOL


BAND_REL_CUBE = 2.0 ** -19     # guard band of the cube threshold, relative to the slot norm (kBandRelCube)


def test_cube_fp32_coefficient_error_is_well_inside_the_guard_band():
    """Outside the guard band the FP32 coefficients decide keep/drop. The cube filter's band for a Haar
    slot is band * ||slot||_F (the slot's normalised Haar combination of the group's patches, whose
    transform is orthonormal), so the FP32 error of every coefficient against the oracle's FP64
    coefficient must stay well below band * ||slot||_F."""
    clean, noisy = _case(64, 64, 31, 12.0, 91)
    prm = dict(ps=8, stride=3, window=15, K=16)
    r = O.denoise(noisy, 12.0, prm)
    out, info = H.denoise_cube(torch.from_numpy(noisy).cuda(), 12.0, prm, return_info=True, coeffs=True)
    coef = info["coeffs"].cpu().numpy().astype(np.float64)
    p = O.Params.of(prm)
    Hk = O.haar_matrix(p.K)
    G = O.gather_groups(noisy, r.idx, p.ps).astype(np.float64)
    S = O.forward_transform(G, r.U, r.V, Hk)
    n = len(r.idx)
    err = np.abs(coef.reshape(n, p.K, -1) - S.reshape(n, p.K, -1)).max(axis=2)
    slots = np.tensordot(Hk, G, axes=([1], [1])).transpose(1, 0, 2, 3, 4)       # [n, m, i, j, band]
    nrm = np.sqrt((slots.reshape(n, p.K, -1) ** 2).sum(axis=2))
    worst = float((err / np.maximum(nrm, 1e-30)).max())
    print(f"cube FP32 coefficient error: max |S32 - S64| / ||slot||_F = 2^{np.log2(worst):.2f}")
    assert worst <= BAND_REL_CUBE / 4, worst

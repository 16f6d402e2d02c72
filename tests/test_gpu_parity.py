"""GPU path vs the FP64 oracle through the C ABI (needs a GB300 and the built library).

Bar: match indices and threshold masks bit-exact (masks: except coefficients the oracle
itself finds within 1e-9 of tau, expected none); pixels within 1e-3 on the [0, 255]
scale; PSNR within 0.01 dB; basis within 1e-9.
"""
import math

import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth
from tests._common import PIX_TOL, PSNR_TOL, max_abs, oracle_run, pack_masks, psnr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run_gpu(noisy, sigma, prm, **kw):
    out, info = H.denoise(_dev(noisy), sigma, prm, return_info=True, masks=True, weights=True, basis=True, **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy(), {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in info.items()}


def _basis_from_gpu(b):
    z = b[..., 0] + 1j * b[..., 1]            # (2, C, 8, 8)
    return z[0], z[1]


def _compare(noisy, sigma, prm, r, clean=None):
    out, info = _run_gpu(noisy, sigma, prm)
    # grouping
    np.testing.assert_array_equal(info["idx"].astype(np.int64), r.idx)
    # bases
    U, V = _basis_from_gpu(info["basis"])
    assert np.abs(U - r.U).max() < 1e-9 and np.abs(V - r.V).max() < 1e-9
    # masks
    om = pack_masks(r.masks)
    gm = info["masks"].view(np.uint32)[:, :om.shape[1]]
    diff = np.nonzero(om != gm)
    bad = 0
    if diff[0].size:
        amb = {(int(g), int(i)) for g, i in r.ambiguous}
        for g, wd in zip(*diff):
            x = int(om[g, wd]) ^ int(gm[g, wd])
            for b in range(32):
                if (x >> b) & 1 and (int(g), int(wd) * 32 + b) not in amb:
                    bad += 1
    assert bad == 0, f"{bad} mask bits differ outside the ambiguity band"
    # pixels
    err = max_abs(out, r.out)
    assert err <= PIX_TOL, f"max abs pixel error {err}"
    if clean is not None:
        assert abs(psnr(out, clean) - psnr(r.out, clean)) <= PSNR_TOL
    return out, info


def test_gray128_parity():
    clean, noisy, sigma, prm, r = oracle_run("gray128")
    out, info = _compare(noisy, sigma, prm, r, clean)
    assert psnr(out, clean) > psnr(noisy, clean) + 6


def test_rgb512_parity_with_estimated_sigma():
    clean, noisy, sigma, prm, r = oracle_run("rgb512")
    out, info = _compare(noisy, None, prm, r, clean)
    assert abs(info["sigma"] - sigma) <= 1e-9 * sigma
    assert psnr(out, clean) > psnr(noisy, clean) + 6


@pytest.mark.parametrize("shape,prm,sigma", [
    ((37, 45, 3), dict(ps=8, stride=3, window=11, K=8), 20.0),          # ragged tail in both axes
    ((50, 29, 1), dict(ps=8, stride=4, window=9, K=16), 15.0),
    ((20, 26, 3), dict(ps=8, stride=2, window=31, K=32), 30.0),         # image smaller than the window
    ((64, 70, 3), dict(ps=8, stride=5, window=17, K=4, match_mode="full"), 25.0),
    ((64, 48, 3), dict(ps=8, stride=3, window=15, K=16, agg_mode="sparsity"), 25.0),
    ((33, 40, 3), dict(ps=8, stride=1, window=7, K=2), 10.0),
    ((61, 75, 3), dict(ps=8, stride=3, window=15, K=16, tile=7), 20.0),  # forced filter tiles (ragged)
    # windows wider than 32: 9..16 candidate quads per lane row, 2 or 3 strips per warp
    ((72, 88, 3), dict(ps=8, stride=5, window=45, K=16), 20.0),
    ((80, 80, 1), dict(ps=8, stride=6, window=64, K=32), 25.0),                # the largest window built
    ((64, 72, 3), dict(ps=8, stride=5, window=37, K=8, match_mode="full"), 20.0),
    ((47, 52, 1), dict(ps=8, stride=2, window=13, K=8, tile=3), 20.0),
])
def test_small_images_parity(shape, prm, sigma):
    Hh, Ww, C = shape
    clean = synth.clean_image(Hh, Ww, C, 77)
    noisy = synth.add_gaussian(clean, sigma, 77)
    # the filter tile is a launch choice of the GPU path: the oracle has no such parameter
    r = O.denoise(noisy, sigma, {k: v for k, v in prm.items() if k != "tile"}, keep_masks=True)
    out, info = _compare(noisy, sigma, prm, r)
    if prm.get("agg_mode") == "sparsity":
        # w_g = 1 / max(1, #kept): the kept counts are integers and must agree exactly
        np.testing.assert_array_equal(np.rint(1.0 / info["weights"]), np.rint(1.0 / r.weights))


def test_tied_distances_lowest_index():
    tile = np.random.default_rng(3).integers(0, 256, size=(8, 8, 3), dtype=np.uint8)
    noisy = np.ascontiguousarray(np.tile(tile, (6, 6, 1)))
    prm = dict(ps=8, stride=4, window=21, K=16)
    r = O.denoise(noisy, 20.0, prm, keep_masks=True)
    _compare(noisy, 20.0, prm, r)


def test_zero_threshold_is_identity_on_gpu():
    clean, noisy, sigma, prm = synth.workload_rgb512()
    out = H.denoise(_dev(noisy), 0.0, prm).cpu().numpy()
    assert max_abs(out, noisy) <= 2e-3


def test_huge_threshold_gives_zero():
    _, noisy, _, prm = synth.workload_gray128()
    out = H.denoise(_dev(noisy), 1e30, prm).cpu().numpy()
    assert np.abs(out).max() == 0.0


def test_constant_image():
    img = np.full((40, 40, 3), 91, dtype=np.uint8)
    out = H.denoise(_dev(img), 25.0, dict(ps=8, stride=3, window=9, K=8)).cpu().numpy()
    assert max_abs(out, 91.0) <= PIX_TOL


def test_deterministic_bitwise():
    _, noisy, sigma, prm = synth.workload_gray128()
    a = H.denoise(_dev(noisy), sigma, prm).cpu().numpy()
    b = H.denoise(_dev(noisy), sigma, prm).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("shape,prm", [
    ((96, 80, 3), dict(ps=8, stride=3, window=15, K=16)),
    ((70, 90, 1), dict(ps=8, stride=2, window=13, K=8)),
])
def test_bases_from_the_full_moment_equal_the_direct_ones(shape, prm):
    # with sigma estimated the row/column moments are summed from the full second moment; with
    # sigma given they are read from the image: both are exact integer sums, so the bases agree bitwise
    img = synth.quantize(synth.add_gaussian(synth.clean_image(*shape, seed=77), 20.0, seed=78))
    x = _dev(img)
    _, est = H.denoise(x, None, prm, return_info=True, basis=True)
    _, giv = H.denoise(x, 20.0, prm, return_info=True, basis=True)
    torch.cuda.synchronize()
    assert torch.equal(est["basis"], giv["basis"])


def test_estimate_sigma_matches_oracle():
    clean, noisy, sigma, prm, r = oracle_run("rgb512")
    s = H.estimate_sigma(_dev(noisy), prm)
    assert abs(s - sigma) <= 1e-9 * sigma


def test_estimate_sigma_adaptive_matches_oracle():
    clean = synth.clean_image(160, 192, 3, 5)
    noisy = synth.add_gaussian(clean, 35.0, 5)
    prm = dict(ps=8, stride=3, window=15, K=32, adapt=True)
    s_or, det = O.estimate_sigma(noisy, prm, return_details=True)
    s = H.estimate_sigma(_dev(noisy), prm)
    assert abs(s - s_or) <= 1e-9 * s_or


def test_float_input_matches_oracle():
    clean = synth.clean_image(64, 72, 3, 9)
    x = synth.add_gaussian_float(clean, 25.0, 9)
    prm = dict(ps=8, stride=3, window=15, K=16)
    r = O.denoise(x, 25.0, prm, keep_masks=True)
    out, info = H.denoise_f32(_dev(x), 25.0, prm, return_info=True)
    np.testing.assert_array_equal(info["idx"].cpu().numpy().astype(np.int64), r.idx)
    assert max_abs(out.cpu().numpy(), r.out) <= PIX_TOL


def test_batch_matches_single_calls_and_replays():
    """One persistent launch per phase over uneven images (graph-captured), against single calls;
    the tile shapes may differ (autotuned), so the tile partials add in another order."""
    shapes = [(64, 80), (96, 40), (48, 48), (130, 200)]
    imgs, sig = [], []
    for j, (h, w) in enumerate(shapes):
        c, n = synth.batch_image(j, h, w, 15.0 + 10 * j)
        imgs.append(_dev(n))
        sig.append(15.0 + 10 * j)
    prm = dict(ps=8, stride=3, window=31, K=32)
    outs = H.denoise_batch(imgs, sig, prm)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    outs2 = H.denoise_batch(imgs, sig, prm, outs=outs)          # same batch: graph replay
    torch.cuda.synchronize()
    for t, s, o, f in zip(imgs, sig, outs2, first):
        ref = H.denoise(t, s, prm)
        assert float((ref - o).abs().max()) <= PIX_TOL
        assert torch.equal(o, f)


def test_batch_rejects_mixed_channels():
    a = _dev(np.zeros((32, 32, 3), dtype=np.uint8))
    b = _dev(np.zeros((32, 32, 1), dtype=np.uint8))
    with pytest.raises(RuntimeError):
        H.denoise_batch([a, b], [10.0, 10.0], dict(ps=8, stride=3, window=9, K=8))


@pytest.mark.parametrize("shape,prm,sigma", [
    ((96, 120, 3), dict(ps=8, stride=2, window=15, K=32), 20.0),
    ((80, 64, 1), dict(ps=8, stride=1, window=13, K=16), 35.0),
    ((72, 72, 3), dict(ps=8, stride=3, window=11, K=8), 8.0),
])
def test_sampled_group_ranks_match_oracle(shape, prm, sigma):
    """Eigen-rank of lambda_{K/2} among the circulant eigenvalues of every 8th group per axis
    (Sec. III-D), element by element against the oracle."""
    import ctypes
    import torch
    import paper_2508_10307_gb300 as H
    Hh, Ww, C = shape
    noisy = synth.add_gaussian(synth.clean_image(Hh, Ww, C, 53), sigma, 53)
    _, det = O.estimate_sigma(noisy, dict(prm, adapt=True), return_details=True)
    lib = H.load_library()
    f = lib.htsvd_internal_sampled_ranks
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_int32]
    f.restype = ctypes.c_int32
    cp = H.HtsvdParams.of(prm).c()
    x = torch.from_numpy(noisy).cuda()
    out = np.zeros(4096, np.int32)
    n = f(x.data_ptr(), Hh, Ww, C, ctypes.addressof(cp), out.ctypes.data, out.size)
    assert n == det["ranks"].size
    np.testing.assert_array_equal(out[:n], det["ranks"])


BAND_REL = 2.0 ** -19     # guard band of the threshold decision, relative to ||G||_F (kBandRel in kernels.h)


def _coefficient_errors(key):
    """FP32 coefficients of the GPU path against the oracle's FP64 coefficients on sampled groups:
    (|S32 - S64| [n, K, 64*C], ||G||_F [n], ||G restricted to the Haar support of row m||_F [n, K])."""
    clean, noisy, sigma, prm, r = oracle_run(key)
    out, info = H.denoise(_dev(noisy), sigma, prm, return_info=True, coeffs=True)
    coef = info["coeffs"].cpu().numpy()
    p = O.Params.of(prm)
    Hk = O.haar_matrix(p.K)
    rng = np.random.default_rng(0)
    sample = rng.choice(len(r.idx), size=min(2048, len(r.idx)), replace=False)
    G = O.gather_groups(noisy, r.idx[sample], p.ps).astype(np.float64)
    S = O.forward_transform(G, r.U, r.V, Hk)
    n = len(sample)
    err = np.abs(coef[sample].astype(np.float64) - S).reshape(n, p.K, -1)
    pk = (G.reshape(n, p.K, -1) ** 2).sum(axis=2)              # squared norm per patch (group order)
    supp = (np.abs(Hk) > 0).astype(np.float64)                 # [m, k]: patch k in the support of row m
    return err, np.sqrt(pk.sum(axis=1)), np.sqrt(pk @ supp.T)


@pytest.mark.parametrize("key", ["gray128", "rgb512"])
def test_fp32_coefficient_error_is_well_inside_the_guard_band(key):
    """Outside the guard band the FP32 coefficients decide keep/drop, so their error against the
    oracle's FP64 coefficients must stay well below band * ||G||_F, and below band * ||G_m||_F with
    G_m the patches in the Haar support of the coefficient's row."""
    err, nrm, nrm_m = _coefficient_errors(key)
    worst = float((err.max(axis=2) / nrm[:, None]).max())
    worst_m = float((err.max(axis=2) / nrm_m).max())
    assert worst <= BAND_REL / 4, f"max |S32 - S64| / ||G|| = {worst:.3e}"
    assert worst_m <= BAND_REL / 4, f"max |S32 - S64| / ||G_m|| = {worst_m:.3e}"


def test_strict_basis_rejects_a_constant_image_like_the_oracle():
    img = np.full((40, 48, 3), 77, np.uint8)
    prm = dict(ps=8, stride=3, window=9, K=8, strict_basis=True)
    with pytest.raises(O.DegenerateBasis):
        O.denoise(img, 25.0, prm)
    from paper_2508_10307_gb300 import _lib
    with pytest.raises(_lib.DegenerateBasisError):
        H.denoise(_dev(img), 25.0, prm)
    out = H.denoise(_dev(img), 25.0, dict(prm, strict_basis=False)).cpu().numpy()   # default mode runs
    assert max_abs(out, 77.0) <= 1e-3


@pytest.mark.parametrize("key", ["gray128", "rgb512"])
def test_basis_gap_matches_the_oracle(key):
    clean, noisy, sigma, prm, r = oracle_run(key)
    out, info = H.denoise(_dev(noisy), sigma, dict(prm, strict_basis=True), return_info=True, basis_gap=True)
    torch.cuda.synchronize()
    want = r.extra["basis_gap"]
    assert want > 1e-9 and abs(info["basis_gap"] - want) <= 1e-6 * want

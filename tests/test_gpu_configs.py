"""GPU parity at the geometries the benchmarked workloads run (needs a GB300 and the built library).

- a 512 x 768 crop of the 3840 x 2160 Poisson-Gaussian workload (stride 3, window 31, K 32,
  sigma = sqrt(b)) filtered with the tile edge the 4K frame takes;
- the batched form (htsvd_denoise_batch) against the oracle image by image, on uneven images
  (one wider than 1024 px) with sigma across [10, 50];
- the hand-written VJP at the differentiation workload's K 32 / stride 2 / window 31 against the
  FP64 adjoint, and against central differences of the CUDA forward itself at perturbations that
  leave the grouping and the threshold masks unchanged.
Bar: indices and masks bit-exact, pixels within 1e-3, PSNR within 0.01 dB, adjoint within 1e-4.
"""
import ctypes

import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth
from tests._common import PIX_TOL, PSNR_TOL, max_abs, psnr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402
from tests.test_gpu_parity import _compare  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _filter_tile(Hh, Ww, C, prm):
    cp = H.HtsvdParams.of(prm).c()
    return int(H.load_library().htsvd_internal_filter_tile(Hh, Ww, C, ctypes.byref(cp)))


def test_rgb4k_geometry_crop_parity():
    prm = dict(ps=8, stride=3, window=31, K=32)
    clean = np.ascontiguousarray(synth.clean_image(2160, 3840, 3, 1003)[824:1336, 1536:2304])
    noisy = synth.add_poisson_gaussian(clean, 0.01, 25.0 ** 2, 1003)
    tile = _filter_tile(2160, 3840, 3, prm)                  # the tile edge the full frame takes
    assert 1 <= tile <= 16
    r = O.denoise(noisy, 25.0, prm, keep_masks=True)
    _compare(noisy, 25.0, dict(prm, tile=tile), r, synth.quantize(clean))


def test_batch_matches_the_oracle_image_by_image():
    shapes = [(72, 1040), (96, 130), (130, 200), (64, 64), (200, 72), (88, 150)]     # (H, W)
    sigmas = [10.0, 18.0, 26.0, 34.0, 42.0, 50.0]
    prm = dict(ps=8, stride=3, window=31, K=32)
    imgs, cleans, idx = [], [], []
    for j, ((h, w), s) in enumerate(zip(shapes, sigmas)):
        c, n = synth.batch_image(40 + j, h, w, s)
        cleans.append(c)
        imgs.append(n)
        idx.append(torch.empty((H.num_groups(h, w, prm), 32), dtype=torch.int32, device="cuda"))
    outs = H.denoise_batch([_dev(n) for n in imgs], sigmas, prm, idx_outs=idx)
    torch.cuda.synchronize()
    for n, c, s, o, ix in zip(imgs, cleans, sigmas, outs, idx):
        r = O.denoise(n, s, prm)
        np.testing.assert_array_equal(ix.cpu().numpy().astype(np.int64), r.idx)
        out = o.cpu().numpy()
        assert max_abs(out, r.out) <= PIX_TOL
        assert abs(psnr(out, c) - psnr(r.out, c)) <= PSNR_TOL


def _vjp_problem(seed=17):
    """96 x 96 x 3 float image of the differentiation workload (Gaussian noise, sigma 25), with every
    value at least 0.3 away from a rounding boundary so that small perturbations keep the rounded
    image, and with it the grouping and the bases, unchanged."""
    clean = synth.clean_image(96, 96, 3, seed)
    x = synth.add_gaussian_float(clean, 25.0, seed).astype(np.float64)
    q = np.clip(np.rint(x), 0, 255)
    x = (q + np.clip(x - q, -0.2, 0.2)).astype(np.float32)
    return clean, x, dict(ps=8, stride=2, window=31, K=32)


def test_vjp_at_the_differentiation_workload_geometry():
    clean, x, prm = _vjp_problem()
    rng = np.random.default_rng(5)
    r = O.denoise(x.astype(np.float64), 25.0, prm, keep_masks=True)
    w = rng.uniform(0.5, 1.5, size=len(r.idx))
    gout = rng.standard_normal(x.shape)
    gx_o, gw_o = O.denoise_fixed_vjp(x.astype(np.float64), gout, r.idx, r.masks, r.U, r.V, w, 8)
    xt = _dev(x)
    wt = torch.from_numpy(w.astype(np.float32)).cuda()
    out, info = H.denoise_f32(xt, 25.0, prm, w=wt, return_info=True)
    np.testing.assert_array_equal(info["idx"].cpu().numpy().astype(np.int64), r.idx)
    gx, gw = H.denoise_vjp(xt, 25.0, info["idx"], wt, out, _dev(gout.astype(np.float32)), prm)
    gx, gw = gx.cpu().numpy(), gw.cpu().numpy()
    assert np.abs(gx - gx_o).max() <= 1e-4 * np.abs(gx_o).max()
    assert np.abs(gw - gw_o).max() <= 1e-4 * max(1.0, np.abs(gw_o).max())


def test_vjp_matches_central_differences_of_the_cuda_forward():
    """<u, (f(x + h v) - f(x - h v)) / 2h> against <J^T u, v> from the CUDA adjoint, and likewise for
    the per-group weights. The threshold is put in the middle of the widest gap between the
    oracle's coefficient magnitudes in [100, 1000] (a valid tau like any other), and h is a quarter of
    that gap over the largest norm of v on a group: the projection is orthonormal, so no coefficient
    moves by more than a quarter gap and the masks stay those of x (the device masks are checked too);
    the rounded image, grouping and bases stay put because every value of x lies within 0.2 of an
    integer and |h v| < 0.1. Along v the map is then linear and the central difference exact up to
    FP32 rounding (the weights enter through out = N / D, whose central difference is exact to
    second order in the step)."""
    clean, x, prm = _vjp_problem(23)
    rng = np.random.default_rng(6)
    v64 = rng.uniform(-1.0, 1.0, size=x.shape)
    r0 = O.denoise(x.astype(np.float64), 25.0, prm, keep_coeffs=True)
    vals = np.unique(r0.coeffs.ravel())
    sel = vals[(vals > 100.0) & (vals < 1000.0)]
    i = int(np.argmax(np.diff(sel)))
    tau, gap = 0.5 * (sel[i] + sel[i + 1]), sel[i + 1] - sel[i]
    Gv = O.gather_groups(v64, r0.idx, 8)
    bound = float(np.sqrt((Gv ** 2).reshape(len(r0.idx), -1).sum(axis=1)).max())
    h = min(0.1, 0.25 * gap / bound)
    assert h > 1e-3, (gap, bound)
    prm = dict(prm, tau_mult=tau / 25.0)
    n = len(r0.idx)
    u = _dev(rng.standard_normal(x.shape).astype(np.float32))
    v = _dev(v64.astype(np.float32))
    w = torch.from_numpy(rng.uniform(0.5, 1.5, size=n).astype(np.float32)).cuda()
    dw = torch.from_numpy(rng.uniform(-1.0, 1.0, size=n).astype(np.float32)).cuda()
    xt = _dev(x)
    out, info = H.denoise_f32(xt, 25.0, prm, w=w, return_info=True, masks=True)
    np.testing.assert_array_equal(info["idx"].cpu().numpy().astype(np.int64), r0.idx)
    assert int(info["masks"].ne(0).sum()) > 0                 # the threshold keeps some coefficients
    gx, gw = H.denoise_vjp(xt, 25.0, info["idx"], w, out, u, prm)
    fwd = {}
    for sgn in (1.0, -1.0):
        o, inf = H.denoise_f32(xt + sgn * h * v, 25.0, prm, w=w, return_info=True, masks=True)
        assert torch.equal(inf["idx"], info["idx"]) and torch.equal(inf["masks"], info["masks"])
        fwd[sgn] = o.double()
    # FP32 rounding of the outputs (at most 255 x 2^-24 each) over 2h, summed against u: the scale of
    # the difference the central difference alone makes; the bound allows four times it
    unorm = float(u.double().norm())
    fd_x = float(((fwd[1.0] - fwd[-1.0]) / (2 * h) * u.double()).sum())
    ad_x = float((gx.double() * v.double()).sum())
    assert abs(fd_x - ad_x) <= 1e-3 * abs(ad_x) + 4 * unorm * 255 * 2.0 ** -24 / (2 * h)
    assert abs(ad_x) > 40 * unorm * 255 * 2.0 ** -24 / (2 * h)      # well above that scale
    hw = 0.05
    fw = [H.denoise_f32(xt, 25.0, prm, w=w + sgn * hw * dw).double() for sgn in (1.0, -1.0)]
    fd_w = float(((fw[0] - fw[1]) / (2 * hw) * u.double()).sum())
    ad_w = float((gw.double() * dw.double()).sum())
    assert abs(fd_w - ad_w) <= 1e-3 * abs(ad_w) + 4 * unorm * 255 * 2.0 ** -24 / (2 * hw)

"""A-Haar-tSVD (Alg. 2) through the C ABI against the oracle: per-subimage sigma estimates and
per-subimage denoising."""
import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth
from tests._common import PIX_TOL, PSNR_TOL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _quadrant_noise(Hh, Ww, C, sigmas, seed):
    """Clean synthetic image with a different Gaussian noise level in each quadrant."""
    clean = synth.clean_image(Hh, Ww, C, seed)
    noisy = np.empty(clean.shape, np.uint8)
    h2, w2 = Hh // 2, Ww // 2
    quads = [(slice(0, h2), slice(0, w2)), (slice(0, h2), slice(w2, Ww)),
             (slice(h2, Hh), slice(0, w2)), (slice(h2, Hh), slice(w2, Ww))]
    for k, (ys, xs) in enumerate(quads):
        noisy[ys, xs] = synth.add_gaussian(np.ascontiguousarray(clean[ys, xs]), sigmas[k], seed + k)
    return synth.quantize(clean), noisy


@pytest.mark.parametrize("shape,sub,prm", [
    ((96, 112, 3), (48, 56), dict(ps=8, stride=3, window=11, K=8, adapt=True)),
    ((80, 72, 1), (40, 36), dict(ps=8, stride=2, window=9, K=16)),
    ((100, 118, 3), (48, 56), dict(ps=8, stride=2, window=9, K=8, match_mode="full")),  # 50x59 subimages
    # 35x45 subimages: 130 references for 192 patch entries, so the covariance is rank-deficient and
    # sigma is zero up to rounding on both sides (the absolute tolerance below)
    ((70, 90, 3), (30, 40), dict(ps=8, stride=3, window=9, K=8)),
])
def test_adaptive_matches_oracle(shape, sub, prm):
    import paper_2508_10307_gb300 as H
    Hh, Ww, C = shape
    clean, noisy = _quadrant_noise(Hh, Ww, C, (6.0, 15.0, 25.0, 40.0), 31)
    ref, ref_sig = O.a_haar_tsvd(noisy, sub[0], sub[1], prm)
    x = torch.from_numpy(noisy).cuda()
    out, sig = H.denoise_adaptive(x, sub, prm, return_sigmas=True)
    # absolute floor: sqrt of the rounding level of the covariance eigenvalues (~1e-12 of ~1e4)
    np.testing.assert_allclose(np.array(sig), ref_sig, rtol=1e-9, atol=1e-5)
    got = out.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref.reshape(got.shape)).max() <= PIX_TOL
    psnr_g = synth.psnr(got.reshape(clean.shape), clean)
    psnr_o = synth.psnr(ref.reshape(clean.shape), clean)
    assert abs(psnr_g - psnr_o) <= PSNR_TOL


def test_adaptive_single_subimage_equals_plain_estimate_and_denoise():
    import paper_2508_10307_gb300 as H
    noisy = synth.add_gaussian(synth.clean_image(64, 80, 3, 41), 20.0, 41)
    prm = dict(ps=8, stride=3, window=13, K=16, adapt=True)
    x = torch.from_numpy(noisy).cuda()
    out, sig = H.denoise_adaptive(x, (512, 512), prm, return_sigmas=True)
    plain, info = H.denoise(x, None, prm, return_info=True)
    assert len(sig) == 1 and sig[0] == pytest.approx(info["sigma"], rel=1e-12)
    assert (out - plain).abs().max().item() <= PIX_TOL

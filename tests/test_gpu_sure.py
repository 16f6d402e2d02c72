"""SURE threshold selection through the C ABI against the oracle (reading R17)."""
import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402


@pytest.mark.parametrize("eps", [0.0, 2.0])
@pytest.mark.parametrize("shape,prm,sigma", [
    ((48, 56, 3), dict(ps=8, stride=3, window=11, K=16), 20.0),
    ((40, 44, 1), dict(ps=8, stride=2, window=9, K=8), 25.0),
])
def test_sure_matches_oracle(shape, prm, sigma, eps):
    y = synth.add_gaussian_float(synth.clean_image(*shape, 801), sigma, 802).astype(np.float32)
    b = np.random.default_rng(803).choice([-1.0, 1.0], size=y.shape).astype(np.float32)
    mults = [1.6, 2.2, 2.8, 3.6]
    ref = O.sure(y, sigma, mults, b, prm, eps=eps)
    got = np.array(H.sure(torch.from_numpy(y).cuda(), sigma, mults, torch.from_numpy(b).cuda(), prm, eps=eps))
    # FP32 estimates within 1e-3 per pixel move each term by far less than 1e-3 of sigma^2
    np.testing.assert_allclose(got, ref, rtol=1e-3, atol=1e-3 * sigma ** 2)
    assert int(np.argmin(got)) == int(np.argmin(ref))


@pytest.mark.parametrize("eps", [0.0, 1.5])
def test_sure_of_a_vanishing_threshold_is_sigma_squared(eps):
    y = synth.add_gaussian_float(synth.clean_image(40, 48, 3, 811), 15.0, 812).astype(np.float32)
    b = np.random.default_rng(813).choice([-1.0, 1.0], size=y.shape).astype(np.float32)
    (s,) = H.sure(torch.from_numpy(y).cuda(), 15.0, [1e-9], torch.from_numpy(b).cuda(),
                  dict(ps=8, stride=3, window=9, K=8), eps=eps)
    assert s == pytest.approx(15.0 ** 2, rel=1e-4)


def test_finite_difference_sure_tracks_the_error_against_the_clean_image():
    """Stein's lemma at a size the oracle does not reach quickly: on Gaussian noise the
    finite-difference SURE of the device path stays close to the device path's own mean squared
    error against the clean image, and both pick the same threshold. SURE is itself an estimate:
    the realisation's noise energy ||y - x||^2 / n - sigma^2 enters every value alike (standard
    deviation sigma^2 sqrt(2 / n), 2.0 here), so the bound is 5% plus three of those."""
    clean = synth.clean_image(256, 256, 3, 821)
    y = synth.add_gaussian_float(clean, 25.0, 822).astype(np.float32)
    b = np.random.default_rng(823).choice([-1.0, 1.0], size=y.shape).astype(np.float32)
    prm = dict(ps=8, stride=2, window=15, K=16)
    mults = [1.5, 2.7, 4.5]
    dy = torch.from_numpy(y).cuda()
    got = np.array(H.sure(dy, 25.0, mults, torch.from_numpy(b).cuda(), prm, eps=2.5))
    x = torch.from_numpy(clean.astype(np.float32)).cuda()
    mse = np.array([float(((H.denoise_f32(dy, 25.0, dict(prm, tau_mult=m)) - x) ** 2).mean()) for m in mults])
    np.testing.assert_allclose(got, mse, rtol=0.05, atol=3 * 25.0 ** 2 * np.sqrt(2 / y.size))
    assert int(np.argmin(got)) == int(np.argmin(mse))

"""SURE of the per-group aggregation weights and its gradient on the GPU against the FP64 oracle
(reading R19), plus the properties that hold at any size (needs a GB300 and the built library).

Bar: SURE within 1e-4 relative, the gradient within 2e-3 of its largest component (FP32 outputs
and adjoint), sum_g w_g grad_g = 0 to FP32 rounding, and central differences of the device SURE."""
import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402


def _case(h=40, w=44, seed=7, sigma=20.0, prm=None):
    clean = synth.clean_image(h, w, 3, seed)
    y = synth.add_gaussian_float(clean, sigma, seed).astype(np.float32)
    rng = np.random.default_rng(seed + 1)
    b = rng.choice([-1.0, 1.0], size=y.shape).astype(np.float32)
    prm = prm or dict(ps=8, stride=3, window=9, K=8)
    n = H.num_groups(h, w, prm)
    return y, b, prm, rng.uniform(0.5, 1.5, n).astype(np.float32), rng


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("shape,prm", [((40, 44), dict(ps=8, stride=3, window=9, K=8)),
                                       ((72, 80), dict(ps=8, stride=3, window=31, K=32))])
def test_sure_weights_match_the_oracle(shape, prm):
    y, b, prm, w, _ = _case(*shape, prm=prm)
    s_o, g_o = O.sure_weights(y, 20.0, w.astype(np.float64), b, prm, eps=2.0)
    s_g, g_g = H.sure_weights(_dev(y), 20.0, _dev(w), _dev(b), prm, eps=2.0)
    g_g = g_g.cpu().numpy().astype(np.float64)
    assert abs(s_g - s_o) <= 1e-4 * abs(s_o), (s_g, s_o)
    assert np.abs(g_g - g_o).max() <= 2e-3 * np.abs(g_o).max()


def test_device_sure_weight_gradient_is_scale_free_and_matches_differences():
    y, b, prm, w, rng = _case(48, 52, seed=21)
    yt, bt, wt = _dev(y), _dev(b), _dev(w)
    s0, g = H.sure_weights(yt, 20.0, wt, bt, prm, eps=2.0)
    g = g.double()
    wd = wt.double()
    assert abs(float((wd * g).sum())) <= 1e-4 * float((wd * g).abs().sum())
    s1, _ = H.sure_weights(yt, 20.0, 2.5 * wt, bt, prm, eps=2.0)
    assert abs(s1 - s0) <= 1e-5 * abs(s0)
    d = torch.from_numpy(rng.standard_normal(w.size).astype(np.float32)).cuda()
    h = 0.02
    sp, _ = H.sure_weights(yt, 20.0, wt + h * d, bt, prm, eps=2.0)
    sm, _ = H.sure_weights(yt, 20.0, wt - h * d, bt, prm, eps=2.0)
    fd, ad = (sp - sm) / (2 * h), float((g * d.double()).sum())
    # second-order term of the central difference plus FP32 rounding of SURE (about 1e-6 relative)
    assert abs(fd - ad) <= 2e-2 * abs(ad) + 2e-6 * abs(s0) / h, (fd, ad)


def test_device_weight_tuning_follows_the_oracle():
    y, b, prm, _, _ = _case(40, 44, seed=17)
    w_o, tr_o = O.tune_weights(y, 20.0, b, prm, eps=2.0, steps=3, step=0.3)
    w_g, tr_g = H.tune_weights(_dev(y), 20.0, _dev(b), prm, eps=2.0, steps=3, step=0.3)
    tr_g = np.array(tr_g)
    assert np.all(np.diff(tr_g) < 0), tr_g
    np.testing.assert_allclose(tr_g, tr_o, rtol=2e-4)
    w_g = w_g.cpu().numpy()
    assert np.all(w_g > 0)
    np.testing.assert_allclose(w_g, w_o, rtol=2e-3)


def test_sure_weights_refuse_bad_arguments():
    y, b, prm, w, _ = _case()
    yt, bt, wt = _dev(y), _dev(b), _dev(w)
    for kw in (dict(sigma=0.0, eps=2.0), dict(sigma=20.0, eps=0.0), dict(sigma=20.0, eps=-1.0)):
        with pytest.raises(RuntimeError):
            H.sure_weights(yt, kw["sigma"], wt, bt, prm, eps=kw["eps"])
    with pytest.raises(RuntimeError):
        H.tune_weights(yt, 20.0, bt, prm, eps=2.0, steps=2, step=0.0)

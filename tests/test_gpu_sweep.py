"""Threshold sweeps with cached grouping and noisy coefficients: every output equals a plain
htsvd_denoise call at that threshold, bitwise, and the oracle within the pixel tolerance."""
import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth
from tests._common import PIX_TOL, max_abs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402


@pytest.mark.parametrize("shape,prm,sigma", [
    ((64, 72, 3), dict(ps=8, stride=3, window=15, K=32), 20.0),
    ((56, 60, 1), dict(ps=8, stride=2, window=11, K=16), 25.0),
    ((72, 80, 3), dict(ps=8, stride=3, window=11, K=8, agg_mode="sparsity"), None),
])
def test_sweep_equals_plain_calls(shape, prm, sigma):
    noisy = synth.add_gaussian(synth.clean_image(*shape, seed=321), 20.0 if sigma is None else sigma, seed=322)
    x = torch.from_numpy(noisy).cuda()
    mults = [0.0, 1.5, 2.2, 2.7, 3.4]
    outs, sg = H.denoise_tau_sweep(x, mults, sigma, prm, return_sigma=True)
    torch.cuda.synchronize()
    for i, m in enumerate(mults):
        if m == 0.0:
            # tau = 0 keeps every coefficient: the sweep reproduces its input (plain calls cannot ask
            # for tau_mult 0, which selects the default multiplier)
            # (the FP32 round trip of projections and Haar, as in the plain zero-threshold test)
            assert max_abs(outs[i].cpu().numpy(), noisy.astype(np.float64).reshape(outs[i].shape)) <= 2e-3
            continue
        plain = H.denoise(x, sg, dict(prm, tau_mult=m))
        assert torch.equal(outs[i], plain), m
    ref = O.denoise(noisy, sg, dict(prm, tau_mult=mults[2]))
    assert max_abs(outs[2].cpu().numpy(), ref.out) <= PIX_TOL

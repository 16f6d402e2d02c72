"""Hand-written VJP (GPU) vs the FP64 oracle's frozen-mask adjoint, and the autograd wrapper."""
import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402


def _problem(C, shape=(48, 56), seed=13, K=16):
    clean = synth.clean_image(shape[0], shape[1], C, seed)
    x = synth.add_gaussian_float(clean, 25.0, seed)
    prm = dict(ps=8, stride=3, window=13, K=K)
    return clean, x, prm


@pytest.mark.parametrize("C", [1, 3])
def test_vjp_matches_oracle_adjoint(C):
    clean, x, prm = _problem(C)
    rng = np.random.default_rng(4)
    r = O.denoise(x.astype(np.float64), 25.0, prm, keep_masks=True)
    w = rng.uniform(0.5, 1.5, size=len(r.idx))
    gout = rng.standard_normal(x.shape)
    gx_o, gw_o = O.denoise_fixed_vjp(x.astype(np.float64), gout, r.idx, r.masks, r.U, r.V, w, 8)

    xt = torch.from_numpy(x).cuda()
    wt = torch.from_numpy(w.astype(np.float32)).cuda()
    out, info = H.denoise_f32(xt, 25.0, prm, w=wt, return_info=True)
    gx, gw = H.denoise_vjp(xt, 25.0, info["idx"], wt, out, torch.from_numpy(gout.astype(np.float32)).cuda(), prm)
    gx, gw = gx.cpu().numpy(), gw.cpu().numpy()
    assert np.abs(gx - gx_o).max() <= 1e-4 * np.abs(gx_o).max()
    assert np.abs(gw - gw_o).max() <= 1e-4 * max(1.0, np.abs(gw_o).max())


def test_autograd_function_gradients():
    clean, x, prm = _problem(3, seed=21)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    n = H.num_groups(x.shape[0], x.shape[1], prm)
    wt = torch.ones(n, device="cuda", requires_grad=True)
    out = H.HtsvdFn.apply(xt, wt, 25.0, prm)
    target = torch.from_numpy(clean.astype(np.float32)).cuda()
    loss = ((out - target) ** 2).mean()
    loss.backward()
    assert xt.grad is not None and torch.isfinite(xt.grad).all()
    assert wt.grad is not None and torch.isfinite(wt.grad).all()
    # against the oracle adjoint of the same loss
    r = O.denoise(x.astype(np.float64), 25.0, prm, keep_masks=True)
    gout = 2.0 * (r.out - clean) / r.out.size
    gx_o, gw_o = O.denoise_fixed_vjp(x.astype(np.float64), gout, r.idx, r.masks, r.U, r.V, np.ones(n), 8)
    assert np.abs(xt.grad.cpu().numpy() - gx_o).max() <= 1e-4 * np.abs(gx_o).max()
    assert np.abs(wt.grad.cpu().numpy() - gw_o).max() <= 1e-4 * max(1e-12, np.abs(gw_o).max())

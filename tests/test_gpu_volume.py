"""MRI volumes (Alg. 1 on 4 x 4 x 4 cubes, reading R20) on the GPU against the FP64 oracle.

Bar as for images: match indices bit-exact, threshold masks bit-exact (except coefficients the
oracle itself finds within 1e-9 of tau), voxels within 1e-3, PSNR within 0.01 dB, bases within 1e-9.
"""
import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth
from tests._common import PIX_TOL, PSNR_TOL, max_abs, pack_masks, psnr

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402
from paper_2508_10307_gb300 import _lib  # noqa: E402


def _case(shape, sigma, seed):
    clean = synth.clean_volume(*shape, seed)
    return synth.quantize(clean), synth.add_gaussian(clean, sigma, seed)


@pytest.mark.parametrize("shape,prm,sigma", [
    ((20, 24, 22), dict(ps=4, stride=2, window=5, K=16), 11.5),
    ((18, 21, 19), dict(ps=4, stride=2, window=3, K=8, agg_mode="sparsity"), 7.65),
    ((24, 26, 28), dict(ps=4, stride=2, window=5, K=32), 11.5),      # the paper's MRI setting
    ((13, 9, 11), dict(ps=4, stride=3, window=4, K=4), 15.0),        # even window, ragged grid
    ((30, 33, 17), dict(ps=4, stride=2, window=6, K=32, tau_mult=2.5), 9.0),
])
def test_volume_parity(shape, prm, sigma):
    clean, noisy = _case(shape, sigma, 80 + shape[0])
    r = O.denoise_volume(noisy, sigma, prm, keep_masks=True)
    x = torch.from_numpy(noisy).cuda()
    out, info = H.denoise_volume(x, sigma, prm, return_info=True, masks=True, weights=True, basis=True)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(info["idx"].cpu().numpy().astype(np.int64), r.idx)
    b = info["basis"].cpu().numpy()
    z = b[..., 0] + 1j * b[..., 1]
    assert np.abs(z[0] - r.U).max() < 1e-9 and np.abs(z[1] - r.V).max() < 1e-9
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
    np.testing.assert_allclose(info["weights"].cpu().numpy(), r.weights, rtol=1e-6)


def test_volume_zero_threshold_is_the_identity_and_repeats_agree():
    _, noisy = _case((17, 19, 23), 10.0, 5)
    x = torch.from_numpy(noisy).cuda()
    prm = dict(ps=4, stride=2, window=5, K=8, tau_mult=1e-12)
    out = H.denoise_volume(x, 10.0, prm)
    assert max_abs(out.cpu().numpy(), noisy) <= PIX_TOL
    a = H.denoise_volume(x, 10.0, dict(ps=4, stride=2, window=5, K=8))
    b = H.denoise_volume(x, 10.0, dict(ps=4, stride=2, window=5, K=8))
    torch.cuda.synchronize()
    assert max_abs(a.cpu().numpy(), b.cpu().numpy()) <= 1e-4       # float atomics: rounding order only


def test_volume_at_the_benchmarked_size():
    """A 176 x 208 x 176 volume (the OASIS T1-weighted size) at the paper's MRI setting: the
    grouping of 400 sampled references against the oracle, the bases against the oracle's from all
    reference cubes, a PSNR gain over the input, and the estimated sigma against the oracle's."""
    clean, noisy = _case((176, 208, 176), 11.5, 3)
    prm = dict(ps=4, stride=2, window=5, K=32)
    x = torch.from_numpy(noisy).cuda()
    out, info = H.denoise_volume(x, 11.5, prm, return_info=True, basis=True)
    torch.cuda.synchronize()
    idx = info["idx"].cpu().numpy().astype(np.int64)
    rng = np.random.default_rng(1)
    pick = np.concatenate([[0, idx.shape[0] - 1], rng.choice(idx.shape[0], 398, replace=False)])
    np.testing.assert_array_equal(idx[pick], O.block_match_volume(noisy, prm, only=pick))
    p = O.Params.of(prm)
    U, V, _, _ = O.global_basis(O.gather_cubes(noisy, O.volume_reference_positions(noisy.shape, p), 4))
    b = info["basis"].cpu().numpy()
    z = b[..., 0] + 1j * b[..., 1]
    assert np.abs(z[0] - U).max() < 1e-9 and np.abs(z[1] - V).max() < 1e-9
    o = out.cpu().numpy()
    assert np.isfinite(o).all()
    assert psnr(o, clean) > psnr(noisy.astype(np.float64), clean) + 3.0
    _, est = H.denoise_volume(x, None, prm, return_info=True)
    torch.cuda.synchronize()
    s_ref = O.estimate_sigma_volume(noisy, prm)
    assert abs(est["sigma"] - s_ref) <= 1e-9 * s_ref


@pytest.mark.parametrize("shape,prm,sigma", [
    ((20, 24, 22), dict(ps=4, stride=2, window=5, K=16), 11.5),
    ((30, 33, 17), dict(ps=4, stride=2, window=5, K=32), 7.65),
])
def test_volume_estimated_sigma_matches_oracle(shape, prm, sigma):
    """sigma < 0: the eigenvalue rule on the reference cubes' covariance (exact integer moments, host
    FP64 eigenvalues) against the oracle's numpy eigvalsh, then the denoiser at that sigma."""
    clean, noisy = _case(shape, sigma, 120 + shape[0])
    s_ref = O.estimate_sigma_volume(noisy, prm)
    r = O.denoise_volume(noisy, s_ref, prm)
    out, info = H.denoise_volume(torch.from_numpy(noisy).cuda(), None, prm, return_info=True)
    torch.cuda.synchronize()
    assert abs(info["sigma"] - s_ref) <= 1e-9 * s_ref
    assert max_abs(out.cpu().numpy(), r.out) <= PIX_TOL


def test_volume_strict_basis_refuses_a_constant_volume():
    x = torch.full((12, 13, 14), 77, dtype=torch.uint8, device="cuda")
    with pytest.raises(_lib.DegenerateBasisError):
        H.denoise_volume(x, 5.0, dict(ps=4, stride=2, window=5, K=8, strict_basis=True))
    out = H.denoise_volume(x, 5.0, dict(ps=4, stride=2, window=5, K=8))      # default mode proceeds
    torch.cuda.synchronize()
    assert max_abs(out.cpu().numpy(), np.full((12, 13, 14), 77.0)) <= PIX_TOL


def test_volume_bad_arguments():
    _, noisy = _case((12, 12, 12), 10.0, 2)
    x = torch.from_numpy(noisy).cuda()
    for prm, code in ((dict(ps=8), 2), (dict(window=9), 1), (dict(K=64), 1), (dict(K=12), 1),
                      (dict(match_mode="gcp"), 1)):
        with pytest.raises(_lib.HtsvdError) as e:
            H.denoise_volume(x, 10.0, prm)
        assert _lib.STATUS_NAMES[code] in str(e.value)
    with pytest.raises(_lib.HtsvdError):
        H.denoise_volume(torch.zeros((3, 12, 12), dtype=torch.uint8, device="cuda"), 10.0)


@pytest.mark.parametrize("shape,sub,prm", [
    ((40, 28, 30), (20, 28, 30), dict(ps=4, stride=2, window=5, K=16)),      # two noise levels along z
    ((24, 26, 29), (12, 13, 14), dict(ps=4, stride=2, window=4, K=8)),       # 2 x 2 x 2 ragged parts
])
def test_volume_adaptive_matches_oracle(shape, sub, prm):
    """A-Haar-tSVD on a volume: per sub-volume sigma (eigenvalue rule) against the oracle's, and the
    composed estimate voxel by voxel against the oracle's adaptive variant."""
    clean = synth.clean_volume(*shape, 140 + shape[0])
    rng = np.random.default_rng(shape[1])
    level = np.where(np.arange(shape[0])[:, None, None] < shape[0] // 2, 5.0, 15.0)
    noisy = np.clip(np.rint(clean + level * rng.standard_normal(shape)), 0, 255).astype(np.uint8)
    ref, s_ref = O.a_haar_tsvd_volume(noisy, sub, prm)
    out, sig = H.denoise_volume_adaptive(torch.from_numpy(noisy).cuda(), sub, prm, return_sigmas=True)
    torch.cuda.synchronize()
    assert len(sig) == len(s_ref)
    assert np.abs(np.array(sig) - s_ref).max() <= 1e-9 * s_ref.max()
    assert max_abs(out.cpu().numpy(), ref) <= PIX_TOL
    if shape[0] == 40:
        assert s_ref[1] > 2.0 * s_ref[0]


def test_volume_adaptive_bad_arguments():
    _, noisy = _case((16, 16, 16), 10.0, 4)
    x = torch.from_numpy(noisy).cuda()
    for sub in ((0, 8, 8), (2, 16, 16)):             # a zero size; parts two voxels deep
        with pytest.raises(_lib.HtsvdError) as e:
            H.denoise_volume_adaptive(x, sub, dict(K=8))
        assert _lib.STATUS_NAMES[1] in str(e.value)

"""Batched basis projection (Sec. III-B.2, Eq. (forward transform) before the Haar step) on the GPU.

htsvd_project_patches runs S = U^T * P * V of a batch of patches as one dense contraction on the
tensor cores (patch bytes exact in FP16, the basis matrix split in two FP16 pieces, FP32
accumulation); htsvd_internal_project_simt runs the structured per-slice FP32 form on the CUDA cores.
Both are compared with the oracle's patch_forward (FP64, its own bases) patch by patch. The bar is a
quarter of the group filter's guard band per patch: |S_gpu - S_oracle| <= 2^-21 ||P||_F, so that a
coefficient computed this way could take the filter's threshold decision (the band is 2^-19 of the
group norm, which bounds every patch norm of the group).
"""
import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2508_10307_gb300 as H  # noqa: E402
from paper_2508_10307_gb300 import _lib  # noqa: E402

BAR = 2.0 ** -21


def _oracle_coefficients(noisy, prm, pos):
    """Oracle patch_forward of the patches at linear positions pos, with the oracle's own bases."""
    p = O.Params.of(prm)
    U, V, _, _ = O.global_basis(O.reference_patches(noisy, p))
    G = O.gather_groups(noisy, pos[:, None].astype(np.int64), 8)[:, 0]       # (n, 8, 8, C)
    S = O.patch_forward(G, U, V).reshape(len(pos), -1)
    norms = np.sqrt((G.astype(np.float64) ** 2).reshape(len(pos), -1).sum(axis=1))
    return S, norms


def _gpu_setup(noisy, prm):
    x = torch.from_numpy(noisy).cuda()
    _, info = H.denoise(x, 20.0, prm, return_info=True, basis=True)
    return x, info["idx"].reshape(-1).contiguous(), info["basis"].reshape(-1).contiguous()


def _check(gpu, ref, norms, what):
    err = np.abs(gpu.astype(np.float64) - ref).max(axis=1) / np.maximum(norms, 1.0)
    worst = float(err.max())
    assert worst <= BAR, f"{what}: worst error {np.log2(worst):.2f} (log2 of a fraction of the patch norm)"
    return worst


@pytest.mark.parametrize("shape,prm", [
    ((40, 48, 1), dict(ps=8, stride=3, window=11, K=8)),
    ((72, 80, 3), dict(ps=8, stride=3, window=15, K=16)),
    ((33, 41, 3), dict(ps=8, stride=2, window=9, K=4)),
])
def test_projection_matches_oracle(shape, prm):
    Hh, Ww, C = shape
    clean = synth.clean_image(Hh, Ww, C, 70 + C)
    noisy = synth.add_gaussian(clean, 20.0, 70 + C)
    x, idx, basis = _gpu_setup(noisy, prm)
    # group members (several MMA tiles and a ragged tail), the four corner patches, and positions whose
    # patch leaves the image (before the first pixel, past the last, across the right and bottom edges)
    corners = [0, Ww - 8, (Hh - 8) * Ww, (Hh - 8) * Ww + Ww - 8]
    bad = [-1, Hh * Ww, Ww - 7, (Hh - 7) * Ww]
    pos_np = np.concatenate([idx.cpu().numpy(), corners, bad]).astype(np.int32)
    assert len(pos_np) % 128 != 0 and len(pos_np) > 2 * 128
    pos = torch.from_numpy(pos_np).cuda()
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    tc = H.project_patches(x, pos, basis, flag=flag)
    st = H.project_patches(x, pos, basis, structured=True)
    torch.cuda.synchronize()
    assert int(flag.item()) == 0
    good = pos_np[: -len(bad)]
    ref, norms = _oracle_coefficients(noisy, prm, good)
    t = tc.cpu().numpy()
    s = st.cpu().numpy()
    _check(t[: len(good)], ref, norms, "tensor cores")
    _check(s[: len(good)], ref, norms, "CUDA cores")
    assert np.isnan(t[len(good):]).all() and np.isnan(s[len(good):]).all()


def test_projection_at_the_benchmarked_geometry():
    """Every member of every group of the 512x512x3 workload (2,048,288 patches, stride 2, window 31,
    K 32), in the launch configuration the benchmark times: the oracle on a sample of 3,000 patches,
    the two GPU forms against each other on all of them, two tensor-core calls bitwise equal."""
    clean, noisy, _, prm = synth.workload_rgb512()
    x = torch.from_numpy(noisy).cuda()
    _, info = H.denoise(x, None, prm, return_info=True, basis=True)
    pos = info["idx"].reshape(-1).contiguous()
    basis = info["basis"].reshape(-1).contiguous()
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    tc = H.project_patches(x, pos, basis, flag=flag)
    tc2 = H.project_patches(x, pos, basis)
    st = H.project_patches(x, pos, basis, structured=True)
    torch.cuda.synchronize()
    assert int(flag.item()) == 0
    assert torch.equal(tc, tc2)
    n = pos.numel()
    rng = np.random.default_rng(5)
    pick = np.sort(rng.choice(n, 3000, replace=False))
    pick[-1] = n - 1
    pos_np = pos.cpu().numpy()
    ref, norms = _oracle_coefficients(noisy, prm, pos_np[pick])
    t = tc.cpu().numpy()
    _check(t[pick], ref, norms, "tensor cores")
    _check(st.cpu().numpy()[pick], ref, norms, "CUDA cores")
    # all patches: the two forms within twice the bar of each other (relative to the patch norm)
    pn = torch.sqrt(_patch_norms2(x, pos)).clamp_min(1.0)
    diff = ((tc - st).abs().amax(dim=1) / pn).max().item()
    assert diff <= 2 * BAR


def _patch_norms2(x, pos):
    """Squared Frobenius norms of the patches at pos (torch on the device; test-side helper)."""
    Hh, Ww, C = x.shape
    xf = x.float()
    p = pos.long()
    y, xx = p // Ww, p % Ww
    out = torch.zeros(pos.numel(), dtype=torch.float32, device=x.device)
    for a in range(8):
        for b in range(8):
            out += (xf[y + a, xx + b] ** 2).sum(dim=-1)
    return out


@pytest.mark.parametrize("shape", [(40, 48, 1), (72, 200, 3), (33, 41, 3), (19, 301, 3)])
def test_projection_of_every_position_matches_oracle(shape):
    """pos = None: every top-left corner, row-major (the im2col batch: tiles of 128 positions of one
    row, the last of a row ragged; rows narrower and wider than a tile)."""
    Hh, Ww, C = shape
    clean = synth.clean_image(Hh, Ww, C, 90 + Ww)
    noisy = synth.add_gaussian(clean, 20.0, 90 + Ww)
    x, _, basis = _gpu_setup(noisy, dict(ps=8, stride=3, window=7, K=4))
    tc = H.project_patches(x, None, basis)
    st = H.project_patches(x, None, basis, structured=True)
    torch.cuda.synchronize()
    ys, xs = np.mgrid[0:Hh - 7, 0:Ww - 7]
    pos = (ys * Ww + xs).ravel()
    ref, norms = _oracle_coefficients(noisy, dict(ps=8, stride=3, window=7, K=4), pos)
    _check(tc.cpu().numpy(), ref, norms, "tensor cores, every position")
    _check(st.cpu().numpy(), ref, norms, "CUDA cores, every position")


def test_projection_of_every_position_at_the_benchmarked_size():
    """Every position of the 512x512x3 workload (255,025 patches) as the benchmark times it: a sample
    against the oracle, the two forms against each other everywhere, two calls bitwise equal, and
    the same coefficients as the position-list form."""
    clean, noisy, _, prm = synth.workload_rgb512()
    x = torch.from_numpy(noisy).cuda()
    _, info = H.denoise(x, None, prm, return_info=True, basis=True)
    basis = info["basis"].reshape(-1).contiguous()
    tc = H.project_patches(x, None, basis)
    tc2 = H.project_patches(x, None, basis)
    st = H.project_patches(x, None, basis, structured=True)
    ys, xs = np.mgrid[0:505, 0:505]
    pos = torch.from_numpy((ys * 512 + xs).ravel().astype(np.int32)).cuda()
    lst = H.project_patches(x, pos, basis)
    torch.cuda.synchronize()
    assert torch.equal(tc, tc2) and torch.equal(tc, lst)
    rng = np.random.default_rng(7)
    pick = np.sort(rng.choice(tc.shape[0], 2000, replace=False))
    ref, norms = _oracle_coefficients(noisy, prm, pos.cpu().numpy()[pick])
    _check(tc.cpu().numpy()[pick], ref, norms, "tensor cores")
    pn = torch.sqrt(_patch_norms2(x, pos)).clamp_min(1.0)
    assert ((tc - st).abs().amax(dim=1) / pn).max().item() <= 2 * BAR


def test_projection_empty_and_bad_arguments():
    noisy = synth.add_gaussian(synth.clean_image(24, 24, 3, 9), 15.0, 9)
    x = torch.from_numpy(noisy).cuda()
    basis = torch.zeros(2 * 3 * 64 * 2, dtype=torch.float64, device="cuda")
    lib = _lib.load()
    out = torch.full((4, 192), 7.0, device="cuda")
    pos = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    import ctypes
    vp = ctypes.c_void_p
    assert lib.htsvd_project_patches(vp(x.data_ptr()), 24, 24, 3, vp(pos.data_ptr()), 0, vp(basis.data_ptr()),
                                     vp(out.data_ptr()), None, vp(s)) == 0
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())
    assert lib.htsvd_project_patches(vp(x.data_ptr()), 24, 24, 2, vp(pos.data_ptr()), 4, vp(basis.data_ptr()),
                                     vp(out.data_ptr()), None, vp(s)) == 1
    assert lib.htsvd_project_patches(vp(x.data_ptr()), 24, 24, 3, vp(pos.data_ptr()), 4, vp(basis.data_ptr()),
                                     vp(out.data_ptr() + 4), None, vp(s)) == 1
    assert lib.htsvd_project_patches(vp(x.data_ptr()), 7, 24, 3, vp(pos.data_ptr()), 4, vp(basis.data_ptr()),
                                     vp(out.data_ptr()), None, vp(s)) == 1
    assert lib.htsvd_project_patches(vp(x.data_ptr()), 24, 24, 3, None, 4, vp(basis.data_ptr()),
                                     vp(out.data_ptr()), None, vp(s)) == 1

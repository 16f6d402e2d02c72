"""Pins of the FP64 oracle to what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a worked example,
a closed form, a definition written out another way, brute force on a tiny input,
or an invariant that a dropped term, wrong sign, wrong index or transposed operand breaks.
"""
import math
import os

import numpy as np
import pytest

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Haar (Sec. II-D)

def test_haar_worked_example_h4():
    rows = [l for l in open(os.path.join(GOLDEN, "haar4.txt")) if not l.startswith("#")]
    x = np.array(rows[0].split(), dtype=float)
    y = np.array(rows[1].split(), dtype=float)
    np.testing.assert_allclose(O.haar_matrix(4) @ x, y, rtol=0, atol=1e-15)


def test_haar_h2_matches_equation():
    np.testing.assert_allclose(O.haar_matrix(2), np.array([[1, 1], [1, -1]]) / math.sqrt(2), atol=0)


@pytest.mark.parametrize("K", [2, 4, 8, 16, 32, 64])
def test_haar_orthonormal_and_first_row(K):
    H = O.haar_matrix(K)
    np.testing.assert_allclose(H @ H.T, np.eye(K), atol=1e-14)
    # Eq. (first eigen) / Sec. III-B.2: u_max = 1/sqrt(K) (1,...,1) is the first Haar row.
    np.testing.assert_allclose(H[0], np.full(K, 1 / math.sqrt(K)), atol=1e-15)
    # rows K/2..K-1 are the pairwise differences of Eq. (H_2N)
    for m in range(K // 2):
        e = np.zeros(K)
        e[2 * m], e[2 * m + 1] = 1 / math.sqrt(2), -1 / math.sqrt(2)
        np.testing.assert_allclose(H[K // 2 + m], e, atol=1e-15)


def test_haar_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        O.haar_matrix(12)


# ---------------------------------------------------------------- t-product (Sec. II-C)

@pytest.mark.parametrize("n3", [1, 3, 4])
def test_t_product_fft_equals_bcirc_definition(n3):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((5, 4, n3))
    B = rng.standard_normal((4, 6, n3))
    np.testing.assert_allclose(O.t_product_fft(A, B), O.t_product_bcirc(A, B), atol=1e-12)
    # bcirc(A*B) = bcirc(A) bcirc(B)
    np.testing.assert_allclose(O.bcirc(O.t_product_bcirc(A, B)), O.bcirc(A) @ O.bcirc(B), atol=1e-12)


def test_t_transpose_is_bcirc_transpose():
    A = np.random.default_rng(1).standard_normal((3, 5, 3))
    np.testing.assert_allclose(O.bcirc(O.t_transpose(A)), O.bcirc(A).T, atol=0)


def _rgb_patches(seed=3, n=400, ps=4):
    clean = synth.clean_image(40, 40, 3, seed)
    noisy = synth.add_gaussian(clean, 20.0, seed)
    p = O.Params(ps=ps, stride=2, window=7, K=8)
    return noisy, p, O.reference_patches(noisy, p)


def test_basis_is_real_orthogonal_tensor():
    _, _, P = _rgb_patches()
    U, V, lu, lv = O.global_basis(P)
    for F in (U, V):
        T = np.fft.ifft(F, axis=0)                      # slices -> real tensor, mode 3 last
        assert np.abs(T.imag).max() < 1e-13
        Tr = np.moveaxis(T.real, 0, -1)                 # (ps, ps, C)
        # U^T * U = identity tensor (Sec. II-C orthogonality), checked through bcirc
        UtU = O.t_product_bcirc(O.t_transpose(Tr), Tr)
        I = np.zeros_like(UtU)
        I[:, :, 0] = np.eye(Tr.shape[0])
        np.testing.assert_allclose(UtU, I, atol=1e-12)
    assert np.all(np.diff(lu[0]) <= 0) and np.all(np.diff(lv[1]) <= 0)


def test_basis_diagonalises_slice_second_moments():
    _, _, P = _rgb_patches()
    U, V, lu, lv = O.global_basis(P)
    PF = np.fft.fft(P, axis=-1)
    for f in range(3):
        A = sum(X @ X.conj().T for X in PF[..., f])      # plain sum over patches
        B = sum(X.conj().T @ X for X in PF[..., f])
        np.testing.assert_allclose(U[f].conj().T @ A @ U[f], np.diag(lu[f]), atol=1e-7 * lu[f][0])
        np.testing.assert_allclose(V[f].conj().T @ B @ V[f], np.diag(lv[f]), atol=1e-7 * lv[f][0])
        # canonical phase: largest-modulus entry real and positive
        for Q in (U[f], V[f]):
            for c in range(Q.shape[1]):
                a = int(np.argmax(np.abs(Q[:, c])))
                assert abs(Q[a, c].imag) < 1e-12 and Q[a, c].real > 0


def test_gray_basis_is_plain_eigenvectors_of_row_and_column_scatter():
    clean = synth.clean_image(48, 48, 1, 5)
    noisy = synth.add_gaussian(clean, 15.0, 5)
    p = O.Params(ps=8, stride=3, window=9, K=8)
    P = O.reference_patches(noisy, p)[..., 0]
    U, V, _, _ = O.global_basis(P[..., None])
    Arow = np.zeros((8, 8))
    Bcol = np.zeros((8, 8))
    for X in P:                                          # textbook 2-D SVD scatter matrices
        Arow += X @ X.T
        Bcol += X.T @ X
    for F, S in ((U[0], Arow), (V[0], Bcol)):
        w, Q = np.linalg.eigh(S)
        Q = Q[:, ::-1]
        np.testing.assert_allclose(np.abs(np.sum(Q * F.real, axis=0)), 1.0, atol=1e-10)


def test_patch_projection_equals_t_products_by_definition():
    noisy, p, P = _rgb_patches()
    U, V, _, _ = O.global_basis(P)
    Ur = np.moveaxis(np.fft.ifft(U, axis=0).real, 0, -1)
    Vr = np.moveaxis(np.fft.ifft(V, axis=0).real, 0, -1)
    X = P[17]
    S_def = O.t_product_bcirc(O.t_product_bcirc(O.t_transpose(Ur), X), Vr)   # U^T * P * V
    np.testing.assert_allclose(O.patch_forward(X, U, V), S_def, atol=1e-10)
    back = O.t_product_bcirc(O.t_product_bcirc(Ur, S_def), O.t_transpose(Vr))  # U * S * V^T
    np.testing.assert_allclose(back, X, atol=1e-10)
    np.testing.assert_allclose(O.patch_inverse(S_def, U, V), X, atol=1e-10)


def test_group_transform_is_orthogonal_and_uses_haar_along_group_mode():
    noisy, p, P = _rgb_patches()
    U, V, _, _ = O.global_basis(P)
    H = O.haar_matrix(8)
    G = P[:8]
    S = O.forward_transform(G, U, V, H)
    np.testing.assert_allclose(np.linalg.norm(S), np.linalg.norm(G), rtol=1e-13)
    np.testing.assert_allclose(O.inverse_transform(S, U, V, H), G, atol=1e-10)
    T = O.patch_forward(G, U, V)
    # coefficient row 0 is the scaled group sum (first principal direction, Eq. first eigen)
    np.testing.assert_allclose(S[0], T.sum(axis=0) / math.sqrt(8), atol=1e-10)
    # last row is the difference of the last pair (Eq. H_2N)
    np.testing.assert_allclose(S[7], (T[6] - T[7]) / math.sqrt(2), atol=1e-10)


# ---------------------------------------------------------------- grouping (Sec. III-A)

def _brute_force_match(img, ry, rx, p):
    """Pure-Python brute force: every candidate, Python integers, full sort on (ssd, index)."""
    H, W, C = img.shape
    ps = p.ps
    npy, npx = H - ps + 1, W - ps + 1
    def win(r, npos):
        if npos <= p.window:
            return range(npos)
        s = min(max(r - (p.window - 1) // 2, 0), npos - p.window)
        return range(s, s + p.window)
    im = img.astype(int).tolist()
    if C == 1:
        plane = [[px[0] for px in row] for row in im]
    else:
        r2 = g2 = b2 = 0
        for i in range(ps):
            for j in range(ps):
                r, g, b = im[ry + i][rx + j]
                r2 += r * r; g2 += g * g; b2 += b * b
        gg = p.gcp_gamma * p.gcp_gamma
        green = gg * g2 >= r2 and gg * g2 >= b2
        plane = [[px[1] if green else px[0] + px[1] + px[2] for px in row] for row in im]
    keys = []
    for y in win(ry, npy):
        for x in win(rx, npx):
            if (y, x) == (ry, rx):
                continue
            d = 0
            for i in range(ps):
                for j in range(ps):
                    t = plane[ry + i][rx + j] - plane[y + i][x + j]
                    d += t * t
            keys.append((d, y * W + x))
    keys.sort()
    return [ry * W + rx] + [k[1] for k in keys[:p.K - 1]]


@pytest.mark.parametrize("C,shape,window,K,stride", [
    (1, (17, 19), 5, 8, 3), (3, (16, 21), 7, 8, 2), (3, (13, 13), 31, 16, 3), (1, (12, 30), 6, 4, 4)])
def test_block_matching_equals_brute_force(C, shape, window, K, stride):
    rng = np.random.default_rng(11)
    img = rng.integers(0, 256, size=shape + (C,), dtype=np.uint8)
    p = O.Params(ps=4, stride=stride, window=window, K=K)
    idx, _ = O.block_match(img, p)
    ys = O.reference_positions(shape[0], 4, stride)
    xs = O.reference_positions(shape[1], 4, stride)
    n = 0
    for ry in ys:
        for rx in xs:
            assert list(idx[n]) == _brute_force_match(img, int(ry), int(rx), p)
            n += 1


def test_block_matching_ties_break_by_lowest_index():
    tile = np.random.default_rng(2).integers(0, 256, size=(4, 4), dtype=np.uint8)
    img = np.tile(tile, (5, 5))[:, :, None]             # many exact duplicates -> SSD ties at 0
    p = O.Params(ps=4, stride=4, window=9, K=8)
    idx, _ = O.block_match(img, p)
    for row in idx:
        W = img.shape[1]
        assert row[0] == idx[list(idx[:, 0]).index(row[0]), 0]
        zeros = [v for v in row[1:]]
        assert zeros == sorted(zeros)                   # all SSD = 0 -> ascending linear index
    # the same through brute force
    assert list(idx[7]) == _brute_force_match(img, int(idx[7, 0] // 20), int(idx[7, 0] % 20), p)


def test_gcp_rule_switches_plane():
    p = np.zeros((4, 4, 3), dtype=np.uint8)
    p[:, :, 0], p[:, :, 1], p[:, :, 2] = 100, 90, 50      # 1.44*90^2 = 11664 >= 10000 -> green
    assert O.gcp_uses_green(p, 0, 0, 4, 1.2)
    p[:, :, 1] = 80                                       # 1.44*80^2 = 9216 < 10000 -> average
    assert not O.gcp_uses_green(p, 0, 0, 4, 1.2)
    p[:, :, 1] = 84                                       # 1.44*7056 = 10160.6 >= 10000 but B large
    p[:, :, 2] = 101
    assert not O.gcp_uses_green(p, 0, 0, 4, 1.2)


def test_reference_grid_and_window():
    assert len(O.reference_positions(128, 8, 3)) == 41
    assert len(O.reference_positions(512, 8, 2)) == 253
    assert len(O.reference_positions(2160, 8, 3)) == 719
    assert len(O.reference_positions(3840, 8, 3)) == 1279
    assert list(O.reference_positions(20, 8, 5)) == [0, 5, 10, 12]
    assert O.window_range(0, 100, 8, 31) == (0, 31)
    assert O.window_range(50, 100, 8, 31) == (35, 31)
    assert O.window_range(92, 100, 8, 31) == (62, 31)
    assert O.window_range(3, 20, 8, 31) == (0, 13)


# ---------------------------------------------------------------- whole filter (Alg. 1)

@pytest.mark.parametrize("C", [1, 3])
def test_zero_threshold_is_identity(C):
    clean = synth.clean_image(24, 26, C, 9)
    noisy = synth.add_gaussian(clean, 20.0, 9)
    r = O.denoise(noisy, 0.0, dict(ps=8, stride=3, window=9, K=8))
    np.testing.assert_allclose(r.out, noisy.astype(float), atol=1e-10)


def test_infinite_threshold_gives_zero():
    noisy = synth.add_gaussian(synth.clean_image(24, 24, 3, 9), 20.0, 9)
    r = O.denoise(noisy, 1e30, dict(ps=8, stride=3, window=9, K=8))
    assert np.abs(r.out).max() == 0.0


def test_constant_image_is_fixed_point():
    img = np.full((24, 24, 3), 77, dtype=np.uint8)
    r = O.denoise(img, 25.0, dict(ps=8, stride=3, window=9, K=8))
    np.testing.assert_allclose(r.out, 77.0, atol=1e-9)


def test_strict_basis_raises_on_coinciding_eigenvalues():
    """Reading R7: a constant image has rank-one slice scatter matrices (seven eigenvalues 0 in slice 0,
    all eight 0 in the colour slice), so its eigenvectors are not unique; strict mode refuses it, the
    default mode runs."""
    img = np.full((24, 24, 3), 77, dtype=np.uint8)
    prm = dict(ps=8, stride=3, window=9, K=8)
    with pytest.raises(O.DegenerateBasis):
        O.denoise(img, 25.0, dict(prm, strict_basis=True))
    r = O.denoise(img, 25.0, prm)
    assert r.extra["basis_gap"] == 0.0
    U, V, lu, lv = O.global_basis(O.reference_patches(img, O.Params.of(prm)))
    assert np.count_nonzero(np.abs(lu[0]) > 1e-6 * lu[0].max()) == 1


def test_basis_gap_of_a_noisy_image_is_far_from_degenerate():
    """Distinct eigenvalues: the gap equals the smallest spacing of the textbook (numpy eigvalsh)
    eigenvalues of the row and column scatter matrices of a gray image (C = 1 reduces the t-SVD to
    the 2-D SVD), and it is far above the 1e-9 threshold."""
    clean = synth.clean_image(64, 64, 1, 9)
    img = synth.add_gaussian(clean, 20.0, 9)
    p = O.Params.of(dict(ps=8, stride=3, window=9, K=8))
    P = O.reference_patches(img, p)[..., 0].astype(np.float64)
    A = np.einsum("nab,ncb->ac", P, P)
    B = np.einsum("nab,nac->bc", P, P)
    want = min(O.basis_gap(np.linalg.eigvalsh(A)), O.basis_gap(np.linalg.eigvalsh(B)))
    r = O.denoise(img, 20.0, dict(ps=8, stride=3, window=9, K=8, strict_basis=True))
    assert abs(r.extra["basis_gap"] - want) <= 1e-9 * want
    assert r.extra["basis_gap"] > 1e-6


def test_aggregation_denominator_counts_covering_patches():
    noisy = synth.add_gaussian(synth.clean_image(20, 22, 1, 4), 20.0, 4)
    p = O.Params(ps=4, stride=3, window=7, K=4)
    idx, _ = O.block_match(noisy, p)
    count = np.zeros((20, 22))
    for row in idx:
        for v in row:
            y, x = divmod(int(v), 22)
            count[y:y + 4, x:x + 4] += 1
    G = O.gather_groups(noisy.astype(float), idx, 4)
    _, den = O.aggregate(noisy.shape, idx, G, np.ones(len(idx)), 4)
    np.testing.assert_array_equal(den, count)
    assert den.min() >= 1


def test_denoiser_improves_psnr_on_gray_workload():
    clean, noisy, sigma, prm = synth.workload_gray128()
    r = O.denoise(noisy, sigma, prm)
    assert synth.psnr(r.out, clean) > synth.psnr(noisy, clean) + 6.0


def test_default_threshold_multiplier():
    assert abs(O.tau_multiplier(O.Params(ps=8, K=32), 3) - 4.176896) < 1e-6
    assert abs(O.tau_multiplier(O.Params(ps=8, K=16, tau_mult=2.7), 1) - 2.7) == 0


def test_sparsity_weights():
    noisy = synth.add_gaussian(synth.clean_image(24, 24, 1, 4), 20.0, 4)
    r = O.denoise(noisy, 20.0, dict(ps=8, stride=3, window=9, K=8, agg_mode="sparsity"), keep_masks=True)
    kept = r.masks.reshape(len(r.idx), -1).sum(axis=1)
    np.testing.assert_allclose(r.weights, 1.0 / np.maximum(1, kept))


# ---------------------------------------------------------------- circulant eigen-analysis (Sec. III-B.2, III-D)

def _circ(G):
    K = G.shape[0]
    p = G.reshape(K, -1)
    return np.vstack([np.concatenate([p[(i - j) % K] for j in range(K)]) for i in range(K)])


def test_circulant_eigenvalues_closed_form():
    rng = np.random.default_rng(4)
    G = rng.integers(0, 256, size=(8, 3, 3, 2)).astype(float)
    C = _circ(G)
    dense = np.sort(np.linalg.eigvalsh(C @ C.T))
    lam = O.circulant_eigenvalues(G)
    np.testing.assert_allclose(np.sort(lam), dense, rtol=1e-10)
    p = G.reshape(8, -1)
    np.testing.assert_allclose(lam[0], np.sum(p.sum(axis=0) ** 2))                            # Eq. (first eigen)
    np.testing.assert_allclose(lam[4], np.sum((((-1.0) ** np.arange(8))[:, None] * p).sum(0) ** 2))  # Eq. (other eigenvalue)
    assert lam[0] == lam.max()                          # non-negative data: lambda_max = ||sum p||^2


def test_rank_position_extremes():
    base = np.random.default_rng(5).integers(0, 256, size=(4, 4, 1)).astype(float)
    smooth = np.stack([base + 0.01 * k for k in range(8)])         # nearly identical patches
    assert O.rank_position(smooth) <= 4
    alt = np.stack([base if k % 2 == 0 else 255 - base for k in range(8)])
    # alternating patches: only lambda_0 and lambda_{K/2} are non-zero and lambda_0 = ||sum p||^2 is the
    # larger for non-negative data, so lambda_hat is the second largest (rank K-1), cf. Fig. (change lambda)
    assert O.rank_position(alt) == 7


# ---------------------------------------------------------------- noise level estimate

@pytest.mark.parametrize("sigma", [5.0, 10.0, 25.0])
def test_sigma_estimate_recovers_pure_noise(sigma):
    rng = np.random.default_rng(int(sigma))
    img = np.clip(np.rint(128 + sigma * rng.standard_normal((256, 256, 1))), 0, 255).astype(np.uint8)
    s = O.estimate_sigma(img, dict(ps=8, stride=2))
    assert abs(s - math.sqrt(sigma ** 2 + 1 / 12)) / sigma < 0.02


def test_sigma_estimate_rgb_pure_noise():
    rng = np.random.default_rng(8)
    img = np.clip(np.rint(128 + 10 * rng.standard_normal((256, 256, 3))), 0, 255).astype(np.uint8)
    s = O.estimate_sigma(img, dict(ps=8, stride=2))
    assert abs(s - 10.0) / 10.0 < 0.02


def test_sigma_rule_on_constructed_spectrum():
    lam = np.concatenate([np.full(50, 4.0), np.linspace(30, 900, 14)])
    assert abs(O.sigma_from_eigenvalues(lam) - 2.0) < 1e-12


def _ramp_zone_image(n=256, stride=4, seed=5):
    """Gray image for the vote-direction pin, high side: random texture everywhere except a 14 x 14 zone
    around every sampled reference (every 8th reference per axis) holding I = 20 + x' + 17 y' in zone
    coordinates. Window 7 (offsets -3..3) keeps every candidate patch of a sampled reference inside its
    zone, where a candidate at offset (dy, dx) is the reference patch plus the constant dx + 17 dy, so
    its SSD is 64 (dx + 17 dy)^2: the three nearest are dx = -1, +1, -2 in that order (equal SSD ->
    lowest index), dy = 0. The texture elsewhere makes the patch covariance full rank (sigma_est > 0)."""
    rng = np.random.default_rng(seed)
    img = rng.integers(0, 256, size=(n, n)).astype(np.int64)
    ys = O.reference_positions(n, 8, stride)[::8]
    for Y0 in ys:
        for X0 in ys:
            y0, x0 = int(Y0) - 3, int(X0) - 3
            for y in range(max(0, y0), min(n, y0 + 14)):
                for x in range(max(0, x0), min(n, x0 + 14)):
                    img[y, x] = 20 + (x - x0) + 17 * (y - y0)
    return img.astype(np.uint8)[:, :, None]


def test_adaptive_vote_divides_when_every_group_ranks_low():
    """Eq. (adjust noise level): sigma_hat = sigma_est / beta when a <= gamma wins the vote. An image tiled
    with one random 8 x 8 texture has, in a window of 25, at least 3 x 3 exact copies of every reference
    patch, so with K = 8 every group is 8 identical patches: lambda_f = 0 for f != 0, hence
    a = 1 + #{f : lambda_f < lambda_4 = 0} = 1 <= gamma = round(13 * 8 / 32) = 3 for every sampled group."""
    tex = np.random.default_rng(11).integers(0, 256, size=(8, 8)).astype(np.uint8)
    img = np.tile(tex, (8, 8))[:, :, None]
    prm = dict(ps=8, stride=3, window=25, K=8)
    p = O.Params.of(prm)
    for ry in O.reference_positions(64, 8, 3)[::8]:
        for rx in O.reference_positions(64, 8, 3)[::8]:
            idx, _, _ = O.block_match_one(img, int(ry), int(rx), p)
            G = O.gather_groups(img, idx[None], 8)[0]
            assert (G == G[0]).all()                      # 8 identical patches
    s_est = O.estimate_sigma(img, prm)
    s_hat, d = O.estimate_sigma(img, dict(prm, adapt=True), return_details=True)
    assert s_est > 1.0
    assert (d["ranks"] == 1).all() and d["high"] == 0
    assert s_hat == s_est / 1.2


def test_adaptive_vote_keeps_sigma_when_groups_rank_high():
    """High side of Eq. (adjust noise level): with K = 4 an interior sampled group is p, p - 1, p + 1, p - 2
    (constants added to one patch p; see _ramp_zone_image), so lambda_2 = 64 (0 + 1 + 1 + 2)^2 = 1024
    exceeds lambda_1 = lambda_3 = 64 ((0 - 1)^2 + (-1 + 2)^2) = 128 and a >= 3 > gamma = round(13 * 4 / 32)
    = 2. Only the sampled references on the first row or column (window clamped at the border) can rank
    low, so a > gamma wins the vote and sigma is left as estimated."""
    img = _ramp_zone_image()
    prm = dict(ps=8, stride=4, window=7, K=4)
    p = O.Params.of(prm)
    idx, _, _ = O.block_match_one(img, 32, 32, p)
    assert (idx - (32 * 256 + 32)).tolist() == [0, -1, 1, -2]
    lam = O.circulant_eigenvalues(O.gather_groups(img, idx[None], 8)[0])
    assert abs(lam[2] - 1024.0) < 1e-6 and abs(lam[1] - 128.0) < 1e-6 and abs(lam[3] - 128.0) < 1e-6
    s_est = O.estimate_sigma(img, prm)
    s_hat, d = O.estimate_sigma(img, dict(prm, adapt=True), return_details=True)
    assert s_est > 1.0
    n_border = 2 * 8 - 1                                 # sampled references with y = 0 or x = 0
    assert d["high"] >= len(d["ranks"]) - n_border > d["low"]
    assert s_hat == s_est


# ---------------------------------------------------------------- frozen-mask map and its adjoint

def _frozen_problem(C=1, seed=6):
    clean = synth.clean_image(16, 18, C, seed)
    x = synth.add_gaussian_float(clean, 20.0, seed).astype(np.float64)
    p = O.Params(ps=4, stride=2, window=7, K=4)
    r = O.denoise(x, 20.0, p, keep_masks=True)
    w = np.random.default_rng(seed).uniform(0.5, 1.5, size=len(r.idx))
    return x, r, w, p


@pytest.mark.parametrize("C", [1, 3])
def test_frozen_map_is_linear_and_adjoint_dot_product(C):
    x, r, w, p = _frozen_problem(C)
    rng = np.random.default_rng(1)
    v, u = rng.standard_normal(x.shape), rng.standard_normal(x.shape)
    f = lambda z: O.denoise_fixed(z, r.idx, r.masks, r.U, r.V, w, p.ps)[0]
    np.testing.assert_allclose(f(2 * v + x), 2 * f(v) + f(x), atol=1e-9)
    gx, _ = O.denoise_fixed_vjp(x, u, r.idx, r.masks, r.U, r.V, w, p.ps)
    assert abs(np.sum(f(v) * u) - np.sum(v * O.denoise_fixed_vjp(v, u, r.idx, r.masks, r.U, r.V, w, p.ps)[0])) < 1e-8
    assert abs(np.sum(f(v) * u) - np.sum(v * gx)) < 1e-8


def test_frozen_map_gradients_match_central_differences():
    x, r, w, p = _frozen_problem(3)
    u = np.random.default_rng(2).standard_normal(x.shape)
    L = lambda z, ww: float(np.sum(O.denoise_fixed(z, r.idx, r.masks, r.U, r.V, ww, p.ps)[0] * u))
    gx, gw = O.denoise_fixed_vjp(x, u, r.idx, r.masks, r.U, r.V, w, p.ps)
    h = 1e-3
    rng = np.random.default_rng(3)
    for _ in range(6):
        pos = tuple(int(rng.integers(0, s)) for s in x.shape)
        e = np.zeros_like(x)
        e[pos] = h
        fd = (L(x + e, w) - L(x - e, w)) / (2 * h)
        assert abs(fd - gx[pos]) < 1e-7 * max(1, abs(fd))
    for g in rng.integers(0, len(w), size=6):
        e = np.zeros_like(w)
        e[g] = h
        fd = (L(x, w + e) - L(x, w - e)) / (2 * h)
        assert abs(fd - gw[g]) < 1e-6 * max(1, abs(fd))


# ---------------------------------------------------------------- A-Haar-tSVD (Alg. 2), reading R15

@pytest.mark.parametrize("n,sub", [(100, 30), (64, 64), (50, 64), (129, 8), (512, 256)])
def test_subimage_bounds_tile_the_axis(n, sub):
    b = O.subimage_bounds(n, sub)
    assert b[0][0] == 0 and b[-1][1] == n
    assert all(b[i][1] == b[i + 1][0] for i in range(len(b) - 1))
    assert len(b) == max(1, n // sub)
    if n >= sub:
        assert all(e - s >= sub for s, e in b)


def test_a_haar_tsvd_single_subimage_is_alg1_with_estimated_sigma():
    """With one subimage, Alg. 2 is Alg. 1 at the image's own estimate."""
    x = synth.add_gaussian(synth.clean_image(40, 48, 3, 21), 15.0, 21)
    p = dict(ps=8, stride=4, window=9, K=8, adapt=True)
    out, sig = O.a_haar_tsvd(x, 64, 64, p)
    s0 = O.estimate_sigma(x, p)
    assert sig.shape == (1,) and sig[0] == s0
    np.testing.assert_array_equal(out, O.denoise(x, s0, p).out)


def test_a_haar_tsvd_estimates_each_subimage_on_its_own():
    """Left half sigma 6, right half sigma 30: the two subimage estimates follow their own
    noise, and each output half is Alg. 1 on that half alone at its estimate."""
    clean = synth.clean_image(96, 192, 1, 22)
    left = synth.add_gaussian(clean[:, :96], 6.0, 22)
    right = synth.add_gaussian(clean[:, 96:], 30.0, 23)
    x = np.ascontiguousarray(np.concatenate([left, right], axis=1))
    p = dict(ps=8, stride=2, window=11, K=8)
    out, sig = O.a_haar_tsvd(x, 96, 96, p)
    assert sig.shape == (2,)
    # (clipping to [0, 255] and the small sample bias the high-noise estimate low)
    assert 4.0 < sig[0] < 8.5 and 20.0 < sig[1] < 36.0 and sig[1] > 3.0 * sig[0]
    np.testing.assert_array_equal(out[:, 96:], O.denoise(np.ascontiguousarray(x[:, 96:]), sig[1], p).out)


# ---------------------------------------------------------------- video (reading R16)

def _clip(F, H, W, C, seed, sigma=15.0):
    return np.stack([synth.add_gaussian(synth.clean_image(H, W, C, seed=seed), sigma, seed=seed + 100 + t)
                     for t in range(F)])


@pytest.mark.parametrize("C", [3, 1])
def test_video_without_temporal_search_is_the_image_denoiser_per_frame(C):
    clip = _clip(3, 24, 20, C, seed=5)
    prm = dict(ps=8, stride=3, window=9, K=8)
    out, res = O.denoise_video(clip, 20.0, prm, T=0)
    for t in range(3):
        r = O.denoise(clip[t], 20.0, prm)
        assert np.array_equal(out[t], r.out)
        assert np.array_equal(res[t].idx - t * 24 * 20, r.idx)


@pytest.mark.parametrize("C,mode", [(3, "gcp"), (3, "full"), (1, "auto")])
def test_video_grouping_against_brute_force(C, mode):
    """Every candidate of every frame in reach enumerated with plain loops: SSD on the plane the
    reference patch selects, keys (SSD, global index), the reference itself excluded."""
    F, H, W, ps = 3, 15, 13, 8
    clip = _clip(F, H, W, C, seed=9, sigma=30.0)
    prm = O.Params.of(dict(ps=ps, stride=3, window=5, K=6, match_mode=mode))
    T = 1
    for t in range(F):
        idx, green = O.block_match_video(clip, t, prm, T)
        ys = O.reference_positions(H, ps, 3)
        xs = O.reference_positions(W, ps, 3)
        n = 0
        for ry in ys:
            for rx in xs:
                y0, ny = O.window_range(int(ry), H, ps, 5)
                x0, nx = O.window_range(int(rx), W, ps, 5)
                x = clip.astype(np.int64)
                ref = x[t, ry:ry + ps, rx:rx + ps, :]
                if C == 1:
                    planes = [0]
                    use_sum = False
                elif mode == "full":
                    planes, use_sum = [0, 1, 2], False
                else:
                    g2 = int((ref[:, :, 1] ** 2).sum())
                    r2, b2 = int((ref[:, :, 0] ** 2).sum()), int((ref[:, :, 2] ** 2).sum())
                    gg = 1.2 * 1.2
                    use_sum = not (gg * g2 >= r2 and gg * g2 >= b2)
                    planes = [1]
                keys = []
                for f in range(max(0, t - T), min(F - 1, t + T) + 1):
                    for y in range(y0, y0 + ny):
                        for xx in range(x0, x0 + nx):
                            if f == t and y == ry and xx == rx:
                                continue
                            cand = x[f, y:y + ps, xx:xx + ps, :]
                            if use_sum:
                                d = int(((cand.sum(axis=2) - ref.sum(axis=2)) ** 2).sum())
                            else:
                                d = sum(int(((cand[:, :, c] - ref[:, :, c]) ** 2).sum()) for c in planes)
                            keys.append((d, f * H * W + y * W + xx))
                keys.sort()
                want = [t * H * W + ry * W + rx] + [k[1] for k in keys[:5]]
                assert list(idx[n]) == want, (t, ry, rx)
                n += 1


def test_video_output_depends_only_on_frames_in_reach():
    clip = _clip(5, 20, 18, 3, seed=21)
    prm = dict(ps=8, stride=3, window=7, K=8)
    a, _ = O.denoise_video(clip, 18.0, prm, T=1)
    other = clip.copy()
    other[4] = synth.add_gaussian(synth.clean_image(20, 18, 3, seed=99), 18.0, seed=7)
    b, _ = O.denoise_video(other, 18.0, prm, T=1)
    for t in range(3):                                  # frames 0..2 cannot reach frame 4
        assert np.array_equal(a[t], b[t])
    assert not np.array_equal(a[3], b[3])


def test_video_zero_threshold_reproduces_the_clip():
    clip = _clip(3, 20, 18, 3, seed=31)
    out, _ = O.denoise_video(clip, 0.0, dict(ps=8, stride=3, window=7, K=8), T=1)
    np.testing.assert_allclose(out, clip.astype(np.float64), rtol=0, atol=1e-9)


def test_video_static_clip_groups_the_reference_copies_first():
    """With identical frames the reference's own copies in frames t-1 and t+1 have distance 0,
    the smallest possible, and come first in global-index order (a textured noisy frame has no
    other zero-distance candidate)."""
    frame = synth.add_gaussian(synth.clean_image(24, 22, 3, seed=41), 25.0, seed=42)
    clip = np.stack([frame] * 3)
    H, W = 24, 22
    idx, _ = O.block_match_video(clip, 1, dict(ps=8, stride=3, window=9, K=8), T=1)
    ref = idx[:, 0] - H * W
    np.testing.assert_array_equal(idx[:, 1], ref)                # frame 0 copy
    np.testing.assert_array_equal(idx[:, 2], ref + 2 * H * W)    # frame 2 copy


# ---------------------------------------------------------------- SURE threshold selection (reading R17)

def _probe(shape, seed):
    return np.random.default_rng(seed).choice([-1.0, 1.0], size=shape)


def test_sure_closed_forms_at_zero_and_infinite_threshold():
    """tau = 0 keeps every coefficient: f(y) = y and J = I, so SURE = -sigma^2 + 2 sigma^2 b^T b / n
    = sigma^2 for a +-1 probe. A threshold above every coefficient gives f = 0 and J = 0, so
    SURE = ||y||^2 / n - sigma^2."""
    y = synth.add_gaussian_float(synth.clean_image(24, 26, 3, 61), 20.0, 62)
    prm = dict(ps=8, stride=3, window=7, K=8)
    b = _probe(y.shape, 63)
    s0, sbig = O.sure(y, 20.0, [1e-12, 1e6], b, prm)
    assert s0 == pytest.approx(20.0 ** 2, rel=1e-9)
    assert sbig == pytest.approx((y.astype(np.float64) ** 2).mean() - 20.0 ** 2, rel=1e-12)
    # finite-difference form: f(z) = z at tau = 0, so the divergence is b^T (z - y) / eps = n up to
    # the float32 rounding of z (|z - y - eps b| <= 2^-24 |z| per entry)
    s0, sbig = O.sure(y, 20.0, [1e-12, 1e6], b, prm, eps=2.0)
    assert s0 == pytest.approx(20.0 ** 2, rel=1e-5)
    assert sbig == pytest.approx((y.astype(np.float64) ** 2).mean() - 20.0 ** 2, rel=1e-12)


def test_sure_finite_difference_tracks_the_true_risk():
    """Stein's lemma: on Gaussian noise the expectation of SURE is the mean squared error against the
    clean image. The finite-difference form counts the threshold's jumps and the bases' dependence
    on y and lands within 15% of the error; the frozen-mask form counts neither and falls below it."""
    x = synth.clean_image(64, 64, 3, 101).astype(np.float64)
    y = synth.add_gaussian_float(synth.clean_image(64, 64, 3, 101), 20.0, 102)
    b = _probe(y.shape, 103)
    prm = dict(ps=8, stride=3, window=9, K=16)
    ms = [1.5, 2.7]
    fd = O.sure(y, 20.0, ms, b, prm, eps=2.0)
    frozen = O.sure(y, 20.0, ms, b, prm)
    for m, a, c in zip(ms, fd, frozen):
        mse = ((O.denoise(y.astype(np.float64), 20.0, O.Params.of(dict(prm, tau_mult=m))).out - x) ** 2).mean()
        assert a == pytest.approx(mse, rel=0.15)
        assert c < mse
    assert fd[1] < fd[0]     # the larger threshold is the better one here, and SURE says so


def test_sure_divergence_is_the_trace_of_the_frozen_map():
    """Summing b^T J^T b over the unit probes e_i gives trace J, computed here column by column from
    the frozen-mask map itself (a linear map in its input)."""
    y = synth.add_gaussian_float(synth.clean_image(12, 12, 1, 71), 25.0, 72)
    prm = O.Params.of(dict(ps=8, stride=2, window=5, K=4, tau_mult=2.0))
    r = O.denoise(y, 25.0, prm, keep_masks=True)
    n = y.size
    tr_cols = 0.0
    tr_vjp = 0.0
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        e = e.reshape(y.shape[0], y.shape[1], 1)
        col, _ = O.denoise_fixed(e, r.idx, r.masks, r.U, r.V, r.weights, prm.ps)
        tr_cols += col.ravel()[i]
        gx, _ = O.denoise_fixed_vjp(y, e, r.idx, r.masks, r.U, r.V, r.weights, prm.ps)
        tr_vjp += gx.ravel()[i]
    assert tr_vjp == pytest.approx(tr_cols, rel=1e-10)
    assert 0.0 < tr_cols < n


# ---------------------------------------------------------------- hyperspectral cubes (reading R18)

def _cube(H, W, N, seed, sigma=12.0):
    """A smooth cube whose bands are affine in one clean image, plus Gaussian noise, as uint8."""
    rng = np.random.default_rng(seed)
    g = synth.clean_image(H, W, 1, seed)[:, :, 0].astype(np.float64)
    cube = np.stack([g * (0.6 + 0.08 * b) + 9.0 * b for b in range(N)], axis=2)
    return np.clip(np.rint(cube + rng.normal(0.0, sigma, cube.shape)), 0, 255).astype(np.uint8)


def test_hsi_auto_matching_is_the_ssd_over_all_bands():
    img = np.random.default_rng(31).integers(0, 256, size=(13, 15, 5), dtype=np.uint8)
    p = O.Params(ps=4, stride=3, window=6, K=8)
    idx, _ = O.block_match(img, p)
    H, W, N = img.shape
    im = img.astype(int).tolist()
    n = 0
    for ry in O.reference_positions(H, 4, 3):
        for rx in O.reference_positions(W, 4, 3):
            ry, rx = int(ry), int(rx)
            ys = range(min(max(ry - 2, 0), H - 4 - 5), min(max(ry - 2, 0), H - 4 - 5) + 6)
            xs = range(min(max(rx - 2, 0), W - 4 - 5), min(max(rx - 2, 0), W - 4 - 5) + 6)
            keys = []
            for y in ys:
                for x in xs:
                    if (y, x) != (ry, rx):
                        d = sum((im[ry + i][rx + j][b] - im[y + i][x + j][b]) ** 2
                                for i in range(4) for j in range(4) for b in range(N))
                        keys.append((d, y * W + x))
            keys.sort()
            assert list(idx[n]) == [ry * W + rx] + [k[1] for k in keys[:7]]
            n += 1


def test_hsi_denoiser_commutes_with_a_cyclic_shift_of_the_bands():
    """The t-SVD is built on circulant structure along the band mode: a cyclic shift of the bands
    multiplies every Fourier slice by a phase, which leaves the scatter matrices and so the bases
    unchanged, and the inverse band transform turns the phase back into the shift."""
    y = _cube(30, 34, 6, 41)
    prm = dict(ps=8, stride=3, window=9, K=8, tau_mult=2.7)
    a = O.denoise(y, 12.0, prm).out
    for s in (1, 4):
        b = O.denoise(np.roll(y, s, axis=2), 12.0, prm).out
        assert np.abs(b - np.roll(a, s, axis=2)).max() <= 1e-9


def test_hsi_identical_bands_reduce_to_the_gray_denoiser():
    """N equal bands put all energy in Fourier slice 0, whose scatter matrices are N^2 times the gray
    ones (same bases), and the inverse band transform returns the gray coefficients in every band;
    the all-band SSD is N times the gray SSD (same groups). With one multiplier for both, every band
    of the result is the gray result."""
    g = _cube(28, 31, 1, 43)
    prm = dict(ps=8, stride=3, window=9, K=8, tau_mult=2.7)
    r1 = O.denoise(g, 12.0, prm).out
    rN = O.denoise(np.repeat(g, 5, axis=2), 12.0, prm).out
    assert np.abs(rN - np.repeat(r1, 5, axis=2)).max() <= 1e-9


def test_hsi_zero_threshold_is_the_identity_and_rgb_modes_refuse_cubes():
    y = _cube(24, 26, 7, 47)
    out = O.denoise(y, 12.0, dict(ps=8, stride=3, window=7, K=4, tau_mult=1e-12)).out
    assert np.abs(out - y).max() <= 1e-9
    for mode in ("gcp", "gray"):
        with pytest.raises(ValueError):
            O.block_match(y, O.Params(ps=8, stride=3, window=7, K=4, match_mode=mode))


# ----------------------------------------------------------------------------- weight tuning (reading R19)

def _sure_w_case(seed=7, sigma=20.0):
    clean = synth.clean_image(40, 44, 3, seed)
    y = synth.add_gaussian_float(clean, sigma, seed).astype(np.float32)
    rng = np.random.default_rng(seed + 1)
    b = rng.choice([-1.0, 1.0], size=y.shape).astype(np.float32)
    prm = dict(ps=8, stride=3, window=9, K=8)
    n = len(O.reference_positions(40, 8, 3)) * len(O.reference_positions(44, 8, 3))
    return clean, y, b, prm, rng.uniform(0.5, 1.5, n), rng


def test_sure_weight_gradient_matches_central_differences():
    """SURE(w) is a ratio of sums linear in w with masks independent of w, so its central difference
    along any direction converges to <grad, d> (a dropped term of the gradient, its z part or a sign
    in the cotangent, fails this)."""
    clean, y, b, prm, w, rng = _sure_w_case()
    _, g = O.sure_weights(y, 20.0, w, b, prm, eps=2.0)
    for _ in range(3):
        d = rng.standard_normal(w.size)
        h = 1e-5
        sp, _ = O.sure_weights(y, 20.0, w + h * d, b, prm, eps=2.0)
        sm, _ = O.sure_weights(y, 20.0, w - h * d, b, prm, eps=2.0)
        fd, ad = (sp - sm) / (2 * h), float(g @ d)
        assert abs(fd - ad) <= 1e-5 * max(1.0, abs(ad)), (fd, ad)


def test_sure_weights_are_scale_free():
    """f_w = N_w / D_w does not change when every weight is scaled, so SURE(c w) = SURE(w) and, by
    Euler's identity for a function homogeneous of degree 0, sum_g w_g dSURE/dw_g = 0."""
    clean, y, b, prm, w, rng = _sure_w_case(11)
    s1, g = O.sure_weights(y, 20.0, w, b, prm, eps=2.0)
    s2, g2 = O.sure_weights(y, 20.0, 3.5 * w, b, prm, eps=2.0)
    assert abs(s1 - s2) <= 1e-9 * abs(s1)
    assert abs(float(w @ g)) <= 1e-9 * float(np.abs(w * g).sum())
    np.testing.assert_allclose(g2 * 3.5, g, rtol=1e-7, atol=1e-12)      # grad scales as 1 / c


def test_sure_weights_do_not_matter_at_zero_threshold():
    """At tau = 0 every coefficient is kept and each group returns its own patches, so f_w(x) = x for
    any w: SURE is sigma^2 (2 / eps) b^T (z - y) / n - sigma^2 and its gradient vanishes."""
    clean, y, b, prm, w, rng = _sure_w_case(13)
    prm = dict(prm, tau_mult=1e-12)
    s, g = O.sure_weights(y, 20.0, w, b, prm, eps=2.0)
    z = O.perturbed(y, b, 2.0)
    n = y.size
    expect = 2.0 * 20.0 ** 2 / (n * 2.0) * float((b.astype(np.float64) * (z - y.astype(np.float64))).sum()) - 20.0 ** 2
    assert abs(s - expect) <= 1e-9 * abs(expect)
    assert np.abs(g).max() <= 1e-10


def test_weight_tuning_lowers_the_risk_estimate():
    """Exponentiated-gradient steps on SURE(w) from uniform weights lower SURE (small steps along
    the negative gradient) and keep every weight positive."""
    clean, y, b, prm, w, rng = _sure_w_case(17)
    wt, trace = O.tune_weights(y, 20.0, b, prm, eps=2.0, steps=3, step=0.3)
    assert np.all(np.diff(trace) < 0), trace
    assert np.all(wt > 0)


# ----------------------------------------------------------------------------- MRI volumes (reading R20)

def _volume(D, Hh, Wd, seed, sigma=11.0):
    return synth.add_gaussian(synth.clean_volume(D, Hh, Wd, seed), sigma, seed)


@pytest.mark.parametrize("spoil", [0.2, 0.004])
def test_volume_grouping_against_brute_force(spoil):
    """Grouping of cubes: exact SSD over the ps^3 voxels of every candidate of the clamped W^3 window,
    written out voxel by voxel in plain Python; a volume with repeated 2 x 2 x 2 tiles, a few voxels
    overwritten, makes many keys tie, which the lowest linear index must break (the sparse case has
    groups whose K - 1 cut falls inside a run of equal keys)."""
    rng = np.random.default_rng(61)
    tile = rng.integers(0, 256, size=(2, 2, 2))
    v = np.tile(tile, (5, 6, 5)).astype(np.int64)
    v[rng.random(v.shape) < spoil] = 9
    v = v.astype(np.uint8)[:9, :11, :10]
    p = O.Params(ps=4, stride=2, window=3, K=6)
    idx = O.block_match_volume(v, p)
    D, Hh, Wd = v.shape
    vv = v.astype(int).tolist()
    n = cut_ties = 0
    for rz in O.reference_positions(D, 4, 2):
        for ry in O.reference_positions(Hh, 4, 2):
            for rx in O.reference_positions(Wd, 4, 2):
                rz, ry, rx = int(rz), int(ry), int(rx)
                st = [min(max(r - 1, 0), n_ - 4 + 1 - 3) for r, n_ in ((rz, D), (ry, Hh), (rx, Wd))]
                keys = []
                for z in range(st[0], st[0] + 3):
                    for y in range(st[1], st[1] + 3):
                        for x in range(st[2], st[2] + 3):
                            if (z, y, x) != (rz, ry, rx):
                                d = sum((vv[rz + c][ry + a][rx + b] - vv[z + c][y + a][x + b]) ** 2
                                        for a in range(4) for b in range(4) for c in range(4))
                                keys.append((d, (z * Hh + y) * Wd + x))
                keys.sort()
                assert list(idx[n]) == [(rz * Hh + ry) * Wd + rx] + [k[1] for k in keys[:5]]
                cut_ties += keys[4][0] == keys[5][0]
                n += 1
    assert n == idx.shape[0]
    if spoil < 0.1:
        assert cut_ties > 0


def test_volume_cube_gather_and_aggregation_counts():
    """A cube is v[z + k, y + i, x + j] at P[i][j][k]; the denominator counts, per voxel, the
    cubes of all groups that cover it (brute force over the placements)."""
    v = np.arange(7 * 8 * 9, dtype=np.int64).reshape(7, 8, 9) % 251
    lin = np.array([(2 * 8 + 3) * 9 + 4])
    P = O.gather_cubes(v.astype(np.uint8), lin, 4)[0]
    for i in range(4):
        for j in range(4):
            for k in range(4):
                assert P[i, j, k] == v[2 + k, 3 + i, 4 + j]
    rng = np.random.default_rng(3)
    idx = rng.integers(0, 4 * 5 * 6, size=(5, 4))
    zz, r = np.divmod(idx, 5 * 6)
    yy, xx = np.divmod(r, 6)
    idx = (zz * 8 + yy) * 9 + xx                                   # top corners with room for the cube
    w = rng.uniform(0.5, 2.0, 5)
    _, den = O.aggregate_volume(v.shape, idx, np.zeros((5, 4, 4, 4, 4)), w, 4)
    ref = np.zeros(v.shape)
    for g in range(5):
        for k in range(4):
            z, rr = divmod(int(idx[g, k]), 8 * 9)
            y, x = divmod(rr, 9)
            ref[z:z + 4, y:y + 4, x:x + 4] += w[g]
    assert np.abs(den - ref).max() <= 1e-12


def test_volume_bases_are_unitary_with_conjugate_tube_slices():
    """Cube bases per tube-Fourier slice (R6 with c = ps = 4): unitary, slice 2 (the Nyquist slice)
    real, slice 3 the conjugate of slice 1, and the t-product U^T * U is the identity tensor."""
    v = _volume(14, 16, 15, 5)
    p = O.Params(ps=4, stride=2, window=5, K=8)
    U, V, _, _ = O.global_basis(O.gather_cubes(v, O.volume_reference_positions(v.shape, p), 4))
    for B in (U, V):
        for f in range(4):
            np.testing.assert_allclose(B[f].conj().T @ B[f], np.eye(4), atol=1e-12)
        assert np.abs(B[0].imag).max() <= 1e-12 and np.abs(B[2].imag).max() <= 1e-12
        np.testing.assert_allclose(B[3], B[1].conj(), atol=0)
        Ut = np.fft.ifft(B, axis=0).real.transpose(1, 2, 0)          # spatial-domain tensor (4, 4, 4)
        I = O.t_product_bcirc(O.t_transpose(Ut), Ut)
        E = np.zeros((4, 4, 4))
        E[:, :, 0] = np.eye(4)
        np.testing.assert_allclose(I, E, atol=1e-12)


def test_volume_zero_and_infinite_threshold():
    v = _volume(12, 13, 14, 7)
    prm = dict(ps=4, stride=2, window=5, K=8)
    assert np.abs(O.denoise_volume(v, 10.0, prm, tau=0.0).out - v).max() <= 1e-9
    assert np.abs(O.denoise_volume(v, 10.0, prm, tau=1e9).out).max() == 0.0


def test_volume_denoiser_commutes_with_transposing_rows_and_columns():
    """Swapping y and x transposes every cube slice: the row and column scatter matrices trade places
    (U_f of the transposed volume is conj(V_f), V_f is conj(U_f)), so every coefficient moves to the
    transposed position and the output is the transposed output. The grouping is held fixed (the
    transposed indices) so that ties of the integer SSD cannot reorder a group."""
    v = _volume(12, 14, 14, 9)
    prm = dict(ps=4, stride=2, window=5, K=8, tau_mult=2.2)
    r = O.denoise_volume(v, 11.0, prm)
    D, Hh, Wd = v.shape
    z, rr = np.divmod(r.idx, Hh * Wd)
    y, x = np.divmod(rr, Wd)
    idx_t = (z * Wd + x) * Hh + y
    # the transposed grid lists the same references in (z, x, y) order: reorder the groups to match
    ng = len(O.reference_positions(Hh, 4, 2))
    order = np.arange(r.idx.shape[0]).reshape(-1, ng, ng).transpose(0, 2, 1).ravel()
    t = O.denoise_volume(np.ascontiguousarray(v.transpose(0, 2, 1)), 11.0, prm, idx=idx_t[order])
    assert np.abs(t.out - r.out.transpose(0, 2, 1)).max() <= 1e-9


def test_volume_denoiser_commutes_with_reversing_the_tube_axis():
    """Reversing z reverses every cube's tube: each tube-Fourier slice becomes a phase times its
    conjugate, so the scatter matrices and bases are conjugated and the coefficients reverse along
    the tube; thresholds keep the same set and the output is the reversed output (grid symmetric:
    (D - ps) divisible by the stride; grouping held fixed as above)."""
    v = _volume(14, 12, 13, 11)
    prm = dict(ps=4, stride=2, window=5, K=8, tau_mult=2.2)
    r = O.denoise_volume(v, 11.0, prm)
    D, Hh, Wd = v.shape
    z, rr = np.divmod(r.idx, Hh * Wd)
    idx_f = (D - 4 - z) * Hh * Wd + rr
    nz = len(O.reference_positions(D, 4, 2))
    order = np.arange(r.idx.shape[0]).reshape(nz, -1)[::-1].ravel()
    f = O.denoise_volume(np.ascontiguousarray(v[::-1]), 11.0, prm, idx=idx_f[order])
    assert np.abs(f.out - r.out[::-1]).max() <= 1e-9


def test_volume_default_threshold_counts_the_cube_voxels():
    """tau = sigma sqrt(2 ln(c K ps^2)) with the tube length c = ps: sqrt(2 ln(ps^3 K))."""
    v = _volume(10, 10, 10, 13)
    r = O.denoise_volume(v, 10.0, dict(ps=4, stride=2, window=5, K=32))
    assert abs(r.tau - 10.0 * math.sqrt(2 * math.log(4 ** 3 * 32))) <= 1e-12


@pytest.mark.parametrize("sigma", [5.0, 10.0])
def test_volume_sigma_estimate_recovers_pure_noise(sigma):
    """Pure Gaussian noise around 128 (no clipping at these levels): the covariance of the reference
    cubes is sigma^2 I up to sampling error, so the rule recovers sigma within 2 %."""
    rng = np.random.default_rng(int(sigma))
    v = np.clip(np.rint(128.0 + sigma * rng.standard_normal((40, 44, 42))), 0, 255).astype(np.uint8)
    s = O.estimate_sigma_volume(v, dict(ps=4, stride=2, window=5, K=8))
    assert abs(s - sigma) <= 0.02 * sigma


def test_volume_sigma_estimate_of_a_noise_free_ramp_is_zero():
    """A linear ramp has a covariance of rank <= 4 (a cube is determined by its corner value and three
    slopes), so at least 60 of its 64 eigenvalues vanish and the rule returns 0."""
    zz, yy, xx = np.mgrid[0:20, 0:22, 0:24]
    v = (10 + 2 * zz + 3 * yy + xx).astype(np.uint8)
    assert O.estimate_sigma_volume(v, dict(ps=4, stride=2, window=5, K=8)) <= 1e-6


def test_adaptive_volume_single_part_is_alg1_with_the_estimated_sigma():
    v = _volume(14, 15, 16, 21)
    prm = dict(ps=4, stride=2, window=5, K=8)
    out, sig = O.a_haar_tsvd_volume(v, (100, 100, 100), prm)
    s = O.estimate_sigma_volume(v, prm)
    assert sig.shape == (1,) and sig[0] == s
    assert np.abs(out - O.denoise_volume(v, s, prm).out).max() == 0.0


def test_adaptive_volume_estimates_each_part_on_its_own():
    """Two halves along z with noise 4 and 16 on a flat volume: each half's estimate follows its own
    level (within 5 %), and each half's output is Alg. 1 of that half alone."""
    rng = np.random.default_rng(22)
    base = np.full((32, 24, 24), 120.0)
    noise = np.concatenate([4.0 * rng.standard_normal((16, 24, 24)), 16.0 * rng.standard_normal((16, 24, 24))])
    v = np.clip(np.rint(base + noise), 0, 255).astype(np.uint8)
    prm = dict(ps=4, stride=2, window=5, K=8)
    out, sig = O.a_haar_tsvd_volume(v, (16, 24, 24), prm)
    assert sig.shape == (2,)
    assert abs(sig[0] - 4.0) <= 0.05 * 4.0 and abs(sig[1] - 16.0) <= 0.05 * 16.0
    lower = np.ascontiguousarray(v[16:])
    assert np.abs(out[16:] - O.denoise_volume(lower, sig[1], prm).out).max() == 0.0


def test_subimage_bounds_are_the_floor_boundaries():
    """Reading R15's boundaries floor(i n / t), worked by hand: a ceiling or rounded variant moves them."""
    assert O.subimage_bounds(41, 20) == [(0, 20), (20, 41)]
    assert O.subimage_bounds(100, 30) == [(0, 33), (33, 66), (66, 100)]
    assert O.subimage_bounds(29, 14) == [(0, 14), (14, 29)]
    assert O.subimage_bounds(26, 13) == [(0, 13), (13, 26)]
    assert O.subimage_bounds(7, 20) == [(0, 7)]


def test_adaptive_volume_places_ragged_parts_where_they_came_from():
    """2 x 1 x 2 ragged parts of a 21 x 12 x 23 volume (bounds worked by hand: z 0|10|21, x 0|11|23):
    every part of the output is Alg. 1 on that part alone at that part's own estimate."""
    v = _volume(21, 12, 23, 23)
    prm = dict(ps=4, stride=2, window=4, K=8)
    out, sig = O.a_haar_tsvd_volume(v, (10, 12, 11), prm)
    assert sig.shape == (4,)
    parts = [((0, 10), (0, 11)), ((0, 10), (11, 23)), ((10, 21), (0, 11)), ((10, 21), (11, 23))]
    for t, ((z0, z1), (x0, x1)) in enumerate(parts):
        part = np.ascontiguousarray(v[z0:z1, :, x0:x1])
        s = O.estimate_sigma_volume(part, prm)
        assert sig[t] == s
        assert np.abs(out[z0:z1, :, x0:x1] - O.denoise_volume(part, s, prm).out).max() == 0.0


def test_rank_gamma_is_13K_over_32_rounded_half_up():
    """Reading R12's default gamma_rank = 13 K / 32 rounded half up, worked by hand (K = 16: 6.5 -> 7)."""
    for K, g in ((2, 1), (4, 2), (8, 3), (16, 7), (32, 13), (64, 26)):
        assert O.rank_gamma(O.Params(K=K)) == g


def test_canonical_phase_takes_the_lowest_index_among_equal_moduli():
    """Reading R7 on matrices whose eigenvectors have two entries of equal modulus (worked by hand):
    [[2, 1], [1, 2]] has (1, 1)/sqrt 2 for 3 and (1, -1)/sqrt 2 for 1; [[2, i], [-i, 2]] has
    (1, -i)/sqrt 2 for 3 and (1, i)/sqrt 2 for 1: the first entry is made real positive."""
    r = 1 / math.sqrt(2)
    w, Q = O.canonical_eigvecs(np.array([[2.0, 1.0], [1.0, 2.0]], dtype=complex))
    assert np.allclose(w, [3.0, 1.0]) and np.allclose(Q, [[r, r], [r, -r]], atol=1e-14)
    w, Q = O.canonical_eigvecs(np.array([[2.0, 1j], [-1j, 2.0]]))
    assert np.allclose(w, [3.0, 1.0]) and np.allclose(Q, [[r, r], [-1j * r, 1j * r]], atol=1e-14)


def test_threshold_keeps_a_coefficient_equal_to_tau():
    """Reading R9: a coefficient whose magnitude equals tau is kept; one ulp below is dropped."""
    tau = 7.25
    below = np.nextafter(tau, 0.0)
    S = np.array([tau, -tau, below, -below, 2 * tau, 0.0])
    assert O.hard_threshold_mask(S, tau).tolist() == [True, True, False, False, True, False]


def test_sigma_rule_takes_the_mean_of_the_largest_qualifying_run():
    """Reading R11 worked by hand. [0.9, 1, 1, 1.05, 40, 90]: the runs r = 1..4 qualify (mean against
    1.02 median: 0.9/0.9, 0.95/0.95, 0.967/1, 0.9875/1), r = 5, 6 do not, so sigma^2 = 0.9875, the run's
    mean (its median is 1). [1] * 4 + [3] * 8: r = 5..7 fail, r = 8..12 qualify again (r = 12: mean
    7/3 <= 1.02 x 3), so r* = 12, the largest qualifying run, not the last before a failure."""
    assert abs(O.sigma_from_eigenvalues(np.array([0.9, 1.0, 1.0, 1.05, 40.0, 90.0])) - math.sqrt(0.9875)) < 1e-12
    assert abs(O.sigma_from_eigenvalues(np.array([1.0] * 4 + [3.0] * 8)) - math.sqrt(7.0 / 3.0)) < 1e-12


def _offset_pair(shape, seed):
    rng = np.random.default_rng(seed)
    base = np.clip(np.rint(60.0 + 25.0 * rng.standard_normal(shape)), 0, 150).astype(np.int64)
    ramp = (np.indices(shape).sum(axis=0) % 7) * 3          # some structure besides the noise
    a = np.clip(base + ramp, 0, 150)
    return a.astype(np.uint8), (a + 100).astype(np.uint8)


def test_sigma_estimate_is_invariant_to_a_constant_offset():
    """The patch covariance is centred (Sec. III-D), so adding a constant to every pixel (no clipping)
    leaves the estimate unchanged; an uncentred second moment would move it."""
    a, b = _offset_pair((96, 104, 3), 31)
    sa, sb = (O.estimate_sigma(x, dict(ps=8, stride=2)) for x in (a, b))
    assert abs(sa - sb) <= 1e-9 * sa


def test_volume_sigma_estimate_is_invariant_to_a_constant_offset():
    a, b = _offset_pair((30, 28, 26), 32)
    prm = dict(ps=4, stride=2, window=5, K=8)
    sa, sb = (O.estimate_sigma_volume(x, prm) for x in (a, b))
    assert abs(sa - sb) <= 1e-9 * sa


def test_float_inputs_are_quantised_by_rounding_to_nearest():
    """Reading R13: q = clip(rint(x)), worked by hand (rint takes halves to even)."""
    x = np.array([[[0.4], [0.6], [254.6], [-3.0]], [[300.0], [2.5], [3.5], [17.49]]])
    assert O._as_quantised(x)[..., 0].tolist() == [[0, 1, 255, 0], [255, 2, 4, 17]]


def test_sparsity_weight_of_a_group_keeping_one_coefficient_is_one():
    """Reading R10: w_g = 1 / max(1, #kept). On a constant image every patch of every group is the same
    constant patch, whose only non-zero coefficient is the DC one (Haar row 0, basis row and column 0),
    so at a small threshold each group keeps exactly one coefficient and its weight is 1."""
    x = np.full((24, 28, 1), 100, dtype=np.uint8)
    r = O.denoise(x, 1.0, dict(ps=8, stride=4, window=9, K=8, tau_mult=1e-3, agg_mode="sparsity"), keep_masks=True)
    assert (r.masks.reshape(r.masks.shape[0], -1).sum(axis=1) == 1).all()
    assert (r.weights == 1.0).all()
    assert np.abs(r.out - 100.0).max() < 1e-9


def test_sparsity_weight_of_a_group_keeping_nothing_is_one():
    """Reading R10's max(1, .): a group that keeps no coefficient still weighs 1 (images and volumes);
    with nothing kept the estimate is zero."""
    x = synth.add_gaussian(synth.clean_image(24, 28, 3, seed=46), 10.0, seed=46)
    r = O.denoise(x, 10.0, dict(ps=8, stride=4, window=9, K=8, tau_mult=1e9, agg_mode="sparsity"))
    assert (r.weights == 1.0).all() and np.abs(r.out).max() == 0.0
    v = _volume(12, 13, 14, 46)
    r = O.denoise_volume(v, 10.0, dict(ps=4, stride=2, window=5, K=8, tau_mult=1e9, agg_mode="sparsity"))
    assert (r.weights == 1.0).all() and np.abs(r.out).max() == 0.0


def test_video_estimates_sigma_frame_by_frame():
    """Reading R16: sigma = None estimates each frame's own level; frames with noise 4 and 16 on the
    same flat frame give estimates in the ratio 4."""
    rng = np.random.default_rng(44)
    base = np.full((96, 96), 120.0)
    clip = np.stack([np.clip(np.rint(base + s * rng.standard_normal(base.shape)), 0, 255) for s in (4.0, 16.0)])
    _, res = O.denoise_video(clip.astype(np.uint8), None, dict(ps=8, stride=4, window=9, K=8), T=0)
    s0, s1 = (r.extra["sigma"] for r in res)
    # 529 reference patches of 64 pixels bias both estimates low alike; their ratio is the noise ratio
    assert abs(s1 / s0 - 4.0) <= 0.05 * 4.0
    assert abs(s0 - 4.0) <= 0.15 * 4.0 and abs(s1 - 16.0) <= 0.15 * 16.0


def test_perturbed_image_is_formed_in_float32():
    """Reading R17: z = y + eps b is formed in float32 with each operation rounded once, so every value
    of z is a float32 number and equals the float32 sum of the float32 product."""
    rng = np.random.default_rng(45)
    y = (255 * rng.random((17, 19, 3))).astype(np.float32)
    b = rng.choice([-1.0, 1.0], size=y.shape) * (1 + rng.random(y.shape))
    z = O.perturbed(y, b, 0.37)
    assert (z.astype(np.float32).astype(np.float64) == z).all()
    assert (z == (y + np.float32(0.37) * b.astype(np.float32)).astype(np.float64)).all()
    assert not (z == y.astype(np.float64) + 0.37 * b).all()


def test_basis_gap_is_relative_to_the_largest_eigenvalue():
    """Reading R7's gap: min |l_i - l_(i+1)| / |l_max|, worked by hand; unchanged by scaling."""
    assert O.basis_gap(np.array([4.0, 1.0, 2.0])) == 0.25
    assert O.basis_gap(np.array([400.0, 100.0, 200.0])) == 0.25
    assert O.basis_gap(np.array([3.0, 3.0, 1.0])) == 0.0


def test_volume_reference_positions_are_z_major():
    """Reading R20: the reference cubes of a 6 x 6 x 6 volume at ps 4, stride 2 (per axis {0, 2}),
    z-major, as linear positions (z H + y) W + x worked by hand."""
    assert O.volume_reference_positions((6, 6, 6), O.Params(ps=4, stride=2)).tolist() == \
        [0, 2, 12, 14, 72, 74, 84, 86]


def test_weight_tuning_step_is_normalised_by_the_largest_gradient():
    """Reading R19's step w <- w exp(-step g / max|g|): from uniform weights one step moves the weight
    with the largest gradient by exactly a factor exp(-+step) and every other weight by less, in the
    direction opposite to its gradient."""
    clean, y, b, prm, w, rng = _sure_w_case(18)
    _, g = O.sure_weights(y, 20.0, np.ones_like(w), b, prm, eps=2.0)
    wt, _ = O.tune_weights(y, 20.0, b, prm, eps=2.0, steps=1, step=0.3)
    lw = np.log(wt)
    assert abs(np.abs(lw).max() - 0.3) < 1e-12
    assert np.argmax(np.abs(lw)) == np.argmax(np.abs(g))
    assert np.all(lw * g <= 0)


def test_reference_patches_in_row_major_grid_order():
    """Reading R3: reference patches of a 10 x 12 image at ps 8, stride 2 (rows {0, 2}, columns
    {0, 2, 4}), row-major, identified by their top-left pixel (the image holds y * 12 + x)."""
    x = (np.arange(10 * 12).reshape(10, 12, 1) % 256).astype(np.uint8)
    P = O.reference_patches(x, O.Params(ps=8, stride=2))
    assert P[:, 0, 0, 0].tolist() == [0, 2, 4, 24, 26, 28]


def test_rgb_green_plane_mode_groups_on_the_green_channel():
    """The green-plane mode on RGB matches on G alone: its grouping is the gray grouping of G."""
    img = synth.add_gaussian(synth.clean_image(40, 44, 3, seed=47), 15.0, seed=47)
    prm = dict(ps=8, stride=3, window=9, K=8)
    idx_rgb, _ = O.block_match(img, O.Params.of(dict(prm, match_mode="gray")))
    idx_g, _ = O.block_match(np.ascontiguousarray(img[:, :, 1:2]), O.Params.of(prm))
    np.testing.assert_array_equal(idx_rgb, idx_g)

"""Host logic of the basis solve (CPU): the library's slice solver, run on the host from
exact integer moments, against the oracle's global bases (numpy eigh on the FFT'd patches)."""
import ctypes

import numpy as np
import pytest

import paper_2508_10307_gb300 as H
from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth


def _moments(P):
    Pi = P.astype(np.int64)
    R = np.einsum("nabc,nxbd->axcd", Pi, Pi, optimize=True)   # sum_r sum_b P[a][b][c] P[a'][b][c']
    Q = np.einsum("nabc,naxd->bxcd", Pi, Pi, optimize=True)   # sum_r sum_a P[a][b][c] P[a][b'][c']
    return np.ascontiguousarray(np.stack([R, Q]).astype(np.uint64))


@pytest.mark.parametrize("C,shape,stride", [(3, (48, 56), 3), (1, (64, 40), 2), (3, (96, 128), 2)])
def test_host_slice_basis_matches_oracle(C, shape, stride):
    lib = H.load_library()
    lib.htsvd_internal_slice_basis.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_void_p]
    lib.htsvd_internal_slice_basis.restype = None
    noisy = synth.add_gaussian(synth.clean_image(shape[0], shape[1], C, 3), 20.0, 3)
    p = O.Params(ps=8, stride=stride, window=15, K=16)
    P = O.reference_patches(noisy, p)
    mom = _moments(P)
    U, V, _, _ = O.global_basis(P.astype(float))
    for which, ref in ((0, U), (1, V)):
        for f in range(C // 2 + 1):
            out = np.zeros(128)
            lib.htsvd_internal_slice_basis(mom.ctypes.data, C, which, f, out.ctypes.data)
            z = (out[0::2] + 1j * out[1::2]).reshape(8, 8)
            assert np.abs(z - ref[f]).max() < 1e-9


def _sigma_hook():
    lib = H.load_library()
    f = lib.htsvd_internal_sigma_from_moments
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_double
    return f


@pytest.mark.parametrize("C,shape,stride,kind", [(3, (64, 72), 3, "natural"), (1, (80, 64), 2, "natural"),
                                                 (3, (40, 48), 1, "flat"), (1, (48, 40), 2, "constant")])
def test_host_sigma_eigenvalues_match_oracle(C, shape, stride, kind):
    """Host tridiagonal-QR eigenvalues of the patch covariance and the sigma rule (Sec. III-D)
    against numpy's eigvalsh and the oracle's estimate, from exact integer moments."""
    f = _sigma_hook()
    if kind == "constant":
        noisy = np.full(shape + (C,), 117, np.uint8)
    else:
        clean = synth.clean_image(shape[0], shape[1], C, 5)
        if kind == "flat":     # low-rank signal: the covariance is dominated by few directions
            clean = np.repeat(clean[:, :1, :], shape[1], axis=1)
        noisy = synth.add_gaussian(clean, 12.0, 5)
    p = O.Params(ps=8, stride=stride, window=15, K=16)
    P = O.reference_patches(noisy, p).reshape(-1, 64 * C).astype(np.int64)
    M = np.ascontiguousarray((P.T @ P).astype(np.uint64))
    S = np.ascontiguousarray(P.sum(axis=0).astype(np.uint64))
    lam = np.zeros(64 * C)
    sig = f(M.ctypes.data, S.ctypes.data, 64 * C, P.shape[0], lam.ctypes.data)
    ref = np.linalg.eigvalsh(O.patch_covariance(noisy, p))
    scale = max(np.abs(ref).max(), 1.0)
    assert np.abs(lam - np.sort(ref)).max() <= 1e-10 * scale
    assert sig == pytest.approx(O.estimate_sigma(noisy, p), rel=1e-9, abs=1e-9)


def test_host_sigma_rejects_bad_args():
    f = _sigma_hook()
    M = np.zeros((64, 64), np.uint64)
    S = np.zeros(64, np.uint64)
    assert f(M.ctypes.data, S.ctypes.data, 64, 0, None) == -1.0
    assert f(None, S.ctypes.data, 64, 5, None) == -1.0


@pytest.mark.parametrize("shape,seed", [((20, 24, 22), 5), ((40, 36, 30), 8)])
def test_host_volume_bases_match_oracle(shape, seed):
    """Bases of the MRI volume path (reading R20), solved on the host from exact integer cube
    moments (4 x 4 Hermitian slices, slice 1 through its real embedding), against the oracle's
    numpy eigh of the tube-Fourier slices of the reference cubes; same canonical phases."""
    lib = H.load_library()
    v = synth.add_gaussian(synth.clean_volume(*shape, seed), 11.0, seed)
    p = O.Params(ps=4, stride=2, window=5, K=8)
    P = O.gather_cubes(v, O.volume_reference_positions(v.shape, p), 4)      # (n, i, j, k)
    mom = _moments(P)
    b = np.zeros(256)
    gap = lib.htsvd_internal_volume_bases(mom.ctypes.data, b.ctypes.data)
    U, V, lu, lv = O.global_basis(P)
    z = (b[0::2] + 1j * b[1::2]).reshape(2, 4, 4, 4)
    assert np.abs(z[0] - U).max() < 1e-9 and np.abs(z[1] - V).max() < 1e-9
    assert abs(gap - O.global_basis_gap(lu, lv)) <= 1e-9 * max(gap, 1e-12)


def test_host_volume_bases_report_a_degenerate_constant_volume():
    """Reading R7 for volumes: a constant volume makes every slice scatter matrix rank one (repeated zero
    eigenvalues), so the smallest relative gap is 0, as the oracle's, and the oracle's strict mode raises."""
    lib = H.load_library()
    v = np.full((12, 13, 14), 77, dtype=np.uint8)
    p = O.Params(ps=4, stride=2, window=5, K=8)
    P = O.gather_cubes(v, O.volume_reference_positions(v.shape, p), 4)
    mom = _moments(P)                      # held: the library reads it through a raw pointer
    b = np.zeros(256)
    gap = lib.htsvd_internal_volume_bases(mom.ctypes.data, b.ctypes.data)
    _, _, lu, lv = O.global_basis(P)
    assert gap == 0.0 and O.global_basis_gap(lu, lv) == 0.0
    with pytest.raises(O.DegenerateBasis):
        O.denoise_volume(v, 5.0, dict(ps=4, stride=2, window=5, K=8, strict_basis=True))


def test_host_volume_bases_take_the_lowest_index_among_equal_moduli():
    """Reading R7's tie rule in the library's 4 x 4 solver: reference cubes closed under swapping rows 0
    and 1 (and columns 0 and 1) make every slice matrix commute with that swap, so its antisymmetric
    eigenvectors have two entries of equal modulus; the first is made real positive, as in the oracle."""
    lib = H.load_library()
    rng = np.random.default_rng(12)
    P0 = rng.integers(0, 256, size=(40, 4, 4, 4)).astype(np.float64)
    Pi = P0[:, [1, 0, 2, 3]]
    P = np.concatenate([P0, Pi, P0[:, :, [1, 0, 2, 3]], Pi[:, :, [1, 0, 2, 3]]])
    mom = _moments(P)                      # held: the library reads it through a raw pointer
    b = np.zeros(256)
    lib.htsvd_internal_volume_bases(mom.ctypes.data, b.ctypes.data)
    U, V, _, _ = O.global_basis(P)
    z = (b[0::2] + 1j * b[1::2]).reshape(2, 4, 4, 4)
    ties = sum(int(np.sum(np.isclose(np.abs(M[f][:, i]), np.abs(M[f][:, i]).max(), rtol=1e-9)) > 1)
               for M in (U, V) for f in range(4) for i in range(4))
    assert ties > 0
    assert np.abs(z[0] - U).max() < 1e-9 and np.abs(z[1] - V).max() < 1e-9


@pytest.mark.parametrize("C", [1, 3])
def test_host_slice_basis_takes_the_lowest_index_among_equal_moduli(C):
    """The image path's slice solver on reference patches closed under swapping rows 0 and 1 (and
    columns 0 and 1): antisymmetric eigenvectors have two entries of equal modulus, and the first is
    made real positive, as in the oracle (reading R7)."""
    lib = H.load_library()
    lib.htsvd_internal_slice_basis.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_void_p]
    lib.htsvd_internal_slice_basis.restype = None
    rng = np.random.default_rng(13 + C)
    sw = [1, 0, 2, 3, 4, 5, 6, 7]
    P0 = rng.integers(0, 256, size=(30, 8, 8, C)).astype(np.int64)
    Pi = P0[:, sw]
    P = np.concatenate([P0, Pi, P0[:, :, sw], Pi[:, :, sw]])
    U, V, _, _ = O.global_basis(P.astype(float))
    mom = _moments(P)
    ties = 0
    for which, ref in ((0, U), (1, V)):
        for f in range(C // 2 + 1):
            out = np.zeros(128)
            lib.htsvd_internal_slice_basis(mom.ctypes.data, C, which, f, out.ctypes.data)
            z = (out[0::2] + 1j * out[1::2]).reshape(8, 8)
            assert np.abs(z - ref[f]).max() < 1e-9
            ties += sum(int(np.sum(np.isclose(np.abs(ref[f][:, i]), np.abs(ref[f][:, i]).max(), rtol=1e-9)) > 1)
                        for i in range(8))
    assert ties > 0

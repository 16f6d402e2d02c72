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

"""Helpers shared by the GPU tests: oracle runs cached per process, mask packing, comparisons."""
from __future__ import annotations

import functools
import math

import numpy as np

from oracle import htsvd_oracle as O
from paper_2508_10307_gb300 import synth

# Tolerances of the parity bar: pixels on the [0, 255] scale, PSNR in dB.
PIX_TOL = 1e-3
PSNR_TOL = 0.01


def pack_masks(masks: np.ndarray) -> np.ndarray:
    """Oracle masks (n, K, ps, ps, C) bool -> (n, words) uint32, bit ((m*ps+i)*ps+j)*C+c."""
    n = masks.shape[0]
    flat = masks.reshape(n, -1)
    pad = (-flat.shape[1]) % 32
    if pad:
        flat = np.concatenate([flat, np.zeros((n, pad), dtype=bool)], axis=1)
    by = np.packbits(flat, axis=1, bitorder="little")
    return by.view("<u4").reshape(n, -1)


def unpack_words(words: np.ndarray, nbits: int) -> np.ndarray:
    by = np.ascontiguousarray(words.astype("<u4")).view(np.uint8)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :nbits].astype(bool)


@functools.lru_cache(maxsize=8)
def oracle_run(key: str):
    """(clean, noisy, sigma, params, oracle Result) of a named workload, computed once per process."""
    if key == "gray128":
        clean, noisy, sigma, prm = synth.workload_gray128()
    elif key == "rgb512":
        clean, noisy, sigma, prm = synth.workload_rgb512()
        sigma = O.estimate_sigma(noisy, prm)
    else:
        raise KeyError(key)
    r = O.denoise(noisy, sigma, prm, keep_masks=True)
    return clean, noisy, sigma, prm, r


def psnr(out, clean) -> float:
    return synth.psnr(out, clean)


def max_abs(a, b) -> float:
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64))))


def sqrt(x):
    return math.sqrt(x)

"""GB300 Haar-tSVD denoising core (Kong, Zhang & Yang, arXiv 2508.10307).

Thin PyTorch-facing binding over the C ABI of libhtsvd.so (include/htsvd.h): it only
moves tensors' device pointers and the current CUDA stream across the boundary. Every
step of the method runs in the library's CUDA kernels; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, fields

from . import _lib

__all__ = ["HtsvdParams", "denoise", "denoise_f32", "estimate_sigma", "denoise_batch", "denoise_adaptive",
           "denoise_video", "denoise_cube", "denoise_tau_sweep", "sure", "sure_weights", "tune_weights", "denoise_vjp", "project_patches", "denoise_volume",
           "num_groups", "HtsvdFn", "load_library"]

_MATCH = {"auto": 0, "gcp": 1, "full": 2, "green": 3}
_AGG = {"uniform": 0, "sparsity": 1}


@dataclass
class HtsvdParams:
    """Method parameters (Sec. IV-A defaults: ps 8, K 32, window 18; tau = sigma sqrt(2 ln(C K ps^2)))."""
    ps: int = 8
    stride: int = 3
    window: int = 18
    K: int = 32
    tau_mult: float = 0.0
    match_mode: str = "auto"
    gcp_gamma: float = 1.2
    agg_mode: str = "uniform"
    adapt: bool = False
    beta: float = 1.2
    rank_gamma: int = 0
    tile: int = 0
    strict_basis: bool = False      # fail with DEGENERATE_BASIS when a basis slice's eigen-gap is below 1e-9

    @staticmethod
    def of(p) -> "HtsvdParams":
        if p is None:
            return HtsvdParams()
        if isinstance(p, HtsvdParams):
            return p
        names = {f.name for f in fields(HtsvdParams)}
        d = dict(p)
        unknown = sorted(set(d) - names)
        if unknown:                       # a misspelt parameter would otherwise fall back to its default
            raise ValueError(f"unknown parameters {unknown}; known: {sorted(names)}")
        return HtsvdParams(**d)

    def c(self) -> _lib.CParams:
        cp = _lib.CParams()
        cp.ps, cp.stride, cp.window, cp.K = self.ps, self.stride, self.window, self.K
        cp.tau_mult = float(self.tau_mult)
        if self.match_mode not in _MATCH or self.agg_mode not in _AGG:
            raise ValueError(f"match_mode must be one of {sorted(_MATCH)} and agg_mode one of {sorted(_AGG)}, "
                             f"got {self.match_mode!r} and {self.agg_mode!r}")
        cp.match_mode = _MATCH[self.match_mode]
        cp.gcp_gamma = float(self.gcp_gamma)
        cp.agg_mode = _AGG[self.agg_mode]
        cp.adapt = int(bool(self.adapt))
        cp.beta = float(self.beta)
        cp.rank_gamma = int(self.rank_gamma)
        cp.tile = int(self.tile)
        cp.strict_basis = int(bool(self.strict_basis))
        return cp


def load_library():
    return _lib.load()


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _hwc(x):
    if x.dim() == 2:
        x = x.unsqueeze(-1)
    if x.dim() != 3 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor of shape (H, W) or (H, W, C)")
    return x


def _need(t, name, shape, dtype, like=None):
    """Checks a buffer the library reads or writes through a bare pointer: its shape (it sets how far
    the kernels index), dtype, contiguity and device. Returns t."""
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    if not t.is_cuda or (like is not None and t.device != like.device):
        raise ValueError(f"{name}: expected a CUDA tensor on {like.device if like is not None else 'the GPU'}")
    return t


def num_groups(H: int, W: int, params=None) -> int:
    lib = _lib.load()
    cp = HtsvdParams.of(params).c()
    return int(lib.htsvd_num_groups(H, W, ctypes.byref(cp)))


def _outputs(x, p, params, want_idx, want_masks, want_weights, want_basis, want_coeffs=False):
    torch = _torch()
    H, W, C = x.shape
    n = num_groups(H, W, p)
    out = torch.empty((H, W, C), dtype=torch.float32, device=x.device)
    info = {}
    idx = torch.empty((n, p.K), dtype=torch.int32, device=x.device) if want_idx else None
    if want_masks:
        info["masks"] = torch.empty((n, (p.K * 64 * C + 31) // 32), dtype=torch.int32, device=x.device)
        params.d_mask_out = info["masks"].data_ptr()
    if want_weights:
        info["weights"] = torch.empty(n, dtype=torch.float32, device=x.device)
        params.d_weights_out = info["weights"].data_ptr()
    if want_basis:
        info["basis"] = torch.empty((2, C, 8, 8, 2), dtype=torch.float64, device=x.device)
        params.d_basis_out = info["basis"].data_ptr()
    if want_coeffs:
        info["coeffs"] = torch.empty((n, p.K, 8, 8, C), dtype=torch.float32, device=x.device)
        params.d_coef_out = info["coeffs"].data_ptr()
    return out, idx, info


def denoise(noisy, sigma=None, params=None, *, return_info=False, masks=False, weights=False, basis=False,
            coeffs=False, basis_gap=False, stream=None):
    """Alg. 1 on a uint8 (H, W[, C]) CUDA tensor. sigma=None estimates it on the device.
    Returns the float32 (H, W, C) estimate, or (estimate, info) with return_info; basis_gap=True adds
    info["basis_gap"], the smallest relative eigen-gap of the basis slices (synchronises)."""
    lib = _lib.load()
    x = _hwc(noisy)
    if x.dtype != _torch().uint8:
        raise TypeError("denoise expects uint8; use denoise_f32 for float images")
    p = HtsvdParams.of(params)
    cp = p.c()
    sig_out = ctypes.c_double(-1.0)
    cp.h_sigma_out = ctypes.pointer(sig_out)
    gap_out = ctypes.c_double(-1.0)
    if basis_gap:
        cp.h_basis_gap_out = ctypes.pointer(gap_out)
    out, idx, info = _outputs(x, p, cp, return_info, masks, weights, basis, coeffs)
    H, W, C = x.shape
    st = lib.htsvd_denoise(_ptr(x), H, W, C, -1.0 if sigma is None else float(sigma), ctypes.byref(cp),
                           _ptr(out), _ptr(idx), _stream_ptr(stream))
    _lib.check(st, "htsvd_denoise")
    if return_info:
        info.update(idx=idx, sigma=sig_out.value)
        if basis_gap:
            info["basis_gap"] = gap_out.value
        return out, info
    return out


def denoise_f32(x, sigma=None, params=None, *, w=None, return_info=False, masks=False, weights=False,
                basis=False, stream=None):
    """Alg. 1 on a float32 image; grouping and bases use the rounded image, the filter uses x."""
    lib = _lib.load()
    x = _hwc(x)
    torch = _torch()
    if x.dtype != torch.float32:
        raise TypeError("denoise_f32 expects float32")
    p = HtsvdParams.of(params)
    cp = p.c()
    sig_out = ctypes.c_double(-1.0)
    cp.h_sigma_out = ctypes.pointer(sig_out)
    out, idx, info = _outputs(x, p, cp, True, masks, weights, basis)
    H, W, C = x.shape
    wt = None if w is None else _need(w.contiguous().float(), "w", (idx.shape[0],), torch.float32, x)
    st = lib.htsvd_denoise_f32(_ptr(x), H, W, C, -1.0 if sigma is None else float(sigma), ctypes.byref(cp),
                               _ptr(wt), _ptr(out), _ptr(idx), _stream_ptr(stream))
    _lib.check(st, "htsvd_denoise_f32")
    if return_info:
        info.update(idx=idx, sigma=sig_out.value)
        return out, info
    return out


def estimate_sigma(noisy, params=None, stream=None) -> float:
    """Noise level from the covariance eigenvalues of the reference patches (optionally adjusted by
    the eigen-rank vote of Sec. III-D). Synchronises the stream."""
    lib = _lib.load()
    x = _hwc(noisy)
    if x.dtype != _torch().uint8:
        raise TypeError("estimate_sigma expects uint8")
    p = HtsvdParams.of(params)
    cp = p.c()
    s = ctypes.c_double(0.0)
    H, W, C = x.shape
    _lib.check(lib.htsvd_estimate_sigma(_ptr(x), H, W, C, ctypes.byref(cp), ctypes.byref(s), _stream_ptr(stream)),
               "htsvd_estimate_sigma")
    return s.value


def denoise_batch(images, sigmas, params=None, outs=None, stream=None, idx_outs=None):
    """Denoises a list of uint8 (H, W, C) CUDA tensors of any sizes with per-image sigma.
    idx_outs: optional list of int32 (N_groups, K) CUDA tensors that receive each image's grouping."""
    lib = _lib.load()
    torch = _torch()
    imgs = [_hwc(t) for t in images]
    sigmas = list(sigmas)
    if len(sigmas) != len(imgs):
        raise ValueError(f"denoise_batch: {len(imgs)} images but {len(sigmas)} sigmas")
    for t in imgs:
        if t.dtype != torch.uint8:
            raise TypeError("denoise_batch expects uint8 images")
    if outs is None:
        outs = [torch.empty(t.shape, dtype=torch.float32, device=t.device) for t in imgs]
    if len(outs) != len(imgs):
        raise ValueError(f"denoise_batch: {len(imgs)} images but {len(outs)} outputs")
    for i, (t, o) in enumerate(zip(imgs, outs)):
        _need(o if o.dim() == 3 else o.unsqueeze(-1), f"outs[{i}]", t.shape, torch.float32, t)
    p = HtsvdParams.of(params)
    if idx_outs is not None:
        if len(idx_outs) != len(imgs):
            raise ValueError(f"denoise_batch: {len(imgs)} images but {len(idx_outs)} index buffers")
        for i, (t, ix) in enumerate(zip(imgs, idx_outs)):
            _need(ix, f"idx_outs[{i}]", (num_groups(t.shape[0], t.shape[1], p), p.K), torch.int32, t)
    arr = (_lib.CImage * len(imgs))()
    for i, (t, s, o) in enumerate(zip(imgs, sigmas, outs)):
        arr[i].d_in = t.data_ptr()
        arr[i].H, arr[i].W, arr[i].C = t.shape
        arr[i].sigma = float(s)
        arr[i].d_out = o.data_ptr()
        arr[i].d_idx_out = idx_outs[i].data_ptr() if idx_outs is not None else None
    cp = p.c()
    _lib.check(lib.htsvd_denoise_batch(arr, len(imgs), ctypes.byref(cp), _stream_ptr(stream)),
               "htsvd_denoise_batch")
    return outs


def subimage_bounds(n: int, n_sub: int):
    """Subimage boundaries of one axis used by denoise_adaptive: t = max(1, n // n_sub) parts,
    boundaries floor(i n / t)."""
    t = max(1, n // n_sub)
    return [((i * n) // t, ((i + 1) * n) // t) for i in range(t)]


def denoise_adaptive(noisy, sub=(256, 256), params=None, *, return_sigmas=False, stream=None):
    """A-Haar-tSVD (Alg. 2) on a uint8 (H, W[, C]) CUDA tensor: per-subimage noise estimates
    (eigenvalue rule; the eigen-rank vote when params.adapt) and per-subimage denoising.
    Returns the float32 (H, W, C) estimate, and the subimage sigmas (row-major) if asked."""
    lib = _lib.load()
    torch = _torch()
    x = _hwc(noisy)
    if x.dtype != torch.uint8:
        raise TypeError("denoise_adaptive expects uint8")
    H, W, C = x.shape
    cp = HtsvdParams.of(params).c()
    out = torch.empty((H, W, C), dtype=torch.float32, device=x.device)
    n = len(subimage_bounds(H, int(sub[0]))) * len(subimage_bounds(W, int(sub[1])))
    sig = (ctypes.c_double * n)()
    _lib.check(lib.htsvd_denoise_adaptive(_ptr(x), H, W, C, int(sub[0]), int(sub[1]), ctypes.byref(cp), _ptr(out),
                                          sig, _stream_ptr(stream)), "htsvd_denoise_adaptive")
    return (out, [float(v) for v in sig]) if return_sigmas else out


def denoise_cube(cube, sigma, params=None, *, return_info=False, masks=False, weights=False, basis=False,
                 coeffs=False, stream=None):
    """Alg. 1 on a hyperspectral uint8 (H, W, N) CUDA tensor (N bands, 2..64) at the given sigma; the
    t-SVD runs along the band mode. Returns the float32 (H, W, N) estimate, or (estimate, info)."""
    lib = _lib.load()
    x = _hwc(cube)
    if x.dtype != _torch().uint8:
        raise TypeError("denoise_cube expects uint8")
    p = HtsvdParams.of(params)
    cp = p.c()
    out, idx, info = _outputs(x, p, cp, return_info, masks, weights, False, coeffs)
    H, W, N = x.shape
    if basis:
        info["basis"] = _torch().empty((2, N, 8, 8, 2), dtype=_torch().float64, device=x.device)
        cp.d_basis_out = info["basis"].data_ptr()
    st = lib.htsvd_denoise_cube(_ptr(x), H, W, N, float(sigma), ctypes.byref(cp), _ptr(out), _ptr(idx),
                                _stream_ptr(stream))
    _lib.check(st, "htsvd_denoise_cube")
    if return_info:
        info.update(idx=idx)
        return out, info
    return out


VOLUME_DEFAULTS = dict(ps=4, stride=2, window=5, K=32)


def denoise_volume(vol, sigma=None, params=None, *, return_info=False, masks=False, weights=False, basis=False,
                   stream=None):
    """Alg. 1 on a uint8 (D, H, W) CUDA volume with 4 x 4 x 4 cubes (the t-SVD tube along z) at the
    given sigma (None: estimated from the reference cubes' covariance eigenvalues); params default to
    the paper's MRI setting (ps 4, K 32, window 5; stride 2). Returns the float32 (D, H, W) estimate,
    or (estimate, info)."""
    lib = _lib.load()
    torch = _torch()
    if vol.dim() != 3 or not vol.is_cuda or not vol.is_contiguous() or vol.dtype != torch.uint8:
        raise ValueError("denoise_volume expects a contiguous uint8 CUDA tensor (D, H, W)")
    if params is None or isinstance(params, dict):
        params = dict(VOLUME_DEFAULTS, **(params or {}))
    p = HtsvdParams.of(params)
    cp = p.c()
    D, H, W = vol.shape
    nz, ny, nx = (len(range(0, n - p.ps + 1, p.stride)) + (1 if (n - p.ps) % p.stride else 0) for n in (D, H, W))
    n = nz * ny * nx
    out = torch.empty((D, H, W), dtype=torch.float32, device=vol.device)
    idx = torch.empty((n, p.K), dtype=torch.int32, device=vol.device)
    info = {}
    if masks:
        info["masks"] = torch.empty((n, 2 * p.K), dtype=torch.int32, device=vol.device)
        cp.d_mask_out = info["masks"].data_ptr()
    if weights:
        info["weights"] = torch.empty(n, dtype=torch.float32, device=vol.device)
        cp.d_weights_out = info["weights"].data_ptr()
    if basis:
        info["basis"] = torch.empty((2, 4, 4, 4, 2), dtype=torch.float64, device=vol.device)
        cp.d_basis_out = info["basis"].data_ptr()
    gap = ctypes.c_double(0.0)
    used = ctypes.c_double(0.0)
    cp.h_basis_gap_out = ctypes.pointer(gap)
    cp.h_sigma_out = ctypes.pointer(used)
    st = lib.htsvd_denoise_volume(_ptr(vol), D, H, W, -1.0 if sigma is None else float(sigma), ctypes.byref(cp),
                                  _ptr(out), _ptr(idx), _stream_ptr(stream))
    _lib.check(st, "htsvd_denoise_volume")
    if return_info:
        info.update(idx=idx, basis_gap=gap.value, sigma=used.value)
        return out, info
    return out


def denoise_volume_adaptive(vol, sub=(88, 104, 88), params=None, *, return_sigmas=False, stream=None):
    """A-Haar-tSVD (Alg. 2) on a uint8 (D, H, W) CUDA volume: each axis cut into parts at least
    sub long, a sigma per sub-volume by the eigenvalue rule on its reference cubes, and Alg. 1 of
    denoise_volume on each part at its sigma. Returns the float32 (D, H, W) estimate, and the
    sub-volume sigmas (z-major) if asked."""
    lib = _lib.load()
    torch = _torch()
    if vol.dim() != 3 or not vol.is_cuda or not vol.is_contiguous() or vol.dtype != torch.uint8:
        raise ValueError("denoise_volume_adaptive expects a contiguous uint8 CUDA tensor (D, H, W)")
    if params is None or isinstance(params, dict):
        params = dict(VOLUME_DEFAULTS, **(params or {}))
    cp = HtsvdParams.of(params).c()
    D, H, W = vol.shape
    sd, sh, sw = (int(v) for v in sub)
    n = 1
    for length, part in ((D, sd), (H, sh), (W, sw)):
        n *= len(subimage_bounds(length, max(part, 1)))
    out = torch.empty((D, H, W), dtype=torch.float32, device=vol.device)
    sig = (ctypes.c_double * n)()
    st = lib.htsvd_denoise_volume_adaptive(_ptr(vol), D, H, W, sd, sh, sw, ctypes.byref(cp), _ptr(out), sig,
                                           _stream_ptr(stream))
    _lib.check(st, "htsvd_denoise_volume_adaptive")
    return (out, [float(v) for v in sig]) if return_sigmas else out


def denoise_video(frames, sigma=None, params=None, *, T=1, return_info=False, stream=None):
    """A clip of uint8 frames (F, H, W[, C]) on the GPU, frame by frame with spatio-temporal grouping
    over frames t-T..t+T; sigma=None estimates it per frame. Returns float32 (F, H, W, C), or
    (estimate, info) with return_info: info["idx"] (F, N, K) global group indices, info["sigmas"]."""
    lib = _lib.load()
    torch = _torch()
    v = frames if frames.dim() == 4 else frames.unsqueeze(-1)
    if v.dim() != 4 or not v.is_cuda:
        raise ValueError("denoise_video expects a CUDA tensor of shape (F, H, W) or (F, H, W, C)")
    if v.dtype != torch.uint8:
        raise TypeError("denoise_video expects uint8")
    v = v.contiguous()
    F, H, W, C = v.shape
    p = HtsvdParams.of(params)
    out = torch.empty((F, H, W, C), dtype=torch.float32, device=v.device)
    idx = torch.empty((F, num_groups(H, W, p), p.K), dtype=torch.int32, device=v.device) if return_info else None
    cp = p.c()
    sig = (ctypes.c_double * F)()
    _lib.check(lib.htsvd_denoise_video(_ptr(v), F, H, W, C, int(T), -1.0 if sigma is None else float(sigma),
                                       ctypes.byref(cp), _ptr(out), _ptr(idx), sig, _stream_ptr(stream)),
               "htsvd_denoise_video")
    if return_info:
        return out, {"idx": idx, "sigmas": [float(s) for s in sig]}
    return out


def denoise_tau_sweep(noisy, tau_mults, sigma=None, params=None, *, return_sigma=False, stream=None):
    """Alg. 1 on a uint8 (H, W[, C]) CUDA tensor at every tau = tau_mults[i] * sigma, with the grouping,
    bases, sigma and noisy coefficients computed once. Returns float32 (n, H, W, C)."""
    lib = _lib.load()
    torch = _torch()
    x = _hwc(noisy)
    if x.dtype != torch.uint8:
        raise TypeError("denoise_tau_sweep expects uint8")
    H, W, C = x.shape
    m = [float(t) for t in tau_mults]
    outs = torch.empty((len(m), H, W, C), dtype=torch.float32, device=x.device)
    cp = HtsvdParams.of(params).c()
    sig = ctypes.c_double(-1.0)
    _lib.check(lib.htsvd_denoise_tau_sweep(_ptr(x), H, W, C, -1.0 if sigma is None else float(sigma),
                                           (ctypes.c_double * len(m))(*m), len(m), ctypes.byref(cp), _ptr(outs),
                                           ctypes.byref(sig), _stream_ptr(stream)), "htsvd_denoise_tau_sweep")
    return (outs, sig.value) if return_sigma else outs


def sure(y, sigma, tau_mults, probe, params=None, eps=None, stream=None):
    """SURE of each threshold multiplier on a float32 (H, W[, C]) CUDA image y along probe (same
    shape; e.g. a +-1 Rademacher vector). eps > 0 (default sigma / 10): the divergence is the finite
    difference of the whole denoiser at y + eps * probe; eps = 0: the frozen-mask VJP applied to
    probe (biased low: it omits the threshold's jumps). Returns a list of floats; synchronises the
    stream."""
    lib = _lib.load()
    torch = _torch()
    x = _hwc(y)
    if x.dtype != torch.float32:
        raise TypeError("sure expects float32")
    b = _need(probe if probe.dim() == 3 else probe.unsqueeze(-1), "probe", x.shape, torch.float32, x)
    H, W, C = x.shape
    m = [float(t) for t in tau_mults]
    res = (ctypes.c_double * len(m))()
    cp = HtsvdParams.of(params).c()
    e = 0.1 * float(sigma) if eps is None else float(eps)
    _lib.check(lib.htsvd_sure(_ptr(x), H, W, C, float(sigma), (ctypes.c_double * len(m))(*m), len(m),
                              _ptr(b), e, ctypes.byref(cp), res, _stream_ptr(stream)), "htsvd_sure")
    return [float(v) for v in res]


def sure_weights(y, sigma, w, probe, params=None, eps=None, stream=None):
    """SURE of the denoiser aggregating with per-group weights w (float32 CUDA tensor of num_groups
    values > 0) on the float32 (H, W[, C]) CUDA image y, and its gradient in w (htsvd_sure_weights;
    eps > 0, default sigma / 10). Returns (sure: float, grad_w: tensor); synchronises the stream."""
    lib = _lib.load()
    torch = _torch()
    x = _hwc(y)
    if x.dtype != torch.float32:
        raise TypeError("sure_weights expects float32")
    b = _need(probe if probe.dim() == 3 else probe.unsqueeze(-1), "probe", x.shape, torch.float32, x)
    H, W, C = x.shape
    p = HtsvdParams.of(params)
    n = num_groups(H, W, p)
    wt = _need(w.contiguous(), "w", (n,), torch.float32, x)
    g = torch.empty(n, dtype=torch.float32, device=x.device)
    res = ctypes.c_double()
    cp = p.c()
    e = 0.1 * float(sigma) if eps is None else float(eps)
    _lib.check(lib.htsvd_sure_weights(_ptr(x), H, W, C, float(sigma), _ptr(wt), _ptr(b), e,
                                      ctypes.byref(cp), ctypes.byref(res), _ptr(g), _stream_ptr(stream)),
               "htsvd_sure_weights")
    return float(res.value), g


def tune_weights(y, sigma, probe, params=None, eps=None, steps=3, step=0.5, w0=None, stream=None):
    """Per-group weights tuned by exponentiated-gradient steps on their SURE (htsvd_tune_weights),
    from w0 (default all ones). Returns (w, trace) with trace the SURE before each step and after the
    last."""
    lib = _lib.load()
    torch = _torch()
    x = _hwc(y)
    if x.dtype != torch.float32:
        raise TypeError("tune_weights expects float32")
    b = _need(probe if probe.dim() == 3 else probe.unsqueeze(-1), "probe", x.shape, torch.float32, x)
    H, W, C = x.shape
    p = HtsvdParams.of(params)
    n = num_groups(H, W, p)
    w = (torch.ones(n, dtype=torch.float32, device=x.device) if w0 is None
         else _need(w0.contiguous(), "w0", (n,), torch.float32, x).clone())
    trace = (ctypes.c_double * (int(steps) + 1))()
    cp = p.c()
    e = 0.1 * float(sigma) if eps is None else float(eps)
    _lib.check(lib.htsvd_tune_weights(_ptr(x), H, W, C, float(sigma), _ptr(b), e,
                                      int(steps), float(step), ctypes.byref(cp), _ptr(w), trace, _stream_ptr(stream)),
               "htsvd_tune_weights")
    return w, [float(v) for v in trace]


def denoise_vjp(x, sigma, idx, w, out, grad_out, params=None, want_grad_w=True, stream=None):
    """Vector-Jacobian product of denoise_f32 at x (grouping, bases, tau and masks held fixed)."""
    lib = _lib.load()
    torch = _torch()
    x = _hwc(x)
    if x.dtype != torch.float32:
        raise TypeError("denoise_vjp expects float32")
    H, W, C = x.shape
    p = HtsvdParams.of(params)
    n = num_groups(H, W, p)
    idx = _need(idx.contiguous(), "idx", (n, p.K), torch.int32, x)
    out = _need(out.contiguous().view(x.shape) if out.numel() == x.numel() else out, "out", x.shape, torch.float32, x)
    grad_out = _need(grad_out.contiguous().view(x.shape) if grad_out.numel() == x.numel() else grad_out,
                     "grad_out", x.shape, torch.float32, x)
    gx = torch.empty_like(x)
    gw = torch.empty(n, dtype=torch.float32, device=x.device) if want_grad_w else None
    cp = p.c()
    wt = None if w is None else _need(w.contiguous().float(), "w", (n,), torch.float32, x)
    st = lib.htsvd_denoise_vjp(_ptr(x), H, W, C, float(sigma), ctypes.byref(cp), _ptr(idx), _ptr(wt),
                               _ptr(out), _ptr(grad_out), _ptr(gx), _ptr(gw), _stream_ptr(stream))
    _lib.check(st, "htsvd_denoise_vjp")
    return gx, gw


def project_patches(img, pos, basis, *, out=None, flag=None, stream=None, structured=False):
    """Coefficients S = U^T * P * V (64 C per patch, mask-bit order) of the 8 x 8 patches of a uint8
    HWC image at linear top-left positions pos (int32), or of every position (row-major over the
    (H - 7) x (W - 7) corners) when pos is None, with the FP64 bases `basis` (the layout of
    denoise(..., basis=True)). The tensor-core path by default; structured=True runs the per-slice
    FP32 form on the CUDA cores (internal comparison hook)."""
    lib = _lib.load()
    torch = _torch()
    img = _hwc(img)
    if img.dtype != torch.uint8:
        raise TypeError("project_patches expects a uint8 image")
    H, W, C = img.shape
    if pos is None:
        n = (H - 7) * (W - 7)
    else:
        pos = _need(pos.contiguous().view(-1), "pos", (pos.numel(),), torch.int32, img)
        n = pos.numel()
    basis = _need(basis.contiguous(), "basis", (2 * C * 64 * 2,) if basis.dim() == 1 else tuple(basis.shape),
                  torch.float64, img)
    if basis.numel() != 2 * C * 64 * 2:
        raise ValueError(f"basis must hold {2 * C * 64 * 2} doubles")
    if out is None:
        out = torch.empty((n, 64 * C), dtype=torch.float32, device=img.device)
    out = _need(out, "out", (n, 64 * C), torch.float32, img)
    if structured:
        st = lib.htsvd_internal_project_simt(_ptr(img), H, W, C, _ptr(pos), n, _ptr(basis), _ptr(out),
                                             _stream_ptr(stream))
        _lib.check(st, "htsvd_internal_project_simt")
    else:
        if flag is not None:
            flag = _need(flag, "flag", (1,), torch.int32, img)
        st = lib.htsvd_project_patches(_ptr(img), H, W, C, _ptr(pos), n, _ptr(basis), _ptr(out), _ptr(flag),
                                       _stream_ptr(stream))
        _lib.check(st, "htsvd_project_patches")
    return out


def _make_fn():
    torch = _torch()

    class HtsvdFn(torch.autograd.Function):
        """out = Haar-tSVD(x; w) with a hand-written VJP for x and the per-group weights w.
        The grouping, bases, tau and masks are held fixed; the backward recomputes the group
        tensors instead of storing them."""

        @staticmethod
        def forward(ctx, x, w, sigma, params):
            p = HtsvdParams.of(params)
            out, info = denoise_f32(x.contiguous(), sigma, p, w=w, return_info=True)
            ctx.save_for_backward(x, w, info["idx"], out)
            ctx.sigma = info["sigma"]
            ctx.params = p
            return out

        @staticmethod
        def backward(ctx, grad_out):
            x, w, idx, out = ctx.saved_tensors
            gx, gw = denoise_vjp(x, ctx.sigma, idx, w, out, grad_out.contiguous(), ctx.params,
                                 want_grad_w=ctx.needs_input_grad[1])
            return gx, gw, None, None

    return HtsvdFn


def __getattr__(name):
    if name == "HtsvdFn":
        fn = _make_fn()
        globals()["HtsvdFn"] = fn
        return fn
    raise AttributeError(name)

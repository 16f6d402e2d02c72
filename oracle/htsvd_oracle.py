"""FP64 CPU oracle for the Haar-tSVD denoising core (Kong, Zhang & Yang, arXiv 2508.10307).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import or execute this
module; only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg use it. It shares no code with the CUDA path.

Every function restates a step of the paper in plain numpy, float64 unless the
quantity is an exact integer, without blocking or fusion beyond what the
definition states:

* grouping by green-channel-prior block matching       -- Sec. III-A, Eq. (GCP distance)
* global t-SVD bases from all reference patches        -- Sec. III-B.1, Eqs. (BCR nonlocal SVD), Alg. 1 Step 2(1)
* t-product via mode-3 FFT                               -- Sec. II-C, Def. T-product, Eqs. (FFT product, FFT third mode)
* Haar matrix                                            -- Sec. II-D, Eqs. (H_2), (H_2N)
* forward transform, hard threshold, inverse           -- Sec. III-B.2, Eqs. (forward transform), (hard thresholding), (backward transform)
* aggregation                                            -- Sec. II-B, Eq. (aggregation); Alg. 1 Step 3
* circulant eigen-analysis and sigma adjustment         -- Sec. III-D, Eqs. (other eigenvalue), (adjust noise level)
* eigenvalue noise-level estimate (patch-covariance rule, used in place of the paper's CNN)

Readings where the paper is silent or ambiguous:
  R1 distance = exact integer SSD on the chosen plane; the "avg" branch uses the
     R+G+B sum plane (SSD = 9x the SSD of the average, same order).
  R2 the GCP test is evaluated on the reference patch with raw L2 norms, in
     float64 as (gamma*gamma)*|G|^2 >= |R|^2 and likewise for B.
  R3 reference grid per axis = {0, s, 2s, ...} U {n - ps}.
  R4 window = W x W candidate top-left positions, start clamped so the window
     lies inside the image; all positions if fewer than W exist.
  R5 slot 0 is the reference; slots 1..K-1 are the K-1 smallest (SSD, y*W+x)
     keys among the other candidates (ties -> lowest linear index).
  R6 global bases: per Fourier slice f, U_f = eigenvectors of sum_r P_f P_f^H,
     V_f = eigenvectors of sum_r P_f^H P_f (uncentred, reference patches);
     slice C-f := conj(slice f).
  R7 eigenvector convention: eigenvalues descending, each eigenvector's
     largest-modulus entry made real positive (ties within 1e-6 relative ->
     lowest index). Where two eigenvalues of a slice lie within 1e-9 of each other
     (relative to the largest) the eigenvectors are not unique; strict mode raises
     DegenerateBasis there (a test mode: without it the call proceeds).
  R8 coefficients along the group mode are H_K applied to each K-fibre
     (U_Haar = H_K^T); the inverse is H_K^T.
  R9 tau = tau_mult * sigma; tau_mult <= 0 means sqrt(2 ln(C K ps^2)); the
     threshold applies to every coefficient and |S| == tau is kept.
  R10 aggregation weights: 1 per group (uniform), or 1/max(1, #kept) (sparsity),
     or caller-given per-group weights.
  R11 noise estimate: covariance of reference patches, ascending eigenvalues,
     r* = max{r : mean(l_1..r) <= 1.02 median(l_1..r)}, sigma = sqrt(mean(l_1..r*)).
  R12 adaptive adjustment: groups of every 8th reference per axis; rank
     a = 1 + #{f : lambda_f < lambda_{K/2}}; majority of a <= gamma_rank divides
     sigma by beta; gamma_rank defaults to 13 K / 32 rounded half up (13 at K = 32).
  R13 float inputs: matching, bases and sigma use q = clip(rint(x)); the
     transforms use x.
  R14 vector-Jacobian product: grouping, bases, tau and masks held fixed (masks
     taken at x), so the map is linear in x and its adjoint is the transposed chain.
  R15 A-Haar-tSVD (Alg. 2) subimages: each axis of length n is cut into
     t = max(1, floor(n / n_sub)) parts with boundaries floor(i n / t), so every
     subimage is at least n_sub long; each subimage gets its own noise estimate
     (R11, with R12 when adapt is set) and is denoised on its own (Alg. 1).
  R16 video (Sec. IV, real-world color video denoising; the paper states only that
     the patch search covers space and time and that the noise estimate runs frame
     by frame): output frame t is Alg. 1 on frame t with frame t's own bases (R6)
     and sigma; the candidates of a reference of frame t are the positions of its
     spatial window (R4) in every frame max(0, t-T) .. min(F-1, t+T), the
     reference itself excluded, compared on the plane its own patch selects (R1,
     R2 on frame t); keys (SSD, f*H*W + y*W + x), ties -> lowest global index;
     only the estimated patches that lie in frame t are aggregated into it.
  R17 threshold selection by Stein's unbiased risk estimate (the paper only notes that tuning is
     sped up by caching indices and coefficients, Sec. III-E): for each multiplier m,
     f = Alg. 1 at tau = m sigma on a float image y (R13), n = H W C,
     SURE(m) = ||f - y||^2 / n - sigma^2 + (2 sigma^2 / n) div, b a caller-given probe (a Rademacher
     vector makes b^T J b an unbiased estimate of trace J). With a step eps > 0 the divergence is the
     Monte-Carlo finite difference of the whole denoiser (Ramani, Blu and Unser, 2008),
     div = b^T (f(z) - f(y)) / eps with z = y + eps b rounded to float32 as the device forms it
     (round(eps), then round(eps b), then round(y + eps b)); f(z) regroups and re-solves the bases,
     so the threshold's jumps and the bases' dependence on y are counted. With eps = 0 it is
     b^T J^T b, J the Jacobian of the frozen-mask map at y (R14), which counts neither: hard
     thresholding makes that form biased low (the jump terms grow as tau falls).
  R18 hyperspectral cubes (Sec. III-E, extension to other imaging; Sec. IV, real-world HSI
     denoising): an H x W x N cube is Alg. 1 with C = N, so a patch is a ps x ps x N tube and the
     t-SVD runs along the band mode (N Fourier slices); the paper is silent on matching for HSI,
     so 'auto' matching takes the SSD over all bands (exact integers); tau = sigma sqrt(2 ln(N K
     ps^2)) (Sec. IV-A with c = N, as R9). The paper's band-mean noise estimate goes through its
     CNN, so for cubes sigma is an input.
  R19 per-group weight tuning by SURE (the aggregation weights of R10 as free parameters, tuned
     through the vector-Jacobian product; the paper's tuning remark in Sec. III-E): for weights
     w > 0, f_w(x) = N_w(x) / D_w with the grouping, bases and masks of x (none depends on w),
     SURE(w) = ||f_w(y) - y||^2 / n - sigma^2 + (2 sigma^2 / n) b^T (f_w(z) - f_w(y)) / eps with z as
     in R17 (eps > 0), and its gradient is exact through the weight part G_x of the adjoint (R14):
     dSURE/dw = G_y((2/n)(f_w(y) - y) - (2 sigma^2 / (n eps)) b) + G_z((2 sigma^2 / (n eps)) b).
     Tuning takes exponentiated-gradient steps w <- w exp(-step g / max|g|), which keep w > 0.
  R20 MRI volumes (Sec. III-E, extension to other imaging: an MRI patch is a ps x ps x ps cube;
     Sec. IV, MRI denoising: ps = 4, K = 32, W = 5): a (D, H, W) volume (slices z, rows y,
     columns x) is Alg. 1 on cubes P[i][j][k] = v[z + k, y + i, x + j], i.e. a cube is a ps x ps x
     c tensor whose tube (the t-SVD's Fourier mode) runs along z, c = ps; the reference grid is R3
     per axis, the window W x W x W candidate positions clamped per axis (R4), the distance the
     exact integer SSD over the ps^3 voxels, keys (SSD, (z H + y) W + x), slot 0 the reference
     (R5); bases per tube-Fourier slice as R6/R7; tau = sigma sqrt(2 ln(ps^3 K)) (R9 with c = ps);
     aggregation into the volume as R10. The paper's Rician noise goes through variance-
     stabilising transforms, which are outside this core: sigma is the (stabilised) noise level,
     given or estimated by R11 on the covariance of the reference cubes (in place of the CNN).
  R21 the adaptive variant on MRI (Sec. IV runs A-Haar-tSVD on volumes; Alg. 2 is written for
     subimages): each volume axis is cut as R15 cuts image axes; per part sigma by R11 on its own
     reference cubes and Alg. 1 of R20 on the part alone; the eigen-rank vote of R12 is given for
     image groups and is not applied to volumes.

Parity pins for every function are in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from numpy.lib.stride_tricks import sliding_window_view


# --------------------------------------------------------------------------- params

@dataclass
class Params:
    ps: int = 8
    stride: int = 3
    window: int = 18
    K: int = 32
    tau_mult: float = 0.0          # <= 0 -> sqrt(2 ln(C K ps^2))   (Sec. IV-A)
    match_mode: str = "auto"       # auto | gcp | full | gray
    gcp_gamma: float = 1.2         # Sec. III-A
    agg_mode: str = "uniform"      # uniform | sparsity
    adapt: bool = False            # Sec. III-D adjustment
    beta: float = 1.2
    rank_gamma: int = 0            # 0 -> 13 K / 32 rounded half up (reading R12)
    strict_basis: bool = False     # raise DegenerateBasis when a basis slice has coinciding eigenvalues

    @staticmethod
    def of(d: dict | "Params" | None) -> "Params":
        if d is None:
            return Params()
        if isinstance(d, Params):
            return d
        return Params(**d)


def tau_multiplier(p: Params, C: int) -> float:
    """Universal threshold multiplier sqrt(2 log(c K ps^2)) (Sec. IV-A), natural log."""
    if p.tau_mult > 0:
        return float(p.tau_mult)
    return math.sqrt(2.0 * math.log(C * p.K * p.ps * p.ps))


def rank_gamma(p: Params) -> int:
    return p.rank_gamma if p.rank_gamma > 0 else (13 * p.K + 16) // 32


# --------------------------------------------------------------------------- Haar

def haar_matrix(K: int) -> np.ndarray:
    """H_K built recursively from H_2 (Sec. II-D):
    H_2N = 1/sqrt(2) [ H_N kron [1, 1] ; I_N kron [1, -1] ]."""
    if K < 2 or K & (K - 1):
        raise ValueError("K must be a power of two >= 2")
    H = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
    n = 2
    while n < K:
        top = np.kron(H, np.array([[1.0, 1.0]]))
        bot = np.kron(np.eye(n), np.array([[1.0, -1.0]]))
        H = np.vstack([top, bot]) / math.sqrt(2.0)
        n *= 2
    return H


# --------------------------------------------------------------------------- geometry

def reference_positions(n: int, ps: int, stride: int) -> np.ndarray:
    """Reading R3: {0, s, 2s, ...} U {n - ps} along one axis."""
    last = n - ps
    pos = list(range(0, last + 1, stride))
    if pos[-1] != last:
        pos.append(last)
    return np.array(pos, dtype=np.int64)


def window_range(r: int, n: int, ps: int, W: int) -> tuple[int, int]:
    """Reading R4: (start, count) of candidate top-left positions along one axis."""
    npos = n - ps + 1
    if npos <= W:
        return 0, npos
    start = min(max(r - (W - 1) // 2, 0), npos - W)
    return start, W


# --------------------------------------------------------------------------- grouping (Sec. III-A)

def resolve_match_mode(mode: str, C: int) -> str:
    """The matching mode used for a C-channel image: 'auto' is the gray plane for one channel, the
    GCP choice (Eq. GCP distance) for RGB and, reading R18, the SSD over all bands for a
    hyperspectral cube. The GCP and green-plane modes name RGB planes and need C in {1, 3}."""
    if mode == "auto":
        return "gray" if C == 1 else ("gcp" if C == 3 else "full")
    if mode in ("gcp", "gray") and C not in (1, 3):
        raise ValueError(f"match mode {mode!r} needs 1 or 3 channels, got {C}")
    return mode


def match_planes(img: np.ndarray):
    """Integer planes the distance of Eq. (GCP distance) is taken on.
    Returns (green_or_gray, rgb_sum); rgb_sum is None for one channel."""
    x = img.astype(np.int64)
    if x.shape[2] == 1:
        return x[:, :, 0], None
    return x[:, :, 1], x[:, :, 0] + x[:, :, 1] + x[:, :, 2]


def gcp_uses_green(img: np.ndarray, ry: int, rx: int, ps: int, gamma: float) -> bool:
    """Eq. (GCP distance) condition on the reference patch:
    ||P^G|| >= max(||P^R||/gamma, ||P^B||/gamma), evaluated as (gamma*gamma)*|G|^2 >= |R|^2, |B|^2."""
    p = img[ry:ry + ps, rx:rx + ps, :].astype(np.int64)
    r2, g2, b2 = (int((p[:, :, c] ** 2).sum()) for c in range(3))
    g = float(gamma) * float(gamma)
    return (g * float(g2) >= float(r2)) and (g * float(g2) >= float(b2))


def _match_plane_ssd(planes, ry, rxs, y0, ny, x0s, nx, ps):
    """SSD of the reference patches at (ry, rxs[n]) against every candidate of their windows:
    (n, ny, nx) int64, summed over the given integer planes."""
    ssd = np.zeros((len(rxs), ny, nx), dtype=np.int64)
    cols = x0s[:, None] + np.arange(nx)[None, :]                       # (n, nx)
    for pl in planes:
        views = sliding_window_view(pl, (ps, ps))                       # [y, x, i, j]
        cand = views[y0:y0 + ny][:, cols]                               # (ny, n, nx, i, j)
        ref = views[ry, rxs]                                            # (n, i, j)
        d = cand - ref[None, :, None]
        ssd += np.einsum("ynxij,ynxij->nyx", d, d)
    return ssd


def _match_row(img: np.ndarray, ry: int, rxs: np.ndarray, p: Params):
    """Grouping for the references (ry, rxs[n]) of one reference row (Alg. 1 Step 1)."""
    H, Wd, C = img.shape
    ps, K = p.ps, p.K
    y0, ny = window_range(ry, H, ps, p.window)
    xw = [window_range(int(rx), Wd, ps, p.window) for rx in rxs]
    x0s = np.array([a for a, _ in xw], dtype=np.int64)
    nx = xw[0][1]
    if ny * nx < K:
        raise ValueError("search window holds fewer than K candidates")
    mode = resolve_match_mode(p.match_mode, C)
    x = img.astype(np.int64)
    n = len(rxs)
    if mode == "full":
        ssd = _match_plane_ssd([x[:, :, c] for c in range(C)], ry, rxs, y0, ny, x0s, nx, ps)
        green = np.zeros(n, dtype=bool)
    elif C == 1 or mode == "gray":
        ssd = _match_plane_ssd([x[:, :, 0] if C == 1 else x[:, :, 1]], ry, rxs, y0, ny, x0s, nx, ps)
        green = np.ones(n, dtype=bool)
    else:
        green = np.array([gcp_uses_green(img, ry, int(rx), ps, p.gcp_gamma) for rx in rxs])
        g, s = match_planes(img)
        ssd = np.where(green[:, None, None],
                       _match_plane_ssd([g], ry, rxs, y0, ny, x0s, nx, ps),
                       _match_plane_ssd([s], ry, rxs, y0, ny, x0s, nx, ps))
    lin = ((y0 + np.arange(ny))[None, :, None] * Wd + (x0s[:, None, None] + np.arange(nx)[None, None, :]))
    lin = np.broadcast_to(lin, ssd.shape).reshape(n, -1)
    ssd = ssd.reshape(n, -1)
    ref_lin = ry * Wd + rxs
    idx = np.empty((n, K), dtype=np.int64)
    dist = np.empty((n, K), dtype=np.int64)
    for r in range(n):
        keep = lin[r] != ref_lin[r]
        cl, cs = lin[r][keep], ssd[r][keep]
        order = np.lexsort((cl, cs))[:K - 1]                 # ascending SSD, ties -> lowest index
        idx[r, 0], dist[r, 0] = ref_lin[r], 0
        idx[r, 1:], dist[r, 1:] = cl[order], cs[order]
    return idx, dist, green


def block_match_one(img: np.ndarray, ry: int, rx: int, p: Params):
    """Group of one reference patch: its own position in slot 0, then the K-1 nearest other
    candidates of its search window by (SSD, linear index).  Returns (linear indices[K], ssd[K], uses_green)."""
    idx, dist, green = _match_row(img, int(ry), np.array([rx], dtype=np.int64), p)
    return idx[0], dist[0], bool(green[0])


def block_match(img: np.ndarray, p: Params):
    """Alg. 1 Step 1 for every reference patch, row-major over the reference grid.
    Returns idx (N_ref, K) int64 linear indices y*W+x and the per-reference green flags."""
    H, Wd, _ = img.shape
    ys = reference_positions(H, p.ps, p.stride)
    xs = reference_positions(Wd, p.ps, p.stride)
    rows = [_match_row(img, int(ry), xs, p) for ry in ys]
    return np.concatenate([r[0] for r in rows]), np.concatenate([r[2] for r in rows])


def gather_groups(x: np.ndarray, idx: np.ndarray, ps: int) -> np.ndarray:
    """Stack the K patches named by each row of idx: (n, K, ps, ps, C) float64."""
    H, Wd, C = x.shape
    views = sliding_window_view(x.astype(np.float64), (ps, ps), axis=(0, 1))  # [y, x, C, i, j]
    g = views[idx // Wd, idx % Wd]                                              # [n, K, C, i, j]
    return np.ascontiguousarray(np.moveaxis(g, 2, -1))


def reference_patches(x: np.ndarray, p: Params) -> np.ndarray:
    """All reference patches (N_ref, ps, ps, C) in reference-grid order."""
    H, Wd, C = x.shape
    ys = reference_positions(H, p.ps, p.stride)
    xs = reference_positions(Wd, p.ps, p.stride)
    lin = (ys[:, None] * Wd + xs[None, :]).ravel()
    return gather_groups(x, lin[:, None], p.ps)[:, 0]


# --------------------------------------------------------------------------- t-product algebra (Sec. II-C)

def bcirc(A: np.ndarray) -> np.ndarray:
    """Block circulant matrix of the frontal slices A[:, :, k] (Sec. II-C)."""
    n1, n2, n3 = A.shape
    B = np.zeros((n1 * n3, n2 * n3), dtype=A.dtype)
    for i in range(n3):
        for j in range(n3):
            B[i * n1:(i + 1) * n1, j * n2:(j + 1) * n2] = A[:, :, (i - j) % n3]
    return B


def t_transpose(A: np.ndarray) -> np.ndarray:
    """Tensor transpose: each frontal slice transposed, slices 2..n3 in reverse order,
    so that bcirc(A^T) = bcirc(A)^T."""
    n3 = A.shape[2]
    return np.stack([A[:, :, (-k) % n3].T for k in range(n3)], axis=2)


def t_product_bcirc(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Definition T-product: bcirc(C) = bcirc(A) bcirc(B); C is read off the first block column."""
    n1, _, n3 = A.shape
    n2 = B.shape[1]
    first_col = bcirc(A) @ np.concatenate([B[:, :, k] for k in range(n3)], axis=0)
    return np.stack([first_col[k * n1:(k + 1) * n1] for k in range(n3)], axis=2).reshape(n1, n2, n3)


def t_product_fft(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """T-product computed slice-wise after an FFT along mode 3 (Eqs. FFT product, FFT third mode)."""
    AF = np.fft.fft(A, axis=2)
    BF = np.fft.fft(B, axis=2)
    CF = np.einsum("abk,bck->ack", AF, BF)
    return np.fft.ifft(CF, axis=2).real


# --------------------------------------------------------------------------- global bases (Sec. III-B.1)

def canonical_eigvecs(A: np.ndarray):
    """Reading R7: eigenpairs of a Hermitian matrix, eigenvalues descending, each eigenvector scaled by a
    unit phase so its largest-modulus entry (lowest index within 1e-6 relative) is real positive."""
    w, Q = np.linalg.eigh(A)
    w, Q = w[::-1].copy(), Q[:, ::-1].copy()
    for c in range(Q.shape[1]):
        mod = np.abs(Q[:, c])
        a = int(np.nonzero(mod >= mod.max() * (1.0 - 1e-6))[0][0])
        Q[:, c] *= np.conj(Q[a, c]) / abs(Q[a, c])
    return w, Q


def global_basis(ref_patches: np.ndarray):
    """Global projections U, V of Eq. (BCR nonlocal SVD simplified), read as the 2-D SVD of the
    reference patches per Fourier slice (reading R6).  Returns complex (C, ps, ps) arrays
    U_F, V_F of the Fourier slices, plus the eigenvalues."""
    C = ref_patches.shape[-1]
    PF = np.fft.fft(ref_patches.astype(np.float64), axis=-1)      # (N, ps, ps, C)
    ps = ref_patches.shape[1]
    U = np.zeros((C, ps, ps), dtype=np.complex128)
    V = np.zeros((C, ps, ps), dtype=np.complex128)
    lu = np.zeros((C, ps))
    lv = np.zeros((C, ps))
    for f in range(C // 2 + 1):
        X = PF[..., f]                                  # (N, a, b)
        Xr = X.transpose(1, 0, 2).reshape(ps, -1)       # rows a against (n, b)
        Xc = X.transpose(2, 0, 1).reshape(ps, -1)       # columns b against (n, a)
        A = Xr @ Xr.conj().T                            # sum_r P_f P_f^H   (rows)
        B = Xc.conj() @ Xc.T                            # sum_r P_f^H P_f   (columns)
        lu[f], U[f] = canonical_eigvecs(A)
        lv[f], V[f] = canonical_eigvecs(B)
    for f in range(C // 2 + 1, C):
        U[f], V[f] = U[C - f].conj(), V[C - f].conj()
        lu[f], lv[f] = lu[C - f], lv[C - f]
    return U, V, lu, lv


def basis_gap(lam: np.ndarray) -> float:
    """Smallest relative gap between consecutive eigenvalues (degeneracy check of reading R7)."""
    top = max(abs(lam.max()), 1e-300)
    return float(np.min(np.abs(np.diff(np.sort(lam)))) / top) if lam.size > 1 else 1.0


DEGENERATE_GAP = 1e-9


class DegenerateBasis(ValueError):
    """Reading R7: two eigenvalues of a basis slice lie within DEGENERATE_GAP (relative to the largest), so
    the slice's eigenvectors, and with them the coefficients that are thresholded, are not unique."""


def global_basis_gap(lu: np.ndarray, lv: np.ndarray) -> float:
    """Smallest basis_gap over the U and V slices f = 0 .. C // 2 (slices C - f repeat f)."""
    C = lu.shape[0]
    return min(min(basis_gap(lu[f]), basis_gap(lv[f])) for f in range(C // 2 + 1))


# --------------------------------------------------------------------------- group transform (Sec. III-B.2)

def patch_forward(G: np.ndarray, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """U^T * P * V for every patch P = G[..., k, :, :, :] (t-products in the Fourier domain):
    S_f = U_f^H P_f V_f, then the inverse FFT along the channel mode."""
    GF = np.fft.fft(G, axis=-1)
    SF = np.empty_like(GF)
    for f in range(GF.shape[-1]):
        Y = np.tensordot(GF[..., f], U[f].conj(), axes=([-2], [0]))     # (..., b, i) = (U_f^H P_f)^T
        SF[..., f] = np.tensordot(Y, V[f], axes=([-2], [0]))            # (U_f^H P_f) V_f
    return np.fft.ifft(SF, axis=-1).real


def patch_inverse(S: np.ndarray, U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """U * S * V^T per patch: P_f = U_f S_f V_f^H."""
    SF = np.fft.fft(S, axis=-1)
    GF = np.empty_like(SF)
    for f in range(SF.shape[-1]):
        Y = np.tensordot(SF[..., f], U[f].T, axes=([-2], [0]))          # (..., j, a) = (U_f S_f)^T
        GF[..., f] = np.tensordot(Y, V[f].conj().T, axes=([-2], [0]))   # (U_f S_f) V_f^H
    return np.fft.ifft(GF, axis=-1).real


def forward_transform(G: np.ndarray, U, V, H: np.ndarray) -> np.ndarray:
    """Eq. (forward transform): S = U^T * G * V x_4 U_Haar^T, with coefficient m = sum_k H[m,k] (.)_k.
    G has shape (..., K, ps, ps, C)."""
    T = patch_forward(G, U, V)
    return np.moveaxis(np.tensordot(H, T, axes=([1], [-4])), 0, -4)     # sum_k H[m, k] T_k


def inverse_transform(S: np.ndarray, U, V, H: np.ndarray) -> np.ndarray:
    """Eq. (backward transform) read as the exact inverse (reading R8): x_4 H_K^T then U * . * V^T."""
    T = np.moveaxis(np.tensordot(H.T, S, axes=([1], [-4])), 0, -4)   # sum_m H[m, k] S_m
    return patch_inverse(T, U, V)


def hard_threshold_mask(S: np.ndarray, tau: float) -> np.ndarray:
    """Eq. (hard thresholding): keep |S| >= tau."""
    return np.abs(S) >= tau


# --------------------------------------------------------------------------- aggregation (Eq. aggregation)

def aggregate(shape, idx: np.ndarray, Ghat: np.ndarray, w: np.ndarray, ps: int):
    """Weighted write-back of every estimated patch: num[p] += w_g Ghat, den[p] += w_g."""
    H, Wd, C = shape
    yy, xx = idx // Wd, idx % Wd                                        # (n, K)
    ii, jj = np.mgrid[0:ps, 0:ps]
    pix = ((yy[:, :, None, None] + ii) * Wd + (xx[:, :, None, None] + jj)).ravel()
    wk = np.broadcast_to(w[:, None, None, None], (w.size, idx.shape[1], ps, ps)).ravel()
    num = np.stack([np.bincount(pix, weights=(Ghat[..., c] * w[:, None, None, None]).ravel(),
                                minlength=H * Wd) for c in range(C)], axis=-1).reshape(H, Wd, C)
    den = np.bincount(pix, weights=wk, minlength=H * Wd).reshape(H, Wd)
    return num, den


# --------------------------------------------------------------------------- full denoiser (Alg. 1)

@dataclass
class Result:
    out: np.ndarray
    idx: np.ndarray
    tau: float
    U: np.ndarray
    V: np.ndarray
    weights: np.ndarray
    masks: np.ndarray | None = None       # (n, K, ps, ps, C) bool
    coeffs: np.ndarray | None = None      # |S| values
    ambiguous: np.ndarray | None = None   # (group, flat coefficient index) with | |S| - tau | <= 1e-9 max(tau, 1)
    den: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


def _as_quantised(x: np.ndarray) -> np.ndarray:
    if x.dtype == np.uint8:
        return x
    return np.clip(np.rint(x.astype(np.float64)), 0, 255).astype(np.uint8)


def denoise(x: np.ndarray, sigma: float, params=None, *, idx=None, weights=None,
            keep_masks=False, keep_coeffs=False, chunk=2048, tau=None, basis=None) -> Result:
    """Alg. 1: grouping, global bases, forward transform, hard threshold, inverse, aggregation.

    x: (H, W, C) uint8 or float image on the [0, 255] scale.  For float input the matching and the
    bases use the quantised image (reading R13) and the transforms use x itself.  idx restricts the
    filter to the given groups; basis = global_basis(...) of this image skips its recomputation."""
    p = Params.of(params)
    if x.ndim == 2:
        x = x[:, :, None]
    H, Wd, C = x.shape
    q = _as_quantised(x)
    if idx is None:
        idx, _ = block_match(q, p)
    U, V, lu, lv = global_basis(reference_patches(q, p)) if basis is None else basis
    gap = global_basis_gap(lu, lv)
    if p.strict_basis and not gap >= DEGENERATE_GAP:
        raise DegenerateBasis(f"smallest relative eigen-gap {gap:.3g} < {DEGENERATE_GAP:g}")
    Hk = haar_matrix(p.K)
    if tau is None:
        tau = tau_multiplier(p, C) * float(sigma)
    xf = x.astype(np.float64)
    n = idx.shape[0]
    w = np.ones(n) if weights is None else np.asarray(weights, dtype=np.float64)
    num = np.zeros((H, Wd, C))
    den = np.zeros((H, Wd))
    masks = np.zeros((n, p.K, p.ps, p.ps, C), dtype=bool) if keep_masks else None
    coeffs = np.zeros((n, p.K, p.ps, p.ps, C)) if keep_coeffs else None
    w_out = w.copy()
    amb = []
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        G = gather_groups(xf, idx[a:b], p.ps)
        S = forward_transform(G, U, V, Hk)
        m = hard_threshold_mask(S, tau)
        near = np.nonzero(np.abs(np.abs(S.reshape(b - a, -1)) - tau) <= 1e-9 * max(tau, 1.0))
        amb.extend(zip((near[0] + a).tolist(), near[1].tolist()))
        if weights is None and p.agg_mode == "sparsity":
            w_out[a:b] = 1.0 / np.maximum(1, m.reshape(b - a, -1).sum(axis=1))
        Ghat = inverse_transform(S * m, U, V, Hk)
        nu, de = aggregate((H, Wd, C), idx[a:b], Ghat, w_out[a:b], p.ps)
        num += nu
        den += de
        if keep_masks:
            masks[a:b] = m
        if keep_coeffs:
            coeffs[a:b] = np.abs(S)
    out = num / den[:, :, None]
    return Result(out=out, idx=idx, tau=tau, U=U, V=V, weights=w_out, masks=masks,
                  coeffs=coeffs, den=den, ambiguous=np.array(amb, dtype=np.int64).reshape(-1, 2),
                  extra={"basis_gap": gap})


# --------------------------------------------------------------------------- frozen-mask linear map and its adjoint

def denoise_fixed(x: np.ndarray, idx: np.ndarray, masks: np.ndarray, U, V, w: np.ndarray, ps: int):
    """Reading R14: the denoiser with grouping, bases and masks held fixed: out = N(x) / D,
    N(x) = sum_g w_g Scatter_g T^-1 (M_g . T Gather_g x), D = sum_g w_g Scatter_g 1.  Linear in x."""
    if x.ndim == 2:
        x = x[:, :, None]
    H, Wd, C = x.shape
    K = idx.shape[1]
    Hk = haar_matrix(K)
    G = gather_groups(x.astype(np.float64), idx, ps)
    Ghat = inverse_transform(forward_transform(G, U, V, Hk) * masks, U, V, Hk)
    num, den = aggregate((H, Wd, C), idx, Ghat, w, ps)
    return num / den[:, :, None], den


def denoise_fixed_vjp(x: np.ndarray, gout: np.ndarray, idx: np.ndarray, masks: np.ndarray, U, V,
                      w: np.ndarray, ps: int):
    """Reading R14: adjoint of denoise_fixed at x for cotangent gout.
    d/dx  = sum_g w_g Gather_g^T T^T (M_g . T Gather_g (gout / D))
    d/dw_g = sum over g's patches of (gout/D)[q] * (Ghat_g[q] - out[q])."""
    if x.ndim == 2:
        x = x[:, :, None]
    if gout.ndim == 2:
        gout = gout[:, :, None]
    H, Wd, C = x.shape
    K = idx.shape[1]
    Hk = haar_matrix(K)
    out, den = denoise_fixed(x, idx, masks, U, V, w, ps)
    r = gout.astype(np.float64) / den[:, :, None]
    Gr = gather_groups(r, idx, ps)
    back = inverse_transform(forward_transform(Gr, U, V, Hk) * masks, U, V, Hk)
    gx, _ = aggregate((H, Wd, C), idx, back, w, ps)
    Gx = gather_groups(x.astype(np.float64), idx, ps)
    Ghat = inverse_transform(forward_transform(Gx, U, V, Hk) * masks, U, V, Hk)
    Gout = gather_groups(out, idx, ps)
    gw = ((Ghat - Gout) * Gr).reshape(idx.shape[0], -1).sum(axis=1)
    return gx, gw


# --------------------------------------------------------------------------- noise level (Sec. III-D + reading R11/R12)

def patch_covariance(q: np.ndarray, p: Params) -> np.ndarray:
    P = reference_patches(q, p).reshape(-1, p.ps * p.ps * q.shape[2])
    mu = P.mean(axis=0)
    return P.T @ P / P.shape[0] - np.outer(mu, mu)


def sigma_from_eigenvalues(lam: np.ndarray) -> float:
    """Reading R11: the largest leading run of ascending eigenvalues whose mean stays within 2% of
    its median is taken as the noise subspace; sigma = sqrt(mean of that run)."""
    lam = np.sort(lam)
    rstar = 1
    for r in range(1, lam.size + 1):
        if lam[:r].mean() <= 1.02 * np.median(lam[:r]):
            rstar = r
    return float(math.sqrt(max(lam[:rstar].mean(), 0.0)))


def circulant_eigenvalues(G: np.ndarray) -> np.ndarray:
    """Eigenvalues of circ(G) circ(G)^T in closed form: lambda_f = || sum_m p_m exp(-2 pi i f m / K) ||^2
    (Sec. III-B.2; lambda_0 = ||sum p||^2 is Eq. (first eigen), lambda_{K/2} is Eq. (other eigenvalue))."""
    K = G.shape[0]
    P = G.reshape(K, -1).astype(np.float64)
    F = np.fft.fft(P, axis=0)
    return (np.abs(F) ** 2).sum(axis=1)


def rank_position(G: np.ndarray) -> int:
    """a = rank of lambda_hat = lambda_{K/2} among the K eigenvalues in ascending order (Sec. III-D)."""
    lam = circulant_eigenvalues(G)
    K = G.shape[0]
    return 1 + int(np.sum(lam < lam[K // 2]))


def estimate_sigma(x: np.ndarray, params=None, return_details=False):
    """Noise level from the patch covariance (reading R11), optionally adjusted by the
    eigen-rank vote of Eq. (adjust noise level) over sampled groups (reading R12)."""
    p = Params.of(params)
    if x.ndim == 2:
        x = x[:, :, None]
    q = _as_quantised(x)
    lam = np.linalg.eigvalsh(patch_covariance(q, p))
    sigma = sigma_from_eigenvalues(lam)
    det = {"lam": lam, "sigma_est": sigma}
    if p.adapt:
        H, Wd, C = q.shape
        ys = reference_positions(H, p.ps, p.stride)[::8]
        xs = reference_positions(Wd, p.ps, p.stride)[::8]
        gam = rank_gamma(p)
        low = high = 0
        ranks = []
        for ry in ys:
            for rx in xs:
                idx1, _, _ = block_match_one(q, int(ry), int(rx), p)
                a = rank_position(gather_groups(q, idx1[None], p.ps)[0])
                ranks.append(a)
                if a <= gam:
                    low += 1
                else:
                    high += 1
        if low > high:
            sigma = sigma / p.beta
        det.update(ranks=np.array(ranks), low=low, high=high)
    return (sigma, det) if return_details else sigma


# --------------------------------------------------------------------------- A-Haar-tSVD (Alg. 2)

def subimage_bounds(n: int, n_sub: int) -> list[tuple[int, int]]:
    """Reading R15: t = max(1, floor(n / n_sub)) parts of one axis, boundaries floor(i n / t)."""
    t = max(1, n // n_sub)
    return [((i * n) // t, ((i + 1) * n) // t) for i in range(t)]


def a_haar_tsvd(x: np.ndarray, sub_h: int, sub_w: int, params=None):
    """Alg. 2 (A-Haar-tSVD) with the eigenvalue noise estimate (R11, R12) in place of the CNN:
    Step 1 estimates sigma per subimage, Step 2 denoises each subimage with Alg. 1 at its sigma.
    Returns (output (H, W, C) float64, per-subimage sigmas in row-major subimage order)."""
    p = Params.of(params)
    if x.ndim == 2:
        x = x[:, :, None]
    H, Wd, C = x.shape
    out = np.zeros((H, Wd, C))
    sigmas = []
    for (y0, y1) in subimage_bounds(H, sub_h):
        for (x0, x1) in subimage_bounds(Wd, sub_w):
            sub = np.ascontiguousarray(x[y0:y1, x0:x1])
            sg = estimate_sigma(sub, p)
            sigmas.append(sg)
            out[y0:y1, x0:x1] = denoise(sub, sg, p).out
    return out, np.array(sigmas)


# --------------------------------------------------------------------------- video (Sec. IV, reading R16)

def _match_plane_ssd_pair(ref_planes, cand_planes, ry, rxs, y0, ny, x0s, nx, ps):
    """As _match_plane_ssd, with the reference patches taken from ref_planes and the candidates
    from cand_planes (another frame): (n, ny, nx) int64."""
    ssd = np.zeros((len(rxs), ny, nx), dtype=np.int64)
    cols = x0s[:, None] + np.arange(nx)[None, :]
    for rp, cp in zip(ref_planes, cand_planes):
        cand = sliding_window_view(cp, (ps, ps))[y0:y0 + ny][:, cols]     # (ny, n, nx, i, j)
        ref = sliding_window_view(rp, (ps, ps))[ry, rxs]                 # (n, i, j)
        d = cand - ref[None, :, None]
        ssd += np.einsum("ynxij,ynxij->nyx", d, d)
    return ssd


def _guide_planes(img: np.ndarray, mode: str):
    """The integer planes of one frame for each matching mode: (byte planes, R+G+B plane)."""
    x = img.astype(np.int64)
    C = x.shape[2]
    if mode == "full":
        return [x[:, :, c] for c in range(C)], None
    if C == 1:
        return [x[:, :, 0]], None
    return [x[:, :, 1]], x[:, :, 0] + x[:, :, 1] + x[:, :, 2]


def _match_row_video(video: np.ndarray, t: int, ry: int, rxs: np.ndarray, p: Params, T: int):
    """Reading R16: groups of the references (ry, rxs[n]) of frame t over frames t-T..t+T."""
    F, H, Wd, C = video.shape
    ps, K = p.ps, p.K
    y0, ny = window_range(ry, H, ps, p.window)
    xw = [window_range(int(rx), Wd, ps, p.window) for rx in rxs]
    x0s = np.array([a for a, _ in xw], dtype=np.int64)
    nx = xw[0][1]
    mode = resolve_match_mode(p.match_mode, C)
    n = len(rxs)
    if mode == "full" or C == 1 or mode == "gray":
        green = np.ones(n, dtype=bool) if mode != "full" else np.zeros(n, dtype=bool)
    else:
        green = np.array([gcp_uses_green(video[t], ry, int(rx), ps, p.gcp_gamma) for rx in rxs])
    rb, rs = _guide_planes(video[t], mode)
    if mode == "gray" and C == 3:
        rb = [video[t].astype(np.int64)[:, :, 1]]
    f0, f1 = max(0, t - T), min(F - 1, t + T)
    ssds, lins = [], []
    for f in range(f0, f1 + 1):
        cb, cs = _guide_planes(video[f], mode)
        if mode == "gray" and C == 3:
            cb = [video[f].astype(np.int64)[:, :, 1]]
        sb = _match_plane_ssd_pair(rb, cb, ry, rxs, y0, ny, x0s, nx, ps)
        if rs is not None and mode == "gcp":
            ss = _match_plane_ssd_pair([rs], [cs], ry, rxs, y0, ny, x0s, nx, ps)
            sb = np.where(green[:, None, None], sb, ss)
        lin = (f * H * Wd + (y0 + np.arange(ny))[None, :, None] * Wd
               + (x0s[:, None, None] + np.arange(nx)[None, None, :]))
        ssds.append(sb.reshape(n, -1))
        lins.append(np.broadcast_to(lin, sb.shape).reshape(n, -1))
    ssd = np.concatenate(ssds, axis=1)
    lin = np.concatenate(lins, axis=1)
    ref_lin = t * H * Wd + ry * Wd + rxs
    if ssd.shape[1] - 1 < K - 1:
        raise ValueError("search window holds fewer than K candidates")
    idx = np.empty((n, K), dtype=np.int64)
    for r in range(n):
        keep = lin[r] != ref_lin[r]
        cl, cs = lin[r][keep], ssd[r][keep]
        order = np.lexsort((cl, cs))[:K - 1]                 # ascending SSD, ties -> lowest global index
        idx[r, 0] = ref_lin[r]
        idx[r, 1:] = cl[order]
    return idx, green


def block_match_video(video: np.ndarray, t: int, params=None, T: int = 1):
    """Reading R16 for every reference patch of frame t (row-major reference grid): global
    indices f*H*W + y*W + x (N_ref, K), slot 0 the reference, and the per-reference green flags."""
    p = Params.of(params)
    if video.ndim == 3:
        video = video[..., None]
    F, H, Wd, C = video.shape
    ys = reference_positions(H, p.ps, p.stride)
    xs = reference_positions(Wd, p.ps, p.stride)
    rows = [_match_row_video(video, t, int(ry), xs, p, T) for ry in ys]
    return np.concatenate([r[0] for r in rows]), np.concatenate([r[1] for r in rows])


def gather_groups_video(xv: np.ndarray, idx: np.ndarray, ps: int) -> np.ndarray:
    """Stack the K patches named by global indices f*H*W + y*W + x: (n, K, ps, ps, C) float64."""
    F, H, Wd, C = xv.shape
    views = sliding_window_view(xv.astype(np.float64), (ps, ps), axis=(1, 2))    # [f, y, x, C, i, j]
    f, rem = idx // (H * Wd), idx % (H * Wd)
    g = views[f, rem // Wd, rem % Wd]                                              # [n, K, C, i, j]
    return np.ascontiguousarray(np.moveaxis(g, 2, -1))


def aggregate_frame(shape, t: int, idx: np.ndarray, Ghat: np.ndarray, w: np.ndarray, ps: int):
    """Eq. (aggregation) restricted to frame t (reading R16): the estimated patches whose global
    index lies in frame t are written back with their group's weight; the others are dropped."""
    H, Wd, C = shape
    inf = (idx // (H * Wd)) == t
    loc = idx % (H * Wd)
    g_i, k_i = np.nonzero(inf)
    yy, xx = loc[g_i, k_i] // Wd, loc[g_i, k_i] % Wd
    ii, jj = np.mgrid[0:ps, 0:ps]
    pix = ((yy[:, None, None] + ii) * Wd + (xx[:, None, None] + jj)).ravel()
    wg = w[g_i]
    num = np.stack([np.bincount(pix, weights=(Ghat[g_i, k_i, :, :, c] * wg[:, None, None]).ravel(),
                                minlength=H * Wd) for c in range(C)], axis=-1).reshape(H, Wd, C)
    den = np.bincount(pix, weights=np.broadcast_to(wg[:, None, None], (wg.size, ps, ps)).ravel(),
                      minlength=H * Wd).reshape(H, Wd)
    return num, den


def denoise_video(video: np.ndarray, sigma=None, params=None, T: int = 1, *, keep_masks=False, chunk=2048):
    """Reading R16: a uint8 clip (F, H, W, C) denoised frame by frame with spatio-temporal grouping.
    sigma None -> estimated per frame (R11, R12); else used for every frame.
    Returns (output (F, H, W, C) float64, per-frame Results with global idx, masks and ambiguity)."""
    p = Params.of(params)
    if video.ndim == 3:
        video = video[..., None]
    F, H, Wd, C = video.shape
    xv = video.astype(np.float64)
    Hk = haar_matrix(p.K)
    out = np.zeros((F, H, Wd, C))
    results = []
    for t in range(F):
        frame = video[t]
        sg = estimate_sigma(frame, p) if sigma is None else float(sigma)
        idx, _ = block_match_video(video, t, p, T)
        U, V, _, _ = global_basis(reference_patches(frame, p))
        tau = tau_multiplier(p, C) * sg
        n = idx.shape[0]
        num = np.zeros((H, Wd, C))
        den = np.zeros((H, Wd))
        masks = np.zeros((n, p.K, p.ps, p.ps, C), dtype=bool) if keep_masks else None
        w_out = np.ones(n)
        amb = []
        for a in range(0, n, chunk):
            b = min(n, a + chunk)
            G = gather_groups_video(xv, idx[a:b], p.ps)
            S = forward_transform(G, U, V, Hk)
            m = hard_threshold_mask(S, tau)
            near = np.nonzero(np.abs(np.abs(S.reshape(b - a, -1)) - tau) <= 1e-9 * max(tau, 1.0))
            amb.extend(zip((near[0] + a).tolist(), near[1].tolist()))
            if p.agg_mode == "sparsity":
                w_out[a:b] = 1.0 / np.maximum(1, m.reshape(b - a, -1).sum(axis=1))
            Ghat = inverse_transform(S * m, U, V, Hk)
            nu, de = aggregate_frame((H, Wd, C), t, idx[a:b], Ghat, w_out[a:b], p.ps)
            num += nu
            den += de
            if keep_masks:
                masks[a:b] = m
        out[t] = num / den[:, :, None]
        results.append(Result(out=out[t], idx=idx, tau=tau, U=U, V=V, weights=w_out, masks=masks, den=den,
                              ambiguous=np.array(amb, dtype=np.int64).reshape(-1, 2), extra={"sigma": sg}))
    return out, results


# --------------------------------------------------------------------------- threshold selection (reading R17)

def sure(x: np.ndarray, sigma: float, tau_mults, probe: np.ndarray, params=None, eps: float = 0.0) -> np.ndarray:
    """Reading R17: SURE(m) for every multiplier m. x: float (H, W, C) image on the [0, 255] scale
    (float32 values); probe: same shape. eps > 0: the divergence is the finite difference of the
    whole denoiser along the probe; eps = 0: the frozen-mask adjoint applied to the probe."""
    p = Params.of(params)
    if x.ndim == 2:
        x = x[:, :, None]
    if probe.ndim == 2:
        probe = probe[:, :, None]
    xf = x.astype(np.float64)
    b = probe.astype(np.float64)
    n = xf.size
    z = None
    if eps > 0:
        # the perturbed image in float32, each operation rounded once
        z = (x.astype(np.float32) + np.float32(eps) * probe.astype(np.float32)).astype(np.float64)
    res = []
    for m in tau_mults:
        pm = Params.of(dict(p.__dict__, tau_mult=float(m)))
        r = denoise(xf, sigma, pm, keep_masks=eps == 0)
        if eps > 0:
            div = float((b * (denoise(z, sigma, pm).out - r.out)).sum()) / eps
        else:
            gx, _ = denoise_fixed_vjp(xf, b, r.idx, r.masks, r.U, r.V, r.weights, pm.ps)
            div = float((b * gx).sum())
        res.append(((r.out - xf) ** 2).sum() / n - sigma ** 2 + 2.0 * sigma ** 2 / n * div)
    return np.array(res)


# --------------------------------------------------------------------------- weight tuning (reading R19)

def perturbed(x: np.ndarray, probe: np.ndarray, eps: float) -> np.ndarray:
    """z = y + eps b formed in float32 as the device forms it (reading R17)."""
    return (x.astype(np.float32) + np.float32(eps) * probe.astype(np.float32)).astype(np.float64)


def sure_weights(x: np.ndarray, sigma: float, w: np.ndarray, probe: np.ndarray, params=None,
                 eps: float = 1.0):
    """Reading R19: SURE of the denoiser with per-group weights w (tau = tau_mult sigma) and its
    gradient in w. Returns (sure, grad_w)."""
    p = Params.of(params)
    if x.ndim == 2:
        x = x[:, :, None]
    if probe.ndim == 2:
        probe = probe[:, :, None]
    xf = x.astype(np.float64)
    b = probe.astype(np.float64)
    w = np.asarray(w, dtype=np.float64)
    n = xf.size
    z = perturbed(x, probe, eps)
    ry = denoise(xf, sigma, p, weights=w, keep_masks=True)
    rz = denoise(z, sigma, p, weights=w, keep_masks=True)
    beta = 2.0 * sigma ** 2 / (n * eps)
    sure_w = ((ry.out - xf) ** 2).sum() / n - sigma ** 2 + beta * float((b * (rz.out - ry.out)).sum())
    _, gy = denoise_fixed_vjp(xf, 2.0 / n * (ry.out - xf) - beta * b, ry.idx, ry.masks, ry.U, ry.V, w, p.ps)
    _, gz = denoise_fixed_vjp(z, beta * b, rz.idx, rz.masks, rz.U, rz.V, w, p.ps)
    return float(sure_w), gy + gz


def tune_weights(x: np.ndarray, sigma: float, probe: np.ndarray, params=None, eps: float = 1.0,
                 steps: int = 3, step: float = 0.5, w0=None):
    """Reading R19: `steps` exponentiated-gradient steps on SURE(w) from w0 (default all ones).
    Returns (w, trace) with trace the SURE before each step and after the last."""
    p = Params.of(params)
    n_groups = len(reference_positions(x.shape[0], p.ps, p.stride)) * len(reference_positions(x.shape[1], p.ps, p.stride))
    w = np.ones(n_groups) if w0 is None else np.asarray(w0, dtype=np.float64).copy()
    trace = []
    for it in range(steps + 1):
        sv, g = sure_weights(x, sigma, w, probe, p, eps)
        trace.append(sv)
        if it == steps:
            break
        gm = np.abs(g).max()
        if gm > 0:
            w = w * np.exp(-step * g / gm)
    return w, np.array(trace)


# --------------------------------------------------------------------------- MRI volumes (reading R20)

def volume_reference_positions(shape, p: Params) -> np.ndarray:
    """Linear positions (z H + y) W + x of the reference cubes, z-major over the grid of R3 per axis."""
    D, Hh, Wd = shape
    zs, ys, xs = (reference_positions(n, p.ps, p.stride) for n in (D, Hh, Wd))
    return ((zs[:, None, None] * Hh + ys[None, :, None]) * Wd + xs[None, None, :]).ravel()


def gather_cubes(v: np.ndarray, idx: np.ndarray, ps: int) -> np.ndarray:
    """The cubes at linear positions idx as (..., ps, ps, ps) float64 tensors P[i][j][k] =
    v[z + k, y + i, x + j] (rows along y, columns along x, the tube along z)."""
    D, Hh, Wd = v.shape
    views = sliding_window_view(v.astype(np.float64), (ps, ps, ps))      # [z, y, x, dz, dy, dx]
    z, r = np.divmod(idx, Hh * Wd)
    y, x = np.divmod(r, Wd)
    return np.ascontiguousarray(np.moveaxis(views[z, y, x], -3, -1))


def block_match_volume(v: np.ndarray, params=None, only=None) -> np.ndarray:
    """Grouping of a (D, H, W) uint8 volume (reading R20): for every reference cube of the grid,
    itself in slot 0, then the K - 1 other candidates of its W x W x W window with the smallest
    (exact integer SSD over the ps^3 voxels, linear index) keys. Returns (N_ref, K) int64; with
    `only` (group numbers, z-major over the grid) just those groups, in that order."""
    p = Params.of(params)
    D, Hh, Wd = v.shape
    ps = p.ps
    views = sliding_window_view(v.astype(np.int64), (ps, ps, ps))
    zs, ys, xs = (reference_positions(n, ps, p.stride) for n in (D, Hh, Wd))
    if only is None:
        only = np.arange(len(zs) * len(ys) * len(xs))
    out = np.empty((len(only), p.K), dtype=np.int64)
    for g, gi in enumerate(np.asarray(only, dtype=np.int64)):
        iz, r = divmod(int(gi), len(ys) * len(xs))
        iy, ix = divmod(r, len(xs))
        z, y, x = int(zs[iz]), int(ys[iy]), int(xs[ix])
        z0, nz = window_range(z, D, ps, p.window)
        y0, ny = window_range(y, Hh, ps, p.window)
        x0, nx = window_range(x, Wd, ps, p.window)
        ref = views[z, y, x]
        cand = views[z0:z0 + nz, y0:y0 + ny, x0:x0 + nx]
        ssd = ((cand - ref) ** 2).sum(axis=(3, 4, 5)).ravel()
        cz, cy, cx = np.meshgrid(np.arange(z0, z0 + nz), np.arange(y0, y0 + ny), np.arange(x0, x0 + nx),
                                 indexing="ij")
        lin = ((cz * Hh + cy) * Wd + cx).ravel()
        me = (z * Hh + y) * Wd + x
        keep = lin != me
        order = np.lexsort((lin[keep], ssd[keep]))
        if order.size < p.K - 1:
            raise ValueError("the search window holds fewer than K cubes")
        out[g, 0] = me
        out[g, 1:] = lin[keep][order[:p.K - 1]]
    return out


def aggregate_volume(shape, idx: np.ndarray, Ghat: np.ndarray, w: np.ndarray, ps: int):
    """Weighted write-back of every estimated cube into the volume: num += w_g Ghat, den += w_g."""
    D, Hh, Wd = shape
    z, r = np.divmod(idx, Hh * Wd)
    y, x = np.divmod(r, Wd)
    ii, jj, kk = np.meshgrid(np.arange(ps), np.arange(ps), np.arange(ps), indexing="ij")
    e = (slice(None), slice(None), None, None, None)
    vox = ((z[e] + kk) * Hh + (y[e] + ii)) * Wd + (x[e] + jj)                  # (n, K, i, j, k)
    we = w[:, None, None, None, None]
    wg = np.broadcast_to(we, vox.shape)
    num = np.bincount(vox.ravel(), weights=(Ghat * we).ravel(), minlength=D * Hh * Wd)
    den = np.bincount(vox.ravel(), weights=wg.ravel(), minlength=D * Hh * Wd)
    return num.reshape(D, Hh, Wd), den.reshape(D, Hh, Wd)


def denoise_volume(v: np.ndarray, sigma: float, params=None, *, idx=None, keep_masks=False, tau=None,
                   chunk=1024, basis=None) -> Result:
    """Alg. 1 on a (D, H, W) uint8 volume with ps x ps x ps cubes (reading R20): grouping, global
    bases of the reference cubes per tube-Fourier slice, forward transform, hard threshold,
    inverse, aggregation. idx fixes the grouping (as block_match_volume would return it); basis =
    global_basis(...) of this volume's reference cubes skips its recomputation."""
    p = Params.of(params)
    D, Hh, Wd = v.shape
    ps = p.ps
    if idx is None:
        idx = block_match_volume(v, p)
    if basis is None:
        basis = global_basis(gather_cubes(v, volume_reference_positions(v.shape, p), ps))
    U, V, lu, lv = basis
    gap = global_basis_gap(lu, lv)
    if p.strict_basis and not gap >= DEGENERATE_GAP:
        raise DegenerateBasis(f"smallest relative eigen-gap {gap:.3g} < {DEGENERATE_GAP:g}")
    Hk = haar_matrix(p.K)
    if tau is None:
        tau = tau_multiplier(p, ps) * float(sigma)
    n = idx.shape[0]
    w = np.ones(n)
    num = np.zeros((D, Hh, Wd))
    den = np.zeros((D, Hh, Wd))
    masks = np.zeros((n, p.K, ps, ps, ps), dtype=bool) if keep_masks else None
    amb = []
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        G = gather_cubes(v, idx[a:b], ps)
        S = forward_transform(G, U, V, Hk)
        m = hard_threshold_mask(S, tau)
        near = np.nonzero(np.abs(np.abs(S.reshape(b - a, -1)) - tau) <= 1e-9 * max(tau, 1.0))
        amb.extend(zip((near[0] + a).tolist(), near[1].tolist()))
        if p.agg_mode == "sparsity":
            w[a:b] = 1.0 / np.maximum(1, m.reshape(b - a, -1).sum(axis=1))
        Ghat = inverse_transform(S * m, U, V, Hk)
        nu, de = aggregate_volume(v.shape, idx[a:b], Ghat, w[a:b], ps)
        num += nu
        den += de
        if keep_masks:
            masks[a:b] = m
    return Result(out=num / den, idx=idx, tau=tau, U=U, V=V, weights=w, masks=masks, den=den,
                  ambiguous=np.array(amb, dtype=np.int64).reshape(-1, 2), extra={"basis_gap": gap})


def estimate_sigma_volume(v: np.ndarray, params=None) -> float:
    """Noise level of a volume (reading R20 with R11): the eigenvalue rule on the covariance of the
    reference cubes, each flattened in (i, j, k) order."""
    p = Params.of(params)
    P = gather_cubes(v, volume_reference_positions(v.shape, p), p.ps).reshape(-1, p.ps ** 3)
    mu = P.mean(axis=0)
    return sigma_from_eigenvalues(np.linalg.eigvalsh(P.T @ P / P.shape[0] - np.outer(mu, mu)))


def a_haar_tsvd_volume(v: np.ndarray, sub: tuple, params=None):
    """Alg. 2 on a volume (reading R21, the paper's adaptive variant on MRI): each axis cut
    into sub-volumes as R15 cuts image axes; per sub-volume the noise level by the eigenvalue rule on
    its reference cubes (estimate_sigma_volume) and Alg. 1 at that level. The eigen-rank vote of R12
    is not applied to volumes. Returns (output (D, H, W) float64, sigmas in z-major sub-volume order)."""
    p = Params.of(params)
    out = np.zeros(v.shape)
    sigmas = []
    for (z0, z1) in subimage_bounds(v.shape[0], sub[0]):
        for (y0, y1) in subimage_bounds(v.shape[1], sub[1]):
            for (x0, x1) in subimage_bounds(v.shape[2], sub[2]):
                part = np.ascontiguousarray(v[z0:z1, y0:y1, x0:x1])
                sg = estimate_sigma_volume(part, p)
                sigmas.append(sg)
                out[z0:z1, y0:y1, x0:x1] = denoise_volume(part, sg, p).out
    return out, np.array(sigmas)

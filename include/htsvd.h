/*
 * htsvd.h — C ABI of the GB300 Haar-tSVD denoising core.
 *
 * Method: Kong, Zhang & Yang, "Efficient Image Denoising Using Global and Local
 * Circulant Representation" (arXiv 2508.10307), Algorithm 1 (Haar-tSVD) and the
 * eigenvalue analysis of Sec. III-D.
 *
 * Conventions shared by every entry point
 *  - Images are contiguous row-major H x W x C (HWC), C in {1, 3}, on the
 *    [0, 255] scale (hyperspectral cubes take C = N bands and MRI volumes are
 *    D x H x W: see those calls). Pointers named d_* are DEVICE pointers owned by
 *    the caller; pointers named h_* or documented as host are HOST pointers.
 *  - Patches are ps x ps with ps = 8 (the paper's value, Sec. IV-A; other sizes
 *    return HTSVD_ERR_UNSUPPORTED; volumes use 4 x 4 x 4 cubes). K is a power of
 *    two in [2, 32].
 *  - Reference patches sit on the grid {0, s, 2s, ...} U {n - ps} of each axis,
 *    row-major; group g belongs to the g-th reference of that order.
 *  - Match indices are int32 linear top-left positions y * W + x, K per group;
 *    slot 0 is the reference itself, slots 1..K-1 the K-1 nearest other
 *    candidates of its search window by (SSD, linear index) ascending.
 *  - Calls are asynchronous on `stream` except where a host result is
 *    returned (documented per call). The library owns a workspace cached per
 *    (device, stream); it grows with cudaMalloc on first use at a size. Calls
 *    on different streams may run from different host threads at once; calls
 *    on one stream share its workspace, so host threads that issue them must
 *    serialise them (stream order then keeps their kernels apart).
 *  - No exceptions cross this ABI; every call returns an htsvd_status.
 */
#ifndef HTSVD_H
#define HTSVD_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum htsvd_status {
    HTSVD_OK = 0,
    HTSVD_ERR_INVALID_ARG = 1,   /* bad size, pointer or parameter */
    HTSVD_ERR_UNSUPPORTED = 2,   /* valid for the method, not built here (ps != 8, K > 32, window > 64) */
    HTSVD_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    HTSVD_ERR_OOM = 4,           /* workspace allocation failed */
    HTSVD_ERR_TIMEOUT = 5,       /* reserved: no kernel of this library waits on another CTA, so no call returns it */
    HTSVD_ERR_DEGENERATE_BASIS = 6, /* strict mode only: a global-basis slice has a relative eigen-gap below 1e-9,
                                       so its eigenvectors (and the coefficients) are not unique (Sec. III-B.1) */
} htsvd_status;

typedef enum htsvd_match_mode {
    HTSVD_MATCH_AUTO = 0,   /* C=1: the gray plane; C=3: green-channel prior (GCP) */
    HTSVD_MATCH_GCP = 1,    /* Sec. III-A, Eq. (GCP distance): G plane if ||G|| >= max(||R||,||B||)/gamma on the
                               reference patch, else the R+G+B plane (same order as the channel average) */
    HTSVD_MATCH_FULL = 2,   /* SSD summed over all channels */
    HTSVD_MATCH_GREEN = 3,  /* always the G plane (C=3) */
} htsvd_match_mode;

typedef enum htsvd_agg_mode {
    HTSVD_AGG_UNIFORM = 0,  /* every group weighs 1: the plain average of Alg. 1 Step 3 */
    HTSVD_AGG_SPARSITY = 1, /* w_g = 1 / max(1, number of kept coefficients of g), Eq. (aggregation) weights */
} htsvd_agg_mode;

/* Parameters. A zero-filled struct means the paper's defaults (Sec. IV-A):
 * ps 8, K 32, window 18, stride 3, tau = sigma * sqrt(2 ln(C K ps^2)), gamma 1.2,
 * beta 1.2, rank gamma 13 (scaled by K/32). */
typedef struct htsvd_params {
    int32_t ps;            /* patch size; 0 -> 8 */
    int32_t stride;        /* reference grid step; 0 -> 3 */
    int32_t window;        /* search window W (candidate top-left positions per axis); 0 -> 18, at most 64 */
    int32_t K;             /* patches per group; 0 -> 32 */
    double  tau_mult;      /* tau = tau_mult * sigma; <= 0 -> sqrt(2 ln(C K ps^2)) (Sec. IV-A) */
    int32_t match_mode;    /* htsvd_match_mode */
    double  gcp_gamma;     /* <= 0 -> 1.2 (Sec. III-A) */
    int32_t agg_mode;      /* htsvd_agg_mode */
    int32_t adapt;         /* sigma estimation: apply the eigen-rank vote of Eq. (adjust noise level) */
    double  beta;          /* <= 0 -> 1.2 (Sec. III-D) */
    int32_t rank_gamma;    /* <= 0 -> 13 K / 32 rounded half up, (13 K + 16) / 32 (Sec. III-D) */
    int32_t tile;          /* reference tile edge for the filter (0 -> automatic), at most 16 */
    /* Optional outputs (may be NULL). */
    double*   h_sigma_out;   /* HOST: the sigma actually used (estimated when sigma < 0) */
    uint32_t* d_mask_out;    /* DEVICE: threshold masks, per group ceil(K*ps*ps*C/32) words, bit index
                                ((m*ps + i)*ps + j)*C + c for Haar row m, pixel (i, j), channel c */
    float*    d_weights_out; /* DEVICE: per-group aggregation weights actually used */
    double*   d_basis_out;   /* DEVICE: 2*C*ps*ps complex values (re, im): U_F slices then V_F slices,
                                each slice row-major [a][i] (column i = i-th eigenvector) */
    float*    d_coef_out;    /* DEVICE: FP32 coefficients S before thresholding, K*ps*ps*C floats per group,
                                same index as the mask bits (for accuracy checks) */
    /* Eigen-gap check of the global bases (Sec. III-B.1: the bases are eigenvectors of the per-slice
     * scatter matrices; where two eigenvalues coincide the eigenvectors, and so the thresholded
     * coefficients, are not unique). The gap of a slice is min_i |l_i - l_{i+1}| / |l_max| over its
     * eigenvalues; the check takes the smallest over all U and V slices. Either field makes the call
     * synchronise `stream` once after the basis solve. Honoured by htsvd_denoise, htsvd_denoise_f32,
     * htsvd_denoise_noalloc, htsvd_denoise_cube and htsvd_denoise_volume; htsvd_denoise_volume_adaptive
     * applies strict_basis to every part and does not report a gap. */
    int32_t   strict_basis;  /* nonzero: return HTSVD_ERR_DEGENERATE_BASIS (before the filter runs, d_out
                                unwritten) when that gap is below 1e-9; zero: no check (production) */
    double*   h_basis_gap_out; /* HOST (may be NULL): receives that smallest relative gap */
} htsvd_params;

/* One image of a batch. */
typedef struct htsvd_image {
    const uint8_t* d_in;   /* H x W x C uint8 */
    int32_t H, W, C;
    double sigma;          /* noise level; must be >= 0 in a batch */
    float* d_out;          /* H x W x C float32 */
    int32_t* d_idx_out;    /* optional (may be NULL): N_groups x K int32 match indices of this image, as the
                              d_idx_out of htsvd_denoise (the batch then groups into this buffer) */
} htsvd_image;

/* Alg. 1 (Haar-tSVD) on a uint8 image.
 * sigma >= 0: the given noise level; sigma < 0: estimated on the device with the
 * eigenvalue rule of htsvd_estimate_sigma (one host synchronisation, overlapped with
 * block matching).
 * d_out: H*W*C float32, the aggregated estimate, unclipped.
 * d_idx_out: optional N_groups*K int32 match indices (see conventions).
 * Errors: INVALID_ARG if H or W < ps, C not 1 or 3, K not a power of two, stride < 1,
 * window < 1, or the search window holds fewer than K positions. */
htsvd_status htsvd_denoise(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, double sigma,
                           const htsvd_params* p, float* d_out, int32_t* d_idx_out, cudaStream_t stream);

/* Alg. 1 on a float32 image x (H x W x C on the [0, 255] scale). Grouping, the global
 * bases and an estimated sigma use q = clip(rint(x), 0, 255); the transforms use x.
 * d_w: optional per-group aggregation weights (N_groups floats); NULL uses p->agg_mode.
 * Other arguments as htsvd_denoise. */
htsvd_status htsvd_denoise_f32(const float* d_x, int32_t H, int32_t W, int32_t C, double sigma,
                               const htsvd_params* p, const float* d_w, float* d_out, int32_t* d_idx_out,
                               cudaStream_t stream);

/* Color video (Sec. IV, real-world color video denoising: the patch search covers space and
 * time, the noise estimate runs frame by frame). d_video: F frames of H x W x C uint8, frame-major
 * (DEVICE); d_out: the same shape in float32 (DEVICE). Output frame t is Alg. 1 on frame t with
 * frame t's own global bases and sigma (estimated from frame t when sigma < 0, else sigma for
 * every frame), except that grouping searches the spatial window in frames t - T .. t + T
 * (clipped to the clip) and only the patches lying in frame t are aggregated into it. Group
 * indices are global, f * H * W + y * W + x; ties break towards the lowest. T = 0 gives
 * htsvd_denoise on every frame. d_idx_out (DEVICE, may be NULL): the groups of every frame,
 * F x N_groups x K int32 (frame-major, each frame as htsvd_denoise's d_idx_out). h_sigmas (HOST,
 * may be NULL) receives the F sigmas used.
 * Synchronises `stream` once per frame when sigma is estimated. Errors: INVALID_ARG for a null
 * pointer, F < 1, T < 0 or a frame that fails the checks of htsvd_denoise; UNSUPPORTED when
 * F * H * W reaches 2^31; optional outputs of p are ignored. */
htsvd_status htsvd_denoise_video(const uint8_t* d_video, int32_t F, int32_t H, int32_t W, int32_t C, int32_t T,
                                 double sigma, const htsvd_params* p, float* d_out, int32_t* d_idx_out,
                                 double* h_sigmas, cudaStream_t stream);

/* A sweep of thresholds (parameter tuning, Sec. III-E: the grouping and the noisy coefficients
 * are computed once and cached). d_noisy: H x W x C uint8 (DEVICE); h_tau_mults: n_tau >= 1
 * threshold multipliers (HOST, each finite and >= 0); d_outs: n_tau x H x W x C float32 (DEVICE).
 * Output i equals htsvd_denoise at tau = h_tau_mults[i] * sigma (sigma < 0: estimated once,
 * returned in h_sigma, HOST, may be NULL). The cache takes N_groups x K x 64 C floats of device
 * memory in the stream's workspace. Errors: INVALID_ARG for a null pointer, n_tau < 1, a negative or
 * non-finite multiplier, or an image that fails the checks of htsvd_denoise; UNSUPPORTED for
 * K < 8; optional outputs of p are ignored. Synchronises `stream` once when sigma is estimated. */
htsvd_status htsvd_denoise_tau_sweep(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, double sigma,
                                     const double* h_tau_mults, int32_t n_tau, const htsvd_params* p,
                                     float* d_outs, double* h_sigma, cudaStream_t stream);

/* Threshold selection by Stein's unbiased risk estimate (tuning, Sec. III-E). For each multiplier
 * m = h_tau_mults[i] > 0: f = htsvd_denoise_f32 at tau = m * sigma on d_y (H x W x C float32 on the
 * [0, 255] scale, DEVICE), n = H W C, b = d_probe (H x W x C float32, DEVICE; a +-1 Rademacher
 * vector makes the divergence below an unbiased estimate of trace J), and
 *   h_sure[i] = ||f - y||^2 / n - sigma^2 + (2 sigma^2 / n) div.
 * eps > 0: div = b^T (f(z) - f(y)) / eps, the Monte-Carlo finite difference of the whole denoiser
 * (Ramani, Blu and Unser, 2008) with z = y + eps b formed in float32, each operation rounded once;
 * f(z) groups and solves the bases of z, so the hard threshold's jumps and the bases' dependence
 * on y are counted (eps about sigma / 10 suits the [0, 255] scale). eps = 0: div = b^T J^T b with
 * J^T b the vector-Jacobian product of htsvd_denoise_vjp (grouping, bases, tau and masks held
 * fixed), which counts neither and so falls below the true risk. Sums in FP64. sigma > 0 is
 * required. h_sure: n_tau doubles (HOST). Synchronises `stream`. Errors: INVALID_ARG for a null
 * pointer, n_tau < 1, sigma or a multiplier not positive and finite, eps negative, not finite or
 * vanishing in float32, or an image that fails the checks of htsvd_denoise; optional outputs of p
 * are ignored. */
htsvd_status htsvd_sure(const float* d_y, int32_t H, int32_t W, int32_t C, double sigma, const double* h_tau_mults,
                        int32_t n_tau, const float* d_probe, double eps, const htsvd_params* p, double* h_sure,
                        cudaStream_t stream);

/* Per-group aggregation weights scored by Stein's unbiased risk estimate (tuning, Sec. III-E, with
 * the weights of the aggregation, Sec. II-B, as the free parameters). For weights w (d_w: N_groups
 * floats > 0, DEVICE, N_groups = htsvd_num_groups) let f_w(x) be htsvd_denoise_f32 of x aggregated
 * with w (tau = tau_mult * sigma; the grouping, bases and masks of x, none of which depends on w).
 * With y = d_y (H x W x C float32 on the [0, 255] scale, DEVICE), b = d_probe (same shape, DEVICE; a
 * +-1 Rademacher vector), n = H W C and z = y + eps b formed in float32 as in htsvd_sure:
 *   h_sure = ||f_w(y) - y||^2 / n - sigma^2 + (2 sigma^2 / n) b^T (f_w(z) - f_w(y)) / eps,
 *   d_grad_w = dSURE/dw = G_y((2/n)(f_w(y) - y) - (2 sigma^2 / (n eps)) b) + G_z((2 sigma^2 / (n eps)) b),
 * G_x(u) the weight gradient of htsvd_denoise_vjp at x for the cotangent u. f_w is a ratio of sums
 * linear in w, so this is the exact gradient of SURE for the groupings and masks of y and z.
 * h_sure: HOST double; d_grad_w: N_groups floats (DEVICE). Synchronises `stream`. Errors:
 * INVALID_ARG for a null pointer, sigma not positive and finite, eps not positive, finite and
 * non-zero in float32, or an image that fails the checks of htsvd_denoise; optional outputs of p are
 * ignored. */
htsvd_status htsvd_sure_weights(const float* d_y, int32_t H, int32_t W, int32_t C, double sigma, const float* d_w,
                                const float* d_probe, double eps, const htsvd_params* p, double* h_sure,
                                float* d_grad_w, cudaStream_t stream);

/* n_steps exponentiated-gradient steps on the SURE of htsvd_sure_weights: from d_w (in: start, out:
 * tuned; N_groups floats > 0, DEVICE), w <- w exp(-step g / max|g|) with g the gradient, which keeps
 * every weight positive (nothing moves when g vanishes). The groupings and bases of y and z are formed
 * once. h_sure: n_steps + 1 doubles (HOST): SURE before each step and after the last. step > 0 and
 * finite, n_steps >= 0; otherwise errors as htsvd_sure_weights. Synchronises `stream` once per step. */
htsvd_status htsvd_tune_weights(const float* d_y, int32_t H, int32_t W, int32_t C, double sigma, const float* d_probe,
                                double eps, int32_t n_steps, double step, const htsvd_params* p, float* d_w,
                                double* h_sure, cudaStream_t stream);

/* Noise level from the eigenvalues of the covariance of the reference patches:
 * ascending eigenvalues l_1..l_d, r* = max{r : mean(l_1..r) <= 1.02 median(l_1..r)},
 * sigma = sqrt(mean(l_1..r*)). With p->adapt the eigen-rank vote of Sec. III-D,
 * Eq. (adjust noise level), over groups of every 8th reference per axis divides it by beta.
 * h_sigma: HOST output. Synchronises `stream`. */
htsvd_status htsvd_estimate_sigma(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C,
                                  const htsvd_params* p, double* h_sigma, cudaStream_t stream);

/* A-Haar-tSVD (Alg. 2), with the patch-covariance eigenvalue estimate (and, when p->adapt is
 * set, the eigen-rank vote of Eq. (adjust noise level)) in place of the paper's CNN estimator.
 * The uint8 image d_noisy (H x W x C, DEVICE) is cut into subimages: each axis of length n into
 * t = max(1, n / n_sub) parts with boundaries floor(i n / t), so every part is at least n_sub
 * long (sub_h, sub_w >= 1). Step 1 estimates sigma per subimage; Step 2 denoises every
 * subimage on its own (Alg. 1, its own grouping, bases and threshold) at that sigma, all in one
 * batched pass (htsvd_denoise_batch), and writes it into d_out (H x W x C float32, DEVICE).
 * h_sigmas (HOST, may be NULL) receives the subimage sigmas in row-major subimage order.
 * Synchronises `stream` once (host eigenvalue step). Errors: INVALID_ARG for a null pointer,
 * sub_h or sub_w < 1, or a subimage that fails the checks of htsvd_denoise; optional outputs of p
 * are ignored. */
htsvd_status htsvd_denoise_adaptive(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, int32_t sub_h,
                                    int32_t sub_w, const htsvd_params* p, float* d_out, double* h_sigmas,
                                    cudaStream_t stream);

/* Alg. 1 on n uint8 images of any sizes (one C for the whole batch) with per-image sigma
 * (>= 0). Each phase (moments, bases, grouping, filter, reduction) is one persistent launch
 * whose CTAs take (image, tile) work items from a queue over all images; the sequence is
 * captured into a CUDA graph that later calls with the same images, sizes, sigmas and
 * parameters replay. The first call for a new batch shape also times candidate tile shapes
 * (autotuning) and synchronises `stream`; replays do not synchronise. If `stream` cannot be
 * captured (for instance because the caller is capturing it), the sequence runs eagerly.
 * Optional outputs of p are ignored. */
htsvd_status htsvd_denoise_batch(const htsvd_image* h_imgs, int32_t n, const htsvd_params* p,
                                 cudaStream_t stream);

/* Alg. 1 on a hyperspectral cube (Sec. III-E, extension to other imaging; Sec. IV, real-world HSI
 * denoising): a patch is a ps x ps x N tube and the t-SVD runs along the band mode (N Fourier
 * slices); tau = tau_mult * sigma with tau_mult <= 0 meaning sqrt(2 ln(N K ps^2)).
 * d_cube: H x W x N uint8, band-interleaved (pixel-major) on the [0, 255] scale (DEVICE); N in [2, 64].
 * sigma: the noise level (>= 0, finite; the paper's band-mean estimate goes through its CNN, so it is
 * an input here). Grouping takes the SSD summed over all bands (exact integers; the paper is silent
 * on matching for cubes): match_mode must be AUTO or FULL.
 * d_out: H x W x N float32 (DEVICE). d_idx_out (DEVICE, may be NULL): N_groups x K int32 indices as
 * in htsvd_denoise. Optional outputs of p are honoured (d_mask_out: ceil(K 64 N / 32) words per group;
 * d_coef_out: K 64 N floats per group; d_basis_out: 2 N 64 complex values). The aggregation adds
 * with float atomics, so repeated calls agree to rounding rather than bit for bit.
 * Errors: INVALID_ARG for a null pointer, N outside [2, 64], H or W < ps, a negative or non-finite
 * sigma, a match mode other than AUTO or FULL, or a search window with fewer than K positions;
 * UNSUPPORTED when H W N reaches 2^31. */
htsvd_status htsvd_denoise_cube(const uint8_t* d_cube, int32_t H, int32_t W, int32_t N, double sigma,
                                const htsvd_params* p, float* d_out, int32_t* d_idx_out, cudaStream_t stream);

/* Alg. 1 on an MRI volume (Sec. III-E, extension to other imaging: an MRI patch is a ps x ps x ps
 * cube; Sec. IV, MRI denoising with ps 4, K 32, W 5). d_vol: D x H x W uint8 (slices z, rows y,
 * columns x; DEVICE, 4-byte aligned). A cube P[i][j][k] = v[z + k][y + i][x + j] is a 4 x 4 x 4 tensor
 * whose tube (the t-SVD's Fourier mode, 4 slices) runs along z; the reference grid is {0, s, 2s, ...}
 * U {n - 4} per axis, the search window W x W x W candidate cubes clamped per axis, the distance the
 * exact integer SSD over the 64 voxels with ties broken by the lowest linear index (z H + y) W + x,
 * the reference itself in slot 0; tau = tau_mult * sigma, tau_mult <= 0 meaning sqrt(2 ln(4^3 K)).
 * sigma: the noise level (>= 0; for Rician MRI data, the level after a variance-stabilising
 * transform, which is the caller's), or < 0 to estimate it with the eigenvalue rule of
 * htsvd_estimate_sigma on the covariance of the reference cubes (64 x 64, host FP64; the paper's CNN
 * estimator is replaced as for images; the used value goes to h_sigma_out). Parameters: ps 0 or 4 (others UNSUPPORTED), stride 0 -> 2,
 * window 0 -> 5 (at most 8), K 0 -> 32 (a power of two, at most 32); match_mode AUTO or FULL.
 * d_out: D x H x W float32 (DEVICE). d_idx_out (DEVICE, may be NULL): N_groups x K int32 linear
 * indices, groups z-major over the grid. Optional outputs of p are honoured (d_mask_out: 2 K words
 * per group, bit m 64 + (i 4 + j) 4 + k for Haar row m; d_weights_out; d_basis_out: 2 x 4 x 16
 * complex values, U slices then V slices, each [a][i]; h_sigma_out; strict_basis and
 * h_basis_gap_out as in htsvd_denoise). The bases are solved on the host (one synchronisation on
 * an event, overlapped with the grouping). The aggregation adds with float atomics, so repeated
 * calls agree to rounding rather than bit for bit.
 * Errors: INVALID_ARG for a null or misaligned pointer, a non-finite sigma, D, H or W below 4, K not a power of two in [2, 32], window outside [1, 8], a window with fewer than K
 * cubes, or another match or aggregation mode; UNSUPPORTED for ps other than 4 or D H W >= 2^31. */
htsvd_status htsvd_denoise_volume(const uint8_t* d_vol, int32_t D, int32_t H, int32_t W, double sigma,
                                  const htsvd_params* p, float* d_out, int32_t* d_idx_out, cudaStream_t stream);

/* A-Haar-tSVD (Alg. 2) on an MRI volume (Sec. IV, MRI denoising: the adaptive variant with ps 4,
 * K 32, W 5). d_vol: D x H x W uint8 (DEVICE). Each axis of length n is cut into t = max(1, n / n_sub)
 * parts with boundaries floor(i n / t), as the image axes of htsvd_denoise_adaptive (sub_d, sub_h,
 * sub_w >= 1). Step 1 estimates sigma per sub-volume with the eigenvalue rule on its reference cubes'
 * covariance (as htsvd_denoise_volume with sigma < 0; the eigen-rank vote is not applied to
 * volumes); Step 2 denoises every sub-volume on its own (Alg. 1 of htsvd_denoise_volume: its own
 * grouping, bases and threshold) at that sigma and writes it into d_out (D x H x W float32, DEVICE).
 * h_sigmas (HOST, may be NULL) receives the sigmas in z-major sub-volume order. Synchronises
 * `stream` once per sub-volume (host eigenvalue step). Errors: INVALID_ARG for a null pointer, a
 * sub size < 1, or a sub-volume that fails the checks of htsvd_denoise_volume (each part must be
 * at least 4 long and hold K cubes in its window); UNSUPPORTED as for htsvd_denoise_volume. Every
 * part is checked before any device work, so on these errors d_out is left untouched. The
 * per-volume optional outputs of p (masks, weights, basis, gap, sigma) are ignored. */
htsvd_status htsvd_denoise_volume_adaptive(const uint8_t* d_vol, int32_t D, int32_t H, int32_t W, int32_t sub_d,
                                           int32_t sub_h, int32_t sub_w, const htsvd_params* p, float* d_out,
                                           double* h_sigmas, cudaStream_t stream);

/* Batched forward projection of patches onto the global t-SVD bases (Sec. III-B.2, Eq. (forward
 * transform) before the Haar transform along the group mode; Sec. II-C, Def. T-product): for each
 * of n patches, S = U^T * P * V of the ps x ps x C uint8 patch P whose top-left corner is d_pos[t]
 * (linear index y * W + x), i.e. per channel-Fourier slice f, U_f^H P_f V_f, then the inverse DFT
 * along the channel mode. d_img: H x W x C uint8 (DEVICE, 4-byte aligned); d_pos: n int32 (DEVICE), or
 * NULL for every position of the image, row-major over the (H - 7) x (W - 7) top-left corners (n must
 * then be (H - 7)(W - 7); a tile is then 128 consecutive positions of one row, im2col-style);
 * d_basis: the FP64 bases in the layout of htsvd_params.d_basis_out (DEVICE; e.g. from htsvd_denoise
 * of the same image); d_coef: n x 64 C float32 (DEVICE, 16-byte aligned), coefficient
 * (i * 8 + j) * C + c of patch t at d_coef[t * 64 C + ...] (the order of the mask bits).
 * The map P -> S is one real (64 C) x (64 C) matrix; it runs on the tensor cores as a dense
 * contraction: the patch bytes are exact in FP16, the matrix (scaled by 2^14) is split into two
 * FP16 pieces (the second the rounding of what the first leaves), FP32 accumulation, so the
 * coefficients carry an FP32-level error (tested against 2^-21 of the patch norm). A position whose patch does not
 * lie inside the image gives NaN coefficients. d_flag (DEVICE, may be NULL): bit 0 is set if a wait
 * for the tensor cores ran out (about two seconds; the affected tile is not written).
 * Errors: INVALID_ARG for C not 1 or 3, H or W < 8, n < 0, a null image, basis or output pointer with
 * n > 0, a null d_pos with n other than (H - 7)(W - 7), or a misaligned d_img or d_coef;
 * UNSUPPORTED when H W C reaches 2^31. Asynchronous on stream. */
htsvd_status htsvd_project_patches(const uint8_t* d_img, int32_t H, int32_t W, int32_t C, const int32_t* d_pos,
                                   int64_t n, const double* d_basis, float* d_coef, int32_t* d_flag,
                                   cudaStream_t stream);

/* Vector-Jacobian product of htsvd_denoise_f32 at x with the grouping (d_idx), the
 * global bases, tau and the threshold masks held fixed (masks are recomputed at x).
 * d_w: per-group weights used by the forward (NULL = all ones); d_out: the forward's
 * output at x; d_grad_out: cotangent of the output (H*W*C).
 * d_grad_x: H*W*C float32 output; d_grad_w: optional N_groups float32 output.
 * sigma must be >= 0 (pass the sigma the forward used). */
htsvd_status htsvd_denoise_vjp(const float* d_x, int32_t H, int32_t W, int32_t C, double sigma,
                               const htsvd_params* p, const int32_t* d_idx, const float* d_w,
                               const float* d_out, const float* d_grad_out, float* d_grad_x,
                               float* d_grad_w, cudaStream_t stream);

/* Size of the fixed device array used by htsvd_denoise_noalloc. */
#define HTSVD_NOALLOC_SCRATCH_BYTES (32u << 20)
/* Square RGB edges that array holds at stride 3, window 18, K 32 on a 152-SM GB300 (see below). */
#define HTSVD_NOALLOC_SAME_TILES_RGB_EDGE 305
#define HTSVD_NOALLOC_MAX_RGB_EDGE 821

/* The plain uint8 denoiser of htsvd_denoise, without any device-memory allocation. The paper has
 * no counterpart: this call serves callers that must not let a library allocate. A host whose own
 * caching allocator has reserved the device memory cannot have a library call cudaMalloc behind it,
 * and a latency-bound processing loop cannot take the device-wide synchronisation that cudaFree
 * implies. This call runs the same kernels as htsvd_denoise with the same parameter checks; it takes
 * the same filter tiles (so the same output, bit for bit) whenever their tile partials fit, else the
 * largest tile edge whose shared memory fits a CTA (equal output up to rounding order). It keeps
 * every temporary (match indices, moments, bases, eigen-gaps, tile partials) in one array of
 * HTSVD_NOALLOC_SCRATCH_BYTES (32 MiB) that the
 * library declares in device memory; every GPU that loads the library holds that array until the
 * process exits. It calls no cudaMalloc, cudaFree or allocating library routine.
 * sigma must be given (>= 0, finite); there is no estimation and no d_idx_out. Every field of p is
 * honoured as in htsvd_denoise (optional outputs, tile, strict_basis, h_basis_gap_out).
 * Images whose temporaries do not fit the array return HTSVD_ERR_INVALID_ARG before any device work.
 * At stride 3, window 18, K 32 on a 152-SM GB300, square RGB images up to
 * HTSVD_NOALLOC_SAME_TILES_RGB_EDGE take the tiles of htsvd_denoise and images up to
 * HTSVD_NOALLOC_MAX_RGB_EDGE fit at all (htsvd_internal_noalloc_bytes gives the need of any size).
 * The first call on a device looks up the array's device address (with that device current); make
 * that first call before any stream capture. All calls share the one array and it keeps the last
 * call's contents (each call clears what it accumulates); calls that can overlap on the GPU (other
 * streams, other host threads) race on it and must be serialised by the caller. */
htsvd_status htsvd_denoise_noalloc(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, double sigma,
                                   const htsvd_params* p, float* d_out, cudaStream_t stream);

/* Number of groups (reference patches) of an H x W image, or -1 on bad arguments. */
int64_t htsvd_num_groups(int32_t H, int32_t W, const htsvd_params* p);

/* Static description of a status code. */
const char* htsvd_status_string(htsvd_status s);

/* Benchmark instrumentation (not needed for correct use). While enabled, every kernel
 * launch of the library is bracketed by CUDA events on its stream.
 * htsvd_profile_collect waits for the recorded events and writes, for up to max_kernels
 * kernel names, the name (NUL-terminated, name_len bytes per entry, HOST), the number of
 * launches and their total device time in ms (HOST arrays); it then clears the record and
 * returns the number of entries written, or -1 if an event could not be read. The host part
 * of the noise-level estimate (the covariance eigenvalues) is recorded as "sigma_host" with
 * its wall-clock time. */
htsvd_status htsvd_profile_enable(int32_t enable);
int32_t htsvd_profile_collect(int32_t max_kernels, char* names, int32_t name_len, int64_t* launches,
                              double* total_ms);

/* Releases the workspaces of the calling thread's current device. */
htsvd_status htsvd_release_workspace(void);

#ifdef __cplusplus
}
#endif
#endif /* HTSVD_H */

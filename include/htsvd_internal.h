/*
 * htsvd_internal.h — test hooks of libhtsvd (not part of the stable API).
 *
 * They expose single steps of the path so that tests can check them in isolation.
 */
#ifndef HTSVD_INTERNAL_H
#define HTSVD_INTERNAL_H

#include <stdint.h>
#include "htsvd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* HOST computation of one global-basis slice (Sec. III-B.1): from the integer row (which = 0)
 * or column (which = 1) moments `mom` ([2][8][8][C][C] uint64, host memory), the slice-f scatter
 * matrix and its canonical eigenvectors, written to out[64][2] (row-major [a][i], re/im).
 * Uses the same complex Jacobi method as the device solver (cyclic pair order here, round-robin
 * order on the device), so the two agree to rounding. No errors are reported. */
void htsvd_internal_slice_basis(const unsigned long long* mom, int C, int which, int f, double* out);

/* DEVICE: integer row/column moments of the reference patches of a uint8 image (d_img) with the
 * given grid stride into d_mom (2*64*C*C uint64, device); synchronises the device.
 * Returns 0 on success, 1 on a CUDA error. */
int htsvd_internal_moments(const uint8_t* d_img, int H, int W, int C, int stride, unsigned long long* d_mom);

/* DEVICE: basis solve from device moments; d_b64 receives 2*2*C*64 doubles (see d_basis_out of
 * htsvd_params), d_b32 512 floats (the filter's packed FP32 copy); synchronises the device.
 * Returns 0 on success, 1 on a CUDA error. */
int htsvd_internal_basis(const unsigned long long* d_mom, int C, double* d_b64, float* d_b32);

/* HOST noise level of Sec. III-D from the integer patch moments of the reference patches:
 * M (d x d uint64, sum over references of x x^T) and S (d uint64, sum of x), n references,
 * d = 64 C (patch entries in (row, column, channel) order). The covariance M/n - (S/n)(S/n)^T
 * is reduced to tridiagonal form and its eigenvalues found by shifted QR (FP64); if lam is not
 * NULL it receives the d eigenvalues in ascending order (host). Returns sigma, or -1 on a bad
 * argument or if the iteration did not converge. */
double htsvd_internal_sigma_from_moments(const unsigned long long* M, const unsigned long long* S, int d, int64_t n,
                                         double* lam);

/* DEVICE + HOST: the eigen-rank vote inputs of Sec. III-D for a uint8 image (d_img, DEVICE):
 * grouping of every 8th reference per axis, then for each such group the rank
 * a = 1 + #{f : lambda_f < lambda_{K/2}} of its circulant eigenvalues, written row-major to
 * h_ranks (HOST, max_ranks entries). Synchronises the device. Returns the number of groups, or
 * -1 on a bad argument, too small an array or a CUDA error. */
int32_t htsvd_internal_sampled_ranks(const uint8_t* d_img, int32_t H, int32_t W, int32_t C, const htsvd_params* p,
                                     int32_t* h_ranks, int32_t max_ranks);

/* Tile edge (references per tile side) that the forward filter of htsvd_denoise takes for an H x W x C
 * uint8 image with parameters p on the current device (it follows the SM count), or -1 on bad
 * arguments. Host only; launches nothing. */
int32_t htsvd_internal_filter_tile(int32_t H, int32_t W, int32_t C, const htsvd_params* p);

/* Bytes of the static scratch array that htsvd_denoise_noalloc would use for an H x W x C image
 * with parameters p on the current device (the filter tiles depend on its SM count), or -1 when
 * the arguments fail the checks of htsvd_denoise. Host only; launches nothing. */
int64_t htsvd_internal_noalloc_bytes(int32_t H, int32_t W, int32_t C, const htsvd_params* p);

/* DEVICE: the projection of htsvd_project_patches (same arguments, same output) in the structured
 * per-slice form on the CUDA cores in FP32 (channel DFT, U_f^H X_f, (.) V_f, inverse channel DFT),
 * the arithmetic of the group filter's projection stages; for comparison with the tensor-core form.
 * Asynchronous on stream; errors as htsvd_project_patches. */
htsvd_status htsvd_internal_project_simt(const uint8_t* d_img, int32_t H, int32_t W, int32_t C, const int32_t* d_pos,
                                         int64_t n, const double* d_basis, float* d_coef, cudaStream_t stream);

/* HOST: the global bases of htsvd_denoise_volume from its integer cube moments mom (HOST, 512 uint64:
 * rows R[a][a'][c][c'] = sum over reference cubes and columns b of P[a][b][c] P[a'][b][c'], then
 * columns Q[b][b'][c][c'] = sum over reference cubes and rows a of P[a][b][c] P[a][b'][c'], each
 * [4][4][4][4] row-major; P[a][b][c] = v[z + c][y + a][x + b]). b64 (HOST) receives 256 doubles in the
 * layout of htsvd_params.d_basis_out. Returns the smallest relative eigen-gap of the slices 0..2. */
double htsvd_internal_volume_bases(const unsigned long long* mom, double* b64);

/* DEVICE probe of an arithmetic pipe's issue rate on the current device: 2 CTAs of 512 threads per
 * SM, each thread running 8 independent chains of one instruction for 32 * iters steps (op 0: FP32
 * fused multiply-add, 1: 32-bit integer multiply-add, 2: 4-way byte dot product with accumulate).
 * Returns the mean over SMs of operations per SM clock (clock64 spans per SM), or -1 on a bad
 * argument or a CUDA error. Synchronises the device; allocates two small buffers. */
double htsvd_internal_alu_probe(int32_t op, int32_t iters);

#ifdef __cplusplus
}
#endif
#endif /* HTSVD_INTERNAL_H */

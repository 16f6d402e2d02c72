// Internal launch interface between the C-ABI layer (api.cu) and the kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"

namespace htsvd {

enum MatchMode { MM_GRAY = 0, MM_GCP = 1, MM_FULL = 2, MM_GREEN = 3 };

// Streaming multiprocessors of the calling thread's current device (cudaDevAttrMultiProcessorCount,
// looked up once per device); grids and wave counts are sized from it.
int device_sm_count();

// ---- block matching (bm.cu)
struct BMArgs {
    const uint8_t* img;
    Geo g;
    int mode;            // MatchMode (resolved: gray for C = 1)
    double gamma2;       // gcp_gamma^2
    int rstep;           // reference subsampling (1 = every reference)
    int nry_s, nrx_s;    // references per axis after subsampling
    int TRy, TRx;        // references per tile
    int32_t* idx;        // out [nry_s * nrx_s][K]
    // Spatio-temporal search (video): candidates also come from frames f0 .. f0 + nfr - 1 of the
    // clip at vid (frame stride fstride bytes); img is frame fref. Indices are global,
    // f * H * W + y * W + x. nfr = 0 (the default) searches img alone, with frame-local indices.
    const uint8_t* vid;
    long long fstride;
    int f0, nfr, fref;
};
size_t bm_smem_bytes(const BMArgs& a);
// Halves the tile (TRx, TRy) until its shared-memory footprint leaves room for two CTAs per SM.
void bm_fit_tiles(BMArgs& a);
cudaError_t launch_block_match(const BMArgs& a, cudaStream_t s);

// ---- second moments and bases (moments.cu)
// Row/column second moments of the reference patches, exact:
//   R[a][a'][c][c'] = sum_r sum_b P_r[a][b][c] P_r[a'][b][c']
//   Q[b][b'][c][c'] = sum_r sum_a P_r[a][b][c] P_r[a][b'][c']
// stored as uint64 [2][8][8][C][C] (R then Q).
cudaError_t launch_moments(const uint8_t* img, const Geo& g, unsigned long long* d_mom, cudaStream_t s);
// Row and column moments derived exactly from the full second moment (lower triangle) that
// launch_full_moment wrote; replaces launch_moments where the full moment is already formed.
cudaError_t launch_moments_from_full(const unsigned long long* d_M, int C, unsigned long long* d_mom, cudaStream_t s);
// Full second moment M[u][v] = sum_r p_r[u] p_r[v] (d = 64 C) and s[u] = sum_r p_r[u], uint64.
cudaError_t launch_full_moment(const uint8_t* img, const Geo& g, unsigned long long* d_M,
                               unsigned long long* d_s, cudaStream_t s);
// FP64 eigen-solve of the per-slice row/column scatter matrices -> canonical bases.
//   basis64: [2 (U,V)][C][8][8] complex (re, im), slice f, row a, column i.
//   basis32: packed float slices for the filter (U0r, [U1r, U1i], V0r, [V1r, V1i]), each [a][i].
//   gap (optional): per solved problem (U slices f = 0 .. C/2, then V slices; basis_problems(C) of them)
//   the smallest gap between consecutive eigenvalues relative to the largest eigenvalue.
inline int basis_problems(int C) { return 2 * (C / 2 + 1); }
cudaError_t launch_basis(const unsigned long long* d_mom, int C, double* d_basis64, float* d_basis32,
                         cudaStream_t s, double* d_gap = nullptr);
// Row and column moments (layout as launch_moments) of a cube with any number of bands g.C.
cudaError_t launch_cube_moments(const uint8_t* img, const Geo& g, unsigned long long* d_mom, cudaStream_t s);
// Floats of the packed FP32 basis: C in {1, 3}: 512 (the filter's layout); cubes (other C):
// [2 (U, V)][C/2 + 1 slices][re, im][8][8].
inline int basis32_floats(int C) { return (C == 1 || C == 3) ? 512 : 2 * (C / 2 + 1) * 2 * 64; }
// Quantise a float image: q = clip(rint(x), 0, 255).
cudaError_t launch_quantize(const float* x, int64_t n, uint8_t* q, cudaStream_t s);

// ---- group filter and aggregation (filter.cu)
enum FilterMode { FM_FORWARD = 0, FM_DENOM = 1, FM_ADJOINT = 2, FM_VIDEO = 3, FM_ANALYZE = 4, FM_SYNTH = 5 };

// Guard band of the threshold decision: a coefficient whose FP32 value lies within
// kBandRel * ||G||_F + kBandTau * tau of tau is decided again in FP64 (||G||_F: Frobenius
// norm of the group's inputs; kBandTau covers tau rounded to FP32).
constexpr float kBandRel = 1.9073486328125e-06f;      // 2^-19
constexpr double kBandTau = 2.384185791015625e-07;    // 2^-22
// Cubes: band relative to the norm of the Haar slot being thresholded (its FP32 coefficient error,
// measured on 31-band cubes: 2^-23 of that norm).
constexpr float kBandRelCube = 1.9073486328125e-06f;   // 2^-19
struct FilterArgs {
    const void* img;         // uint8 or float H x W x C (the values that are filtered)
    int img_is_float;
    Geo g;
    int TR, ntx, nty;        // references per tile edge, tiles per axis
    int FHmax, FWmax;        // partial-footprint strides
    const int32_t* idx;      // [N][K]
    const float* basis32;
    const double* basis64;
    float tau32;
    double tau64;
    float band_rel;          // guard band: |S| within band_rel*||G||_F + band_abs of tau -> FP64 decision
    float band_abs;
    const float* w_in;       // optional per-group weights
    int agg_mode;
    float* partials;         // [ntiles][FHmax][FWmax][C+1]
    uint32_t* mask_out;      // optional
    float* weights_out;      // optional
    float* coef_out;         // optional FP32 coefficients, K*64*C per group (accuracy checks)
    int mode;                // FilterMode
    // adjoint inputs
    const float* r_img;      // (gout / D) image that is filtered with the masks of img (FM_ADJOINT)
    const float* out_img;    // forward output (FM_ADJOINT, for the weight gradient)
    float* grad_w;           // FM_ADJOINT, per group
    // FM_VIDEO (forward over a clip, uint8): groups of frame fref may hold patches of frames
    // f0 .. f0 + nfr - 1 of vid (frame stride fstride elements, indices f * H * W + y * W + x);
    // only the patches of frame fref are aggregated. img is frame fref.
    const void* vid;
    long long fstride;
    int f0, nfr, fref;
    // Coefficient cache of the noisy groups (threshold sweeps): FM_ANALYZE writes, FM_SYNTH reads
    // the Haar-domain coefficients of every group ([N][K][64 C] floats, unnormalised Haar, slot
    // order of the in-place transform), the per-patch squared norms ([N][32]) and ||G||_F^2 ([N],
    // the filter's own integer or float-bit representation).
    float* cache_coef;
    float* cache_pn;
    int* cache_nrm;
};
size_t filter_smem_bytes(const FilterArgs& a);
cudaError_t launch_filter(const FilterArgs& a, cudaStream_t s);
// out[p] = sum_tiles num / sum_tiles den (deterministic tile order). If den_out is set, the
// denominator plane is written too; if num_only, out = sum num (no division).
cudaError_t launch_reduce(const float* partials, const Geo& g, int TR, int ntx, int nty, int FHmax, int FWmax,
                          float* out, float* den_out, int num_only, const float* den_in, cudaStream_t s);
// z = y + eps b over n floats, each operation rounded once (the finite-difference SURE's perturbed image).
cudaError_t launch_perturb(const float* y, const float* b, float eps, int64_t n, float* z, cudaStream_t s);
// SURE terms in FP64: res[0] = sum (out - x)^2, res[1] = sum b * g over n floats (deterministic
// two-level reduction; scratch: sure_scratch_doubles() doubles).
size_t sure_scratch_doubles();
// Weight tuning (SURE of the per-group weights): u = alpha (f - x) - beta b; acc += a;
// w <- w exp(-step g / max|g|) (scratch: one unsigned, for max|g|).
cudaError_t launch_sure_cotangent(const float* f, const float* x, const float* b, float alpha, float beta, int64_t n,
                                  float* u, cudaStream_t s);
cudaError_t launch_add(const float* a, float* acc, int64_t n, cudaStream_t s);
cudaError_t launch_eg_update(float* w, const float* g, int64_t n, float step, unsigned* scratch, cudaStream_t s);
cudaError_t launch_sure_terms(const float* out, const float* x, const float* b, const float* g, int64_t n,
                              double* scratch, double* res, cudaStream_t s);
// Adjoint helper: r = gout / den.
cudaError_t launch_div(const float* gout, const float* den, int64_t npix, int C, float* r, cudaStream_t s);

// ---- batched patch projection (project.cu): S = U^T * P * V per patch, 64 C coefficients in the
// order n = (i * 8 + j) * C + c; positions are linear top-left indices y * W + x (outside: NaN).
// Bytes of the split BF16 basis matrix (three pieces, both halves) that launch_project_split writes.
size_t project_pieces_bytes(int C);
cudaError_t launch_project_split(const double* d_b64, int C, void* d_pieces, cudaStream_t s);
// Tensor cores (C in {1, 3}); flag (may be null) gets bit 0 set if a wait for the tensor cores ran out.
cudaError_t launch_project_tc(const uint8_t* img, int H, int W, int C, const int32_t* pos, long long n,
                              const void* d_pieces, float* coef, int* flag, cudaStream_t s);
// Structured per-slice FP32 form on the CUDA cores.
cudaError_t launch_project_simt(const uint8_t* img, int H, int W, int C, const int32_t* pos, long long n,
                                const double* d_b64, float* coef, cudaStream_t s);

// ---- MRI volumes (volume.cu): Alg. 1 on 4 x 4 x 4 cubes of a D x H x W uint8 volume, the t-SVD
// tube along z (cube P[i][j][k] = v[z + k][y + i][x + j]); linear indices (z H + y) W + x.
struct VolGeo {
    int D, H, W;
    int s, win, K;
    int nrz, nry, nrx;       // references per axis
    int npz, npy, npx;       // candidate positions per axis
    int wnz, wny, wnx;       // window extent per axis
};
VolGeo make_vol_geo(int D, int H, int W, int s, int win, int K);
int volume_max_window();
cudaError_t launch_block_match_volume(const uint8_t* vol, const VolGeo& g, int32_t* idx, cudaStream_t s);
// uint64 [2][4][4][4][4]: rows R[a][a'][c][c'] then columns Q[b][b'][c][c'] of the reference cubes.
cudaError_t launch_volume_moments(const uint8_t* vol, const VolGeo& g, unsigned long long* d_mom, cudaStream_t s);
// HOST: canonical bases from the moments: b64 [2 (U, V)][4 slices][4][4] complex (re, im), slice 3 the
// conjugate of slice 1; returns the smallest relative eigen-gap over the slices 0..2 of U and V.
double volume_bases_host(const unsigned long long* mom, double* b64);
// Full second moment M (64 x 64) and sums S (64) of the reference cubes (uint64, exact), for the noise
// estimate; entry order u = (a * 4 + b) * 4 + c.
cudaError_t launch_volume_full_moment(const uint8_t* vol, const VolGeo& g, unsigned long long* d_M,
                                      unsigned long long* d_S, cudaStream_t s);
struct VolFilterArgs {
    const uint8_t* vol;
    VolGeo g;
    const int32_t* idx;      // [N][K]
    const double* basis64;   // device copy of the host bases
    float tau32;
    double tau64;
    float band_rel, band_abs;
    const float* w_in;       // optional per-group weights
    int agg_mode;
    float* num;              // D H W, zeroed by the caller
    float* den;
    uint32_t* mask_out;      // optional, 2 K words per group (bit m * 64 + (i * 4 + j) * 4 + k)
    float* weights_out;      // optional
};
size_t volume_filter_smem_bytes(const VolGeo& g);
cudaError_t launch_volume_filter(const VolFilterArgs& a, cudaStream_t s);
cudaError_t launch_volume_finalize(const float* num, const float* den, long long n, float* out, cudaStream_t s);

// ---- hyperspectral cubes (cube.cu): Alg. 1 with C = N bands, one Haar slot of a group at a time
struct CubeArgs {
    const uint8_t* img;      // H x W x N uint8
    Geo g;                   // g.C = N
    const int32_t* idx;      // [groups][K]
    const float* basis32;    // basis32_floats(N) floats, cube layout
    const double* basis64;   // [2][N][8][8] complex
    float tau32;
    double tau64;
    float band_rel, band_abs; // guard band: |S| within band_rel ||G||_F + band_abs of tau -> FP64 decision
    const float* w_in;       // optional per-group weights
    int agg_mode;
    float* scratch;          // grid x K x 64 N floats (spatial Haar slots per CTA)
    float* num;              // H x W x N, zeroed by the launcher
    float* den;              // H x W, zeroed by the launcher
    float* out;              // H x W x N = num / den
    uint32_t* mask_out;      // optional: ceil(K 64 N / 32) words per group (bit (m 64 + p) N + c)
    float* weights_out;      // optional
    float* coef_out;         // optional: K 64 N floats per group
};
size_t cube_smem_bytes(int C, int K);
// CTAs of the persistent cube filter (a few per SM, at most one per group).
int cube_grid(int C, int K, int64_t ngroups);
cudaError_t launch_cube_filter(const CubeArgs& a, int grid, cudaStream_t s);

// ---- persistent batch forms over many images (work items -> image by prefix sums)
int bm_tiles(const BMArgs& a);
cudaError_t launch_block_match_batch(const BMArgs* d_args, const int* d_prefix, int nimg, size_t smem, int grid,
                                     int* d_counter, cudaStream_t s);
int moments_chunks(const Geo& g);
cudaError_t launch_moments_batch(int C, const BMArgs* d_args, unsigned long long* const* d_moms, const int* d_prefix,
                                 int nimg, int grid, cudaStream_t s);
cudaError_t launch_basis_batch(int C, const FilterArgs* d_fargs, unsigned long long* const* d_moms, int nimg,
                               cudaStream_t s);
cudaError_t launch_filter_batch(int K, int C, const FilterArgs* d_args, const int* d_prefix, int nimg, size_t smem,
                                int grid, int* d_counter, cudaStream_t s);
cudaError_t launch_reduce_batch(int C, const FilterArgs* d_args, float* const* d_outs, const int* d_prefix, int nimg,
                                int grid, cudaStream_t s);

// ---- sigma adjustment (moments.cu)
// Rank position a = 1 + #{f : lambda_f < lambda_{K/2}} of each sampled group (Sec. III-D).
cudaError_t launch_group_rank(const uint8_t* img, const Geo& g, const int32_t* idx, int ngroups, int32_t* ranks,
                              cudaStream_t s);

}  // namespace htsvd

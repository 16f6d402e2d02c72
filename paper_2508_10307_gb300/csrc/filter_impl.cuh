// Collaborative filter and aggregation (Alg. 1 Steps 2(2)-(4) and 3).
//
// Per group (Sec. III-B.2):
//   S = U^T * G * V  x_4 H_K            (Eq. (forward transform); t-products evaluated per
//                                         Fourier slice after an FFT along channels)
//   S_t = S . [|S| >= tau]               (Eq. (hard thresholding))
//   G^ = U * S_t * V^T  x_4 H_K^T        (Eq. (backward transform), exact inverse)
// and every estimated patch is written back with weight w_g (Eq. (aggregation)).
//
// One CTA (256 threads, 8 warps) per tile of TR x TR references. The CTA stages the
// image footprint of the tile (union of its search windows) in shared memory and keeps
// a numerator/denominator accumulator for that footprint; groups are processed one at a
// time, all data of a group living in shared memory / registers:
//   A  thread (k, b): column b of patch k -> channel DFT -> Y_f = U_f^H X_f
//   B  thread (i, k): row i -> S_f = Y_f V_f -> inverse channel DFT (real S)
//   C  thread = fibre (i, j, c): Haar butterflies along the K patches (in place, one register
//      array), threshold, inverse butterflies. Coefficients whose FP32 value lies inside a
//      guard band around tau get their keep/drop decision recomputed in FP64 (one warp per
//      entry). In the forward mode each warp's 32 fibres sit on 32 distinct banks.
//   D  thread (i, k): channel DFT -> Z_f = T_f V_f^H   (outer products, transposed basis)
//   E  thread (k, b): G_f = U_f Z_f -> inverse channel DFT (real estimate), likewise
//   F  warp w owns footprint rows r with r mod 8 == w: it adds row (w - y_k) mod 8 of
//      every patch k, k ascending. No atomics, fixed order: bitwise reproducible.
// The forward mode (filter_tile_fwd) pipelines these over the tile's groups with two group
// buffers and two CTA barriers per group: [D, E(q) on warps 0-3 | A, B(q+1) on warps 4-7], then
// [F(q), C(q+1)]; there each thread of A, B, D, E owns two columns or two rows of a patch. The
// same routine serves video groups (stacked frame footprints) and the analysis / synthesis passes
// of a threshold sweep; the sequential routine (filter_tile) serves the VJP's passes.
// The tile's accumulator is written to a partial buffer; reduce_kernel sums the
// overlapping tile partials in fixed tile order and divides.
#pragma once
#include "kernels.h"

namespace htsvd {

constexpr int FT_THREADS = 256;
constexpr float F_S3H = 0.866025403784438646763723170752936183f;   // sqrt(3)/2
constexpr float F_SQ3 = 1.73205080756887729352744634150587237f;    // sqrt(3)
constexpr float F_R2 = 0.707106781186547524400844362104849039f;    // 1/sqrt(2)
constexpr float F_THIRD = 0.333333333333333333333333333333333333f;

template <int C>
struct FCfg {
    static constexpr int RWF = PS * C;                 // floats of data per patch row
    static constexpr int ROW = (C == 3) ? 28 : 12;     // padded row stride: an odd number of 16-byte units,
                                                       // so the 128-bit row loads of 8 consecutive rows hit
                                                       // distinct bank groups
    static constexpr int PATCH = PS2 * C;              // floats per patch (fibres of the Haar stage)
    static constexpr int GS = (C == 3) ? 232 : 104;    // stride between patches, = 8 (mod 32) words: the column
                                                       // accesses of stages A and E (lanes = 4 patches x 8
                                                       // columns) then fall on 32 distinct banks
    static constexpr int ACC = (C == 3) ? 4 : 2;       // floats per footprint pixel (C numerators + 1 denominator)
    static constexpr int NBAS = (C == 3) ? 384 : 128;  // packed FP32 basis floats
};

// Shared-memory layout (bytes), identical on host and device.
struct FLayout {
    int off_bas, off_gb, off_pos, off_band, off_rkeep, off_misc, off_acc, off_img, off_r, total;
};
template <int K, int C>
__host__ __device__ inline FLayout f_layout(int FH, int FW, int in_bytes, int mode) {
    using G = FCfg<C>;
    FLayout L;
    int o = 0;
    L.off_bas = o; o += 2 * 384 * 4;           // basis rows, then the transposed copies
    L.off_gb = o; o += K * G::GS * 4;
    L.off_pos = o; o += 64 * 4;
    L.off_band = o; o += 192 * 4;
    L.off_rkeep = o; o += 192 * 4;
    L.off_misc = o; o += 16 * 4;
    L.off_acc = o; o += FH * FW * G::ACC * 4;
    L.off_img = o; o += ((mode == FM_DENOM ? 0 : FH * FW * C * in_bytes) + 15) / 16 * 16;
    L.off_r = o; o += (mode == FM_ADJOINT) ? FH * FW * C * 4 : 0;
    L.total = o;
    return L;
}

// Shared-memory layout of the pipelined forward filter: two group buffers (group q+1 is projected
// while group q is inverted and aggregated), three position and counter sets, no band bitmaps. The
// fixed part's offsets are compile-time constants (FwdOff), so the kernel addresses it without
// holding a register per array.
template <int K, int C>
struct FwdOff {
    static constexpr int bas = 0;                                   // basis rows, then the transposed copies
    static constexpr int gb = bas + 2 * 384 * 4;
    static constexpr int pos = gb + 2 * K * FCfg<C>::GS * 4;         // positions of three groups (q, q+1, q+2)
    static constexpr int band = pos + 3 * 64 * 4;                    // per-patch squared norms, two groups
    static constexpr int nz = band + 2 * 32 * 4;                     // basis-row masks per Haar slot, two groups
    static constexpr int dlist = nz + 2 * 32 * 4;                    // stage-D work list (256 entries)
    static constexpr int dcount = dlist + 256;
    static constexpr int misc = dcount + 16;                         // counters of three groups
    static constexpr int aofs = misc + 3 * 16 * 4;                   // aggregation offsets [32][8] int2
    static constexpr int acc = aofs + 32 * 8 * 8;
};
template <int K, int C>
__host__ __device__ inline FLayout f_layout_fwd(int FH, int FW, int in_bytes, int nfr = 1) {
    using G = FCfg<C>;
    using O = FwdOff<K, C>;
    FLayout L;
    int o = O::acc;
    L.off_bas = O::bas;
    L.off_gb = O::gb;
    L.off_pos = O::pos;
    L.off_band = O::band;
    L.off_rkeep = O::nz;
    L.off_misc = O::misc;
    L.off_acc = o; o += FH * FW * G::ACC * 4;
    L.off_img = o; o += (nfr * FH * FW * C * in_bytes + 15) / 16 * 16;   // footprints of nfr frames, stacked
    L.off_r = o;
    L.total = o;
    return L;
}

// Haar analysis along the group mode, o = H_K a (Eq. (H_2N) applied recursively), in place on
// one array: at the level of length n the values sit at stride K/n, so the detail o[n/2 + m]
// lands in slot (2m+1) K/n and the approximation o[0] in slot 0.
// Calls f(mo, slot) for every coefficient o[mo] and its slot in the in-place array. Each level
// is its own template instance, so every loop has a constant trip count, unrolls fully, and
// every index is a compile-time constant: the array stays in registers.
template <int K>
__host__ __device__ constexpr int haar_levels() { return K <= 1 ? 0 : 1 + haar_levels<K / 2>(); }
template <int K, int L, typename F>
__device__ __forceinline__ void haar_each_level(F& f) {       // level L: n = 2^(L+1), details o[2^L + m]
    if constexpr (L >= 0) {
        haar_each_level<K, L - 1>(f);
#pragma unroll
        for (int m = 0; m < (1 << L); ++m) f((1 << L) + m, (2 * m + 1) * (K >> (L + 1)), K >> L);
    }
}
// f(mo, slot, support): support = number of patches the row of o[mo] combines (K for mo = 0 and 1).
template <int K, typename F>
__device__ __forceinline__ void haar_for_each(F&& f) {
    f(0, 0, K);
    haar_each_level<K, haar_levels<K>() - 1>(f);
}
template <int K, int L>
__device__ __forceinline__ void haar_fwd_level(float (&v)[K]) {  // levels L, L-1, ..., 0 (n = K first)
    if constexpr (L >= 0) {
        constexpr int st = K >> (L + 1);
#pragma unroll
        for (int m = 0; m < (1 << L); ++m) {
            const float x = v[2 * m * st], y = v[(2 * m + 1) * st];
            v[(2 * m + 1) * st] = (x - y) * F_R2;
            v[2 * m * st] = (x + y) * F_R2;
        }
        haar_fwd_level<K, L - 1>(v);
    }
}
template <int K, int L>
__device__ __forceinline__ void haar_inv_level(float (&v)[K]) {  // levels L, L+1, ..., (n = 2 first)
    if constexpr ((2 << L) <= K) {
        constexpr int st = K >> (L + 1);
#pragma unroll
        for (int m = (1 << L) - 1; m >= 0; --m) {
            const float sa = v[2 * m * st], d = v[(2 * m + 1) * st];
            v[2 * m * st] = (sa + d) * F_R2;
            v[(2 * m + 1) * st] = (sa - d) * F_R2;
        }
        haar_inv_level<K, L + 1>(v);
    }
}
// Unnormalised forms (sums and differences only): the coefficient of row m comes out multiplied by
// sqrt(L_m), L_m its support, and synthesis of coefficients scaled by 1 / L_m gives H_K^T o.
template <int K, int L>
__device__ __forceinline__ void haar_fwd_level_sum(float (&v)[K]) {
    if constexpr (L >= 0) {
        constexpr int st = K >> (L + 1);
#pragma unroll
        for (int m = 0; m < (1 << L); ++m) {
            const float x = v[2 * m * st], y = v[(2 * m + 1) * st];
            v[(2 * m + 1) * st] = x - y;
            v[2 * m * st] = x + y;
        }
        haar_fwd_level_sum<K, L - 1>(v);
    }
}
template <int K, int L>
__device__ __forceinline__ void haar_inv_level_sum(float (&v)[K]) {
    if constexpr ((2 << L) <= K) {
        constexpr int st = K >> (L + 1);
#pragma unroll
        for (int m = (1 << L) - 1; m >= 0; --m) {
            const float sa = v[2 * m * st], d = v[(2 * m + 1) * st];
            v[2 * m * st] = sa + d;
            v[(2 * m + 1) * st] = sa - d;
        }
        haar_inv_level_sum<K, L + 1>(v);
    }
}
template <int K>
__device__ __forceinline__ void haar_fwd_inplace(float (&v)[K]) { haar_fwd_level<K, haar_levels<K>() - 1>(v); }
template <int K>
__device__ __forceinline__ void haar_inv_inplace(float (&v)[K]) { haar_inv_level<K, 0>(v); }
template <int K>
__device__ __forceinline__ void haar_fwd_sum(float (&v)[K]) { haar_fwd_level_sum<K, haar_levels<K>() - 1>(v); }
template <int K>
__device__ __forceinline__ void haar_inv_sum(float (&v)[K]) { haar_inv_level_sum<K, 0>(v); }

template <typename T>
__device__ __forceinline__ float ldv(const T* p) { return (float)p[0]; }

// Eight consecutive floats of a 32-byte aligned shared-memory row (two 128-bit loads).
__device__ __forceinline__ void load8(const float* p, float (&r)[8]) {
    const float4 a = reinterpret_cast<const float4*>(p)[0], b = reinterpret_cast<const float4*>(p)[1];
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
}

// FP64 value of one coefficient S[m][i][j][c] of the group, from the staged inputs:
// S = T(sum_k H[m,k] P_k) with T the real t-SVD projection; returns |S| >= tau.
// Lane l handles the pixels (a, b) = l and l + 32 of the combined patch Q = sum_k H[m,k] P_k;
// for uint8 inputs the signed sum of the patches is exact in int32.
template <int K, int C, typename Tin>
__device__ __forceinline__ bool refine_keep(int m, int e, const Tin* img_s, int FW, const int* pos,
                                            const double* __restrict__ b64, double tau64, int lane) {
    int k0, L;
    if (m == 0) {
        k0 = 0;
        L = K;
    } else {
        const int l = 31 - __clz(m);
        L = K >> l;
        k0 = (m - (1 << l)) * L;
    }
    const int half = (m == 0) ? L : L / 2;
    // 1/sqrt(L) for L = 2^e: a power of two, times 1/sqrt(2) when e is odd
    const int e2 = 31 - __clz(L);
    const double h = ldexp((e2 & 1) ? 0.70710678118654752440 : 1.0, -(e2 >> 1));
    const int pix = e / C, ch = e - pix * C;
    const int i = pix / PS, j = pix % PS;
    double s0 = 0.0, s1r = 0.0, s1i = 0.0;
    const double s3h = 0.5 * sqrt(3.0);
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
        const int p = lane + 32 * rep;
        const int aa = p / PS, bb = p % PS;
        double q[C];
        if constexpr (sizeof(Tin) == 1) {
            int qi[C];
#pragma unroll
            for (int c = 0; c < C; ++c) qi[c] = 0;
            // L is even and k0 a multiple of L: the positions of patches kk, kk+1 are one aligned int4
            for (int kk = k0; kk < k0 + L; kk += 2) {
                const int4 pp = *reinterpret_cast<const int4*>(pos + 2 * kk);
                const Tin* s0p = img_s + ((pp.x + aa) * FW + pp.y + bb) * C;
                const Tin* s1p = img_s + ((pp.z + aa) * FW + pp.w + bb) * C;
                const bool p0 = kk - k0 < half, p1 = kk + 1 - k0 < half;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int x0 = (int)s0p[c], x1 = (int)s1p[c];
                    qi[c] += (p0 ? x0 : -x0) + (p1 ? x1 : -x1);
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) q[c] = (double)qi[c] * h;
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) q[c] = 0.0;
            for (int kk = k0; kk < k0 + L; ++kk) {
                const Tin* src = img_s + ((pos[2 * kk] + aa) * FW + pos[2 * kk + 1] + bb) * C;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const double v = (double)src[c];
                    q[c] += (kk - k0 < half) ? v : -v;
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) q[c] *= h;
        }
        const double u0 = b64[(0 * C + 0) * 2 * PS2 + 2 * (aa * PS + i)];
        const double v0 = b64[(1 * C + 0) * 2 * PS2 + 2 * (bb * PS + j)];
        if constexpr (C == 3) {
            const double Q0 = q[0] + q[1] + q[2];
            const double Q1r = q[0] - 0.5 * (q[1] + q[2]);
            const double Q1i = s3h * (q[2] - q[1]);
            s0 += u0 * Q0 * v0;
            const double u1r = b64[(0 * C + 1) * 2 * PS2 + 2 * (aa * PS + i)];
            const double u1i = b64[(0 * C + 1) * 2 * PS2 + 2 * (aa * PS + i) + 1];
            const double v1r = b64[(1 * C + 1) * 2 * PS2 + 2 * (bb * PS + j)];
            const double v1i = b64[(1 * C + 1) * 2 * PS2 + 2 * (bb * PS + j) + 1];
            const double tr = u1r * Q1r + u1i * Q1i;       // conj(u1) * Q1
            const double ti = u1r * Q1i - u1i * Q1r;
            s1r += tr * v1r - ti * v1i;
            s1i += tr * v1i + ti * v1r;
        } else {
            s0 += u0 * q[0] * v0;
        }
    }
    // the requested channel is a fixed linear combination of the three slice sums: combine per
    // lane, then reduce one value
    double S;
    if constexpr (C == 3) {
        const double sq3 = sqrt(3.0);
        const double third = 1.0 / 3.0;
        S = (ch == 0) ? (s0 + 2.0 * s1r) * third : (ch == 1) ? (s0 - s1r - sq3 * s1i) * third
                                                              : (s0 - s1r + sq3 * s1i) * third;
    } else {
        S = s0;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) S += __shfl_xor_sync(0xffffffffu, S, off);
    return fabs(S) >= tau64;
}

// Basis rows in shared memory (each [a][i], row a = 8 consecutive floats):
// C = 3: U0 at 0, U1r at 64, U1i at 128, V0 at 192, V1r at 256, V1i at 320; C = 1: U0 at 0, V0 at 64.

// Stage A: thread (k, b) -> Y_f[:, b] = U_f^H X_f[:, b] of patch k. Returns the sum of squares of its inputs.
template <int K, int C, typename Tin>
__device__ __forceinline__ float stage_a(const Tin* img_s, int FW, const int* pos, const float* bas, float* gb,
                                         int k, int b) {
    using G = FCfg<C>;
    const Tin* src = img_s + (pos[2 * k] * FW + pos[2 * k + 1] + b) * C;
    float x[PS][C];
    float nrm = 0.f;
#pragma unroll
    for (int i = 0; i < PS; ++i)
#pragma unroll
        for (int c = 0; c < C; ++c) {
            x[i][c] = ldv(src + i * FW * C + c);
            nrm = fmaf(x[i][c], x[i][c], nrm);
        }
    float* dst = gb + k * G::GS + b * C;
    if constexpr (C == 3) {
        float y0[PS], yr[PS], yi[PS];
#pragma unroll
        for (int ii = 0; ii < PS; ++ii) y0[ii] = yr[ii] = yi[ii] = 0.f;
#pragma unroll
        for (int a = 0; a < PS; ++a) {
            const float X0 = x[a][0] + x[a][1] + x[a][2];
            const float X1r = x[a][0] - 0.5f * (x[a][1] + x[a][2]);
            const float X1i = F_S3H * (x[a][2] - x[a][1]);
            float u0[8], ur[8], ui[8];
            load8(bas + a * PS, u0);
            load8(bas + 64 + a * PS, ur);
            load8(bas + 128 + a * PS, ui);
#pragma unroll
            for (int ii = 0; ii < PS; ++ii) {
                y0[ii] = fmaf(u0[ii], X0, y0[ii]);
                yr[ii] = fmaf(ur[ii], X1r, fmaf(ui[ii], X1i, yr[ii]));
                yi[ii] = fmaf(ur[ii], X1i, fmaf(-ui[ii], X1r, yi[ii]));
            }
        }
#pragma unroll
        for (int ii = 0; ii < PS; ++ii) {
            dst[ii * G::ROW + 0] = y0[ii];
            dst[ii * G::ROW + 1] = yr[ii];
            dst[ii * G::ROW + 2] = yi[ii];
        }
    } else {
        float y0[PS];
#pragma unroll
        for (int ii = 0; ii < PS; ++ii) y0[ii] = 0.f;
#pragma unroll
        for (int a = 0; a < PS; ++a) {
            float u0[8];
            load8(bas + a * PS, u0);
#pragma unroll
            for (int ii = 0; ii < PS; ++ii) y0[ii] = fmaf(u0[ii], x[a][0], y0[ii]);
        }
#pragma unroll
        for (int ii = 0; ii < PS; ++ii) dst[ii * G::ROW] = y0[ii];
    }
    return nrm;
}

// Stage B: thread (i, k): S_f[i, :] = Y_f[i, :] V_f, inverse channel DFT, in place on row i of patch k.
template <int C>
__device__ __forceinline__ void stage_b(const float* bas, float* gb, int k, int i) {
    using G = FCfg<C>;
    float4* row = reinterpret_cast<float4*>(gb + k * G::GS + i * G::ROW);
    float y[G::RWF];
#pragma unroll
    for (int q = 0; q < G::RWF / 4; ++q) {
        float4 v = row[q];
        y[4 * q] = v.x; y[4 * q + 1] = v.y; y[4 * q + 2] = v.z; y[4 * q + 3] = v.w;
    }
    float o[G::RWF];
    if constexpr (C == 3) {
        float s0[PS], sr[PS], si[PS];
#pragma unroll
        for (int j = 0; j < PS; ++j) s0[j] = sr[j] = si[j] = 0.f;
#pragma unroll
        for (int b = 0; b < PS; ++b) {
            float v0[8], vr[8], vi[8];
            load8(bas + 192 + b * PS, v0);
            load8(bas + 256 + b * PS, vr);
            load8(bas + 320 + b * PS, vi);
            const float y0 = y[3 * b], yr = y[3 * b + 1], yi = y[3 * b + 2];
#pragma unroll
            for (int j = 0; j < PS; ++j) {
                s0[j] = fmaf(y0, v0[j], s0[j]);
                sr[j] = fmaf(yr, vr[j], fmaf(-yi, vi[j], sr[j]));
                si[j] = fmaf(yr, vi[j], fmaf(yi, vr[j], si[j]));
            }
        }
#pragma unroll
        for (int j = 0; j < PS; ++j) {
            o[3 * j + 0] = (s0[j] + 2.f * sr[j]) * F_THIRD;
            o[3 * j + 1] = (s0[j] - sr[j] - F_SQ3 * si[j]) * F_THIRD;
            o[3 * j + 2] = (s0[j] - sr[j] + F_SQ3 * si[j]) * F_THIRD;
        }
    } else {
#pragma unroll
        for (int j = 0; j < PS; ++j) o[j] = 0.f;
#pragma unroll
        for (int b = 0; b < PS; ++b) {
            float v0[8];
            load8(bas + 64 + b * PS, v0);
#pragma unroll
            for (int j = 0; j < PS; ++j) o[j] = fmaf(y[b], v0[j], o[j]);
        }
    }
#pragma unroll
    for (int q = 0; q < G::RWF / 4; ++q) row[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
}

// Copies the packed FP32 basis into shared memory, followed by the transpose of each 8x8 block
// (at NBAS): stages D and E read the bases by columns, as outer products.
template <int C>
__device__ __forceinline__ void stage_basis(const float* __restrict__ src, float* bas, int tid) {
    using G = FCfg<C>;
    for (int t = tid; t < G::NBAS; t += FT_THREADS) {
        const float x = src[t];
        bas[t] = x;
        bas[G::NBAS + (t & ~63) + (t & 7) * PS + ((t >> 3) & 7)] = x;
    }
}

// Stage D: thread (i, k): channel DFT, Z_f[i, :] = T_f[i, :] V_f^H, in place on row i of patch k.
// Outer-product order (column j of T_f times row j of the transposed basis) keeps 3 x 8
// independent accumulators; each output sums its terms in the same order as a dot product.
template <int C>
__device__ __forceinline__ void stage_d(const float* bas, float* gb, int k, int i) {
    using G = FCfg<C>;
    float4* row = reinterpret_cast<float4*>(gb + k * G::GS + i * G::ROW);
    float t[G::RWF];
#pragma unroll
    for (int q = 0; q < G::RWF / 4; ++q) {
        float4 v = row[q];
        t[4 * q] = v.x; t[4 * q + 1] = v.y; t[4 * q + 2] = v.z; t[4 * q + 3] = v.w;
    }
    const float* bt = bas + G::NBAS;          // transposed blocks
    float o[G::RWF];
    if constexpr (C == 3) {
        float z0[PS], zr[PS], zi[PS];
#pragma unroll
        for (int b = 0; b < PS; ++b) z0[b] = zr[b] = zi[b] = 0.f;
#pragma unroll
        for (int j = 0; j < PS; ++j) {
            const float T0 = t[3 * j] + t[3 * j + 1] + t[3 * j + 2];
            const float T1r = t[3 * j] - 0.5f * (t[3 * j + 1] + t[3 * j + 2]);
            const float T1i = F_S3H * (t[3 * j + 2] - t[3 * j + 1]);
            float v0[8], vr[8], vi[8];                // column j of V_0, V_1 (re, im)
            load8(bt + 192 + j * PS, v0);
            load8(bt + 256 + j * PS, vr);
            load8(bt + 320 + j * PS, vi);
#pragma unroll
            for (int b = 0; b < PS; ++b) {
                z0[b] = fmaf(T0, v0[b], z0[b]);
                zr[b] = fmaf(T1r, vr[b], fmaf(T1i, vi[b], zr[b]));
                zi[b] = fmaf(T1i, vr[b], fmaf(-T1r, vi[b], zi[b]));
            }
        }
#pragma unroll
        for (int b = 0; b < PS; ++b) {
            o[3 * b] = z0[b]; o[3 * b + 1] = zr[b]; o[3 * b + 2] = zi[b];
        }
    } else {
#pragma unroll
        for (int b = 0; b < PS; ++b) o[b] = 0.f;
#pragma unroll
        for (int j = 0; j < PS; ++j) {
            float v0[8];
            load8(bt + 64 + j * PS, v0);
#pragma unroll
            for (int b = 0; b < PS; ++b) o[b] = fmaf(t[j], v0[b], o[b]);
        }
    }
#pragma unroll
    for (int q = 0; q < G::RWF / 4; ++q) row[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
}

// Stage E: thread (k, b): G_f[:, b] = U_f Z_f[:, b], inverse channel DFT, in place on column b of patch k.
// Outer-product order as in stage D.
template <int C>
__device__ __forceinline__ void stage_e(const float* bas, float* gb, int k, int b) {
    using G = FCfg<C>;
    float* col = gb + k * G::GS + b * C;
    const float* bt = bas + G::NBAS;
    if constexpr (C == 3) {
        float g0[PS], gr[PS], gi[PS];
#pragma unroll
        for (int a = 0; a < PS; ++a) g0[a] = gr[a] = gi[a] = 0.f;
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const float Z0 = col[i * G::ROW], Zr = col[i * G::ROW + 1], Zi = col[i * G::ROW + 2];
            float u0[8], ur[8], ui[8];                // column i of U_0, U_1 (re, im)
            load8(bt + i * PS, u0);
            load8(bt + 64 + i * PS, ur);
            load8(bt + 128 + i * PS, ui);
#pragma unroll
            for (int a = 0; a < PS; ++a) {
                g0[a] = fmaf(u0[a], Z0, g0[a]);
                gr[a] = fmaf(ur[a], Zr, fmaf(-ui[a], Zi, gr[a]));
                gi[a] = fmaf(ur[a], Zi, fmaf(ui[a], Zr, gi[a]));
            }
        }
#pragma unroll
        for (int a = 0; a < PS; ++a) {
            col[a * G::ROW + 0] = (g0[a] + 2.f * gr[a]) * F_THIRD;
            col[a * G::ROW + 1] = (g0[a] - gr[a] - F_SQ3 * gi[a]) * F_THIRD;
            col[a * G::ROW + 2] = (g0[a] - gr[a] + F_SQ3 * gi[a]) * F_THIRD;
        }
    } else {
        float g0[PS];
#pragma unroll
        for (int a = 0; a < PS; ++a) g0[a] = 0.f;
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const float Z = col[i * G::ROW];
            float u0[8];
            load8(bt + i * PS, u0);
#pragma unroll
            for (int a = 0; a < PS; ++a) g0[a] = fmaf(u0[a], Z, g0[a]);
        }
#pragma unroll
        for (int a = 0; a < PS; ++a) col[a * G::ROW] = g0[a];
    }
}

// Two-wide forms of stages A, B, D, E for the pipelined forward filter: thread (k, p), p < 4, owns
// columns 2p, 2p+1 (A, E) or rows r0(p), r0(p) + 2 (B, D) of patch k, so each basis value read
// from shared memory feeds two columns or rows. Each output sums its terms in the same order as
// the one-wide forms. Row pairs start at r0 in {0, 1, 4, 5}: with a patch stride of 8 (mod 32)
// words and row strides of 28 (C = 3) or 12 (C = 1) words, the 128-bit row accesses of a quarter
// warp (2 patches x 4 row pairs) fall on 8 distinct bank groups; the 64-bit column-pair accesses
// of a half warp (4 patches x 4 column pairs) on 32 distinct banks.
__device__ __forceinline__ int row_pair_first(int p) { return (p & 1) + 4 * (p >> 1); }

// Stage A, two columns. Returns the sum of squares of the thread's inputs.
template <int K, int C, typename Tin>
__device__ __forceinline__ float stage_a2(const Tin* img_s, int FW, const int* pos, const float* bas, float* gb,
                                          int k, int p) {
    using G = FCfg<C>;
    const Tin* src = img_s + (pos[2 * k] * FW + pos[2 * k + 1] + 2 * p) * C;
    float* dst = gb + k * G::GS + 2 * p * C;
    float nrm = 0.f;
    if constexpr (C == 3) {
        float y0[2][PS], yr[2][PS], yi[2][PS];
#pragma unroll
        for (int w = 0; w < 2; ++w)
#pragma unroll
            for (int ii = 0; ii < PS; ++ii) y0[w][ii] = yr[w][ii] = yi[w][ii] = 0.f;
#pragma unroll 1
        for (int a = 0; a < PS; ++a) {
            float X0[2], X1r[2], X1i[2];
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                const float x0 = ldv(src + a * FW * C + w * C), x1 = ldv(src + a * FW * C + w * C + 1),
                            x2 = ldv(src + a * FW * C + w * C + 2);
                nrm = fmaf(x0, x0, nrm);
                nrm = fmaf(x1, x1, nrm);
                nrm = fmaf(x2, x2, nrm);
                X0[w] = x0 + x1 + x2;
                X1r[w] = x0 - 0.5f * (x1 + x2);
                X1i[w] = F_S3H * (x2 - x1);
            }
            float u0[8], ur[8], ui[8];
            load8(bas + a * PS, u0);
            load8(bas + 64 + a * PS, ur);
            load8(bas + 128 + a * PS, ui);
#pragma unroll
            for (int ii = 0; ii < PS; ++ii)
#pragma unroll
                for (int w = 0; w < 2; ++w) {
                    y0[w][ii] = fmaf(u0[ii], X0[w], y0[w][ii]);
                    yr[w][ii] = fmaf(ur[ii], X1r[w], fmaf(ui[ii], X1i[w], yr[w][ii]));
                    yi[w][ii] = fmaf(ur[ii], X1i[w], fmaf(-ui[ii], X1r[w], yi[w][ii]));
                }
        }
#pragma unroll
        for (int ii = 0; ii < PS; ++ii) {
            float2* d = reinterpret_cast<float2*>(dst + ii * G::ROW);
            d[0] = make_float2(y0[0][ii], yr[0][ii]);
            d[1] = make_float2(yi[0][ii], y0[1][ii]);
            d[2] = make_float2(yr[1][ii], yi[1][ii]);
        }
    } else {
        float y0[2][PS];
#pragma unroll
        for (int w = 0; w < 2; ++w)
#pragma unroll
            for (int ii = 0; ii < PS; ++ii) y0[w][ii] = 0.f;
#pragma unroll 1
        for (int a = 0; a < PS; ++a) {
            const float x0 = ldv(src + a * FW), x1 = ldv(src + a * FW + 1);
            nrm = fmaf(x0, x0, nrm);
            nrm = fmaf(x1, x1, nrm);
            float u0[8];
            load8(bas + a * PS, u0);
#pragma unroll
            for (int ii = 0; ii < PS; ++ii) {
                y0[0][ii] = fmaf(u0[ii], x0, y0[0][ii]);
                y0[1][ii] = fmaf(u0[ii], x1, y0[1][ii]);
            }
        }
#pragma unroll
        for (int ii = 0; ii < PS; ++ii)
            *reinterpret_cast<float2*>(dst + ii * G::ROW) = make_float2(y0[0][ii], y0[1][ii]);
    }
    return nrm;
}

// Six consecutive floats 6*bb .. 6*bb+5 of a 16-byte aligned C = 3 row (one 128-bit and one 64-bit
// load); odd = bb & 1, a constant at every call site once the loops unroll.
__device__ __forceinline__ void load6(const float* row, int bb, int odd, float (&r)[6]) {
    if (odd == 0) {
        const float4 a = *reinterpret_cast<const float4*>(row + 6 * bb);
        const float2 b = *reinterpret_cast<const float2*>(row + 6 * bb + 4);
        r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w; r[4] = b.x; r[5] = b.y;
    } else {
        const float2 a = *reinterpret_cast<const float2*>(row + 6 * bb);
        const float4 b = *reinterpret_cast<const float4*>(row + 6 * bb + 2);
        r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y; r[4] = b.z; r[5] = b.w;
    }
}

// Stage B, two rows (S_f[i, :] = Y_f[i, :] V_f, inverse channel DFT).
template <int C>
__device__ __forceinline__ void stage_b2(const float* bas, float* gb, int k, int p) {
    using G = FCfg<C>;
    const int r0 = row_pair_first(p);
    float* rows[2] = {gb + k * G::GS + r0 * G::ROW, gb + k * G::GS + (r0 + 2) * G::ROW};
    if constexpr (C == 3) {
        float s0[2][PS], sr[2][PS], si[2][PS];
#pragma unroll
        for (int w = 0; w < 2; ++w)
#pragma unroll
            for (int j = 0; j < PS; ++j) s0[w][j] = sr[w][j] = si[w][j] = 0.f;
#pragma unroll 1
        for (int bb2 = 0; bb2 < PS / 2; bb2 += 2)
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            const int bb = bb2 + par;
            float y[2][6];
            load6(rows[0], bb, par, y[0]);
            load6(rows[1], bb, par, y[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int b = 2 * bb + h;
                float v0[8], vr[8], vi[8];
                load8(bas + 192 + b * PS, v0);
                load8(bas + 256 + b * PS, vr);
                load8(bas + 320 + b * PS, vi);
#pragma unroll
                for (int j = 0; j < PS; ++j)
#pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        const float y0 = y[w][3 * h], yr = y[w][3 * h + 1], yi = y[w][3 * h + 2];
                        s0[w][j] = fmaf(y0, v0[j], s0[w][j]);
                        sr[w][j] = fmaf(yr, vr[j], fmaf(-yi, vi[j], sr[w][j]));
                        si[w][j] = fmaf(yr, vi[j], fmaf(yi, vr[j], si[w][j]));
                    }
            }
        }
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            float o[G::RWF];
#pragma unroll
            for (int j = 0; j < PS; ++j) {
                o[3 * j + 0] = (s0[w][j] + 2.f * sr[w][j]) * F_THIRD;
                o[3 * j + 1] = (s0[w][j] - sr[w][j] - F_SQ3 * si[w][j]) * F_THIRD;
                o[3 * j + 2] = (s0[w][j] - sr[w][j] + F_SQ3 * si[w][j]) * F_THIRD;
            }
            float4* r4 = reinterpret_cast<float4*>(rows[w]);
#pragma unroll
            for (int q = 0; q < G::RWF / 4; ++q) r4[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        }
    } else {
        float y[2][PS], o[2][PS];
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            load8(rows[w], y[w]);
#pragma unroll
            for (int j = 0; j < PS; ++j) o[w][j] = 0.f;
        }
#pragma unroll
        for (int b = 0; b < PS; ++b) {
            float v0[8];
            load8(bas + 64 + b * PS, v0);
#pragma unroll
            for (int j = 0; j < PS; ++j)
#pragma unroll
                for (int w = 0; w < 2; ++w) o[w][j] = fmaf(y[w][b], v0[j], o[w][j]);
        }
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            float4* r4 = reinterpret_cast<float4*>(rows[w]);
            r4[0] = make_float4(o[w][0], o[w][1], o[w][2], o[w][3]);
            r4[1] = make_float4(o[w][4], o[w][5], o[w][6], o[w][7]);
        }
    }
}

// Stage D for one row of a Haar slot in the sparse inverse: thread -> Z_f[i, :] = T_f[i, :] V_f^H of
// slot k, in place on row i. Same terms and order as stage D, but the row is streamed two columns at
// a time (load6) and the outer column loop stays rolled, so that the transposed basis rows are not
// all loaded ahead (with them the kernel outgrew its 128 registers).
template <int C>
__device__ __forceinline__ void stage_d_row(const float* bas, float* gb, int k, int i) {
    using G = FCfg<C>;
    float* row = gb + k * G::GS + i * G::ROW;
    const float* bt = bas + G::NBAS;
    if constexpr (C == 3) {
        float z0[PS], zr[PS], zi[PS];
#pragma unroll
        for (int b = 0; b < PS; ++b) z0[b] = zr[b] = zi[b] = 0.f;
#pragma unroll 1
        for (int jj2 = 0; jj2 < PS / 2; jj2 += 2)
#pragma unroll
        for (int par = 0; par < 2; ++par) {
            const int jj = jj2 + par;
            float t[6];
            load6(row, jj, par, t);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = 2 * jj + h;
                const float T0 = t[3 * h] + t[3 * h + 1] + t[3 * h + 2];
                const float T1r = t[3 * h] - 0.5f * (t[3 * h + 1] + t[3 * h + 2]);
                const float T1i = F_S3H * (t[3 * h + 2] - t[3 * h + 1]);
                float v0[8], vr[8], vi[8];
                load8(bt + 192 + j * PS, v0);
                load8(bt + 256 + j * PS, vr);
                load8(bt + 320 + j * PS, vi);
#pragma unroll
                for (int b = 0; b < PS; ++b) {
                    z0[b] = fmaf(T0, v0[b], z0[b]);
                    zr[b] = fmaf(T1r, vr[b], fmaf(T1i, vi[b], zr[b]));
                    zi[b] = fmaf(T1i, vr[b], fmaf(-T1r, vi[b], zi[b]));
                }
            }
        }
        float4* r4 = reinterpret_cast<float4*>(row);
#pragma unroll
        for (int q = 0; q < G::RWF / 4; ++q) {
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int n = 4 * q + e, b = n / 3, c = n % 3;
                o[e] = c == 0 ? z0[b] : (c == 1 ? zr[b] : zi[b]);
            }
            r4[q] = make_float4(o[0], o[1], o[2], o[3]);
        }
    } else {
        stage_d<C>(bas, gb, k, i);
    }
}

// Sparse form of stage E for the inverse of one Haar slot: thread (k, b) -> G_f[:, b] = U_f Z_f[:, b],
// summing only over the basis rows i set in nzrows (the other rows of Z are zero), then the inverse
// channel DFT, written in place on column b of slot k. Terms are added in ascending i as in stage E,
// so the result equals stage E on the same slot bit for bit.
template <int C>
__device__ __forceinline__ void stage_e_sparse(const float* bas, float* gb, int k, int b, uint32_t nzrows) {
    using G = FCfg<C>;
    float* col = gb + k * G::GS + b * C;
    const float* bt = bas + G::NBAS;
    if constexpr (C == 3) {
        float g0[PS], gr[PS], gi[PS];
#pragma unroll
        for (int a = 0; a < PS; ++a) g0[a] = gr[a] = gi[a] = 0.f;
#pragma unroll 1
        for (uint32_t m = nzrows; m; m &= m - 1) {
            const int i = __ffs(m) - 1;
            const float Z0 = col[i * G::ROW], Zr = col[i * G::ROW + 1], Zi = col[i * G::ROW + 2];
            float u0[8], ur[8], ui[8];
            load8(bt + i * PS, u0);
            load8(bt + 64 + i * PS, ur);
            load8(bt + 128 + i * PS, ui);
#pragma unroll
            for (int a = 0; a < PS; ++a) {
                g0[a] = fmaf(u0[a], Z0, g0[a]);
                gr[a] = fmaf(ur[a], Zr, fmaf(-ui[a], Zi, gr[a]));
                gi[a] = fmaf(ur[a], Zi, fmaf(ui[a], Zr, gi[a]));
            }
        }
#pragma unroll
        for (int a = 0; a < PS; ++a) {
            col[a * G::ROW + 0] = (g0[a] + 2.f * gr[a]) * F_THIRD;
            col[a * G::ROW + 1] = (g0[a] - gr[a] - F_SQ3 * gi[a]) * F_THIRD;
            col[a * G::ROW + 2] = (g0[a] - gr[a] + F_SQ3 * gi[a]) * F_THIRD;
        }
    } else {
        float g0[PS];
#pragma unroll
        for (int a = 0; a < PS; ++a) g0[a] = 0.f;
#pragma unroll 1
        for (uint32_t m = nzrows; m; m &= m - 1) {
            const int i = __ffs(m) - 1;
            const float Z = col[i * G::ROW];
            float u0[8];
            load8(bt + i * PS, u0);
#pragma unroll
            for (int a = 0; a < PS; ++a) g0[a] = fmaf(u0[a], Z, g0[a]);
        }
#pragma unroll
        for (int a = 0; a < PS; ++a) col[a * G::ROW] = g0[a];
    }
}

// Fibre of virtual warp vw, lane l in the Haar stages: the vw-th fibre (in patch-row order) whose
// group-buffer column falls on bank l, so the 32 fibres a warp handles use 32 distinct banks (each
// bank holds NF/32 fibres: the rows start ROW words apart and cover RWF words). -1 if none.
template <int C>
__device__ __forceinline__ int bank_fibre(int vw, int lane) {
    using G = FCfg<C>;
    for (int i = 0, cnt = 0; i < PS; ++i) {
        const int e = (lane - G::ROW * i) & 31;
        if (e < G::RWF) {
            if (cnt == vw) return i * G::RWF + e;
            ++cnt;
        }
    }
    return -1;
}

__device__ __forceinline__ void bar_sync_lower_half() {       // warps 0 .. 3 only (named barrier 1)
    asm volatile("bar.sync 1, 128;" ::: "memory");
}
// Named barrier 3, all 256 threads: the fibre warps arrive after the C phase, the aggregation warps
// wait for it (they build the next group's stage-D work list from its finished row masks).
__device__ __forceinline__ void bar_arrive_cdone() { asm volatile("bar.arrive 3, 256;" ::: "memory"); }
__device__ __forceinline__ void bar_sync_cdone() { asm volatile("bar.sync 3, 256;" ::: "memory"); }

// Forward filter of one tile, software-pipelined over its groups with two CTA barriers per group:
// [inverse of q on the first half of the CTA | A, B(q+1) on the second half] then [F(q) aggregation
// on all warps, C(q+1) Haar analysis and threshold]. The inverse runs in the Haar domain: the Haar
// transform along the group mode and the per-patch t-SVD projection commute, so C leaves the
// thresholded coefficients of every Haar slot in place (scaled for the unnormalised synthesis) and
// records which basis rows of each slot hold a kept coefficient; the first half then applies stage D
// to those rows only (a compacted work list), stage E summing over those rows only, and the Haar
// synthesis per fibre, separated by a named barrier of its four warps. After the threshold most
// slots keep coefficients in two or three basis rows, so this inverse does a fraction of the dense
// one's work and gives the same values up to rounding order; the forward half then sets the pace. Group buffers alternate; positions and
// counters rotate over three slots (those of q+2 are written while q and q+1 are in flight).
// Guard-band entries are re-decided in FP64 by the warp that owns the fibre (no CTA barrier).
// MF: video groups (FM_VIDEO). The footprints of the clip's frames f0 .. f0 + nfr - 1 are staged
// one above the other, the reference frame's first (slot 0, rows [0, FH)), the others after it in
// frame order; a patch's staged row is slot * FH + its row in the footprint, so every stage reads
// it as in one image, and the aggregation adds the slot-0 patches only.
// VAR: 0 the whole filter; 1 (FM_ANALYZE) projections and Haar analysis only, the coefficients,
// patch norms and ||G||_F^2 written to the cache; 2 (FM_SYNTH) the cached coefficients loaded in
// place of the projections, then threshold, synthesis and aggregation as in the whole filter.
template <int K, int C, typename Tin, bool MF, int VAR = 0>
__device__ __forceinline__ void filter_tile_fwd(const FilterArgs& a, const int tile, unsigned char* smem) {
    using G = FCfg<C>;
    constexpr int NF = G::PATCH;
    constexpr int NBW = K * NF / 32;
    constexpr int NU = 4 * K;                    // threads of a two-wide stage: K patches x 4
    constexpr int AB0 = FT_THREADS / 2;          // first thread of the A, B half
    static_assert(NU <= AB0, "two-wide stages need 4K <= half the CTA");
    constexpr unsigned kU = (NU >= 32) ? 0xffffffffu : ((1u << NU) - 1u);
    const Geo& g = a.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
    int FY0, FY1, FX0, FX1;
    tile_span(ty, a.TR, g.nry, g.s, g.H, g.npy, g.wny, g.win, FY0, FY1);
    tile_span(tx, a.TR, g.nrx, g.s, g.W, g.npx, g.wnx, g.win, FX0, FX1);
    const int FH = FY1 - FY0, FW = FX1 - FX0;
    const int nfr = MF ? a.nfr : 1;
    const FLayout L = f_layout_fwd<K, C>(a.FHmax, a.FWmax, (int)sizeof(Tin), nfr);
    using O = FwdOff<K, C>;
    float* bas = reinterpret_cast<float*>(smem + O::bas);
    float* gbb = reinterpret_cast<float*>(smem + O::gb);
    int* posb = reinterpret_cast<int*>(smem + O::pos);
    int* miscb = reinterpret_cast<int*>(smem + O::misc);
    float* pnb = reinterpret_cast<float*>(smem + O::band);
    uint32_t* nzb = reinterpret_cast<uint32_t*>(smem + O::nz);                // [2][32] basis-row masks
    unsigned char* dlist = smem + O::dlist;                                  // stage-D work list (k << 3 | i)
    int* dcount = reinterpret_cast<int*>(smem + O::dcount);
    int2* aofs = reinterpret_cast<int2*>(smem + O::aofs);                     // [patch][row class]
    float* acc = reinterpret_cast<float*>(smem + O::acc);
    Tin* img_s = reinterpret_cast<Tin*>(smem + L.off_img);
    // frame of staging slot sl (slot 0: the reference frame, then the others in order)
    auto slot_frame = [&](int sl) {
        if (!MF) return 0;
        const int f = a.f0 + sl - 1;
        return sl == 0 ? a.fref : (f >= a.fref ? f + 1 : f);
    };

    stage_basis<C>(a.basis32, bas, tid);
    {
        const int rowb = FW * C;
        for (int t = tid; t < nfr * FH * rowb; t += FT_THREADS) {
            const int sl = t / (FH * rowb), tt = t - sl * (FH * rowb);
            const int r = tt / rowb, cb = tt - r * rowb;
            const Tin* img = MF ? reinterpret_cast<const Tin*>(a.vid) + (size_t)slot_frame(sl) * a.fstride
                                : reinterpret_cast<const Tin*>(a.img);
            img_s[t] = img[((size_t)(FY0 + r) * g.W + FX0) * C + cb];
        }
    }
    for (int t = tid; t < FH * FW * G::ACC; t += FT_THREADS) acc[t] = 0.f;

    const int iy0 = ty * a.TR, ix0 = tx * a.TR;
    const int th = min(a.TR, g.nry - iy0), tw = min(a.TR, g.nrx - ix0);
    const int ngr = th * tw;
    auto group_of = [&](int q) { return (iy0 + q / tw) * g.nrx + ix0 + q % tw; };
    // Positions come from the grouping of this geometry and lie in the footprint; a caller-given
    // index outside it is clamped so that no access leaves the staged region.
    auto store_pos = [&](int v, int* pos) {
        if (tid < K) {
            int sl = 0;
            if (MF) {                                 // frame -> staging slot (clamped to the staged frames)
                const int hw = g.H * g.W;
                const int f = min(max(v / hw, a.f0), a.f0 + a.nfr - 1);
                v = max(v - (v / hw) * hw, 0);
                sl = f == a.fref ? 0 : (f < a.fref ? f - a.f0 + 1 : f - a.f0);
            }
            const int y = v / g.W, x = v - y * g.W;
            pos[2 * tid] = sl * FH + min(max(y - FY0, 0), FH - PS);
            pos[2 * tid + 1] = min(max(x - FX0, 0), FW - PS);
        }
    };
    auto fetch_idx = [&](int q) { return tid < K ? a.idx[(size_t)group_of(q) * K + tid] : 0; };
    // slots: group buffer and patch norms alternate, positions and counters rotate over three
    auto gb_of = [&](int q) { return gbb + (q & 1) * K * G::GS; };
    auto pn_of = [&](int q) { return pnb + (q & 1) * 32; };
    auto pos_of = [&](int q) { return posb + (q % 3) * 64; };
    auto misc_of = [&](int q) { return miscb + (q % 3) * 16; };
    auto nz_of = [&](int q) { return nzb + (q & 1) * 32; };
    // A, B of group q by thread u < NU of the second half; ||G||_F^2 into misc[5] (uint8, exact) or
    // misc[2] (float), and the squared norm of each patch into pn[k]
    auto project = [&](int u, int q) {
        float* gbq = gb_of(q);
        int* misc = misc_of(q);
        const float nrm = stage_a2<K, C, Tin>(img_s, FW, pos_of(q), bas, gbq, u >> 2, u & 3);
        {
            float pk = nrm;                               // the 4 column pairs of patch k are 4 adjacent lanes
            pk += __shfl_xor_sync(kU, pk, 1);
            pk += __shfl_xor_sync(kU, pk, 2);
            if ((u & 3) == 0) pn_of(q)[u >> 2] = pk;
        }
        if constexpr (sizeof(Tin) == 1) {
            const int wsum = __reduce_add_sync(kU, (int)nrm);
            if (lane == 0) atomicAdd(&misc[5], wsum);
        } else {
            float v = nrm;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                if (off < NU) v += __shfl_xor_sync(kU, v, off);
            if (lane == 0) atomicAdd(reinterpret_cast<float*>(&misc[2]), v);
        }
        __syncwarp(kU);                                   // stage B reads the rows the 4 lanes of patch k wrote
        stage_b2<C>(bas, gbq, u >> 2, u & 3);
    };

    // Fibre of this thread in the C phase: thread (w, l) takes the w-th fibre (in patch-row order)
    // whose group-buffer column falls on bank l, so the 32 fibres of a warp use 32 distinct banks
    // (each bank holds NF/32 fibres: the rows start ROW words apart and cover RWF words).
    int fib = -1, foff = 0;
    if (tid < NF) {
        fib = bank_fibre<C>(warp, lane);
        foff = (fib / G::RWF) * G::ROW + (fib % G::RWF);
    }
    auto clear_masks = [&](int q) {                     // mask words of group q, before its C phase
        if (a.mask_out && tid < NBW) a.mask_out[(size_t)group_of(q) * NBW + tid] = 0u;
    };

    // F(q) on two warps: warp h adds the footprint rows r with r % 8 in {4h, ..., 4h + 3}; lane
    // (row class 4h + lane / 8, pixel lane % 8) adds that pixel's C numerators and its weight as one
    // vector. The four row classes of a warp are four different footprint rows, so the lanes of one
    // instruction never share an address; patches go in ascending order (no atomics), and these
    // warps run beside the C phase of the next group on the others.
    auto aggregate2 = [&](const int q, const int h) {
        const int grp = group_of(q);
        const float* gbq = gb_of(q);
        const int* misc = misc_of(q);
        float wg = 1.f;
        if (a.w_in) wg = a.w_in[grp];
        else if (a.agg_mode == 1) wg = 1.f / (float)max(1, misc[1]);
        if (h == 0 && lane == 0 && a.weights_out) a.weights_out[grp] = wg;
        const int rc = 4 * h + (lane >> 3), j = lane & 7;
        constexpr int CH = K < 4 ? K : 4;             // patches whose offsets and values are fetched ahead
        static_assert(K % CH == 0, "the chunks cover the group exactly");
#pragma unroll 1
        for (int k0 = 0; k0 < K; k0 += CH) {
            int ao[CH];
            float xv[CH][C];
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int2 o = aofs[(k0 + u) * 8 + rc];   // (accumulator, group-buffer) offsets of the row
                ao[u] = o.x < 0 ? -1 : o.x + j * G::ACC;
                const float* src = gbq + o.y + j * C;
#pragma unroll
                for (int c = 0; c < C; ++c) xv[u][c] = src[c];
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (!MF || ao[u] >= 0) {
                    if constexpr (C == 3) {
                        float4* d = reinterpret_cast<float4*>(acc + ao[u]);
                        float4 t = *d;
                        t.x = fmaf(wg, xv[u][0], t.x);
                        t.y = fmaf(wg, xv[u][1], t.y);
                        t.z = fmaf(wg, xv[u][2], t.z);
                        t.w += wg;
                        *d = t;
                    } else {
                        float2* d = reinterpret_cast<float2*>(acc + ao[u]);
                        float2 t = *d;
                        t.x = fmaf(wg, xv[u][0], t.x);
                        t.y += wg;
                        *d = t;
                    }
                }
                __syncwarp();                         // orders the read-modify-writes of patches k, k+1
            }
        }
    };

    // offsets for aggregate2 of group q, for the four row classes of warp h: patch k's row i with
    // (py + i) % 8 = rc starts at accumulator float ((py + i) FW + px) ACC (-1: a patch of another
    // frame) and group-buffer float k GS + i ROW
    auto agg_offsets = [&](const int q, const int h) {
        const int* pos = pos_of(q);
        for (int e = lane; e < K * 4; e += 32) {
            const int k = e >> 2, rc = 4 * h + (e & 3);
            const int py = pos[2 * k], px = pos[2 * k + 1], i = (rc - py) & 7;
            int ao = ((py + i) * FW + px) * G::ACC;
            if (MF && py >= FH) ao = -1;
            aofs[k * 8 + rc] = make_int2(ao, k * G::GS + i * G::ROW);
        }
    };

    // C(q): Haar analysis, threshold (FP64 inside the guard band), synthesis, by the NF fibre threads
    auto phase_c = [&](const int q) {
        const int grp = group_of(q);
        float* gbq = gb_of(q);
        const int* pos = pos_of(q);
        int* misc = misc_of(q);
        const float* pn = pn_of(q);
        // final keep decisions of the warp's fibres: optional mask output, kept count
        // (nzs: kept coefficients as bits by Haar slot)
        auto keep_finish = [&](uint32_t nzs) {
            if (a.mask_out) {                             // words cleared a phase earlier
                uint32_t keepb = 0;                       // the same bits by Haar row
                haar_for_each<K>([&](int m, int sl, int L) { keepb |= ((nzs >> sl) & 1u) << m; });
                uint32_t* mo = a.mask_out + (size_t)grp * NBW;
                for (uint32_t b = keepb; b; b &= b - 1) {
                    const int m = __ffs(b) - 1;
                    atomicOr(&mo[m * (NF / 32) + (fib >> 5)], 1u << (fib & 31));
                }
            }
            const int wk = __reduce_add_sync(0xffffffffu, __popc(nzs));
            if (lane == 0) atomicAdd(&misc[1], wk);
        };
        // basis row of this fibre into the masks of the Haar slots where it kept a coefficient
        auto mark_rows = [&](uint32_t nzs) {
            uint32_t* nz = nz_of(q);
            for (uint32_t b = nzs; b; b &= b - 1) atomicOr(&nz[__ffs(b) - 1], 1u << (fib / G::RWF));
        };
        if constexpr (VAR == 1) {                     // per-patch norms and ||G||_F^2 of the group
            if (tid < K) a.cache_pn[(size_t)grp * 32 + tid] = pn[tid];
            if (tid == 0) a.cache_nrm[grp] = sizeof(Tin) == 1 ? misc[5] : misc[2];
        }
        if (tid < NF) {
            const float nrm2 = sizeof(Tin) == 1 ? (float)misc[5] : __int_as_float(misc[2]);
            const float delta = a.band_rel * sqrtf(nrm2) + a.band_abs;
            // (the rare guard-band path finishes the fibre in a scope of its own, with a second
            // array reloaded from shared memory, so that no K-register array is live across the
            // FP64 refinement loop: that would push the array to local memory)
            uint32_t nzs = 0, bandb = 0;                  // kept (by Haar slot), inside the band (by Haar row)
            unsigned anyb;
            // The Haar transform runs unnormalised (sums and differences): row m's coefficient is
            // sqrt(L_m) times the normalised one, so threshold and band scale by sqrt(L_m) (one pair of
            // values per support size L = 2^j) and kept coefficients by 1 / L_m before synthesis.
            {
                float v[K];                               // fibre, then its coefficients (haar_for_each slots)
#pragma unroll
                for (int k = 0; k < K; ++k) v[k] = gbq[k * G::GS + foff];
                if constexpr (VAR != 2) haar_fwd_sum<K>(v);
                if constexpr (VAR == 1) {                 // analysis only: cache the coefficients
                    float* cdst = a.cache_coef + (size_t)grp * K * NF + fib;
#pragma unroll
                    for (int k = 0; k < K; ++k) cdst[(size_t)k * NF] = v[k];
                    return;
                }
                if (a.coef_out) {
                    float* cdst = a.coef_out + (size_t)grp * K * NF;
                    haar_for_each<K>([&](int m, int sl, int L) { cdst[m * NF + fib] = v[sl] * rsqrtf((float)L); });
                }
                // decided coefficients are scaled (kept, by 1 / L) or zeroed in place; a coefficient
                // inside the band keeps its raw value until it is decided
                haar_for_each<K>([&](int m, int sl, int L) {
                    const float r = sqrtf((float)L);      // folds to a constant once unrolled
                    const float d = fmaf(-a.tau32, r, fabsf(v[sl]));
                    const bool band = fabsf(d) <= delta * r;
                    const bool kp = !band && d >= 0.f;
                    bandb |= (band ? 1u : 0u) << m;
                    nzs |= (kp ? 1u : 0u) << sl;
                    v[sl] = band ? v[sl] : (kp ? v[sl] * (1.f / (float)L) : 0.f);
                });
#pragma unroll
                for (int k = 0; k < K; ++k) gbq[k * G::GS + foff] = v[k];    // band coefficients still raw
                if (bandb != 0u && (bandb & (bandb - 1u)) == 0u) {
                    // one entry inside the group-wide band (the usual case): the FP32 error of row m
                    // only involves the patches of its Haar support (L = K / 2^level patches from k0),
                    // so the band narrows to their norm. Row m >= 1 of level lv sits in slot
                    // (2 (m - 2^lv) + 1) K / 2^(lv + 1); row 0 in slot 0.
                    const int m = __ffs(bandb) - 1;
                    const int lv = m == 0 ? 0 : 31 - __clz(m);
                    const int L = m == 0 ? K : K >> lv, k0 = m == 0 ? 0 : (m - (1 << lv)) * L;
                    const int sl = m == 0 ? 0 : (2 * (m - (1 << lv)) + 1) * (K >> (lv + 1));
                    float* cm = gbq + sl * G::GS + foff;
                    const float raw = *cm, dm = fmaf(-a.tau32, sqrtf((float)L), fabsf(raw));
                    float sq = 0.f;
                    for (int k = k0; k < k0 + L; ++k) sq += pn[k];
                    if (fabsf(dm) > (a.band_rel * sqrtf(sq) + a.band_abs) * sqrtf((float)L)) {
                        bandb = 0u;
                        const bool kp = dm >= 0.f;
                        *cm = kp ? raw * (1.f / (float)L) : 0.f;
                        nzs |= (kp ? 1u : 0u) << sl;
                    }
                }
                anyb = __ballot_sync(0xffffffffu, bandb != 0u);
                if (!anyb) {
                    keep_finish(nzs);
                    mark_rows(nzs);
                }
            }
            if (anyb) {                                   // warp-uniform
                uint32_t keepb = 0;                       // the kept bits by Haar row, then the FP64 ones
                haar_for_each<K>([&](int m, int sl, int L) { keepb |= ((nzs >> sl) & 1u) << m; });
                __syncwarp();
                do {
                    const int l = __ffs(anyb) - 1;
                    anyb &= anyb - 1;
                    uint32_t bb = __shfl_sync(0xffffffffu, bandb, l);
                    const int fl = __shfl_sync(0xffffffffu, fib, l);
                    while (bb) {
                        const int m = __ffs(bb) - 1;
                        bb &= bb - 1;
                        const bool keep = refine_keep<K, C, Tin>(m, fl, img_s, FW, pos, a.basis64, a.tau64, lane);
                        if (lane == l && keep) keepb |= 1u << m;
                    }
                } while (anyb);
                __syncwarp();
                float w[K];
#pragma unroll
                for (int k = 0; k < K; ++k) w[k] = gbq[k * G::GS + foff];
                uint32_t nzf = 0;
                haar_for_each<K>([&](int m, int sl, int L) {
                    const bool kp = (keepb >> m) & 1u;
                    if ((bandb >> m) & 1u) w[sl] = kp ? w[sl] * (1.f / (float)L) : 0.f;    // the rest is final
                    nzf |= (kp ? 1u : 0u) << sl;
                });
#pragma unroll
                for (int k = 0; k < K; ++k) gbq[k * G::GS + foff] = w[k];
                keep_finish(nzf);
                mark_rows(nzf);
            }
        }
    };

    // iteration q: [inverse of q: D, E, Haar synthesis | A, B(q+1)] then [F(q), C(q+1)]; q = -1 only
    // projects and thresholds group 0
    store_pos(fetch_idx(0), pos_of(0));
    if (tid < 48) miscb[tid] = 0;
    // fibres of the synthesis stage: the first half's warps take the bank-mapped fibres of virtual
    // warps w and w + 4 (NF / 32 of them: 6 for C = 3, 2 for C = 1)
    const int fibA = bank_fibre<C>(warp & 3, lane), fibB = bank_fibre<C>((warp & 3) + 4, lane);
    const int foffA = fibA < 0 ? 0 : (fibA / G::RWF) * G::ROW + (fibA % G::RWF);
    const int foffB = fibB < 0 ? 0 : (fibB / G::RWF) * G::ROW + (fibB % G::RWF);
    __syncthreads();

    for (int q = -1; q < ngr; ++q) {
        // indices of group q+2: loaded here, stored at the end of the second phase
        const int next_idx = q + 2 < ngr ? fetch_idx(q + 2) : 0;

        // ---- inverse of group q on the first half (warps 0-3, named barrier 1) ...
        if constexpr (VAR != 1) {
            if (q >= 0 && tid < 128) {
                float* gbq = gb_of(q);
                const uint32_t* nz = nz_of(q);
                // stage D over the work list of the (Haar slot k, basis row i) pairs holding a kept
                // coefficient (built at the end of the group's C phase)
                const int nd = *dcount;
#pragma unroll 1
                for (int it = tid; it < nd; it += 128) {
                    const int e = dlist[it];
                    stage_d_row<C>(bas, gbq, e >> 3, e & 7);
                }
                bar_sync_lower_half();
#pragma unroll 1
                for (int u = tid; u < K * PS; u += 128) {
                    const uint32_t rows = nz[u >> 3];
                    if (rows) stage_e_sparse<C>(bas, gbq, u >> 3, u & 7, rows);   // slots without a kept
                }                                                               // coefficient stay zero
                bar_sync_lower_half();
                // Haar synthesis along the group mode, per fibre (virtual warps w and w + 4)
#pragma unroll 1
                for (int pass = 0; pass < 2; ++pass) {
                    if (((warp & 3) + 4 * pass) * 32 >= NF) break;               // warp-uniform
                    const int fo = pass == 0 ? foffA : foffB;
                    float v[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) v[k] = gbq[k * G::GS + fo];
                    haar_inv_sum<K>(v);
#pragma unroll
                    for (int k = 0; k < K; ++k) gbq[k * G::GS + fo] = v[k];
                }
            }
        }
        // ... beside A, B(q+1) on the second half
        if (tid >= AB0 && tid < AB0 + NU && q + 1 < ngr) {
            if constexpr (VAR == 2) {
                // the cached coefficients of group q+1, four fibres per 128-bit word (64 C fibres per
                // slot; a run of four never crosses a patch row)
                const int u = tid - AB0;
                const int g1 = group_of(q + 1);
                const float4* src = reinterpret_cast<const float4*>(a.cache_coef + (size_t)g1 * K * NF);
                float* gbn = gb_of(q + 1);
                for (int e4 = u; e4 < K * NF / 4; e4 += NU) {
                    const int k = e4 / (NF / 4), fb = 4 * (e4 - k * (NF / 4));
                    *reinterpret_cast<float4*>(gbn + k * G::GS + (fb / G::RWF) * G::ROW + fb % G::RWF) = src[e4];
                }
                if (u < K) pn_of(q + 1)[u] = a.cache_pn[(size_t)g1 * 32 + u];
                if (u == 0) misc_of(q + 1)[sizeof(Tin) == 1 ? 5 : 2] = a.cache_nrm[g1];
            } else {
                project(tid - AB0, q + 1);
            }
        }
        if (q + 1 < ngr) {
            clear_masks(q + 1);
            if (tid >= AB0 && tid < AB0 + 32) nz_of(q + 1)[tid - AB0] = 0u;
        }
        __syncthreads();
        // ---- F(q) on warps 6, 7 beside C(q+1) on the fibre warps; positions and counters of q+2
        // into the slot that q-1 used
        if (warp >= 6) {
            if (VAR != 1 && q >= 0) aggregate2(q, warp - 6);
            if (VAR != 1 && q + 1 < ngr) {
                __syncwarp();                         // every lane is done with group q's offsets
                agg_offsets(q + 1, warp - 6);
                // stage-D work list of group q+1 once its row masks are final: the (Haar slot k,
                // basis row i) pairs holding a kept coefficient, in (k, i) order
                bar_sync_cdone();
                if (warp == 6) {
                    const uint32_t msk = lane < K ? nz_of(q + 1)[lane] : 0u;
                    const int c = __popc(msk);
                    int incl = c;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int t = __shfl_up_sync(0xffffffffu, incl, off);
                        if (lane >= off) incl += t;
                    }
                    int o = incl - c;
                    for (uint32_t b = msk; b; b &= b - 1) dlist[o++] = (unsigned char)((lane << 3) | (__ffs(b) - 1));
                    if (lane == 31) *dcount = incl;
                }
            }
        } else if (q + 1 < ngr) {
            phase_c(q + 1);
            if (VAR != 1) bar_arrive_cdone();
        }
        if (q + 2 < ngr) {
            store_pos(next_idx, pos_of(q + 2));
            if (tid < 16) misc_of(q + 2)[tid] = 0;
        }
        __syncthreads();
    }
    if constexpr (VAR == 1) return;                   // analysis only: nothing aggregated
    // Write the tile partial.
    float* dst = a.partials + (size_t)tile * a.FHmax * a.FWmax * G::ACC;
    if constexpr (C == 3) {
        const float4* s4 = reinterpret_cast<const float4*>(acc);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int t = tid; t < FH * FW; t += FT_THREADS) {
            const int r = t / FW, c = t - r * FW;
            d4[r * a.FWmax + c] = s4[t];
        }
    } else {
        const float2* s2 = reinterpret_cast<const float2*>(acc);
        float2* d2 = reinterpret_cast<float2*>(dst);
        for (int t = tid; t < FH * FW; t += FT_THREADS) {
            const int r = t / FW, c = t - r * FW;
            d2[r * a.FWmax + c] = s2[t];
        }
    }
}

// One tile of references (tile index t = ty * ntx + tx); smem: f_layout(...).total bytes
// (f_layout_fwd for the forward mode).
template <int K, int C, typename Tin, int MODE>
__device__ __forceinline__ void filter_tile(const FilterArgs& a, const int tile, unsigned char* smem) {
    if constexpr (MODE == FM_FORWARD || MODE == FM_VIDEO) {
        filter_tile_fwd<K, C, Tin, MODE == FM_VIDEO>(a, tile, smem);
        return;
    }
    if constexpr (MODE == FM_ANALYZE || MODE == FM_SYNTH) {
        filter_tile_fwd<K, C, Tin, false, MODE == FM_ANALYZE ? 1 : 2>(a, tile, smem);
        return;
    }
    using G = FCfg<C>;
    constexpr int NF = G::PATCH;                 // fibres
    constexpr int NBW = K * NF / 32;             // bitmap words per group
    // lanes that run the per-patch stages (threads 0 .. 8K-1; K = 2 fills half a warp)
    constexpr unsigned kAB = (8 * K >= 32) ? 0xffffffffu : ((1u << (8 * K)) - 1u);
    const Geo& g = a.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
    int FY0, FY1, FX0, FX1;
    tile_span(ty, a.TR, g.nry, g.s, g.H, g.npy, g.wny, g.win, FY0, FY1);
    tile_span(tx, a.TR, g.nrx, g.s, g.W, g.npx, g.wnx, g.win, FX0, FX1);
    const int FH = FY1 - FY0, FW = FX1 - FX0;
    const FLayout L = f_layout<K, C>(a.FHmax, a.FWmax, (int)sizeof(Tin), MODE);
    float* bas = reinterpret_cast<float*>(smem + L.off_bas);
    float* gb = reinterpret_cast<float*>(smem + L.off_gb);
    int* pos = reinterpret_cast<int*>(smem + L.off_pos);
    uint32_t* band = reinterpret_cast<uint32_t*>(smem + L.off_band);
    uint32_t* rkeep = reinterpret_cast<uint32_t*>(smem + L.off_rkeep);
    int* misc = reinterpret_cast<int*>(smem + L.off_misc);
    float* acc = reinterpret_cast<float*>(smem + L.off_acc);
    Tin* img_s = reinterpret_cast<Tin*>(smem + L.off_img);
    float* r_s = reinterpret_cast<float*>(smem + L.off_r);

    // Stage the basis, the image footprint and clear the accumulator.
    if constexpr (MODE != FM_DENOM) {
        stage_basis<C>(a.basis32, bas, tid);
        const Tin* img = reinterpret_cast<const Tin*>(a.img);
        const int rowb = FW * C;
        for (int t = tid; t < FH * rowb; t += FT_THREADS) {
            const int r = t / rowb, cb = t - r * rowb;
            img_s[t] = img[((size_t)(FY0 + r) * g.W + FX0) * C + cb];
        }
        if constexpr (MODE == FM_ADJOINT) {
            for (int t = tid; t < FH * rowb; t += FT_THREADS) {
                const int r = t / rowb, cb = t - r * rowb;
                r_s[t] = a.r_img[((size_t)(FY0 + r) * g.W + FX0) * C + cb];
            }
        }
    }
    for (int t = tid; t < FH * FW * G::ACC; t += FT_THREADS) acc[t] = 0.f;

    const int iy0 = ty * a.TR, ix0 = tx * a.TR;
    const int th = min(a.TR, g.nry - iy0), tw = min(a.TR, g.nrx - ix0);
    for (int q = 0; q < th * tw; ++q) {
        const int grp = (iy0 + q / tw) * g.nrx + ix0 + q % tw;
        __syncthreads();
        if (tid < K) {
            // Positions come from the grouping of this geometry and lie in the footprint; a caller-given
            // index outside it is clamped so that no access leaves the staged region.
            const int v = a.idx[(size_t)grp * K + tid];
            const int y = v / g.W, x = v - y * g.W;
            pos[2 * tid] = min(max(y - FY0, 0), FH - PS);
            pos[2 * tid + 1] = min(max(x - FX0, 0), FW - PS);
        }
        if (tid < NBW) {
            band[tid] = 0u;
            rkeep[tid] = 0u;
        }
        if (tid < 16) misc[tid] = 0;
        __syncthreads();

        float wg = 1.f;
        float cx[K];          // FM_ADJOINT: coefficients at x of this thread's fibre
        uint32_t keepb = 0;
        if constexpr (MODE != FM_DENOM) {
            // ---- A, B on the filtered image
            // A and B of patch k run on threads 8k..8k+7 of one warp (one column or row per thread;
            // the two-wide forms spill here, where the x coefficients stay live): a warp barrier
            // orders them.
            if (tid < 8 * K) {
                const float nrm = stage_a<K, C, Tin>(img_s, FW, pos, bas, gb, tid >> 3, tid & 7);
                // ||G||_F^2: a warp sum first (exact in int for uint8 inputs), one shared atomic per warp
                if constexpr (sizeof(Tin) == 1) {
                    const int wsum = __reduce_add_sync(kAB, (int)nrm);
                    if (lane == 0) atomicAdd(&misc[5], wsum);
                } else {
                    float v = nrm;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kAB, v, off);
                    if (lane == 0) atomicAdd(reinterpret_cast<float*>(&misc[2]), v);
                }
                __syncwarp(kAB);
                stage_b<C>(bas, gb, tid >> 3, tid & 7);
            }
            __syncthreads();
            // ---- C1: Haar analysis and FP32 decisions with a guard band
            const float nrm2 = sizeof(Tin) == 1 ? (float)misc[5] : __int_as_float(misc[2]);
            const float delta = a.band_rel * sqrtf(nrm2) + a.band_abs;
            float co[K];          // fibre, then its coefficients in place (haar_for_each slots)
            uint32_t bandb = 0;
            // fibre tid = (i*8 + j)*C + c lives at row i, column offset j*C + c of every patch
            const int foff = (tid / G::RWF) * G::ROW + (tid % G::RWF);
            if (tid < NF) {
#pragma unroll
                for (int k = 0; k < K; ++k) co[k] = gb[k * G::GS + foff];
                haar_fwd_inplace<K>(co);
                haar_for_each<K>([&](int m, int sl, int) {
                    const float d = fabsf(co[sl]) - a.tau32;
                    if (fabsf(d) <= delta) bandb |= 1u << m;
                    else if (d >= 0.f) keepb |= 1u << m;
                });
                if (bandb) {
                    atomicAdd(&misc[0], __popc(bandb));
#pragma unroll
                    for (int m = 0; m < K; ++m)
                        if ((bandb >> m) & 1u) atomicOr(&band[(m * NF + tid) >> 5], 1u << (tid & 31));
                }
            }
            __syncthreads();
            // ---- FP64 decisions inside the band (rare)
            if (misc[0] > 0) {
                for (int wi = warp; wi < NBW; wi += FT_THREADS / 32) {
                    uint32_t word = band[wi];
                    while (word) {
                        const int bit = __ffs(word) - 1;
                        word &= word - 1;
                        const int ent = wi * 32 + bit;
                        const int m = ent / NF, e = ent - m * NF;
                        const bool keep = refine_keep<K, C, Tin>(m, e, img_s, FW, pos, a.basis64, a.tau64, lane);
                        if (lane == 0 && keep) atomicOr(&rkeep[wi], 1u << bit);
                    }
                }
                __syncthreads();
            }
            if (tid < NF) {
#pragma unroll
                for (int m = 0; m < K; ++m)
                    if ((bandb >> m) & 1u)
                        if ((rkeep[(m * NF + tid) >> 5] >> (tid & 31)) & 1u) keepb |= 1u << m;
                // (the forward mode runs in filter_tile_fwd; here only the adjoint keeps the
                // kept coefficients at x, for the weight gradient)
                haar_for_each<K>([&](int m, int sl, int) { cx[sl] = ((keepb >> m) & 1u) ? co[sl] : 0.f; });
            }
            __syncthreads();
            if constexpr (MODE == FM_ADJOINT) {
                // ---- second pass on r = gout / D with the masks of x
                if (tid < 8 * K) {
                    stage_a<K, C, float>(r_s, FW, pos, bas, gb, tid >> 3, tid & 7);
                    __syncwarp(kAB);
                    stage_b<C>(bas, gb, tid >> 3, tid & 7);
                    // <Gather(r), Gather(out)> for the weight gradient
                    const int k = tid >> 3, b = tid & 7;
                    const float* rp = r_s + (pos[2 * k] * FW + pos[2 * k + 1] + b) * C;
                    const int gy = pos[2 * k] + FY0, gx = pos[2 * k + 1] + FX0 + b;
                    float dot = 0.f;
#pragma unroll
                    for (int i = 0; i < PS; ++i)
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            dot = fmaf(rp[i * FW * C + c], a.out_img[((size_t)(gy + i) * g.W + gx) * C + c], dot);
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(kAB, dot, off);
                    if (lane == 0) atomicAdd(reinterpret_cast<float*>(&misc[4]), dot);
                }
                __syncthreads();
                if (tid < NF) {
                    float cr[K];      // fibre of the r pass, then its coefficients in place
#pragma unroll
                    for (int k = 0; k < K; ++k) cr[k] = gb[k * G::GS + foff];
                    haar_fwd_inplace<K>(cr);
                    float dot = 0.f;
                    haar_for_each<K>([&](int m, int sl, int) {
                        if (!((keepb >> m) & 1u)) cr[sl] = 0.f;
                        dot = fmaf(cr[sl], cx[sl], dot);
                    });
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
                    if (lane == 0) atomicAdd(reinterpret_cast<float*>(&misc[3]), dot);
                    haar_inv_inplace<K>(cr);
#pragma unroll
                    for (int k = 0; k < K; ++k) gb[k * G::GS + foff] = cr[k];
                }
                __syncthreads();
            }
            // ---- D, E: inverse projection (patch k on threads 8k..8k+7 of one warp)
            if (tid < 8 * K) {
                stage_d<C>(bas, gb, tid >> 3, tid & 7);
                __syncwarp(kAB);
                stage_e<C>(bas, gb, tid >> 3, tid & 7);
            }
        }
        // ---- weight of the group
        if (a.w_in) wg = a.w_in[grp];
        else if (MODE == FM_FORWARD && a.agg_mode == 1) wg = 1.f / (float)max(1, misc[1]);
        if (tid == 0) {
            if (MODE == FM_FORWARD && a.weights_out) a.weights_out[grp] = wg;
            if (MODE == FM_ADJOINT && a.grad_w)
                a.grad_w[grp] = __int_as_float(misc[3]) - __int_as_float(misc[4]);
        }
        __syncthreads();
        // ---- F: aggregation, warp `warp` owns footprint rows r with r % 8 == warp
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            const int py = pos[2 * k], px = pos[2 * k + 1];
            const int i = (warp - py) & 7;
            const int row = py + i;
            float* ap = acc + (row * FW + px) * G::ACC;
            if constexpr (C == 3) {
                if (lane < 24) {
                    if constexpr (MODE != FM_DENOM) {
                        const int j = lane / 3, c = lane - 3 * (lane / 3);
                        ap[j * 4 + c] += wg * gb[k * G::GS + i * G::ROW + lane];
                    }
                } else if (MODE != FM_ADJOINT) {
                    ap[(lane - 24) * 4 + 3] += wg;
                }
            } else {
                if (lane < 8) {
                    if constexpr (MODE != FM_DENOM) ap[lane * 2] += wg * gb[k * G::GS + i * G::ROW + lane];
                } else if (lane < 16 && MODE != FM_ADJOINT) {
                    ap[(lane - 8) * 2 + 1] += wg;
                }
            }
        }
    }
    __syncthreads();
    // Write the tile partial.
    float* dst = a.partials + (size_t)tile * a.FHmax * a.FWmax * G::ACC;
    if constexpr (C == 3) {
        const float4* s4 = reinterpret_cast<const float4*>(acc);
        float4* d4 = reinterpret_cast<float4*>(dst);
        for (int t = tid; t < FH * FW; t += FT_THREADS) {
            const int r = t / FW, c = t - r * FW;
            d4[r * a.FWmax + c] = s4[t];
        }
    } else {
        const float2* s2 = reinterpret_cast<const float2*>(acc);
        float2* d2 = reinterpret_cast<float2*>(dst);
        for (int t = tid; t < FH * FW; t += FT_THREADS) {
            const int r = t / FW, c = t - r * FW;
            d2[r * a.FWmax + c] = s2[t];
        }
    }
}

template <int K, int C, typename Tin, int MODE>
__global__ void __launch_bounds__(FT_THREADS, 2) filter_kernel(FilterArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    filter_tile<K, C, Tin, MODE>(a, blockIdx.x, smem);
}

// Persistent form over the tiles of many images (same K and C): work item w -> image by prefix[].
template <int K, int C>
__global__ void __launch_bounds__(FT_THREADS, 2) filter_batch_kernel(const FilterArgs* __restrict__ args,
                                                                     const int* __restrict__ prefix, int nimg,
                                                                     int* __restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int item;
    const int total = prefix[nimg];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(counter, 1);
        __syncthreads();
        const int w = item;
        if (w >= total) break;
        int lo = 0, hi = nimg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        filter_tile<K, C, uint8_t, FM_FORWARD>(args[lo], w - prefix[lo], smem);
    }
}

template <int K, int C, typename Tin, int MODE>
cudaError_t launch_filter_t(const FilterArgs& a, cudaStream_t s) {
    const FLayout L = (MODE == FM_FORWARD || MODE == FM_ANALYZE || MODE == FM_SYNTH)
                          ? f_layout_fwd<K, C>(a.FHmax, a.FWmax, (int)sizeof(Tin))
                      : MODE == FM_VIDEO ? f_layout_fwd<K, C>(a.FHmax, a.FWmax, (int)sizeof(Tin), a.nfr)
                                         : f_layout<K, C>(a.FHmax, a.FWmax, (int)sizeof(Tin), MODE);
    auto fn = filter_kernel<K, C, Tin, MODE>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    fn<<<a.ntx * a.nty, FT_THREADS, L.total, s>>>(a);
    return cudaGetLastError();
}

}  // namespace htsvd

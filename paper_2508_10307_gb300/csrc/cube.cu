// Alg. 1 on hyperspectral cubes (Sec. III-E, extension to other imaging; Sec. IV, real-world HSI
// denoising): a patch is a ps x ps x N tube and the t-SVD runs along the band mode, with N Fourier
// slices instead of the three of an RGB image.
//
// The group tensor of a cube (K x 64 x N floats: 254 KB at K = 32, N = 31) does not fit a CTA's
// shared memory, so the filter runs over the group one Haar slot at a time. The Haar transform
// along the group mode and the per-patch t-SVD projection commute, so each slot is formed directly
// from the uint8 patches in its Haar support (exact integer sums and differences), projected
//   band DFT -> per slice f: U_f^H X_f V_f -> inverse band DFT,
// thresholded (FP32; FP64 inside a guard band proportional to the slot's own norm), and, if it keeps a
// coefficient, inverted on the kept basis rows only; the 8 x 8 x N spatial slot goes to a per-CTA
// scratch in global memory that stays in L2 (K slots per CTA; slots without a kept coefficient are
// neither written nor read). After the last slot the CTA runs the Haar synthesis per fibre from
// that scratch and adds every estimated patch into the numerator and denominator planes with float
// atomics (the per-CTA footprint accumulator of the image filter would need (W + 7)^2 x (N + 1)
// floats). The summation order of the atomics varies between runs, so outputs agree to rounding,
// not bit for bit.
//
// Layout and arithmetic per slot (C bands, nf = C/2 + 1 Fourier slices of the real band axis):
//   raw slot, folded over the band axis: s_c = x_c + x_{C-c}, d_c = x_c - x_{C-c} (0 < c < C/2),
//     s_c = x_c, d_c = 0 otherwise; exact integers;
//   band DFT: Re X_f = sum_c s_c cos(2 pi f c / C), Im X_f = -sum_c d_c sin(2 pi f c / C), f < nf
//     (half the multiply-adds of the direct sum; the slices f > C/2 are the conjugates);
//   projection per slice and basis row i (one thread): Y_f[i][:] = sum_a conj(U_f[a][i]) X_f[a][:],
//     S_f[i][:] = Y_f[i][:] V_f, stored times w_f / C (w_f = 2 for the slices that stand for a
//     conjugate pair, 1 for f = 0 and f = C/2);
//   inverse band DFT: x_c = A_c + B_c, x_{C-c} = A_c - B_c with A_c = sum_f Re S_f cos(2 pi f c / C)
//     and B_c = -sum_f Im S_f sin(2 pi f c / C).
// Both DFTs are register tiles (2 pixels x 4 frequencies or bands) over a cos table and a -sin
// table that serve both directions (the tables are symmetric in f and c). Rows of 64 pixels are
// RS = 68 floats apart, so that the four slices a warp touches at once fall in different banks.
#include <type_traits>

#include "filter_impl.cuh"

namespace htsvd {

namespace {

constexpr int CB_MAX_THREADS = 256;
// Threads of a CTA: one per DFT tile (2 pixels x 4 frequencies), 32 per frequency quad, within
// [128, 256]: every thread has work in the transform phases, and up to 128 registers each.
__host__ __device__ inline int cube_threads(int C) {
    const int n = 32 * ((C / 2 + 1 + 3) / 4);
    return n < 128 ? 128 : (n > CB_MAX_THREADS ? CB_MAX_THREADS : n);
}
constexpr int RS = 68;       // floats per 64-pixel row (16-byte aligned; consecutive rows 4 banks apart)
constexpr int BS = 136;      // floats per basis block [re, im][a][i] of one (U or V, f) (8 banks apart)
constexpr int NL = 32;       // slots keeping at most NL coefficients take the sparse inverse
constexpr int NB = 16;       // guard-band coefficients decided one at a time by the whole CTA

struct CubeLayout {
    int nf, nfp;                                                  // C/2 + 1 and that rounded up to 4
    int bas, tc, ts, tw64, R, P, Q, stk, lst, blist, red, base, misc, total;   // byte offsets
};
__host__ __device__ inline int log2_of(int K) {
    int l = 0;
    while ((2 << l) <= K) ++l;
    return l;
}
__host__ __device__ inline CubeLayout cube_layout(int C, int K) {
    CubeLayout L;
    L.nf = C / 2 + 1;
    L.nfp = (L.nf + 3) & ~3;
    int o = 0;
    L.bas = o; o += 4 * (2 * L.nf * BS);           // U, V slices f = 0 .. C/2
    L.tc = o; o += 4 * (L.nf * L.nfp);             // cos(2 pi f c / C), [c][f] = [f][c], zero padded
    L.ts = o; o += 4 * (L.nf * L.nfp);             // -sin(2 pi f c / C)
    o = (o + 7) & ~7;
    L.tw64 = o; o += 8 * (2 * C);                   // cos, sin of 2 pi k / C in FP64 (guard band)
    L.R = o; o += 4 * (2 * L.nf * RS);              // folded raw slot s | d; later the spatial slot [c][p]
    L.P = o; o += 4 * (2 * L.nf * RS);              // Fourier slices Re | Im, or folded coefficients
    L.Q = o; o += 4 * (2 * L.nf * RS);
    L.stk = o; o += 4 * (log2_of(K) * L.nf * PS2);  // pending Haar-tree sums, two 16-bit bands per word
    L.lst = o; o += 16 * NL;                        // kept coefficients of a sparse slot: pixel, band, value
    L.blist = o; o += 16 * NB;                      // coefficients inside the guard band: pixel, band, value
    L.red = o; o += 8 * (CB_MAX_THREADS / 32);      // cross-warp sums
    L.base = o; o += 4 * K;                         // pixel index of each patch's corner
    L.misc = o; o += 4 * 16;
    L.total = o;
    return L;
}

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ float comp(const float4& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Haar rows as nodes of a binary tree over the K patches (heap order): row m >= 1 at level
// l = floor(log2 m) has support [k0, k0 + L), L = K >> l, k0 = (m - 2^l) L, and is the sum over its
// first half minus the sum over its second half, i.e. the difference of its children's sums; row 0
// is the sum over all K. Slot sl is where the unnormalised in-place transform stores row m (as
// haar_for_each).
template <int K>
__device__ __forceinline__ void haar_node(int m, int& k0, int& L, int& sl) {
    if (m == 0) {
        k0 = 0; L = K; sl = 0;
        return;
    }
    const int l = 31 - __clz(m), mm = m - (1 << l);
    L = K >> l;
    k0 = mm * L;
    sl = (2 * mm + 1) * (K >> (l + 1));
}
// Rows in post order (children before their parent), then row 0: every child's sum is pushed on a
// stack and its parent pops the two, so each patch is read once per group. First row: K/2.
template <int K>
__device__ __forceinline__ int haar_next(int m) {
    if (m == 1) return 0;
    if (m & 1) return m >> 1;                       // a right child: its parent is next
    m += 1;                                          // a left child: the leftmost lowest row under its sibling
    while (m < K / 2) m <<= 1;
    return m;
}

// TP consecutive floats of a shared-memory row (TP = 2 or 4, 8- or 16-byte aligned).
template <int TP>
__device__ __forceinline__ void ldv(const float* p, float (&r)[TP]) {
    if constexpr (TP == 4) {
        const float4 v = ld4(p);
        r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
    } else {
        const float2 v = *reinterpret_cast<const float2*>(p);
        r[0] = v.x; r[1] = v.y;
    }
}
template <int TP>
__device__ __forceinline__ void stv(float* p, const float (&r)[TP]) {
    if constexpr (TP == 4) *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
    else *reinterpret_cast<float2*>(p) = make_float2(r[0], r[1]);
}

// The DFT tiles: TP pixels x 4 frequencies (or bands); 64 / TP tiles per frequency quad, a warp
// covering one quad when TP = 2.
constexpr int TP = 2;
constexpr int NPT = PS2 / TP;                 // pixel tiles

// Band DFT of a folded real slot: src rows [0, nf) s_c, [nf, 2 nf) d_c; dst rows [0, nf) Re X_f,
// [nf, 2 nf) Im X_f.
__device__ __forceinline__ void band_dft(const float* __restrict__ src, float* __restrict__ dst,
                                         const float* tc, const float* ts, int nf, int nfp, int tid, int nthr) {
    for (int t = tid; t < NPT * (nfp >> 2); t += nthr) {
        const int p0 = (t % NPT) * TP, f0 = (t / NPT) << 2;
        float re[4][TP], im[4][TP];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < TP; ++j) re[i][j] = im[i][j] = 0.f;
#pragma unroll 2
        for (int c = 0; c < nf; ++c) {
            float s[TP], d[TP];
            ldv<TP>(src + c * RS + p0, s);
            ldv<TP>(src + (nf + c) * RS + p0, d);
            const float4 wc = ld4(tc + c * nfp + f0), ws = ld4(ts + c * nfp + f0);
#pragma unroll
            for (int fi = 0; fi < 4; ++fi)
#pragma unroll
                for (int pi = 0; pi < TP; ++pi) {
                    re[fi][pi] = fmaf(s[pi], comp(wc, fi), re[fi][pi]);
                    im[fi][pi] = fmaf(d[pi], comp(ws, fi), im[fi][pi]);
                }
        }
#pragma unroll
        for (int fi = 0; fi < 4; ++fi)
            if (f0 + fi < nf) {
                stv<TP>(dst + (f0 + fi) * RS + p0, re[fi]);
                stv<TP>(dst + (nf + f0 + fi) * RS + p0, im[fi]);
            }
    }
}

// Band DFT of an unfolded real slot (src rows c = 0 .. C-1, band c), folded on load; dst as band_dft.
__device__ __forceinline__ void band_dft_unfolded(const float* __restrict__ src, float* __restrict__ dst,
                                                  const float* tc, const float* ts, int C, int nf, int nfp, int tid,
                                                  int nthr) {
    for (int t = tid; t < NPT * (nfp >> 2); t += nthr) {
        const int p0 = (t % NPT) * TP, f0 = (t / NPT) << 2;
        float re[4][TP], im[4][TP];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < TP; ++j) re[i][j] = im[i][j] = 0.f;
        for (int c = 0; c < nf; ++c) {
            float s[TP], d[TP];
            ldv<TP>(src + c * RS + p0, s);
            if (c > 0 && 2 * c < C) {
                float y[TP];
                ldv<TP>(src + (C - c) * RS + p0, y);
#pragma unroll
                for (int pi = 0; pi < TP; ++pi) {
                    d[pi] = s[pi] - y[pi];
                    s[pi] += y[pi];
                }
            } else {
#pragma unroll
                for (int pi = 0; pi < TP; ++pi) d[pi] = 0.f;
            }
            const float4 wc = ld4(tc + c * nfp + f0), ws = ld4(ts + c * nfp + f0);
#pragma unroll
            for (int fi = 0; fi < 4; ++fi)
#pragma unroll
                for (int pi = 0; pi < TP; ++pi) {
                    re[fi][pi] = fmaf(s[pi], comp(wc, fi), re[fi][pi]);
                    im[fi][pi] = fmaf(d[pi], comp(ws, fi), im[fi][pi]);
                }
        }
#pragma unroll
        for (int fi = 0; fi < 4; ++fi)
            if (f0 + fi < nf) {
                stv<TP>(dst + (f0 + fi) * RS + p0, re[fi]);
                stv<TP>(dst + (nf + f0 + fi) * RS + p0, im[fi]);
            }
    }
}

// One tile of the inverse band DFT of slices stored times w_f / C (src rows Re | Im):
// A[ci][pi] = sum_f Re S_f cos(2 pi f c / C), B[ci][pi] = -sum_f Im S_f sin(2 pi f c / C) at band
// c = c0 + ci and pixel p0 + pi; x_c = A + B and x_{C-c} = A - B.
__device__ __forceinline__ void idft_tile(const float* __restrict__ src, const float* tc, const float* ts, int nf,
                                          int nfp, int p0, int c0, float (&A)[4][TP], float (&B)[4][TP]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TP; ++j) A[i][j] = B[i][j] = 0.f;
#pragma unroll 2
    for (int f = 0; f < nf; ++f) {
        float qr[TP], qi[TP];
        ldv<TP>(src + f * RS + p0, qr);
        ldv<TP>(src + (nf + f) * RS + p0, qi);
        const float4 wc = ld4(tc + f * nfp + c0), ws = ld4(ts + f * nfp + c0);
#pragma unroll
        for (int ci = 0; ci < 4; ++ci)
#pragma unroll
            for (int pi = 0; pi < TP; ++pi) {
                A[ci][pi] = fmaf(qr[pi], comp(wc, ci), A[ci][pi]);
                B[ci][pi] = fmaf(qi[pi], comp(ws, ci), B[ci][pi]);
            }
    }
}

// The same value summed over the whole CTA (every thread calls it with the same (pb, cb) and gets
// the result): thread t takes the (slice, pixel) pairs t, t + nthr, ...; red holds nthr / 32 doubles.
__device__ double coef64_cta(const float* R, const double* t64c, const double* t64s, const double* __restrict__ b64,
                             int C, int nf, int pb, int cb, int tid, int nthr, double* red) {
    const int ib = pb >> 3, jb = pb & 7;
    double acc = 0.0;
    for (int it = tid; it < nf * PS2; it += nthr) {
        const int f = it >> 6, q = it & 63, qa = q >> 3, qb = q & 7;
        double xre = 0.0, xim = 0.0;
        for (int c = 0, k = 0; c < nf; ++c, k = (k + f >= C) ? k + f - C : k + f) {
            xre = fma((double)R[c * RS + q], t64c[k], xre);
            xim = fma(-(double)R[(nf + c) * RS + q], t64s[k], xim);
        }
        const double* u = b64 + 2 * (((size_t)0 * C + f) * PS2 + qa * PS + ib);
        const double* vv = b64 + 2 * (((size_t)1 * C + f) * PS2 + qb * PS + jb);
        const double cr = u[0] * vv[0] + u[1] * vv[1];          // conj(u) v
        const double ci = u[0] * vv[1] - u[1] * vv[0];
        const double pr = cr * xre - ci * xim, pi = cr * xim + ci * xre;
        const int k2 = (f * cb) % C;
        const double wgt = (f == 0 || 2 * f == C) ? 1.0 : 2.0;
        acc += wgt * (t64c[k2] * pr - t64s[k2] * pi);              // Re(w^{-f cb} P_f) terms
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (nthr >> 5); ++w) tot += red[w];
    __syncthreads();
    return tot / (double)C;
}

// Inverse band DFT to a spatial slot in shared memory, [pixel][band] (the layout of the synthesis):
// x_c to dst[p C + c], x_{C-c} to dst[p C + C - c].
__device__ __forceinline__ void band_idft_pc(const float* __restrict__ src, float* __restrict__ dst,
                                             const float* tc, const float* ts, int C, int nf, int nfp, int tid,
                                             int nthr) {
    for (int t = tid; t < NPT * (nfp >> 2); t += nthr) {
        const int p0 = (t % NPT) * TP, c0 = (t / NPT) << 2;
        float A[4][TP], B[4][TP];
        idft_tile(src, tc, ts, nf, nfp, p0, c0, A, B);
#pragma unroll
        for (int ci = 0; ci < 4; ++ci) {
            const int c = c0 + ci;
#pragma unroll
            for (int pi = 0; pi < TP; ++pi) {
                float* o = dst + (p0 + pi) * C;
                if (c < nf) o[c] = A[ci][pi] + B[ci][pi];
                if (c > 0 && 2 * c < C) o[C - c] = A[ci][pi] - B[ci][pi];
            }
        }
    }
}

// FP64 value of the coefficient at pixel pb, band cb of a slot whose folded raw values (exact
// integers) are in R: P_f = sum_{pixels (a, b)} conj(U_f[a][ib]) V_f[b][jb] X_f[a][b] with X_f the
// band DFT, and S = (1/C) sum_{f <= C/2} w_f Re(w^{-f cb} P_f). Every lane of the warp calls it with
// the same (pb, cb); lane l takes pixels l and l + 32.
__device__ __noinline__ double coef64(const float* R, const double* t64c, const double* t64s,
                                      const double* __restrict__ b64, int C, int nf, int pb, int cb, int lane) {
    const int ib = pb >> 3, jb = pb & 7;
    double acc = 0.0;
    for (int f = 0; f < nf; ++f) {
        double pr = 0.0, pi = 0.0;
        for (int q = lane; q < PS2; q += 32) {
            const int qa = q >> 3, qb = q & 7;
            double xre = 0.0, xim = 0.0;
            for (int c = 0, k = 0; c < nf; ++c, k = (k + f >= C) ? k + f - C : k + f) {
                xre = fma((double)R[c * RS + q], t64c[k], xre);
                xim = fma(-(double)R[(nf + c) * RS + q], t64s[k], xim);
            }
            const double* u = b64 + 2 * (((size_t)0 * C + f) * PS2 + qa * PS + ib);
            const double* vv = b64 + 2 * (((size_t)1 * C + f) * PS2 + qb * PS + jb);
            const double cr = u[0] * vv[0] + u[1] * vv[1];      // conj(u) v
            const double ci = u[0] * vv[1] - u[1] * vv[0];
            pr += cr * xre - ci * xim;
            pi += cr * xim + ci * xre;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            pr += __shfl_xor_sync(0xffffffffu, pr, off);
            pi += __shfl_xor_sync(0xffffffffu, pi, off);
        }
        const int k2 = (f * cb) % C;
        const double wgt = (f == 0 || 2 * f == C) ? 1.0 : 2.0;
        acc += wgt * (t64c[k2] * pr - t64s[k2] * pi);          // Re(w^{-f cb} P_f)
    }
    return acc / (double)C;
}

__device__ __forceinline__ void load8s(const float* p, float (&r)[8]) {
    const float4 a = ld4(p), b = ld4(p + 4);
    r[0] = a.x; r[1] = a.y; r[2] = a.z; r[3] = a.w;
    r[4] = b.x; r[5] = b.y; r[6] = b.z; r[7] = b.w;
}
__device__ __forceinline__ void store8s(float* p, const float (&r)[8], float sc) {
    st4(p, r[0] * sc, r[1] * sc, r[2] * sc, r[3] * sc);
    st4(p + 4, r[4] * sc, r[5] * sc, r[6] * sc, r[7] * sc);
}

template <int K>
__global__ void __launch_bounds__(CB_MAX_THREADS, 2) cube_filter_kernel(CubeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Geo& g = a.g;
    const int C = g.C, NE = PS2 * C;
    const CubeLayout Ly = cube_layout(C, K);
    const int nf = Ly.nf, nfp = Ly.nfp, NI = nf * PS2;
    float* bas = reinterpret_cast<float*>(smem + Ly.bas);
    float* tc = reinterpret_cast<float*>(smem + Ly.tc);
    float* ts = reinterpret_cast<float*>(smem + Ly.ts);
    double* t64c = reinterpret_cast<double*>(smem + Ly.tw64);
    double* t64s = t64c + C;
    float* R = reinterpret_cast<float*>(smem + Ly.R);
    float* P = reinterpret_cast<float*>(smem + Ly.P);
    float* Q = reinterpret_cast<float*>(smem + Ly.Q);
    unsigned* stk = reinterpret_cast<unsigned*>(smem + Ly.stk);
    int4* lst = reinterpret_cast<int4*>(smem + Ly.lst);
    int4* blist = reinterpret_cast<int4*>(smem + Ly.blist);
    double* red = reinterpret_cast<double*>(smem + Ly.red);
    int* base = reinterpret_cast<int*>(smem + Ly.base);
    int* misc = reinterpret_cast<int*>(smem + Ly.misc);      // 0 kept in group, 1 kept in slot, 2 row mask,
                                                              // 3 slots holding a kept coefficient, 7 kept listed,
                                                              // 8 the slot has band coefficients, 9 listed,
                                                              // 5, 6 squared slot norms (float, by step parity)
    const int tid = threadIdx.x, lane = tid & 31, nthr = blockDim.x;
    float* scratch = a.scratch + (size_t)blockIdx.x * K * NE;
    const uint8_t* img = a.img;
    const int nbw = (K * NE + 31) / 32;
    // t / nf and t / C as a high multiply (exact for t < 2^16 and divisors up to 64)
    const unsigned mg_nf = 0xffffffffu / (unsigned)nf + 1u, mg_c = 0xffffffffu / (unsigned)C + 1u;

    // the basis, global [U | V][f][re, im][a][i] (128 floats per block) to BS floats per block
    for (int t = tid; t < 2 * nf * 128; t += nthr) bas[(t >> 7) * BS + (t & 127)] = a.basis32[t];
    for (int t = tid; t < nf * nfp; t += nthr) {
        const int r = t / nfp, f = t - r * nfp;
        float sn = 0.f, cs = 0.f;
        if (f < nf) sincospif(2.f * (float)((r * f) % C) / (float)C, &sn, &cs);
        tc[t] = cs;
        ts[t] = -sn;
    }
    for (int t = tid; t < C; t += nthr) {
        double sd, cd;
        sincospi(2.0 * t / C, &sd, &cd);
        t64c[t] = cd;
        t64s[t] = sd;
    }

    for (int grp = blockIdx.x; grp < g.ngroups(); grp += gridDim.x) {
        __syncthreads();
        if (tid < K) {
            // a caller-given index outside the image is clamped so that no access leaves it
            const int v = a.idx[(size_t)grp * K + tid];
            const int y = v / g.W, x = v - y * g.W;
            base[tid] = min(max(y, 0), g.H - PS) * g.W + min(max(x, 0), g.W - PS);
        }
        if (tid < 16) misc[tid] = 0;
        if (a.mask_out)
            for (int t = tid; t < nbw; t += nthr) a.mask_out[(size_t)grp * nbw + t] = 0u;
        __syncthreads();
        int sp = 0;
        for (int step = 0, m = K / 2; step < K; ++step, m = haar_next<K>(m)) {
            int k0, L, sl;
            haar_node<K>(m, k0, L, sl);
            const bool lowest = m != 0 && L == 2;
            const int sp_in = sp;
            sp += lowest ? 1 : -1;
            // raw slot, folded (s | d rows of R), from the children's sums (popped) or, on the lowest
            // level, from the two patches; the row's own sum is pushed. Sums of uint8 values over at
            // most K = 32 patches fit 16 bits, so a word holds the two bands c and C - c and one
            // 32-bit addition adds both.
            float nq = 0.f;
            // the lowest rows read patches k0 and k0 + 1 (b1 bytes after k0; negative if it lies above)
            const uint8_t* img0 = img + (lowest ? (size_t)base[k0] * C : 0);
            const int b1 = lowest ? (base[k0 + 1] - base[k0]) * C : 0;
            auto emit = [&](int t, unsigned lft, unsigned rgt) {
                const int p = __umulhi((unsigned)t, mg_nf), c = t - p * nf;
                const bool paired = c > 0 && 2 * c < C;
                const int s1 = (int)(lft & 0xffffu) - (int)(rgt & 0xffffu);
                const int s2 = paired ? (int)(lft >> 16) - (int)(rgt >> 16) : 0;
                R[c * RS + p] = (float)(s1 + s2);
                R[(nf + c) * RS + p] = (float)(s1 - s2) * (paired ? 1.f : 0.f);
                nq = fmaf((float)s1, (float)s1, fmaf((float)s2, (float)s2, nq));
            };
            if (lowest) {
                // four items' bytes are requested before any is used (the patches come from L2)
                constexpr int U = 4;
                for (int t0 = tid; t0 < NI; t0 += U * nthr) {
                    unsigned lft[U], rgt[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int t = t0 + u * nthr;
                        lft[u] = rgt[u] = 0u;
                        if (t < NI) {
                            const int p = __umulhi((unsigned)t, mg_nf), c = t - p * nf;
                            const uint8_t* i1 = img0 + ((p >> 3) * g.W + (p & 7)) * C + c;
                            const int o2 = (c > 0 && 2 * c < C) ? C - 2 * c : 0;
                            lft[u] = (unsigned)i1[0] | ((unsigned)i1[o2] << 16);
                            rgt[u] = (unsigned)i1[b1] | ((unsigned)i1[b1 + o2] << 16);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int t = t0 + u * nthr;
                        if (t < NI) {
                            stk[sp_in * NI + t] = lft[u] + rgt[u];
                            emit(t, lft[u], rgt[u]);
                        }
                    }
                }
            } else if (m == 0) {
                for (int t = tid; t < NI; t += nthr) emit(t, stk[(sp_in - 1) * NI + t], 0u);
            } else {
                for (int t = tid; t < NI; t += nthr) {
                    const unsigned rgt = stk[(sp_in - 1) * NI + t], lft = stk[(sp_in - 2) * NI + t];
                    stk[(sp_in - 2) * NI + t] = lft + rgt;
                    emit(t, lft, rgt);
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) nq += __shfl_xor_sync(0xffffffffu, nq, off);
            if (tid == 0) { misc[1] = 0; misc[2] = 0; misc[7] = 0; misc[8] = 0; misc[9] = 0; }
            if (lane == 0) atomicAdd(reinterpret_cast<float*>(&misc[5 + (step & 1)]), nq);
            __syncthreads();
            band_dft(R, P, tc, ts, nf, nfp, tid, nthr);
            __syncthreads();
            // S_f[i][:] = (sum_a conj(U_f[a][i]) X_f[a][:]) V_f, one thread per (f, i)
            for (int t = tid; t < nf * PS; t += nthr) {
                const int f = t >> 3, i = t & 7;
                const float* Ub = bas + f * BS;
                const float* Vb = bas + (nf + f) * BS;
                float yr[8], yi[8];
#pragma unroll
                for (int b = 0; b < 8; ++b) yr[b] = yi[b] = 0.f;
#pragma unroll
                for (int a_ = 0; a_ < PS; ++a_) {
                    const float ur = Ub[a_ * 8 + i], ui = Ub[64 + a_ * 8 + i];
                    float xr_[8], xi[8];
                    load8s(P + f * RS + a_ * 8, xr_);
                    load8s(P + (nf + f) * RS + a_ * 8, xi);
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        yr[b] = fmaf(ur, xr_[b], fmaf(ui, xi[b], yr[b]));
                        yi[b] = fmaf(ur, xi[b], fmaf(-ui, xr_[b], yi[b]));
                    }
                }
                float sr[8], si[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) sr[j] = si[j] = 0.f;
#pragma unroll
                for (int b = 0; b < PS; ++b) {
                    float vr[8], vi[8];
                    load8s(Vb + b * 8, vr);
                    load8s(Vb + 64 + b * 8, vi);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        sr[j] = fmaf(yr[b], vr[j], fmaf(-yi[b], vi[j], sr[j]));
                        si[j] = fmaf(yr[b], vi[j], fmaf(yi[b], vr[j], si[j]));
                    }
                }
                const float w = (f == 0 || 2 * f == C ? 1.f : 2.f) / (float)C;
                store8s(Q + f * RS + i * 8, sr, w);
                store8s(Q + (nf + f) * RS + i * 8, si, w);
            }
            __syncthreads();
            // Inverse band DFT with the threshold in its epilogue (the unnormalised slot carries
            // sqrt(L)): a coefficient x is kept when |x| - tau sqrt(L) > band, dropped below -band and
            // decided in FP64 in between (the FP32 error of a slot's coefficients is bounded by a
            // multiple of the slot's own norm, its transform being orthonormal up to the Haar factor,
            // so the band is band_rel x ||slot||_F plus the rounding of tau). Kept values times 1/L,
            // for the unnormalised synthesis, go to row c of P (band c, pixels along the row). The
            // epilogue only flags band coefficients; a slot that has some runs the tiles again and
            // decides them in FP64 (a warp per coefficient).
            {
                const float r = sqrtf((float)L), tl = a.tau32 * r, invL = 1.f / (float)L;
                const float dl = a.band_rel * sqrtf(__int_as_float(misc[5 + (step & 1)])) + a.band_abs * r;
                const int nt = NPT * (nfp >> 2), ntw = (nt + 31) & ~31;
                for (int t = tid; t < ntw; t += nthr) {
                    const bool valid = t < nt;
                    const int p0 = (t % NPT) * TP, c0 = valid ? (t / NPT) << 2 : 0;
                    float A[4][TP], B[4][TP];
                    idft_tile(Q, tc, ts, nf, nfp, p0, c0, A, B);
                    float x[4][TP], y[4][TP];               // kept values times 1/L (band c, band C - c)
                    unsigned km = 0u;                       // which: bit TP ci + pi (c), 4 TP + TP ci + pi (C - c)
                    bool anyband = false;
#pragma unroll
                    for (int ci = 0; ci < 4; ++ci) {
                        const int c = c0 + ci;
                        const bool lo_ok = valid && c < nf, hi_ok = valid && c > 0 && 2 * c < C;
#pragma unroll
                        for (int pi = 0; pi < TP; ++pi) {
                            const float v0 = A[ci][pi] + B[ci][pi], v1 = A[ci][pi] - B[ci][pi];
                            const float d0 = fabsf(v0) - tl, d1 = fabsf(v1) - tl;
                            const bool k0 = d0 > dl, k1 = d1 > dl;
                            anyband |= (lo_ok && fabsf(d0) <= dl) || (hi_ok && fabsf(d1) <= dl);
                            x[ci][pi] = k0 ? v0 * invL : 0.f;
                            y[ci][pi] = k1 ? v1 * invL : 0.f;
                            km |= ((lo_ok && k0) ? 1u : 0u) << (ci * TP + pi);
                            km |= ((hi_ok && k1) ? 1u : 0u) << (4 * TP + ci * TP + pi);
                        }
                        if (lo_ok) stv<TP>(P + c * RS + p0, x[ci]);
                        if (hi_ok) stv<TP>(P + (C - c) * RS + p0, y[ci]);
                    }
                    const int nk = __popc(km);
                    if (nk) {
                        // the kept values, for the sparse inverse (positions past NL are counted only)
                        int at = atomicAdd(&misc[7], nk);
#pragma unroll
                        for (int j = 0; j < 8 * TP; ++j) {
                            if (!((km >> j) & 1u)) continue;
                            const int ci = (j % (4 * TP)) / TP, pi = j % TP, c = c0 + ci;
                            if (at < NL)
                                lst[at] = make_int4(p0 + pi, j >= 4 * TP ? C - c : c,
                                                    __float_as_int(j >= 4 * TP ? y[ci][pi] : x[ci][pi]), 0);
                            ++at;
                        }
                    }
                    const int wk = __reduce_add_sync(0xffffffffu, nk);
                    const unsigned rb = __reduce_or_sync(0xffffffffu, nk ? 1u << (p0 >> 3) : 0u);
                    const bool wb = __any_sync(0xffffffffu, anyband);
                    if (lane == 0) {
                        if (wk) {
                            atomicAdd(&misc[1], wk);
                            atomicOr(&misc[2], (int)rb);
                        }
                        if (wb) misc[8] = 1;
                    }
                }
                if (tid == 0) misc[5 + ((step + 1) & 1)] = 0;   // the next slot's norm accumulator
                __syncthreads();
                if (misc[8] || a.coef_out || a.mask_out) {
                    // the tiles again: list the band coefficients, optional outputs of the FP32 decisions
                    const double tlim = a.tau64 * sqrt((double)L);
                    auto keep_band = [&](int p, int cb, float v) {
                        P[cb * RS + p] = v * invL;
                        atomicAdd(&misc[1], 1);
                        atomicOr(&misc[2], 1 << (p >> 3));
                        const int at = atomicAdd(&misc[7], 1);
                        if (at < NL) lst[at] = make_int4(p, cb, __float_as_int(v * invL), 0);
                        if (a.mask_out) {
                            const size_t bit = (size_t)m * NE + p * C + cb;
                            atomicOr(&a.mask_out[(size_t)grp * nbw + bit / 32], 1u << (bit % 32));
                        }
                    };
                    for (int t = tid; t < nt; t += nthr) {
                        const int p0 = (t % NPT) * TP, c0 = (t / NPT) << 2;
                        float A[4][TP], B[4][TP];
                        idft_tile(Q, tc, ts, nf, nfp, p0, c0, A, B);
#pragma unroll
                        for (int j = 0; j < 8 * TP; ++j) {
                            const int ci = (j % (4 * TP)) / TP, pi = j % TP, c = c0 + ci;
                            const bool hi = j >= 4 * TP;
                            if (!(hi ? (c > 0 && 2 * c < C) : c < nf)) continue;
                            const int cb = hi ? C - c : c, p = p0 + pi;
                            const float v = hi ? A[ci][pi] - B[ci][pi] : A[ci][pi] + B[ci][pi];
                            const float d = fabsf(v) - tl;
                            if (fabsf(d) <= dl) {
                                const int at = atomicAdd(&misc[9], 1);
                                if (at < NB) blist[at] = make_int4(p, cb, __float_as_int(v), 0);
                            }
                            if (a.coef_out) a.coef_out[((size_t)grp * K + m) * NE + p * C + cb] = v / r;
                            if (d > dl && a.mask_out) {
                                const size_t bit = (size_t)m * NE + p * C + cb;
                                atomicOr(&a.mask_out[(size_t)grp * nbw + bit / 32], 1u << (bit % 32));
                            }
                        }
                    }
                    __syncthreads();
                    const int nbl = misc[9];
                    if (nbl <= NB) {
                        // FP64 decisions, each over the whole CTA
                        for (int e = 0; e < nbl; ++e) {
                            const int4 en = blist[e];
                            const double xd = coef64_cta(R, t64c, t64s, a.basis64, C, nf, en.x, en.y, tid, nthr, red);
                            if (tid == 0 && fabs(xd) >= tlim) keep_band(en.x, en.y, __int_as_float(en.z));
                        }
                    } else {
                        // many: each warp decides the band coefficients of its own tiles
                        for (int t = tid; t < ntw; t += nthr) {
                            const bool valid = t < nt;
                            const int p0 = (t % NPT) * TP, c0 = valid ? (t / NPT) << 2 : 0;
                            float A[4][TP], B[4][TP];
                            idft_tile(Q, tc, ts, nf, nfp, p0, c0, A, B);
#pragma unroll
                            for (int j = 0; j < 8 * TP; ++j) {
                                const int ci = (j % (4 * TP)) / TP, pi = j % TP, c = c0 + ci;
                                const bool hi = j >= 4 * TP;
                                const bool ok = valid && (hi ? (c > 0 && 2 * c < C) : c < nf);
                                const int cb = hi ? C - c : c, p = p0 + pi;
                                const float v = hi ? A[ci][pi] - B[ci][pi] : A[ci][pi] + B[ci][pi];
                                unsigned bal = __ballot_sync(0xffffffffu, ok && fabsf(fabsf(v) - tl) <= dl);
                                while (bal) {               // warp-uniform
                                    const int l = __ffs(bal) - 1;
                                    bal &= bal - 1;
                                    const int pl = __shfl_sync(0xffffffffu, p, l), cl = __shfl_sync(0xffffffffu, cb, l);
                                    const double xd = coef64(R, t64c, t64s, a.basis64, C, nf, pl, cl, lane);
                                    if (lane == l && fabs(xd) >= tlim) keep_band(p, cb, v);
                                }
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            // A slot without a kept coefficient is all zeros: nothing is written for it. No barrier is
            // needed on that path: the next slot's writes before its first barrier are the raw slot
            // (read by nobody after the barrier above), the thread's own stack entries and misc[1],
            // misc[2], misc[8], which are zero already or read by nobody.
            if (misc[1] == 0) continue;
            const int rows = misc[2];
            const bool sparse = misc[1] <= NL;
            if (tid == 0) {
                misc[0] += misc[1];
                misc[3] |= 1 << sl;
            }
            if (sparse) {
                // Z_f[i][b] = sum over the listed (i, j, c) of t w^{f c} conj(V_f[b][j]), without the
                // band DFT of the whole slot (to Q)
                const int nl = misc[7];
                for (int t = tid; t < nf * PS; t += nthr) {
                    const int f = t >> 3, b = t & 7;
                    const float* Vb = bas + (nf + f) * BS + b * 8;
                    float* zr = Q + f * RS + b;
                    float* zi = Q + (nf + f) * RS + b;
#pragma unroll
                    for (int i = 0; i < PS; ++i)
                        if ((rows >> i) & 1) zr[i * 8] = zi[i * 8] = 0.f;
                    for (int k = 0; k < nl; ++k) {
                        const int4 en = lst[k];
                        const int i = en.x >> 3, j = en.x & 7, c = en.y;
                        const bool lo = c < nf;                 // w^{f c} from the tables of band c or C - c
                        const int cr = lo ? c : C - c;
                        const float tv = __int_as_float(en.z), sn = ts[cr * nfp + f];
                        const float Tr = tv * tc[cr * nfp + f], Ti = tv * (lo ? sn : -sn);
                        const float vr = Vb[j], vi = Vb[64 + j];
                        zr[i * 8] += fmaf(Tr, vr, Ti * vi);
                        zi[i * 8] += fmaf(Ti, vr, -Tr * vi);
                    }
                }
            } else {
                // band DFT of the kept coefficients (folded on load) to R, then
                // Z_f[i][:] = T_f[i][:] V_f^H on the kept rows i (to Q)
                band_dft_unfolded(P, R, tc, ts, C, nf, nfp, tid, nthr);
                __syncthreads();
                for (int t = tid; t < nf * PS; t += nthr) {
                    const int f = t >> 3, i = t & 7;
                    if (!((rows >> i) & 1)) continue;
                    const float* Vb = bas + (nf + f) * BS;
                    float tr[8], ti[8], zr[8], zi[8];
                    load8s(R + f * RS + i * 8, tr);
                    load8s(R + (nf + f) * RS + i * 8, ti);
#pragma unroll
                    for (int b = 0; b < PS; ++b) {
                        float vr[8], vi[8];
                        load8s(Vb + b * 8, vr);
                        load8s(Vb + 64 + b * 8, vi);
                        float re = 0.f, im = 0.f;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            re = fmaf(tr[j], vr[j], fmaf(ti[j], vi[j], re));
                            im = fmaf(ti[j], vr[j], fmaf(-tr[j], vi[j], im));
                        }
                        zr[b] = re;
                        zi[b] = im;
                    }
                    store8s(Q + f * RS + i * 8, zr, 1.f);
                    store8s(Q + (nf + f) * RS + i * 8, zi, 1.f);
                }
            }
            __syncthreads();
            // G_f[a][:] = sum_{i kept} U_f[a][i] Z_f[i][:] (to P, times w_f / C)
            for (int t = tid; t < nf * PS; t += nthr) {
                const int f = t >> 3, a_ = t & 7;
                float ur[8], ui[8], gr[8], gi[8];
                load8s(bas + f * BS + a_ * 8, ur);
                load8s(bas + f * BS + 64 + a_ * 8, ui);
#pragma unroll
                for (int b = 0; b < 8; ++b) gr[b] = gi[b] = 0.f;
#pragma unroll
                for (int i = 0; i < PS; ++i) {
                    if (!((rows >> i) & 1)) continue;
                    float zr[8], zi[8];
                    load8s(Q + f * RS + i * 8, zr);
                    load8s(Q + (nf + f) * RS + i * 8, zi);
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        gr[b] = fmaf(ur[i], zr[b], fmaf(-ui[i], zi[b], gr[b]));
                        gi[b] = fmaf(ur[i], zi[b], fmaf(ui[i], zr[b], gi[b]));
                    }
                }
                const float w = (f == 0 || 2 * f == C ? 1.f : 2.f) / (float)C;
                store8s(P + f * RS + a_ * 8, gr, w);
                store8s(P + (nf + f) * RS + a_ * 8, gi, w);
            }
            __syncthreads();
            // inverse band DFT to the slot, [p][c], staged in Q and copied to the scratch in 16-byte
            // words (the next slot's first write to Q, its projection, comes after two barriers)
            band_idft_pc(P, Q, tc, ts, C, nf, nfp, tid, nthr);
            __syncthreads();
            {
                const float4* s4 = reinterpret_cast<const float4*>(Q);
                float4* d4 = reinterpret_cast<float4*>(scratch + (size_t)sl * NE);
                for (int e = tid; e < NE / 4; e += nthr) d4[e] = s4[e];
            }
        }
        __syncthreads();
        // weight of the group, then Haar synthesis per fibre (slots without a kept coefficient are
        // zero and not read) and aggregation
        float wg = 1.f;
        if (a.w_in) wg = a.w_in[grp];
        else if (a.agg_mode == 1) wg = 1.f / (float)max(1, misc[0]);
        if (tid == 0 && a.weights_out) a.weights_out[grp] = wg;
        const unsigned nzs = (unsigned)misc[3];
        // VW consecutive bands of a pixel per thread (2 when C is even: 8-byte vector atomics)
        auto synthesis = [&](auto vw_tag) {
            constexpr int VW = decltype(vw_tag)::value;
            using VT = typename std::conditional<VW == 2, float2, float>::type;
            for (int e = tid * VW; e < NE; e += nthr * VW) {
                const int p = __umulhi((unsigned)e, mg_c), c = e - p * C, pa = p >> 3, pb = p & 7;
                if (nzs) {
                    // after the first level of the synthesis (slots 0 and K/2) the two halves of the
                    // in-place layout are independent: K = 32 runs as two syntheses of 16
                    constexpr int KH = K > 16 ? K / 2 : K;
#pragma unroll 1
                    for (int h = 0; h < K / KH; ++h) {
                        float v[VW][KH];
                        auto ld = [&](int sk, float (&o)[VW]) {
                            if ((nzs >> sk) & 1u) {
                                const VT x = *reinterpret_cast<const VT*>(scratch + (size_t)sk * NE + e);
                                if constexpr (VW == 2) { o[0] = x.x; o[1] = x.y; }
                                else o[0] = x;
                            } else {
#pragma unroll
                                for (int w = 0; w < VW; ++w) o[w] = 0.f;
                            }
                        };
#pragma unroll
                        for (int k = 0; k < KH; ++k) {
                            float o[VW];
                            ld(k == 0 ? 0 : h * KH + k, o);
#pragma unroll
                            for (int w = 0; w < VW; ++w) v[w][k] = o[w];
                        }
                        if constexpr (K > KH) {
                            float sh[VW];
                            ld(KH, sh);
#pragma unroll
                            for (int w = 0; w < VW; ++w) v[w][0] = h == 0 ? v[w][0] + sh[w] : v[w][0] - sh[w];
                        }
#pragma unroll
                        for (int w = 0; w < VW; ++w) haar_inv_sum<KH>(v[w]);
#pragma unroll
                        for (int k = 0; k < KH; ++k) {
                            const size_t pix = (size_t)base[h * KH + k] + pa * g.W + pb;
                            if constexpr (VW == 2)
                                atomicAdd(reinterpret_cast<float2*>(a.num + pix * C + c),
                                          make_float2(wg * v[0][k], wg * v[1][k]));
                            else
                                atomicAdd(&a.num[pix * C + c], wg * v[0][k]);
                        }
                    }
                }
                if (c == 0)
#pragma unroll
                    for (int k = 0; k < K; ++k) atomicAdd(&a.den[(size_t)base[k] + pa * g.W + pb], wg);
            }
        };
        if ((C & 1) == 0) synthesis(std::integral_constant<int, 2>{});
        else synthesis(std::integral_constant<int, 1>{});
    }
}

__global__ void cube_finalize_kernel(const float* __restrict__ num, const float* __restrict__ den, int64_t npix,
                                     int C, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix * C; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = num[i] / den[i / C];
}

template <int K>
cudaError_t launch_cube_t(const CubeArgs& a, int grid, cudaStream_t s) {
    const int smem = cube_layout(a.g.C, K).total;
    auto fn = cube_filter_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, cube_threads(a.g.C), smem, s>>>(a);
    return cudaGetLastError();
}

// resident CTAs per SM of the filter for C bands (registers and shared memory), at least 1
template <int K>
int cube_per_sm(int C) {
    const int smem = cube_layout(C, K).total;
    auto fn = cube_filter_kernel<K>;
    int n = 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, cube_threads(C), smem) != cudaSuccess)
        n = 1;
    return n < 1 ? 1 : n;
}

}  // namespace

size_t cube_smem_bytes(int C, int K) { return (size_t)cube_layout(C, K).total; }

int cube_grid(int C, int K, int64_t ngroups) {
    int per_sm = 1;
    switch (K) {
        case 2: per_sm = cube_per_sm<2>(C); break;
        case 4: per_sm = cube_per_sm<4>(C); break;
        case 8: per_sm = cube_per_sm<8>(C); break;
        case 16: per_sm = cube_per_sm<16>(C); break;
        case 32: per_sm = cube_per_sm<32>(C); break;
        default: break;
    }
    const int64_t grid = (int64_t)per_sm * device_sm_count();
    return (int)(grid < ngroups ? grid : ngroups);
}

cudaError_t launch_cube_filter(const CubeArgs& a, int grid, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.num, 0, sizeof(float) * (size_t)a.g.H * a.g.W * a.g.C, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.den, 0, sizeof(float) * (size_t)a.g.H * a.g.W, s);
    if (e != cudaSuccess) return e;
    switch (a.g.K) {
        case 2: e = launch_cube_t<2>(a, grid, s); break;
        case 4: e = launch_cube_t<4>(a, grid, s); break;
        case 8: e = launch_cube_t<8>(a, grid, s); break;
        case 16: e = launch_cube_t<16>(a, grid, s); break;
        case 32: e = launch_cube_t<32>(a, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int64_t n = (int64_t)a.g.H * a.g.W * a.g.C;
    int blocks = (int)((n + 255) / 256);
    if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
    cube_finalize_kernel<<<blocks, 256, 0, s>>>(a.num, a.den, (int64_t)a.g.H * a.g.W, a.g.C, a.out);
    return cudaGetLastError();
}

}  // namespace htsvd

// MRI volumes (Sec. III-E, extension to other imaging: an MRI patch is a ps x ps x ps cube;
// Sec. IV, MRI denoising with ps = 4, K = 32, W = 5). A (D, H, W) uint8 volume is denoised by
// Alg. 1 on cubes P[i][j][k] = v[z + k, y + i, x + j]: the cube is a 4 x 4 x 4 tensor whose tube
// (the t-SVD's Fourier mode) runs along z.
//
// * block_match_volume_kernel: one warp per reference cube; exact SSD of every candidate of the
//   clamped W x W x W window (byte rows through __vabsdiffu4 + DP4A), keys (SSD, linear index) in
//   shared memory; the (K-1)-th smallest SSD by a ballot binary search, then the keys at or below it
//   ranked among themselves (keys are unique) for the K - 1 kept slots.
// * volume_moments_kernel: exact row and column moments of the reference cubes per (tube index
//   pair), from which the host forms the per-slice scatter matrices (Sec. III-B.1, Eq. (BCR
//   nonlocal SVD simplified), read as a 2-D SVD per tube-Fourier slice).
// * volume_bases_host: FP64 Jacobi eigenvectors of the 4 x 4 slice matrices (real slices 0 and 2,
//   the complex slice 1 through its real 8 x 8 embedding), canonical phase, slice 3 = conj(1).
// * volume_filter_kernel: one warp per group, lane k holding cube k of the group. Per row i of
//   the cube's coefficients, the forward projection (Sec. III-B.2, Eq. (forward transform)) in
//   registers, the Haar transform along the group mode across the lanes (normalised butterflies
//   through shuffles: Sec. II-D, Eqs. (H_2), (H_2N)), the hard threshold (Eq. (hard thresholding)),
//   FP32 with an FP64 decision inside a guard band; then per row the inverse Haar and the inverse
//   projection accumulated over the rows (Eq. (backward transform)); estimates added with shared
//   atomics into the CTA's footprint accumulators, which are added to the volume at the end.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "kernels.h"

namespace htsvd {

namespace {

constexpr int VPS = 4;                 // cube edge
constexpr int VTR = 4;                 // references per tile edge of the filter
constexpr int kVolWarps = 6;
constexpr int kMaxCand = 512;          // W^3 <= 512 (W <= 8)
constexpr int kHcBytes = kVolWarps * 32 * 65 * 4;

__host__ __device__ inline int vref_count(int n, int s) {
    const int last = n - VPS;
    return last / s + 1 + ((last % s) != 0 ? 1 : 0);
}
__host__ __device__ inline int vref_pos(int i, int s, int n) {
    const int v = i * s, last = n - VPS;
    return v < last ? v : last;
}

// 4 bytes of a byte array at any offset, from the two aligned words around it. The array must be
// readable up to the aligned word after the last byte (the volume's last word is read bytewise).
__device__ __forceinline__ uint32_t bytes4(const uint8_t* base, long long off, long long total) {
    const long long a = off & ~3ll;
    uint32_t w0, w1;
    if (a + 8 <= total) {
        w0 = __ldg(reinterpret_cast<const uint32_t*>(base + a));
        w1 = __ldg(reinterpret_cast<const uint32_t*>(base + a + 4));
    } else {
        w0 = w1 = 0;
        for (int k = 0; k < 4; ++k) {
            if (a + k < total) w0 |= (uint32_t)base[a + k] << (8 * k);
            if (a + 4 + k < total) w1 |= (uint32_t)base[a + 4 + k] << (8 * k);
        }
    }
    return __funnelshift_r(w0, w1, (int)(off & 3) * 8);
}

// ------------------------------------------------------------------------------ grouping

__global__ void __launch_bounds__(kVolWarps * 32)
block_match_volume_kernel(const uint8_t* __restrict__ vol, VolGeo g, int32_t* __restrict__ idx) {
    __shared__ unsigned long long skey[kVolWarps][kMaxCand];
    __shared__ unsigned long long skey2[kVolWarps][kMaxCand];    // keys that can be kept, compacted
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long total = (long long)g.D * g.H * g.W;
    const long long nref = (long long)g.nrz * g.nry * g.nrx;
    const long long plane = (long long)g.H * g.W;
    for (long long r = (long long)blockIdx.x * kVolWarps + warp; r < nref; r += (long long)gridDim.x * kVolWarps) {
        const int iz = (int)(r / ((long long)g.nry * g.nrx));
        const int rem = (int)(r - (long long)iz * g.nry * g.nrx);
        const int iy = rem / g.nrx, ix = rem - (rem / g.nrx) * g.nrx;
        const int z = vref_pos(iz, g.s, g.D), y = vref_pos(iy, g.s, g.H), x = vref_pos(ix, g.s, g.W);
        const long long me = (long long)z * plane + (long long)y * g.W + x;
        uint32_t ref[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) ref[q] = bytes4(vol, me + (q >> 2) * plane + (q & 3) * (long long)g.W, total);
        const int z0 = win_start(z, g.npz, g.win), y0 = win_start(y, g.npy, g.win), x0 = win_start(x, g.npx, g.win);
        const int ncand = g.wnz * g.wny * g.wnx;
        for (int c = lane; c < ncand; c += 32) {
            const int cz = c / (g.wny * g.wnx), cr = c - cz * (g.wny * g.wnx);
            const int cy = cr / g.wnx, cx = cr - (cr / g.wnx) * g.wnx;
            const long long lin = (long long)(z0 + cz) * plane + (long long)(y0 + cy) * g.W + (x0 + cx);
            unsigned ssd = 0;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const uint32_t d = __vabsdiffu4(ref[q], bytes4(vol, lin + (q >> 2) * plane + (q & 3) * (long long)g.W, total));
                ssd = __dp4a(d, d, ssd);
            }
            skey[warp][c] = lin == me ? ~0ull : (((unsigned long long)ssd << 32) | (unsigned long long)lin);
        }
        __syncwarp();
        // T = the (K-1)-th smallest SSD of the other candidates (binary search over SSD < 2^22 with
        // warp ballots); only keys with SSD <= T can be among the K-1 kept, so only they are ranked,
        // against each other (full keys: ties broken by the linear index)
        const int nslot = (ncand + 31) / 32;
        unsigned lo = 0, hi = 1u << 22;
        while (lo < hi) {
            const unsigned mid = (lo + hi) >> 1;
            int cnt = 0;
            for (int j = 0; j < nslot; ++j) {
                const int c = lane + 32 * j;
                const bool le = c < ncand && (unsigned)(skey[warp][c] >> 32) <= mid;
                cnt += __popc(__ballot_sync(0xffffffffu, le));
            }
            if (cnt >= g.K - 1) hi = mid;
            else lo = mid + 1;
        }
        unsigned long long* sel = skey2[warp];
        int m = 0;
        for (int j = 0; j < nslot; ++j) {
            const int c = lane + 32 * j;
            const unsigned long long k = c < ncand ? skey[warp][c] : ~0ull;
            const bool take = (unsigned)(k >> 32) <= lo;
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            if (take) sel[m + __popc(bal & ((1u << lane) - 1u))] = k;
            m += __popc(bal);
        }
        __syncwarp();
        int32_t* out = idx + r * g.K;
        if (lane == 0) out[0] = (int32_t)me;
        for (int c = lane; c < m; c += 32) {
            const unsigned long long k = sel[c];
            int rank = 0;
            for (int o = 0; o < m; ++o) rank += sel[o] < k ? 1 : 0;
            if (rank < g.K - 1) out[1 + rank] = (int32_t)(k & 0xffffffffull);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------ moments

constexpr int kMomRefs = 64;     // reference cubes staged per round

// mom[0][a][a'][c][c'] = sum_r sum_b P[a][b][c] P[a'][b][c'],  mom[1][b][b'][c][c'] = sum_r sum_a P[a][b][c] P[a][b'][c']
// (a rows, b columns, c tube), uint64, exact. Each thread owns two of the 512 entries.
__global__ void __launch_bounds__(256) volume_moments_kernel(const uint8_t* __restrict__ vol, VolGeo g,
                                                             unsigned long long* __restrict__ mom) {
    __shared__ uint8_t sc[kMomRefs][64];          // staged cubes, [r][(a * 4 + b) * 4 + c]
    const int t = threadIdx.x;
    const long long total = (long long)g.D * g.H * g.W;
    const long long plane = (long long)g.H * g.W;
    const long long nref = (long long)g.nrz * g.nry * g.nrx;
    unsigned long long acc[2] = {0ull, 0ull};
    int e0[2], e1[2], e2[2], e3[2], which[2];
    for (int h = 0; h < 2; ++h) {
        const int e = t + 256 * h;
        which[h] = e >> 8;
        e0[h] = (e >> 6) & 3; e1[h] = (e >> 4) & 3; e2[h] = (e >> 2) & 3; e3[h] = e & 3;
    }
    for (long long base = (long long)blockIdx.x * kMomRefs; base < nref; base += (long long)gridDim.x * kMomRefs) {
        __syncthreads();
        for (int q = t; q < kMomRefs * 16; q += 256) {       // (ref, tube c, row a): 4 bytes along b
            const int rr = q >> 4, c = (q >> 2) & 3, a = q & 3;
            const long long r = base + rr;
            uint32_t w = 0;
            if (r < nref) {
                const int iz = (int)(r / ((long long)g.nry * g.nrx));
                const int rem = (int)(r - (long long)iz * g.nry * g.nrx);
                const int iy = rem / g.nrx, ix = rem - (rem / g.nrx) * g.nrx;
                const long long off = (long long)(vref_pos(iz, g.s, g.D) + c) * plane +
                                      (long long)(vref_pos(iy, g.s, g.H) + a) * g.W + vref_pos(ix, g.s, g.W);
                w = bytes4(vol, off, total);
            }
            for (int b = 0; b < 4; ++b) sc[rr][(a * 4 + b) * 4 + c] = (uint8_t)(w >> (8 * b));
        }
        __syncthreads();
        for (int h = 0; h < 2; ++h) {
            unsigned s = 0;                                   // < 64 * 4 * 255^2 < 2^32
            for (int rr = 0; rr < kMomRefs; ++rr) {
                const uint8_t* P = sc[rr];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    // which 0: a = e0, a' = e1, summed over b = u; which 1: b = e0, b' = e1, summed over a = u
                    const int i0 = which[h] == 0 ? (e0[h] * 4 + u) : (u * 4 + e0[h]);
                    const int i1 = which[h] == 0 ? (e1[h] * 4 + u) : (u * 4 + e1[h]);
                    s += (unsigned)P[i0 * 4 + e2[h]] * (unsigned)P[i1 * 4 + e3[h]];
                }
            }
            acc[h] += s;
        }
    }
    for (int h = 0; h < 2; ++h)
        if (acc[h]) atomicAdd(mom + t + 256 * h, acc[h]);
}

// Full second moment of the reference cubes for the noise estimate: M[u][v] = sum_r P_r[u] P_r[v] and
// S[u] = sum_r P_r[u] (uint64, exact), u = (a * 4 + b) * 4 + c. Each thread owns 16 entries of M.
__global__ void __launch_bounds__(256) volume_full_moment_kernel(const uint8_t* __restrict__ vol, VolGeo g,
                                                                 unsigned long long* __restrict__ M,
                                                                 unsigned long long* __restrict__ S) {
    __shared__ uint8_t sc[kMomRefs][64];
    const int t = threadIdx.x;
    const long long total = (long long)g.D * g.H * g.W;
    const long long plane = (long long)g.H * g.W;
    const long long nref = (long long)g.nrz * g.nry * g.nrx;
    unsigned long long acc[16] = {};
    unsigned long long sacc = 0;
    for (long long base = (long long)blockIdx.x * kMomRefs; base < nref; base += (long long)gridDim.x * kMomRefs) {
        __syncthreads();
        for (int q = t; q < kMomRefs * 16; q += 256) {       // (ref, tube c, row a): 4 bytes along b
            const int rr = q >> 4, c = (q >> 2) & 3, a = q & 3;
            const long long r = base + rr;
            uint32_t w = 0;
            if (r < nref) {
                const int iz = (int)(r / ((long long)g.nry * g.nrx));
                const int rem = (int)(r - (long long)iz * g.nry * g.nrx);
                const int iy = rem / g.nrx, ix = rem - (rem / g.nrx) * g.nrx;
                const long long off = (long long)(vref_pos(iz, g.s, g.D) + c) * plane +
                                      (long long)(vref_pos(iy, g.s, g.H) + a) * g.W + vref_pos(ix, g.s, g.W);
                w = bytes4(vol, off, total);
            }
            for (int b = 0; b < 4; ++b) sc[rr][(a * 4 + b) * 4 + c] = (uint8_t)(w >> (8 * b));
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = t + 256 * q, u = e >> 6, v = e & 63;
            unsigned s = 0;                                   // < 64 * 255^2 < 2^32
            for (int rr = 0; rr < kMomRefs; ++rr) s += (unsigned)sc[rr][u] * (unsigned)sc[rr][v];
            acc[q] += s;
        }
        if (t < 64) {
            unsigned s = 0;
            for (int rr = 0; rr < kMomRefs; ++rr) s += sc[rr][t];
            sacc += s;
        }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
        if (acc[q]) atomicAdd(M + t + 256 * q, acc[q]);
    if (t < 64 && sacc) atomicAdd(S + t, sacc);
}

// ------------------------------------------------------------------------------ filter

// Normalised Haar analysis along the group mode on K values in registers (Sec. II-D, Eqs. (H_2),
// (H_2N)): level by level, (a, b) -> ((a + b) / sqrt 2, (a - b) / sqrt 2) on slots (j, j + st). Slot 0
// ends as row 0 of H_K, slot j > 0 as row K / 2^L + (j >> L), L = ctz(j) + 1. The butterfly is its own
// inverse, so the synthesis runs the same levels in reverse order.
template <int K>
__device__ __forceinline__ void haar_analysis(float (&v)[K]) {
    const float r2 = 0.70710678118654752f;
#pragma unroll
    for (int st = 1; st < K; st <<= 1)
#pragma unroll
        for (int j = 0; j < K; j += 2 * st) {
            const float a = v[j], b = v[j + st];
            v[j] = (a + b) * r2;
            v[j + st] = (a - b) * r2;
        }
}
template <int K>
__device__ __forceinline__ void haar_synthesis(float (&v)[K]) {
    const float r2 = 0.70710678118654752f;
#pragma unroll
    for (int st = K >> 1; st >= 1; st >>= 1)
#pragma unroll
        for (int j = 0; j < K; j += 2 * st) {
            const float a = v[j], b = v[j + st];
            v[j] = (a + b) * r2;
            v[j + st] = (a - b) * r2;
        }
}

__device__ __forceinline__ int haar_row(int j, int K) {
    if (j == 0) return 0;
    const int L = __ffs(j);                // ctz + 1
    return (K >> L) + (j >> L);
}

struct VolSmem {
    __align__(16) float ub[2][3][2][16];   // [U, V][slice 0..2][re, im][i * 4 + a]: columns contiguous
    double ud[2][3][2][16];
};

// Column c of basis w (0: U, 1: V), slice f, real or imaginary part: rows 0..3 in one 128-bit load.
__device__ __forceinline__ float4 ucol(const VolSmem& sm, int w, int f, int ri, int c) {
    return *reinterpret_cast<const float4*>(&sm.ub[w][f][ri][c * 4]);
}

// FP64 coefficient e = (i * 4 + j) * 4 + k of one cube (bytes w[(c * 4 + a)] = row a of tube slice c).
// Out of line: it runs only for coefficients inside the guard band.
__device__ __noinline__ double coef64(const uint32_t (&w)[16], int e, const VolSmem& sm) {
    const int i = e >> 4, j = (e >> 2) & 3, k = e & 3;
    double t0 = 0, t2 = 0, t1r = 0, t1i = 0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            const double p0 = (w[0 * 4 + a] >> (8 * b)) & 0xFF, p1 = (w[1 * 4 + a] >> (8 * b)) & 0xFF;
            const double p2 = (w[2 * 4 + a] >> (8 * b)) & 0xFF, p3 = (w[3 * 4 + a] >> (8 * b)) & 0xFF;
            const double x0 = p0 + p1 + p2 + p3, x2 = p0 - p1 + p2 - p3, xr = p0 - p2, xi = p3 - p1;
            const double u0 = sm.ud[0][0][0][a * 4 + i], v0 = sm.ud[1][0][0][b * 4 + j];
            const double u2 = sm.ud[0][2][0][a * 4 + i], v2 = sm.ud[1][2][0][b * 4 + j];
            t0 += u0 * x0 * v0;
            t2 += u2 * x2 * v2;
            const double ur = sm.ud[0][1][0][a * 4 + i], ui = sm.ud[0][1][1][a * 4 + i];
            const double vr = sm.ud[1][1][0][b * 4 + j], vi = sm.ud[1][1][1][b * 4 + j];
            const double yr = ur * xr + ui * xi, yi = ur * xi - ui * xr;          // conj(u) x
            t1r += yr * vr - yi * vi;
            t1i += yr * vi + yi * vr;
        }
    const double sg = (k & 1) ? -1.0 : 1.0;
    const double c1 = k == 0 ? 2 * t1r : k == 1 ? -2 * t1i : k == 2 ? -2 * t1r : 2 * t1i;
    return 0.25 * (t0 + sg * t2 + c1);
}

// The 16 byte rows of a cube staged in the footprint (zero for an inactive lane).
__device__ __forceinline__ void load_cube(const uint8_t* fb, int fy, int FXp, int oz, int oy, int ox, bool act,
                                          uint32_t (&w)[16]) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            uint32_t v = 0;
            if (act) {
                const int o = ((oz + c) * fy + (oy + a)) * FXp + ox;
                const uint32_t* fw = reinterpret_cast<const uint32_t*>(fb) + (o >> 2);
                v = __funnelshift_r(fw[0], fw[1], (o & 3) * 8);
            }
            w[c * 4 + a] = v;
        }
}

template <int K>
__global__ void __launch_bounds__(kVolWarps * 32, 2)
volume_filter_kernel(VolFilterArgs A) {
    const VolGeo g = A.g;
    __shared__ VolSmem sm;
    extern __shared__ __align__(16) unsigned char dyn[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tile of references and its footprint
    const int nty = (g.nry + VTR - 1) / VTR, ntx = (g.nrx + VTR - 1) / VTR;
    const int tz = blockIdx.x / (nty * ntx), trem = blockIdx.x - tz * (nty * ntx);
    const int ty = trem / ntx, tx = trem - (trem / ntx) * ntx;
    int f0[3], fn[3];
    {
        const int t3[3] = {tz, ty, tx}, nr[3] = {g.nrz, g.nry, g.nrx}, nn[3] = {g.D, g.H, g.W};
        const int np[3] = {g.npz, g.npy, g.npx}, wl[3] = {g.wnz, g.wny, g.wnx};
        for (int d = 0; d < 3; ++d) {
            const int r0 = t3[d] * VTR, r1 = min(r0 + VTR, nr[d]) - 1;
            f0[d] = win_start(vref_pos(r0, g.s, nn[d]), np[d], g.win);
            fn[d] = win_start(vref_pos(r1, g.s, nn[d]), np[d], g.win) + wl[d] + VPS - 1 - f0[d];
        }
    }
    const int FXp = ((fn[2] + 3) & ~3) + 4;            // staged row length: aligned, one spare word
    // the warp's group as a 32 x 65 float block: row k = the coefficients of cube k (lane k writes and
    // reads it), column e = fibre e (lane e % 32 reads it for the Haar transform); the pad of 65 keeps
    // both access patterns free of bank conflicts
    float* hcw = reinterpret_cast<float*>(dyn) + warp * 32 * 65;
    float* hcl = hcw + lane * 65;
    uint8_t* fb = dyn + kHcBytes;                        // footprint bytes [fz][fy][FXp]
    const int nfb = fn[0] * fn[1] * FXp;
    const int nvox = fn[0] * fn[1] * fn[2];
    float* num = reinterpret_cast<float*>(dyn + kHcBytes + ((nfb + 15) & ~15));
    float* org = num + nvox;                             // weights summed at the cubes' first voxel
    float* tmp = org + nvox;
    const long long plane = (long long)g.H * g.W;
    const long long total = (long long)g.D * plane;
    for (int e = tid; e < 2 * 3 * 2 * 16; e += blockDim.x) {
        const int w = e / 96, f = (e / 32) % 3, ri = (e / 16) & 1, ai = e & 15;
        const double v = A.basis64[((w * 4 + f) * 16 + ai) * 2 + ri];
        sm.ud[w][f][ri][ai] = v;
        sm.ub[w][f][ri][(ai & 3) * 4 + (ai >> 2)] = (float)v;
    }
    for (int q = tid; q < fn[0] * fn[1] * (FXp / 4); q += blockDim.x) {
        const int zz = q / (fn[1] * (FXp / 4)), rem = q - zz * (fn[1] * (FXp / 4));
        const int yy = rem / (FXp / 4), xw = rem - (rem / (FXp / 4)) * (FXp / 4);
        const long long off = (long long)(f0[0] + zz) * plane + (long long)(f0[1] + yy) * g.W + f0[2] + 4 * xw;
        uint32_t w = 0;
        // bytes past the footprint's row (or the volume) are staged as zero and never used
        for (int k = 0; k < 4; ++k) {
            const int xx = 4 * xw + k;
            if (xx < fn[2] && off + k < total) w |= (uint32_t)__ldg(A.vol + off + k) << (8 * k);
        }
        reinterpret_cast<uint32_t*>(fb)[q] = w;
    }
    for (int q = tid; q < 2 * nvox; q += blockDim.x) num[q] = 0.f;
    __syncthreads();

    const float tau = A.tau32;
    const int r0z = tz * VTR, r0y = ty * VTR, r0x = tx * VTR;
    const int nz = min(VTR, g.nrz - r0z), ny = min(VTR, g.nry - r0y), nx = min(VTR, g.nrx - r0x);
    for (int q = warp; q < nz * ny * nx; q += kVolWarps) {
        const int qz = q / (ny * nx), qr = q - qz * (ny * nx), qy = qr / nx, qx = qr - (qr / nx) * nx;
        const long long gi = ((long long)(r0z + qz) * g.nry + (r0y + qy)) * g.nrx + (r0x + qx);
        const bool act = lane < K;
        const int lin = act ? A.idx[gi * K + lane] : 0;
        const int cz = (int)(lin / plane), crem = (int)(lin - (long long)cz * plane);
        const int cy = crem / g.W, cx = crem - (crem / g.W) * g.W;
        const int oz = cz - f0[0], oy = cy - f0[1], ox = cx - f0[2];
        uint32_t w[16];                                  // w[c * 4 + a]: row a (bytes along b) of tube slice c
        load_cube(fb, fn[1], FXp, oz, oy, ox, act, w);
        unsigned ss = 0;
#pragma unroll
        for (int q2 = 0; q2 < 16; ++q2) ss = __dp4a(w[q2], w[q2], ss);
        // guard band of the threshold decision from the group's exact squared norm
        unsigned long long ss64 = ss;
        for (int o = 16; o >= 1; o >>= 1) ss64 += __shfl_xor_sync(0xffffffffu, ss64, o);
        const float band = A.band_rel * sqrtf((float)ss64) + A.band_abs;
        // forward projection of cube `lane`: tube DFT X0 (real), X2 (real), X1 = xr + i xi per (a, b)
        float x0[16], x2[16], xr[16], xi[16];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float p0 = (float)((w[0 * 4 + a] >> (8 * b)) & 0xFF), p1 = (float)((w[1 * 4 + a] >> (8 * b)) & 0xFF);
                const float p2 = (float)((w[2 * 4 + a] >> (8 * b)) & 0xFF), p3 = (float)((w[3 * 4 + a] >> (8 * b)) & 0xFF);
                x0[a * 4 + b] = (p0 + p1) + (p2 + p3);
                x2[a * 4 + b] = (p0 - p1) + (p2 - p3);
                xr[a * 4 + b] = p0 - p2;
                xi[a * 4 + b] = p3 - p1;
            }
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {
            // row i of S: Y_f[i][b] = sum_a conj(U_f[a][i]) X_f[a][b]; Z_f[i][j] = sum_b Y_f[i][b] V_f[b][j]
            float y0[4], y2[4], yr[4], yi[4];
            const float4 cu0 = ucol(sm, 0, 0, 0, i), cu2 = ucol(sm, 0, 2, 0, i);
            const float4 cur = ucol(sm, 0, 1, 0, i), cui = ucol(sm, 0, 1, 1, i);
            const float U0[4] = {cu0.x, cu0.y, cu0.z, cu0.w}, U2[4] = {cu2.x, cu2.y, cu2.z, cu2.w};
            const float UR[4] = {cur.x, cur.y, cur.z, cur.w}, UI[4] = {cui.x, cui.y, cui.z, cui.w};
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float s0 = 0.f, s2 = 0.f, sr = 0.f, si = 0.f;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    s0 = fmaf(U0[a], x0[a * 4 + b], s0);
                    s2 = fmaf(U2[a], x2[a * 4 + b], s2);
                    sr = fmaf(UR[a], xr[a * 4 + b], fmaf(UI[a], xi[a * 4 + b], sr));
                    si = fmaf(UR[a], xi[a * 4 + b], fmaf(-UI[a], xr[a * 4 + b], si));
                }
                y0[b] = s0; y2[b] = s2; yr[b] = sr; yi[b] = si;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float z0 = 0.f, z2 = 0.f, zr = 0.f, zi = 0.f;
                const float4 cv0 = ucol(sm, 1, 0, 0, j), cv2 = ucol(sm, 1, 2, 0, j);
                const float4 cvr = ucol(sm, 1, 1, 0, j), cvi = ucol(sm, 1, 1, 1, j);
                const float V0[4] = {cv0.x, cv0.y, cv0.z, cv0.w}, V2[4] = {cv2.x, cv2.y, cv2.z, cv2.w};
                const float VR[4] = {cvr.x, cvr.y, cvr.z, cvr.w}, VI[4] = {cvi.x, cvi.y, cvi.z, cvi.w};
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    z0 = fmaf(y0[b], V0[b], z0);
                    z2 = fmaf(y2[b], V2[b], z2);
                    zr = fmaf(yr[b], VR[b], fmaf(-yi[b], VI[b], zr));
                    zi = fmaf(yr[b], VI[b], fmaf(yi[b], VR[b], zi));
                }
                hcl[i * 16 + j * 4 + 0] = 0.25f * ((z0 + z2) + 2.f * zr);
                hcl[i * 16 + j * 4 + 1] = 0.25f * ((z0 - z2) - 2.f * zi);
                hcl[i * 16 + j * 4 + 2] = 0.25f * ((z0 + z2) - 2.f * zr);
                hcl[i * 16 + j * 4 + 3] = 0.25f * ((z0 - z2) + 2.f * zi);
            }
        }
        __syncwarp();
        // Haar transform along the group mode of fibres e0 = lane and e1 = lane + 32, in registers
        float v0[K], v1[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            v0[k] = hcw[k * 65 + lane];
            v1[k] = hcw[k * 65 + lane + 32];
        }
        haar_analysis(v0);
        haar_analysis(v1);
        unsigned kb0 = 0u, kb1 = 0u, nb0 = 0u, nb1 = 0u, db0 = 0u, db1 = 0u;   // bit j: kept / in band / dropped
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float m0 = fabsf(v0[j]), m1 = fabsf(v1[j]);
            const bool k0 = m0 >= tau, k1 = m1 >= tau, n0 = fabsf(m0 - tau) <= band, n1 = fabsf(m1 - tau) <= band;
            kb0 |= (k0 ? 1u : 0u) << j;
            kb1 |= (k1 ? 1u : 0u) << j;
            nb0 |= (n0 ? 1u : 0u) << j;
            nb1 |= (n1 ? 1u : 0u) << j;
            if (!k0 && !n0) v0[j] = 0.f;
            if (!k1 && !n1) v1[j] = 0.f;
        }
        // FP64 decisions inside the guard band, one coefficient at a time, the whole warp computing it:
        // lane k forms cube k's FP64 coefficient, the Haar row of the slot weighs the cubes
        for (;;) {
            const unsigned bal = __ballot_sync(0xffffffffu, (nb0 | nb1) != 0u);
            if (!bal) break;
            const int owner = __ffs(bal) - 1;
            int code = 0;
            if (lane == owner) code = nb0 ? (__ffs(nb0) - 1) : (64 + __ffs(nb1) - 1);
            code = __shfl_sync(0xffffffffu, code, owner);
            const int j = code & 63, e = owner + ((code >> 6) ? 32 : 0);
            uint32_t wr[16];                             // the cube's bytes again (not kept in registers)
            load_cube(fb, fn[1], FXp, oz, oy, ox, act, wr);
            const double mine = act ? coef64(wr, e, sm) : 0.0;
            double h = 0.0;
            if (act) {
                if (j == 0) h = 1.0 / sqrt((double)K);
                else {
                    const int L = __ffs(j), st = 1 << (L - 1);
                    const double mag = 1.0 / sqrt((double)(1 << L));
                    if (lane >= j - st && lane < j) h = mag;
                    else if (lane >= j && lane < j + st) h = -mag;
                }
            }
            double t = h * mine;
            for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == owner) {
                const unsigned bit = 1u << j;
                const bool keep = fabs(t) >= A.tau64;
                if (code >> 6) {
                    kb1 = keep ? (kb1 | bit) : (kb1 & ~bit);
                    db1 |= keep ? 0u : bit;
                    nb1 &= ~bit;
                } else {
                    kb0 = keep ? (kb0 | bit) : (kb0 & ~bit);
                    db0 |= keep ? 0u : bit;
                    nb0 &= ~bit;
                }
            }
        }
        int kept = __popc(kb0) + __popc(kb1);
        for (int o = 16; o >= 1; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
        const float wgt = A.w_in ? A.w_in[gi] : (A.agg_mode == 1 ? 1.0f / (float)max(1, kept) : 1.0f);
        if (lane == 0 && A.weights_out) A.weights_out[gi] = wgt;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if ((db0 >> j) & 1u) v0[j] = 0.f;
            if ((db1 >> j) & 1u) v1[j] = 0.f;
            if (A.mask_out) {
                const unsigned m0 = __ballot_sync(0xffffffffu, (kb0 >> j) & 1u);
                const unsigned m1 = __ballot_sync(0xffffffffu, (kb1 >> j) & 1u);
                if (lane == 0) {
                    A.mask_out[gi * 2 * K + 2 * haar_row(j, K)] = m0;
                    A.mask_out[gi * 2 * K + 2 * haar_row(j, K) + 1] = m1;
                }
            }
        }
        haar_synthesis(v0);
        haar_synthesis(v1);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            hcw[k * 65 + lane] = v0[k];
            hcw[k * 65 + lane + 32] = v1[k];
        }
        __syncwarp();
        // inverse projection of cube `lane`, row by row: P_f += U_f[:, i] (Z_f[i, :] V_f^H)
        if (act) {
            float p0[16], p2[16], pr[16], pi[16];
#pragma unroll
            for (int q2 = 0; q2 < 16; ++q2) p0[q2] = p2[q2] = pr[q2] = pi[q2] = 0.f;
#pragma unroll 1
            for (int i = 0; i < 4; ++i) {
                float w0[4], w2[4], wrr[4], wi[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) { w0[b] = w2[b] = wrr[b] = wi[b] = 0.f; }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float s0 = hcl[i * 16 + j * 4 + 0], s1 = hcl[i * 16 + j * 4 + 1];
                    const float s2 = hcl[i * 16 + j * 4 + 2], s3 = hcl[i * 16 + j * 4 + 3];
                    const float z0 = (s0 + s1) + (s2 + s3), z2 = (s0 - s1) + (s2 - s3), zr = s0 - s2, zi = s3 - s1;
                    const float4 cv0 = ucol(sm, 1, 0, 0, j), cv2 = ucol(sm, 1, 2, 0, j);
                    const float4 cvr = ucol(sm, 1, 1, 0, j), cvi = ucol(sm, 1, 1, 1, j);
                    const float V0[4] = {cv0.x, cv0.y, cv0.z, cv0.w}, V2[4] = {cv2.x, cv2.y, cv2.z, cv2.w};
                    const float VR[4] = {cvr.x, cvr.y, cvr.z, cvr.w}, VI[4] = {cvi.x, cvi.y, cvi.z, cvi.w};
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        w0[b] = fmaf(z0, V0[b], w0[b]);
                        w2[b] = fmaf(z2, V2[b], w2[b]);
                        wrr[b] = fmaf(zr, VR[b], fmaf(zi, VI[b], wrr[b]));      // z conj(v)
                        wi[b] = fmaf(zi, VR[b], fmaf(-zr, VI[b], wi[b]));
                    }
                }
                const float4 cu0 = ucol(sm, 0, 0, 0, i), cu2 = ucol(sm, 0, 2, 0, i);
                const float4 cur = ucol(sm, 0, 1, 0, i), cui = ucol(sm, 0, 1, 1, i);
                const float U0[4] = {cu0.x, cu0.y, cu0.z, cu0.w}, U2[4] = {cu2.x, cu2.y, cu2.z, cu2.w};
                const float UR[4] = {cur.x, cur.y, cur.z, cur.w}, UI[4] = {cui.x, cui.y, cui.z, cui.w};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        p0[a * 4 + b] = fmaf(U0[a], w0[b], p0[a * 4 + b]);
                        p2[a * 4 + b] = fmaf(U2[a], w2[b], p2[a * 4 + b]);
                        pr[a * 4 + b] = fmaf(UR[a], wrr[b], fmaf(-UI[a], wi[b], pr[a * 4 + b]));
                        pi[a * 4 + b] = fmaf(UR[a], wi[b], fmaf(UI[a], wrr[b], pi[a * 4 + b]));
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int q2 = a * 4 + b;
                    const float v[4] = {0.25f * ((p0[q2] + p2[q2]) + 2.f * pr[q2]), 0.25f * ((p0[q2] - p2[q2]) - 2.f * pi[q2]),
                                        0.25f * ((p0[q2] + p2[q2]) - 2.f * pr[q2]), 0.25f * ((p0[q2] - p2[q2]) + 2.f * pi[q2])};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        atomicAdd(num + ((oz + k) * fn[1] + (oy + a)) * fn[2] + ox + b, wgt * v[k]);
                }
            atomicAdd(org + (oz * fn[1] + oy) * fn[2] + ox, wgt);
        }
        __syncwarp();
    }
    __syncthreads();
    // denominator: the weights of every cube covering a voxel = a 4 x 4 x 4 box sum of the origin weights
    for (int q = tid; q < nvox; q += blockDim.x) {                 // along x
        const int xx = q % fn[2];
        float s = 0.f;
        for (int d = 0; d < 4 && d <= xx; ++d) s += org[q - d];
        tmp[q] = s;
    }
    __syncthreads();
    for (int q = tid; q < nvox; q += blockDim.x) {                 // along y
        const int yy = (q / fn[2]) % fn[1];
        float s = 0.f;
        for (int d = 0; d < 4 && d <= yy; ++d) s += tmp[q - d * fn[2]];
        org[q] = s;
    }
    __syncthreads();
    for (int q = tid; q < nvox; q += blockDim.x) {                 // along z, then into the volume
        const int zz = q / (fn[1] * fn[2]);
        float d = 0.f;
        for (int k = 0; k < 4 && k <= zz; ++k) d += org[q - k * fn[1] * fn[2]];
        if (d == 0.f) continue;
        const int rem = q - zz * (fn[1] * fn[2]);
        const int yy = rem / fn[2], xx = rem - (rem / fn[2]) * fn[2];
        const long long o = (long long)(f0[0] + zz) * plane + (long long)(f0[1] + yy) * g.W + f0[2] + xx;
        atomicAdd(A.num + o, num[q]);
        atomicAdd(A.den + o, d);
    }
}

__global__ void volume_finalize_kernel(const float* __restrict__ num, const float* __restrict__ den, long long n,
                                       float* __restrict__ out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = num[i] / den[i];
}

// ------------------------------------------------------------------------------ host bases

// Cyclic Jacobi on a real symmetric n x n matrix (n <= 8), FP64: eigenvalues in lam, eigenvectors in
// the columns of Q (row-major n x n).
void jacobi_sym(double* M, int n, double* lam, double* Q) {
    for (int i = 0; i < n * n; ++i) Q[i] = (i / n == i % n) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) (p == q ? diag : off) += M[p * n + q] * M[p * n + q];
        if (off <= 1e-34 * diag || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = M[p * n + q];
                if (apq == 0.0) continue;
                const double th = (M[q * n + q] - M[p * n + p]) / (2.0 * apq);
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {          // columns p, q
                    const double mkp = M[k * n + p], mkq = M[k * n + q];
                    M[k * n + p] = c * mkp - s * mkq;
                    M[k * n + q] = s * mkp + c * mkq;
                }
                for (int k = 0; k < n; ++k) {          // rows p, q
                    const double mpk = M[p * n + k], mqk = M[q * n + k];
                    M[p * n + k] = c * mpk - s * mqk;
                    M[q * n + k] = s * mpk + c * mqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double qkp = Q[k * n + p], qkq = Q[k * n + q];
                    Q[k * n + p] = c * qkp - s * qkq;
                    Q[k * n + q] = s * qkp + c * qkq;
                }
            }
    }
    for (int i = 0; i < n; ++i) lam[i] = M[i * n + i];
}

// Canonical eigenvectors of a 4 x 4 Hermitian matrix (re, im row-major): eigenvalues descending,
// each eigenvector's largest-modulus entry (lowest index within 1e-6 relative) real positive.
// out[(a * 4 + i) * 2 + {re, im}] = component a of eigenvector i. Returns the smallest gap between
// consecutive eigenvalues relative to the largest modulus.
double hermitian4_canonical(const double* re, const double* im, bool real_only, double* out) {
    double vr[4][4], vi[4][4], lam[4];
    if (real_only) {
        double M[16], Q[16];
        std::memcpy(M, re, sizeof(M));
        jacobi_sym(M, 4, lam, Q);
        for (int a = 0; a < 4; ++a)
            for (int i = 0; i < 4; ++i) { vr[a][i] = Q[a * 4 + i]; vi[a][i] = 0.0; }
    } else {
        // real embedding [[A, -B], [B, A]] of A + iB: every eigenvalue twice, eigenvectors [x; y] <-> x + iy
        double M[64], Q[64], l8[8];
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                M[a * 8 + b] = re[a * 4 + b];
                M[a * 8 + 4 + b] = -im[a * 4 + b];
                M[(4 + a) * 8 + b] = im[a * 4 + b];
                M[(4 + a) * 8 + 4 + b] = re[a * 4 + b];
            }
        jacobi_sym(M, 8, l8, Q);
        int ord[8];
        for (int i = 0; i < 8; ++i) ord[i] = i;
        for (int i = 0; i < 8; ++i)
            for (int j = i + 1; j < 8; ++j)
                if (l8[ord[j]] > l8[ord[i]]) { const int t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
        int got = 0;
        for (int c = 0; c < 8 && got < 4; ++c) {       // one complex vector per orthogonal direction
            double zr[4], zi[4];
            for (int a = 0; a < 4; ++a) { zr[a] = Q[a * 8 + ord[c]]; zi[a] = Q[(4 + a) * 8 + ord[c]]; }
            for (int p = 0; p < got; ++p) {            // remove the components along the vectors taken
                double dr = 0, di = 0;                 // <v_p, z> = sum conj(v_p) z
                for (int a = 0; a < 4; ++a) {
                    dr += vr[a][p] * zr[a] + vi[a][p] * zi[a];
                    di += vr[a][p] * zi[a] - vi[a][p] * zr[a];
                }
                for (int a = 0; a < 4; ++a) {
                    zr[a] -= dr * vr[a][p] - di * vi[a][p];
                    zi[a] -= dr * vi[a][p] + di * vr[a][p];
                }
            }
            double nn = 0;
            for (int a = 0; a < 4; ++a) nn += zr[a] * zr[a] + zi[a] * zi[a];
            if (nn < 0.25) continue;
            nn = 1.0 / std::sqrt(nn);
            for (int a = 0; a < 4; ++a) { vr[a][got] = zr[a] * nn; vi[a][got] = zi[a] * nn; }
            lam[got] = l8[ord[c]];
            ++got;
        }
    }
    int ord[4] = {0, 1, 2, 3};
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j)
            if (lam[ord[j]] > lam[ord[i]]) { const int t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
    double top = 0;
    for (int i = 0; i < 4; ++i) top = std::fmax(top, std::fabs(lam[i]));
    double gap = 1.0;
    for (int i = 0; i + 1 < 4; ++i) gap = std::fmin(gap, std::fabs(lam[ord[i]] - lam[ord[i + 1]]) / std::fmax(top, 1e-300));
    for (int i = 0; i < 4; ++i) {
        const int c = ord[i];
        double mx = 0;
        for (int a = 0; a < 4; ++a) mx = std::fmax(mx, std::hypot(vr[a][c], vi[a][c]));
        int am = 0;
        for (int a = 0; a < 4; ++a)
            if (std::hypot(vr[a][c], vi[a][c]) >= mx * (1.0 - 1e-6)) { am = a; break; }
        const double m = std::hypot(vr[am][c], vi[am][c]);
        const double hr = vr[am][c] / m, hi = -vi[am][c] / m;       // conj(v_am) / |v_am|
        for (int a = 0; a < 4; ++a) {
            const double r = vr[a][c] * hr - vi[a][c] * hi, s = vr[a][c] * hi + vi[a][c] * hr;
            out[(a * 4 + i) * 2] = r;
            out[(a * 4 + i) * 2 + 1] = real_only ? 0.0 : s;
        }
        out[(am * 4 + i) * 2 + 1] = 0.0;
    }
    return gap;
}

}  // namespace

VolGeo make_vol_geo(int D, int H, int W, int s, int win, int K) {
    VolGeo g;
    g.D = D; g.H = H; g.W = W; g.s = s; g.win = win; g.K = K;
    g.nrz = vref_count(D, s); g.nry = vref_count(H, s); g.nrx = vref_count(W, s);
    g.npz = D - VPS + 1; g.npy = H - VPS + 1; g.npx = W - VPS + 1;
    g.wnz = win_len(g.npz, win); g.wny = win_len(g.npy, win); g.wnx = win_len(g.npx, win);
    return g;
}

int volume_max_window() { return 8; }

cudaError_t launch_block_match_volume(const uint8_t* vol, const VolGeo& g, int32_t* idx, cudaStream_t s) {
    const long long nref = (long long)g.nrz * g.nry * g.nrx;
    const long long blocks = (nref + kVolWarps - 1) / kVolWarps;
    const long long cap = (long long)device_sm_count() * 16;
    block_match_volume_kernel<<<(int)(blocks < cap ? blocks : cap), kVolWarps * 32, 0, s>>>(vol, g, idx);
    return cudaGetLastError();
}

cudaError_t launch_volume_moments(const uint8_t* vol, const VolGeo& g, unsigned long long* d_mom, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_mom, 0, sizeof(unsigned long long) * 512, s);
    if (e != cudaSuccess) return e;
    const long long nref = (long long)g.nrz * g.nry * g.nrx;
    const long long rounds = (nref + kMomRefs - 1) / kMomRefs;
    const long long cap = (long long)device_sm_count() * 2;
    volume_moments_kernel<<<(int)(rounds < cap ? rounds : cap), 256, 0, s>>>(vol, g, d_mom);
    return cudaGetLastError();
}

cudaError_t launch_volume_full_moment(const uint8_t* vol, const VolGeo& g, unsigned long long* d_M,
                                      unsigned long long* d_S, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_M, 0, sizeof(unsigned long long) * 64 * 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_S, 0, sizeof(unsigned long long) * 64, s);
    if (e != cudaSuccess) return e;
    const long long nref = (long long)g.nrz * g.nry * g.nrx;
    const long long rounds = (nref + kMomRefs - 1) / kMomRefs;
    const long long cap = (long long)device_sm_count() * 2;
    volume_full_moment_kernel<<<(int)(rounds < cap ? rounds : cap), 256, 0, s>>>(vol, g, d_M, d_S);
    return cudaGetLastError();
}

double volume_bases_host(const unsigned long long* mom, double* b64) {
    double gap = 1.0;
    for (int w = 0; w < 2; ++w)
        for (int f = 0; f < 3; ++f) {
            // U: A_f[a][a'] = sum_{c,c'} e^{-2 pi i f (c - c') / 4} R[a][a'][c][c'];
            // V: B_f[b][b'] = sum_{c,c'} e^{+2 pi i f (c - c') / 4} Q[b][b'][c][c']  (exact integers)
            double re[16], im[16];
            for (int a = 0; a < 4; ++a)
                for (int a2 = 0; a2 < 4; ++a2) {
                    double sr = 0, si = 0;
                    for (int c = 0; c < 4; ++c)
                        for (int c2 = 0; c2 < 4; ++c2) {
                            const double m = (double)mom[w * 256 + ((a * 4 + a2) * 4 + c) * 4 + c2];
                            int ph = ((f * (c - c2)) % 4 + 4) % 4;           // e^{-2 pi i ph / 4}
                            if (w == 1) ph = (4 - ph) % 4;
                            sr += ph == 0 ? m : ph == 2 ? -m : 0.0;
                            si += ph == 1 ? -m : ph == 3 ? m : 0.0;
                        }
                    re[a * 4 + a2] = sr;
                    im[a * 4 + a2] = si;
                }
            double vec[32];
            gap = std::fmin(gap, hermitian4_canonical(re, im, f != 1, vec));
            for (int q = 0; q < 32; ++q) b64[(w * 4 + f) * 32 + q] = vec[q];
            if (f == 1)
                for (int q = 0; q < 16; ++q) {     // slice 3 = conj(slice 1)
                    b64[(w * 4 + 3) * 32 + 2 * q] = vec[2 * q];
                    b64[(w * 4 + 3) * 32 + 2 * q + 1] = -vec[2 * q + 1];
                }
        }
    return gap;
}

size_t volume_filter_smem_bytes(const VolGeo& g) {
    const int ext[3] = {g.wnz, g.wny, g.wnx};
    int fn[3];
    for (int d = 0; d < 3; ++d) fn[d] = (VTR - 1) * g.s + ext[d] + VPS - 1;
    const int FXp = ((fn[2] + 3) & ~3) + 4;
    const size_t nfb = (size_t)fn[0] * fn[1] * FXp;
    return kHcBytes + ((nfb + 15) & ~(size_t)15) + sizeof(float) * 3 * (size_t)fn[0] * fn[1] * fn[2];
}

template <int K>
static cudaError_t launch_volume_filter_k(const VolFilterArgs& a, int ntiles, size_t smem, cudaStream_t s) {
    static int configured = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured != dev) {
        e = cudaFuncSetAttribute(volume_filter_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        if (e != cudaSuccess) return e;
        configured = dev;
    }
    volume_filter_kernel<K><<<ntiles, kVolWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_volume_filter(const VolFilterArgs& a, cudaStream_t s) {
    const VolGeo& g = a.g;
    const int ntiles = ((g.nrz + VTR - 1) / VTR) * ((g.nry + VTR - 1) / VTR) * ((g.nrx + VTR - 1) / VTR);
    const size_t smem = volume_filter_smem_bytes(g);
    switch (g.K) {
        case 2: return launch_volume_filter_k<2>(a, ntiles, smem, s);
        case 4: return launch_volume_filter_k<4>(a, ntiles, smem, s);
        case 8: return launch_volume_filter_k<8>(a, ntiles, smem, s);
        case 16: return launch_volume_filter_k<16>(a, ntiles, smem, s);
        case 32: return launch_volume_filter_k<32>(a, ntiles, smem, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_volume_finalize(const float* num, const float* den, long long n, float* out, cudaStream_t s) {
    const long long blocks = (n + 255) / 256;
    const long long cap = (long long)device_sm_count() * 8;
    volume_finalize_kernel<<<(int)(blocks < cap ? blocks : cap), 256, 0, s>>>(num, den, n, out);
    return cudaGetLastError();
}

}  // namespace htsvd

// HOST hook of the volume bases (htsvd_internal.h).
extern "C" double htsvd_internal_volume_bases(const unsigned long long* mom, double* b64) {
    return htsvd::volume_bases_host(mom, b64);
}

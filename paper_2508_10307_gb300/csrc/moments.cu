// Second moments of the reference patches and the global t-SVD bases
// (Alg. 1 Step 2(1); Sec. III-B.1, Eq. (BCR nonlocal SVD simplified)), plus the
// circulant eigen-rank of sampled groups (Sec. III-D, Eq. (other eigenvalue)).
//
// The bases are the eigenvectors of the per-Fourier-slice row and column scatter
// matrices of the reference patches, A_f = sum_r P_f P_f^H and B_f = sum_r P_f^H P_f,
// with P_f the f-th slice of the FFT along the channel mode (Eqs. (FFT product),
// (FFT third mode)). A_f and B_f follow exactly from the integer row/column moments
//   R[a][a'][c][c'] = sum_r sum_b P[a][b][c] P[a'][b][c'],
//   Q[b][b'][c][c'] = sum_r sum_a P[a][b][c] P[a][b'][c'],
// as A_f[a][a'] = sum_{c,c'} w^{f(c-c')} R[a][a'][c][c'] and
//    B_f[b][b'] = sum_{c,c'} w^{f(c'-c)} Q[b][b'][c][c'],   w = exp(-2 pi i / C).
#include "kernels.h"

namespace htsvd {

namespace {

// ----------------------------------------------------------------------------- moments

constexpr int MOM_CHUNK = 256;     // references per CTA (uint32 partials: 256 * 8 * 255^2 < 2^32)
constexpr int MOM_BATCH = 32;      // references staged at once

// Moments of the references [chunk * MOM_CHUNK, (chunk + 1) * MOM_CHUNK) added into out.
template <int C>
__device__ __forceinline__ void moments_chunk(const uint8_t* __restrict__ img, const Geo& g, int chunk,
                                              unsigned long long* __restrict__ out) {
    // rows[j][c][a] = 8 bytes of row a of channel c; cols[j][c][b] = 8 bytes of column b.
    __shared__ uint32_t rows[MOM_BATCH][C][PS][2];
    __shared__ uint32_t cols[MOM_BATCH][C][PS][2];
    constexpr int NE = 2 * PS * PS * C * C;
    constexpr int EPT = (NE + 255) / 256;
    uint32_t acc[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) acc[e] = 0;

    const int N = g.ngroups();
    const int r0 = chunk * MOM_CHUNK;
    const int r1 = min(r0 + MOM_CHUNK, N);
    for (int rb = r0; rb < r1; rb += MOM_BATCH) {
        const int nb = min(MOM_BATCH, r1 - rb);
        __syncthreads();
        // rows: task (reference j, patch row a) reads the row's 8 C bytes as aligned 32-bit words
        // (alignment from the absolute address), shifts them into place and splits the channels
        for (int t = threadIdx.x; t < nb * PS; t += 256) {
            const int j = t >> 3, a = t & 7;
            const int r = rb + j;
            const int iy = r / g.nrx, ix = r - iy * g.nrx;
            const int ry = ref_pos(iy, g.s, g.H), rx = ref_pos(ix, g.s, g.W);
            constexpr int NW = 2 * C;                 // words of one patch row
            const uintptr_t ad = reinterpret_cast<uintptr_t>(img + ((size_t)(ry + a) * g.W + rx) * C);
            const int o = (int)(ad & 3);
            // every word read holds at least one byte of the row, so none leaves the image's aligned words
            const uint32_t* w = reinterpret_cast<const uint32_t*>(ad - o);
            uint32_t wv[NW + 1], al[NW];
#pragma unroll
            for (int k = 0; k < NW; ++k) wv[k] = w[k];
            wv[NW] = o ? w[NW] : 0u;
#pragma unroll
            for (int k = 0; k < NW; ++k) al[k] = __funnelshift_r(wv[k], wv[k + 1], 8 * o);
            if constexpr (C == 1) {
                rows[j][0][a][0] = al[0];
                rows[j][0][a][1] = al[1];
            } else {
                // channel c, pixels 4h .. 4h+3: bytes 12h + c + 3i (i = 0..3) of the row
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        uint32_t v = 0u;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int pb = 12 * h + c + 3 * i;
                            v |= ((al[pb >> 2] >> (8 * (pb & 3))) & 0xffu) << (8 * i);
                        }
                        rows[j][c][a][h] = v;
                    }
            }
        }
        __syncthreads();
        // columns: block (j, c, word w of the column = rows 4w..4w+3, word h of the row = columns
        // 4h..4h+3) is a 4 x 4 byte transpose of four row words
        for (int t = threadIdx.x; t < nb * C * 4; t += 256) {
            const int j = t / (C * 4), rem = t - j * C * 4;
            const int c = rem >> 2, w = (rem >> 1) & 1, h = rem & 1;
            const uint32_t r0 = rows[j][c][4 * w + 0][h], r1 = rows[j][c][4 * w + 1][h];
            const uint32_t r2 = rows[j][c][4 * w + 2][h], r3 = rows[j][c][4 * w + 3][h];
            const uint32_t lo01 = __byte_perm(r0, r1, 0x5140u), hi01 = __byte_perm(r0, r1, 0x7362u);
            const uint32_t lo23 = __byte_perm(r2, r3, 0x5140u), hi23 = __byte_perm(r2, r3, 0x7362u);
            cols[j][c][4 * h + 0][w] = __byte_perm(lo01, lo23, 0x5410u);
            cols[j][c][4 * h + 1][w] = __byte_perm(lo01, lo23, 0x7632u);
            cols[j][c][4 * h + 2][w] = __byte_perm(hi01, hi23, 0x5410u);
            cols[j][c][4 * h + 3][w] = __byte_perm(hi01, hi23, 0x7632u);
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            int ent = threadIdx.x + e * 256;
            if (ent < NE) {
                int which = ent / (PS * PS * C * C);
                int rem = ent - which * PS * PS * C * C;
                int u = rem / (PS * C * C);
                rem -= u * PS * C * C;
                int v = rem / (C * C);
                rem -= v * C * C;
                int c = rem / C, c2 = rem - c * C;
                uint32_t s = 0;
                if (which == 0) {
                    for (int j = 0; j < nb; ++j) {
                        s = __dp4a(rows[j][c][u][0], rows[j][c2][v][0], s);
                        s = __dp4a(rows[j][c][u][1], rows[j][c2][v][1], s);
                    }
                } else {
                    for (int j = 0; j < nb; ++j) {
                        s = __dp4a(cols[j][c][u][0], cols[j][c2][v][0], s);
                        s = __dp4a(cols[j][c][u][1], cols[j][c2][v][1], s);
                    }
                }
                acc[e] += s;
            }
        }
    }
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        int ent = threadIdx.x + e * 256;
        if (ent < NE && acc[e]) atomicAdd(out + ent, (unsigned long long)acc[e]);
    }
    __syncthreads();
}

template <int C>
__global__ void __launch_bounds__(256) moments_kernel(const uint8_t* __restrict__ img, Geo g,
                                                      unsigned long long* __restrict__ out) {
    moments_chunk<C>(img, g, blockIdx.x, out);
}

// Batch form: chunk items of all images, item w -> image by prefix[].
template <int C>
__global__ void __launch_bounds__(256) moments_batch_kernel(const BMArgs* __restrict__ args,
                                                            unsigned long long* const* __restrict__ moms,
                                                            const int* __restrict__ prefix, int nimg) {
    const int total = prefix[nimg];
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        int lo = 0, hi = nimg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        moments_chunk<C>(args[lo].img, args[lo].g, w - prefix[lo], moms[lo]);
    }
}

// Row and column moments of the reference patches of a cube with any number of bands C, in the
// layout of moments_chunk ([2][8][8][C][C]): with the 8-byte vectors r_(a,c) = P[a][0..7][c] and
// q_(b,c) = P[0..7][b][c] of a reference, R[a][a'][c][c'] = sum over references of <r_(a,c), r_(a',c')>
// and Q[b][b'][c][c'] = sum of <q_(b,c), q_(b',c')>: two Gram matrices of 8C vectors per reference,
// accumulated with DP4A. The Gram matrices are symmetric, so only tile pairs tu <= tv are formed and
// an off-diagonal tile also writes its mirror. CTA (x: which, tile pair of 64-vector tiles; y: chunk
// of CM_CHUNK references), 16 x 16 threads with 4 x 4 entries each; uint32 partials per CTA
// (CM_CHUNK * 8 * 255^2 < 2^32), added to uint64 out.
constexpr int CM_T = 64;
constexpr int CM_BATCH = 16;
constexpr int CM_CHUNK = 1024;

__global__ void __launch_bounds__(256) cube_moments_kernel(const uint8_t* __restrict__ img, Geo g, int ntile,
                                                           unsigned long long* __restrict__ out) {
    __shared__ __align__(16) uint2 su[CM_BATCH][CM_T], sv[CM_BATCH][CM_T];
    __shared__ int rbase[CM_BATCH];
    const int C = g.C, D = PS * C;
    const int npair = ntile * (ntile + 1) / 2;
    const int which = blockIdx.x / npair;
    int pr = blockIdx.x - which * npair, tu = 0;
    while (pr >= ntile - tu) {
        pr -= ntile - tu;
        ++tu;
    }
    const int tv = tu + pr;                           // tu <= tv
    const bool diag = tu == tv;
    const int N = g.ngroups();
    const int r0 = blockIdx.y * CM_CHUNK, r1 = min(r0 + CM_CHUNK, N);
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    uint32_t acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0u;
    // the 8 bytes of vector x = (e, c) of the reference whose corner is byte rb: row e, columns 0..7
    // (which = 0) or column e, rows 0..7 (which = 1), band c
    const size_t st = (size_t)(which == 0 ? 1 : g.W) * C;
    auto vec = [&](int rb, int x) -> uint2 {
        if (x >= D) return make_uint2(0u, 0u);
        const int e = x / C, c = x - e * C;
        const uint8_t* p0 = img + rb + (size_t)(which == 0 ? e * g.W : e) * C + c;
        uint32_t w0 = 0u, w1 = 0u;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            w0 |= (uint32_t)p0[t * st] << (8 * t);
            w1 |= (uint32_t)p0[(4 + t) * st] << (8 * t);
        }
        return make_uint2(w0, w1);
    };
    for (int rb0 = r0; rb0 < r1; rb0 += CM_BATCH) {
        const int nb = min(CM_BATCH, r1 - rb0);
        __syncthreads();
        if (threadIdx.x < nb) {
            const int r = rb0 + threadIdx.x, iy = r / g.nrx, ix = r - iy * g.nrx;
            rbase[threadIdx.x] = (ref_pos(iy, g.s, g.H) * g.W + ref_pos(ix, g.s, g.W)) * C;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nb * CM_T; t += 256) {
            const int jj = t / CM_T, x = t - jj * CM_T;
            su[jj][x] = vec(rbase[jj], tu * CM_T + x);
            if (!diag) sv[jj][x] = vec(rbase[jj], tv * CM_T + x);
        }
        __syncthreads();
        const uint2 (*Vs)[CM_T] = diag ? su : sv;
        for (int jj = 0; jj < nb; ++jj) {
            const uint4* pa = reinterpret_cast<const uint4*>(&su[jj][ty * 4]);
            const uint4* pb = reinterpret_cast<const uint4*>(&Vs[jj][tx * 4]);
            const uint4 a01 = pa[0], a23 = pa[1], b01 = pb[0], b23 = pb[1];
            const uint32_t au[4][2] = {{a01.x, a01.y}, {a01.z, a01.w}, {a23.x, a23.y}, {a23.z, a23.w}};
            const uint32_t bv[4][2] = {{b01.x, b01.y}, {b01.z, b01.w}, {b23.x, b23.y}, {b23.z, b23.w}};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    acc[i][q] = __dp4a(au[i][0], bv[q][0], acc[i][q]);
                    acc[i][q] = __dp4a(au[i][1], bv[q][1], acc[i][q]);
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int u = tu * CM_T + ty * 4 + i;
        if (u >= D) continue;
        const int e = u / C, c = u - e * C;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int v = tv * CM_T + tx * 4 + q;
            if (v >= D || acc[i][q] == 0u) continue;
            const int e2 = v / C, c2 = v - e2 * C;
            atomicAdd(out + ((((size_t)which * PS + e) * PS + e2) * C + c) * C + c2, (unsigned long long)acc[i][q]);
            if (!diag)
                atomicAdd(out + ((((size_t)which * PS + e2) * PS + e) * C + c2) * C + c, (unsigned long long)acc[i][q]);
        }
    }
}

// Row and column moments from the full second moment M (entry u = a*8C + b*C + c of the packed
// patch; lower triangle u >= v filled): R[a][a'][c][c'] = sum_b M[(a,b,c)][(a',b,c')] and
// Q[b][b'][c][c'] = sum_a M[(a,b,c)][(a,b',c')]. Integer sums, so the result equals the direct
// moments exactly. One thread per entry, written (not added) in the layout of moments_chunk.
template <int C>
__global__ void __launch_bounds__(256) moments_from_full_kernel(const unsigned long long* __restrict__ M,
                                                                unsigned long long* __restrict__ out) {
    constexpr int d = PS2 * C;
    constexpr int NE = 2 * PS * PS * C * C;
    const int ent = blockIdx.x * blockDim.x + threadIdx.x;
    if (ent >= NE) return;
    const int which = ent / (PS * PS * C * C);
    int rem = ent - which * PS * PS * C * C;
    const int u = rem / (PS * C * C);
    rem -= u * PS * C * C;
    const int v = rem / (C * C);
    rem -= v * C * C;
    const int c = rem / C, c2 = rem - c * C;
    unsigned long long sum = 0;
#pragma unroll
    for (int t = 0; t < PS; ++t) {
        // which 0: rows (a, a') = (u, v), summed over the column t; which 1: columns (b, b') = (u, v), over the row t
        const int i = which == 0 ? u * PS * C + t * C + c : t * PS * C + u * C + c;
        const int j = which == 0 ? v * PS * C + t * C + c2 : t * PS * C + v * C + c2;
        sum += i >= j ? M[(size_t)i * d + j] : M[(size_t)j * d + i];
    }
    out[ent] = sum;
}

// Full second moment: CTA (bx, tile) accumulates a 64x64 tile of M over a chunk of references.
// The patch values of 4 consecutive references are packed per 32-bit word ([u][ref/4]), so one
// dp4a adds the products of 4 references; each thread owns a 4x4 block of the tile. M is
// symmetric: only the tiles on and below the diagonal (tu >= tv) are formed, and readers use the
// lower triangle u >= v.
constexpr int FM_CHUNK_MAX = 16384;    // references per CTA at most (16384 * 255^2 < 2^32)
constexpr int FM_BATCH = 64;           // references staged at once
constexpr int FM_WPAD = FM_BATCH / 4 + 1;

template <int C>
__global__ void __launch_bounds__(256) full_moment_kernel(const uint8_t* __restrict__ img, Geo g, int chunk,
                                                          unsigned long long* __restrict__ M,
                                                          unsigned long long* __restrict__ S) {
    constexpr int d = PS2 * C;
    constexpr int ROWB = PS * C;                 // bytes of one patch row
    int tu = 0, tv = blockIdx.y;                 // blockIdx.y -> (tu, tv), tu >= tv, row-major
    while (tv > tu) {
        tv -= tu + 1;
        ++tu;
    }
    __shared__ uint32_t pk[3 * PS2][FM_WPAD];
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
    uint32_t acc[4][4] = {};
    uint32_t sacc = 0;
    const int N = g.ngroups();
    const int r0 = blockIdx.x * chunk, r1 = min(r0 + chunk, N);
    for (int rb = r0; rb < r1; rb += FM_BATCH) {
        const int nb = min(FM_BATCH, r1 - rb);
        __syncthreads();
        // Task (quad jq, patch row i, part h): the part's HB bytes of row i of references 4jq..4jq+3
        // (contiguous in the image) are read as aligned 32-bit words, shifted into place, and
        // transposed 4 x 4 so that word (u, jq) holds byte u of the four references. Only rows that
        // meet this CTA's two 64-row blocks are staged (the others are never read here).
        {
            constexpr int HB = ROWB / 2;              // bytes per part: 12 (C = 3) or 4 (C = 1)
            constexpr int NWD = HB / 4;               // whole words per part
            const int t = threadIdx.x;
            const int h = t & 1, i = (t >> 1) & 7, jq = t >> 4;
            const int u0 = i * ROWB + h * HB;
            const bool need = (u0 < tu * 64 + 64 && u0 + HB > tu * 64) || (u0 < tv * 64 + 64 && u0 + HB > tv * 64);
            if (jq < FM_BATCH / 4 && need) {
                uint32_t al[4][NWD];                  // [reference][word] aligned row bytes
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = jq * 4 + q;
#pragma unroll
                    for (int wd = 0; wd < NWD; ++wd) al[q][wd] = 0u;
                    if (j < nb) {
                        const int r = rb + j;
                        const int iy = r / g.nrx, ix = r - iy * g.nrx;
                        const int ry = ref_pos(iy, g.s, g.H), rx = ref_pos(ix, g.s, g.W);
                        // alignment from the absolute address: the image may start at any byte
                        const uintptr_t a = reinterpret_cast<uintptr_t>(img + ((size_t)(ry + i) * g.W + rx) * C + h * HB);
                        const int o = (int)(a & 3);
                        // every word read holds at least one byte of the part, so none leaves the image's
                        // aligned words
                        const uint32_t* w = reinterpret_cast<const uint32_t*>(a - o);
                        uint32_t wv[NWD + 1];
#pragma unroll
                        for (int wd = 0; wd < NWD; ++wd) wv[wd] = w[wd];
                        // the word after the part holds needed bytes only when the part is unaligned
                        wv[NWD] = o ? w[NWD] : 0u;
#pragma unroll
                        for (int wd = 0; wd < NWD; ++wd) al[q][wd] = __funnelshift_r(wv[wd], wv[wd + 1], 8 * o);
                    }
                }
#pragma unroll
                for (int wd = 0; wd < NWD; ++wd) {
                    const uint32_t lo01 = __byte_perm(al[0][wd], al[1][wd], 0x5140u);
                    const uint32_t hi01 = __byte_perm(al[0][wd], al[1][wd], 0x7362u);
                    const uint32_t lo23 = __byte_perm(al[2][wd], al[3][wd], 0x5140u);
                    const uint32_t hi23 = __byte_perm(al[2][wd], al[3][wd], 0x7362u);
                    const int u = u0 + wd * 4;
                    pk[u + 0][jq] = __byte_perm(lo01, lo23, 0x5410u);
                    pk[u + 1][jq] = __byte_perm(lo01, lo23, 0x7632u);
                    pk[u + 2][jq] = __byte_perm(hi01, hi23, 0x5410u);
                    pk[u + 3][jq] = __byte_perm(hi01, hi23, 0x7632u);
                }
            }
        }
        __syncthreads();
        const int nw = (nb + 3) >> 2;
        for (int jw = 0; jw < nw; ++jw) {
            uint32_t au[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int u = tu * 64 + ty * 4 + q, v = tv * 64 + tx * 4 + q;
                au[q] = u < d ? pk[u][jw] : 0u;
                bv[q] = v < d ? pk[v][jw] : 0u;
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = __dp4a(au[p], bv[q], acc[p][q]);
        }
        if (tv == 0 && threadIdx.x < 64) {
            const int u = tu * 64 + threadIdx.x;
            if (u < d)
                for (int jw = 0; jw < nw; ++jw) sacc = __dp4a(pk[u][jw], 0x01010101u, sacc);
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int u = tu * 64 + ty * 4 + p, v = tv * 64 + tx * 4 + q;
            if (u < d && v < d && acc[p][q]) atomicAdd(M + (size_t)u * d + v, (unsigned long long)acc[p][q]);
        }
    if (tv == 0 && threadIdx.x < 64) {
        const int u = tu * 64 + threadIdx.x;
        if (u < d && sacc) atomicAdd(S + u, (unsigned long long)sacc);
    }
}

// ----------------------------------------------------------------------------- FP64 Hermitian eigensolver

// Cyclic complex Jacobi on an 8x8 Hermitian matrix held as separate real and imaginary
// parts: each rotation first makes the pivot real with a diagonal phase e = a_pq/|a_pq|,
// then applies a real Jacobi rotation (c, s), i.e. A <- J^H A J with
// J[:,p] = c e_p - s conj(e) e_q and J[:,q] = s e_p + c conj(e) e_q.
// On exit the diagonal of (Ar, Ai) holds the eigenvalues and (Vr, Vi) the eigenvectors (columns).
__host__ __device__ void jacobi_herm8(double (*Ar)[PS], double (*Ai)[PS], double (*Vr)[PS], double (*Vi)[PS]) {
    for (int i = 0; i < PS; ++i)
        for (int j = 0; j < PS; ++j) {
            Vr[i][j] = i == j ? 1.0 : 0.0;
            Vi[i][j] = 0.0;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = 0; i < PS; ++i) {
            dia += Ar[i][i] * Ar[i][i];
            for (int j = i + 1; j < PS; ++j) off += Ar[i][j] * Ar[i][j] + Ai[i][j] * Ai[i][j];
        }
        if (off <= 1e-32 * dia || off == 0.0) break;
        for (int p = 0; p < PS - 1; ++p)
            for (int q = p + 1; q < PS; ++q) {
                const double xr = Ar[p][q], xi = Ai[p][q];
                const double r = sqrt(xr * xr + xi * xi);
                const double app = Ar[p][p], aqq = Ar[q][q];
                if (r == 0.0 || r < 1e-17 * sqrt(fabs(app * aqq))) {
                    Ar[p][q] = Ai[p][q] = Ar[q][p] = Ai[q][p] = 0.0;
                    continue;
                }
                const double er = xr / r, ei = xi / r;            // e = a_pq / |a_pq|
                const double th = (aqq - app) / (2.0 * r);
                double t;
                if (fabs(th) > 1e150) t = 0.5 / th;
                else t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                // columns p, q: a_kp <- c a_kp - s conj(e) a_kq ; a_kq <- s a_kp + c conj(e) a_kq
                for (int k = 0; k < PS; ++k) {
                    const double pr = Ar[k][p], pi = Ai[k][p], qr = Ar[k][q], qi = Ai[k][q];
                    const double mr = er * qr + ei * qi, mi = er * qi - ei * qr;     // conj(e) a_kq
                    Ar[k][p] = c * pr - sn * mr;
                    Ai[k][p] = c * pi - sn * mi;
                    Ar[k][q] = sn * pr + c * mr;
                    Ai[k][q] = sn * pi + c * mi;
                }
                // rows p, q: a_pk <- c a_pk - s e a_qk ; a_qk <- s a_pk + c e a_qk
                for (int k = 0; k < PS; ++k) {
                    const double pr = Ar[p][k], pi = Ai[p][k], qr = Ar[q][k], qi = Ai[q][k];
                    const double mr = er * qr - ei * qi, mi = er * qi + ei * qr;     // e a_qk
                    Ar[p][k] = c * pr - sn * mr;
                    Ai[p][k] = c * pi - sn * mi;
                    Ar[q][k] = sn * pr + c * mr;
                    Ai[q][k] = sn * pi + c * mi;
                }
                Ar[p][p] = app - t * r;
                Ar[q][q] = aqq + t * r;
                Ai[p][p] = Ai[q][q] = 0.0;
                Ar[p][q] = Ai[p][q] = Ar[q][p] = Ai[q][p] = 0.0;
                for (int k = 0; k < PS; ++k) {
                    const double pr = Vr[k][p], pi = Vi[k][p], qr = Vr[k][q], qi = Vi[k][q];
                    const double mr = er * qr + ei * qi, mi = er * qi - ei * qr;     // conj(e) v_kq
                    Vr[k][p] = c * pr - sn * mr;
                    Vi[k][p] = c * pi - sn * mi;
                    Vr[k][q] = sn * pr + c * mr;
                    Vi[k][q] = sn * pi + c * mi;
                }
            }
    }
}

// Eigenvalues descending; each eigenvector scaled so that its largest-modulus entry
// (lowest index within 1e-6 relative) is real and positive. Out[a][col] = (re, im).
__host__ __device__ void canonicalise(double (*Ar)[PS], double (*Vr)[PS], double (*Vi)[PS], double (*Out)[PS][2]) {
    int order[PS];
    for (int i = 0; i < PS; ++i) order[i] = i;
    for (int i = 0; i < PS; ++i)          // selection sort, descending, ties keep the lower index first
        for (int j = i + 1; j < PS; ++j)
            if (Ar[order[j]][order[j]] > Ar[order[i]][order[i]]) {
                const int t = order[i];
                order[i] = order[j];
                order[j] = t;
            }
    for (int col = 0; col < PS; ++col) {
        const int src = order[col];
        double mod[PS], mx = 0.0;
        for (int a = 0; a < PS; ++a) {
            mod[a] = sqrt(Vr[a][src] * Vr[a][src] + Vi[a][src] * Vi[a][src]);
            mx = fmax(mx, mod[a]);
        }
        int as = 0;
        for (int a = 0; a < PS; ++a)
            if (mod[a] >= mx * (1.0 - 1e-6)) {
                as = a;
                break;
            }
        const double hr = Vr[as][src] / mod[as], hi = -Vi[as][src] / mod[as];     // conj(v_a) / |v_a|
        for (int a = 0; a < PS; ++a) {
            Out[a][col][0] = Vr[a][src] * hr - Vi[a][src] * hi;
            Out[a][col][1] = Vr[a][src] * hi + Vi[a][src] * hr;
        }
        Out[as][col][1] = 0.0;
    }
}

// Device form of canonicalise for one warp: lane 0 orders the eigenvalues (the same selection
// sort), then lane c < 8 treats output column c. The largest-modulus entry is found on squared
// moduli and the phase takes one reciprocal square root (FP64 square root and division are long
// sequences on this GPU).
__device__ void canonicalise_warp(double (*Ar)[PS], double (*Vr)[PS], double (*Vi)[PS], double (*Out)[PS][2],
                                  int* order, int lane) {
    if (lane == 0) {
        for (int i = 0; i < PS; ++i) order[i] = i;
        for (int i = 0; i < PS; ++i)          // selection sort, descending, as in canonicalise
            for (int j = i + 1; j < PS; ++j)
                if (Ar[order[j]][order[j]] > Ar[order[i]][order[i]]) {
                    const int t = order[i];
                    order[i] = order[j];
                    order[j] = t;
                }
    }
    __syncwarp();
    if (lane < PS) {
        const int col = lane, src = order[col];
        double mod2[PS], mx2 = 0.0;
#pragma unroll
        for (int a = 0; a < PS; ++a) {
            mod2[a] = Vr[a][src] * Vr[a][src] + Vi[a][src] * Vi[a][src];
            mx2 = fmax(mx2, mod2[a]);
        }
        const double lim = mx2 * ((1.0 - 1e-6) * (1.0 - 1e-6));   // |v_a| >= (1 - 1e-6) max |v|
        int as = PS - 1;
#pragma unroll
        for (int a = PS - 1; a >= 0; --a)
            if (mod2[a] >= lim) as = a;
        const double inv = rsqrt(mod2[as]);
        const double hr = Vr[as][src] * inv, hi = -Vi[as][src] * inv;     // conj(v_a) / |v_a|
#pragma unroll
        for (int a = 0; a < PS; ++a) {
            Out[a][col][0] = Vr[a][src] * hr - Vi[a][src] * hi;
            Out[a][col][1] = Vr[a][src] * hi + Vi[a][src] * hr;
        }
        Out[as][col][1] = 0.0;
    }
    __syncwarp();
}

// Scatter matrix of slice f from the integer moments (rows: which = 0, columns: which = 1),
// then its canonical eigenvectors.
// work: 4 * PS * PS doubles of scratch (Ar, Ai, Vr, Vi).
__host__ __device__ void slice_basis(const unsigned long long* mom, int C, int which, int f, double* work,
                                     double (*Out)[PS][2]) {
    double (*Ar)[PS] = reinterpret_cast<double (*)[PS]>(work);
    double (*Ai)[PS] = reinterpret_cast<double (*)[PS]>(work + PS2);
    double (*Vr)[PS] = reinterpret_cast<double (*)[PS]>(work + 2 * PS2);
    double (*Vi)[PS] = reinterpret_cast<double (*)[PS]>(work + 3 * PS2);
    const unsigned long long* M = mom + (size_t)which * PS * PS * C * C;
    const double s32 = 0.5 * sqrt(3.0);
    for (int u = 0; u < PS; ++u)
        for (int v = 0; v < PS; ++v) {
            double accr = 0.0, acci = 0.0;
            for (int c = 0; c < C; ++c)
                for (int c2 = 0; c2 < C; ++c2) {
                    const double m = (double)M[((u * PS + v) * C + c) * C + c2];
                    // phase w^{f d}, d = c - c2 for rows and c2 - c for columns, w = exp(-2 pi i / C)
                    const int d = which == 0 ? (c - c2) : (c2 - c);
                    const int k = ((f * d) % C + C) % C;
                    double phr = 1.0, phi = 0.0;
                    if (C == 3 && k == 1) { phr = -0.5; phi = -s32; }
                    if (C == 3 && k == 2) { phr = -0.5; phi = s32; }
                    accr += m * phr;
                    acci += m * phi;
                }
            Ar[u][v] = accr;
            Ai[u][v] = u == v ? 0.0 : acci;
        }
    jacobi_herm8(Ar, Ai, Vr, Vi);
    canonicalise(Ar, Vr, Vi, Out);
}

// Device form of the solver: parallel (round-robin) Jacobi. Each sweep runs 7 rounds of 4
// rotations on disjoint index pairs (circle schedule: pairs (p[i], p[7-i]) with p a rotation of
// 1..7 around 0), so the FP64 latency chain per sweep is 7 rotations deep instead of 28.
// Lane i < 4 computes rotation i of a round; lane 8i + k applies it to row/column k.
// The 2x2 block of a pair is touched only by its own rotation, so each rotation zeroes its pivot
// exactly as the cyclic solver's would.
// rot: [5][10] shared scratch: rows 0..3 the rotations of a round
// (er, ei, c, s, t*r, skip, p, q, a_pp, a_qq), row 4 the convergence flag.
__device__ void jacobi_herm8_warp(double (*Ar)[PS], double (*Ai)[PS], double (*Vr)[PS], double (*Vi)[PS],
                                  double (*rot)[10], int lane) {
    if (lane < PS)
        for (int j = 0; j < PS; ++j) {
            Vr[lane][j] = lane == j ? 1.0 : 0.0;
            Vi[lane][j] = 0.0;
        }
    __syncwarp();
    const int pr_i = lane >> 3, k = lane & 7;          // rotation of this lane, row/column it updates
    // lane l < 28 holds the off-diagonal pair (oi, oj), oi < oj, of the convergence test
    int oi = 0, oj = 0;
    if (lane < PS * (PS - 1) / 2) {
        int rem = lane;
        while (rem >= PS - 1 - oi) {
            rem -= PS - 1 - oi;
            ++oi;
        }
        oj = oi + 1 + rem;
    }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = lane < PS * (PS - 1) / 2 ? Ar[oi][oj] * Ar[oi][oj] + Ai[oi][oj] * Ai[oi][oj] : 0.0;
        double dia = lane < PS ? Ar[lane][lane] * Ar[lane][lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if (off <= 1e-32 * dia || off == 0.0) break;      // same value in every lane
        __syncwarp();
        for (int r = 0; r < PS - 1; ++r) {
            // pair of rotation i in round r
            auto at = [r](int j) { return j == 0 ? 0 : 1 + ((j - 1 + r) % (PS - 1)); };
            if (lane < 4) {
                int p = at(lane), q = at(PS - 1 - lane);
                if (p > q) { const int t = p; p = q; q = t; }
                const double xr = Ar[p][q], xi = Ai[p][q];
                const double r2 = xr * xr + xi * xi;
                const double app = Ar[p][p], aqq = Ar[q][q];
                double* R = rot[lane];
                R[6] = p;
                R[7] = q;
                R[8] = app;
                R[9] = aqq;
                // FP64 division and square root are long sequences on this GPU: |a_pq|, its phase and
                // theta share one reciprocal square root, c takes another
                if (r2 == 0.0 || r2 < 1e-34 * fabs(app * aqq)) {
                    R[5] = 1.0;
                } else {
                    const double ir = rsqrt(r2), rr = r2 * ir;
                    const double th = 0.5 * (aqq - app) * ir;
                    double t;
                    if (fabs(th) > 1e150) t = 0.5 / th;
                    else t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                    const double c = rsqrt(t * t + 1.0);
                    R[0] = xr * ir;
                    R[1] = xi * ir;
                    R[2] = c;
                    R[3] = t * c;
                    R[4] = t * rr;
                    R[5] = 0.0;
                }
            }
            __syncwarp();
            const double* R = rot[pr_i];
            const bool skip = R[5] != 0.0;
            const int p = (int)R[6], q = (int)R[7];
            const double er = R[0], ei = R[1], c = R[2], sn = R[3];
            if (!skip) {     // columns p, q: a_kp <- c a_kp - s conj(e) a_kq ; a_kq <- s a_kp + c conj(e) a_kq
                const double pr = Ar[k][p], pi = Ai[k][p], qr = Ar[k][q], qi = Ai[k][q];
                const double mr = er * qr + ei * qi, mi = er * qi - ei * qr;
                Ar[k][p] = c * pr - sn * mr;
                Ai[k][p] = c * pi - sn * mi;
                Ar[k][q] = sn * pr + c * mr;
                Ai[k][q] = sn * pi + c * mi;
            }
            __syncwarp();
            if (!skip) {     // rows p, q: a_pk <- c a_pk - s e a_qk ; a_qk <- s a_pk + c e a_qk ; and V
                const double pr = Ar[p][k], pi = Ai[p][k], qr = Ar[q][k], qi = Ai[q][k];
                const double mr = er * qr - ei * qi, mi = er * qi + ei * qr;
                Ar[p][k] = c * pr - sn * mr;
                Ai[p][k] = c * pi - sn * mi;
                Ar[q][k] = sn * pr + c * mr;
                Ai[q][k] = sn * pi + c * mi;
                const double vpr = Vr[k][p], vpi = Vi[k][p], vqr = Vr[k][q], vqi = Vi[k][q];
                const double nr = er * vqr + ei * vqi, ni = er * vqi - ei * vqr;
                Vr[k][p] = c * vpr - sn * nr;
                Vi[k][p] = c * vpi - sn * ni;
                Vr[k][q] = sn * vpr + c * nr;
                Vi[k][q] = sn * vpi + c * ni;
            }
            __syncwarp();
            if (lane < 4) {
                // the rotated 2x2 block: diagonal a_pp - t r, a_qq + t r (a_pp, a_qq before the round), zero pivot
                const double* Rl = rot[lane];
                const int pl = (int)Rl[6], ql = (int)Rl[7];
                if (Rl[5] == 0.0) {
                    Ar[pl][pl] = Rl[8] - Rl[4];
                    Ar[ql][ql] = Rl[9] + Rl[4];
                    Ai[pl][pl] = Ai[ql][ql] = 0.0;
                }
                Ar[pl][ql] = Ai[pl][ql] = Ar[ql][pl] = Ai[ql][pl] = 0.0;
            }
            __syncwarp();
        }
    }
}

// One warp per (U or V, slice f) problem w, f = 0 .. C/2; writes its slice of the outputs.
__device__ __forceinline__ void basis_problem(const unsigned long long* __restrict__ mom, int C, int w,
                                              double* __restrict__ b64, float* __restrict__ b32,
                                              double* __restrict__ gap_out) {
    __shared__ double Res[PS][PS][2];
    __shared__ double work[4 * PS2];
    __shared__ double rot[5][10];
    const int nf = C / 2 + 1;
    const int lane = threadIdx.x & 31;
    const int which = w / nf, f = w % nf;
    double (*Ar)[PS] = reinterpret_cast<double (*)[PS]>(work);
    double (*Ai)[PS] = reinterpret_cast<double (*)[PS]>(work + PS2);
    double (*Vr)[PS] = reinterpret_cast<double (*)[PS]>(work + 2 * PS2);
    double (*Vi)[PS] = reinterpret_cast<double (*)[PS]>(work + 3 * PS2);
    const unsigned long long* M = mom + (size_t)which * PS * PS * C * C;
    // w^k, w = exp(-2 pi i / C), k < C: exact constants for C = 3, the library's cospi / sinpi otherwise
    __shared__ double phr[64], phi[64];
    for (int k = lane; k < C; k += 32) {
        double cr = 1.0, ci = 0.0;
        if (C == 3) {
            const double s32 = 0.5 * sqrt(3.0);
            if (k == 1) { cr = -0.5; ci = -s32; }
            if (k == 2) { cr = -0.5; ci = s32; }
        } else if (k != 0) {
            double sn, cs;
            sincospi(2.0 * k / C, &sn, &cs);
            cr = cs;
            ci = -sn;
        }
        phr[k] = cr;
        phi[k] = ci;
    }
    __syncwarp();
    // A_f[u][v] = sum_{c, c2} M[u v][c][c2] w^{f (c - c2)} (U) or w^{f (c2 - c)} (V): the moments of one
    // band difference d = c - c2 (mod C) share the phase, so they are summed first, exactly in
    // integers, and each difference takes one complex product
    for (int e = lane; e < PS2; e += 32) {
        const int u = e / PS, v = e % PS;
        const unsigned long long* Me = M + (size_t)(u * PS + v) * C * C;
        double accr = 0.0, acci = 0.0;
        for (int d = 0; d < C; ++d) {
            unsigned long long sd = 0;
            for (int c = 0, c2 = C - d; c < C; ++c, ++c2) {
                if (c2 >= C) c2 -= C;                        // c2 = (c - d) mod C
                sd += Me[c * C + c2];
            }
            const int dd = which == 0 ? d : (C - d) % C;
            const int k = (f * dd) % C;
            accr += (double)sd * phr[k];
            acci += (double)sd * phi[k];
        }
        Ar[u][v] = accr;
        Ai[u][v] = u == v ? 0.0 : acci;
    }
    __syncwarp();
    jacobi_herm8_warp(Ar, Ai, Vr, Vi, rot, lane);
    __shared__ int order[PS];
    canonicalise_warp(Ar, Vr, Vi, Res, order, lane);
    if (gap_out && lane == 0) {
        // smallest gap between consecutive eigenvalues (descending order) relative to the largest
        double gmin = fabs(Ar[order[0]][order[0]] - Ar[order[1]][order[1]]);
        for (int i = 1; i + 1 < PS; ++i) gmin = fmin(gmin, fabs(Ar[order[i]][order[i]] - Ar[order[i + 1]][order[i + 1]]));
        gap_out[w] = gmin / fmax(fabs(Ar[order[0]][order[0]]), 1e-300);
    }
    // FP64 slice f (and its conjugate slice C - f) of U or V, and the packed FP32 copy used by the filter.
    for (int ai = lane; ai < PS2; ai += 32) {
        const double re = Res[ai / PS][ai % PS][0], im = Res[ai / PS][ai % PS][1];
        double* o = b64 + 2 * ((size_t)(which * C + f) * PS2 + ai);
        o[0] = re;
        o[1] = im;
        if (f != 0 && C - f != f) {
            double* oc = b64 + 2 * ((size_t)(which * C + (C - f)) * PS2 + ai);
            oc[0] = re;
            oc[1] = -im;
        }
        if (C == 1 || C == 3) {
            const int per = (C == 3) ? 3 * PS2 : PS2;
            float* o32 = b32 + which * per;
            if (f == 0) o32[ai] = (float)re;
            else {
                o32[PS2 + ai] = (float)re;
                o32[2 * PS2 + ai] = (float)im;
            }
        } else {                                    // cubes: [which][f][re, im][a][i]
            float* o32 = b32 + ((size_t)which * nf + f) * 2 * PS2;
            o32[ai] = (float)re;
            o32[PS2 + ai] = (float)im;
        }
    }
}

__global__ void basis_kernel(const unsigned long long* __restrict__ mom, int C, double* __restrict__ b64,
                             float* __restrict__ b32, double* __restrict__ gap) {
    basis_problem(mom, C, blockIdx.x, b64, b32, gap);
}

// Batch form: block b -> image b / (2 (C/2 + 1)), problem b % (2 (C/2 + 1)).
__global__ void basis_batch_kernel(const FilterArgs* __restrict__ fargs, unsigned long long* const* __restrict__ moms,
                                   int C) {
    const int np = 2 * (C / 2 + 1);
    const int i = blockIdx.x / np;
    const FilterArgs& a = fargs[i];
    basis_problem(moms[i], C, blockIdx.x % np, const_cast<double*>(a.basis64), const_cast<float*>(a.basis32), nullptr);
}

__global__ void quantize_kernel(const float* __restrict__ x, int64_t n, uint8_t* __restrict__ q) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float v = rintf(x[i]);
        v = fminf(fmaxf(v, 0.0f), 255.0f);
        q[i] = (uint8_t)v;
    }
}

// lambda_f = || sum_m p_m exp(-2 pi i f m / K) ||^2 over the full-channel patch vectors of a
// group (the eigenvalues of circ(G) circ(G)^T), then the rank of lambda_{K/2}. FP64, one CTA per group.
// Rank of lambda_{K/2} among the circulant eigenvalues lambda_f = sum_u |sum_m p_m[u] w^{-fm}|^2
// of one sampled group (Sec. III-D; the group is real, so lambda_{K-f} = lambda_f and only
// f = 0 .. K/2 are formed). lambda_{K/2} = sum_u (sum_m (-1)^m p_m[u])^2 is an exact integer. The
// others are formed in FP32 together with an absolute error bound, and any lambda_f whose bound
// reaches lambda_{K/2} is recomputed in FP64 before the comparison.
__global__ void __launch_bounds__(256) group_rank_kernel(const uint8_t* __restrict__ img, Geo g,
                                                         const int32_t* __restrict__ idx,
                                                         int32_t* __restrict__ ranks) {
    const int grp = blockIdx.x;
    const int K = g.K;
    const int d = PS2 * g.C;
    const int NFQ = K / 2 + 1;                  // f = 0 .. K/2
    __shared__ uint8_t pv[32][3 * PS2];
    __shared__ float tcf[32], tsf[32];
    __shared__ float lam32[17], bnd[17];
    __shared__ unsigned long long half_sq;
    __shared__ double lam64, tc64[32], ts64[32];
    for (int t = threadIdx.x; t < K * d; t += blockDim.x) {
        const int m = t / d, u = t - m * d;
        const int pix = u / g.C, c = u - pix * g.C;
        const int v = idx[(size_t)grp * K + m];
        const int y = v / g.W, x = v - y * g.W;
        pv[m][u] = img[((size_t)(y + pix / PS) * g.W + x + pix % PS) * g.C + c];
    }
    if (threadIdx.x < K) {
        float sn, cs;
        sincospif(-2.0f * threadIdx.x / K, &sn, &cs);
        tcf[threadIdx.x] = cs;
        tsf[threadIdx.x] = sn;
    }
    if (threadIdx.x < NFQ) lam32[threadIdx.x] = bnd[threadIdx.x] = 0.f;
    if (threadIdx.x == 0) half_sq = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // exact lambda_{K/2}
    {
        unsigned long long acc = 0ull;
        for (int u = threadIdx.x; u < d; u += blockDim.x) {
            int a = 0;
            for (int m = 0; m < K; ++m) a += (m & 1) ? -(int)pv[m][u] : (int)pv[m][u];
            acc += (unsigned long long)((long long)a * a);
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0 && acc) atomicAdd(&half_sq, acc);
    }
    // FP32 lambda_f, f < K/2, and a bound on its error: |X| <= 255 K per entry, each of the K
    // products and sums rounds by at most 2^-24 of that and the twiddle by 2^-24 of 255, so each
    // of Re, Im is off by at most e = 2 K 255 K 2^-24; |X|^2 then by 2 sqrt(2) e |X| + 2 e^2.
    // thread t: frequency t % (K/2), entries u = t / (K/2), + 256/(K/2), ... (partial sums per thread,
    // one shared atomic per thread and frequency)
    {
        const float e = 2.f * K * 255.f * K * 5.9604645e-8f;
        const int nf = NFQ - 1, f = threadIdx.x % nf, u0 = threadIdx.x / nf, du = blockDim.x / nf;
        float lsum = 0.f, bsum = 0.f;
        if (u0 < du)
            for (int u = u0; u < d; u += du) {
                float re = 0.f, im = 0.f;
                for (int m = 0; m < K; ++m) {
                    const int k = (f * m) & (K - 1);
                    re = fmaf((float)pv[m][u], tcf[k], re);
                    im = fmaf((float)pv[m][u], tsf[k], im);
                }
                const float mag2 = re * re + im * im;
                lsum += mag2;
                bsum += 2.8284272f * e * sqrtf(mag2) + 2.f * e * e + 1e-6f * mag2;
            }
        if (u0 < du) {
            atomicAdd(&lam32[f], lsum);
            atomicAdd(&bnd[f], bsum);
        }
    }
    if (threadIdx.x < K) sincospi(-2.0 * threadIdx.x / K, &ts64[threadIdx.x], &tc64[threadIdx.x]);
    __syncthreads();
    const double lh = (double)half_sq;
    // count lambda_f < lambda_{K/2} over all K frequencies (f and K - f count twice)
    int a = 1;
    for (int f = 0; f < NFQ - 1; ++f) {
        const int mult = (f == 0) ? 1 : 2;
        // summing the (positive) terms of lambda_f in FP32 adds at most 2^-24 relative per term:
        // 3e-5 covers the 192 terms with room to spare
        const double l32 = (double)lam32[f], b = 2.0 * (double)bnd[f] + 3e-5 * fabs(l32);
        if (l32 + b < lh) {
            a += mult;
        } else if (l32 - b < lh) {
            // too close to decide in FP32: lambda_f in FP64
            if (threadIdx.x == 0) lam64 = 0.0;
            __syncthreads();
            double part = 0.0;
            for (int u = threadIdx.x; u < d; u += blockDim.x) {
                double re = 0.0, im = 0.0;
                for (int m = 0; m < K; ++m) {
                    const int k = (f * m) & (K - 1);
                    re += pv[m][u] * tc64[k];
                    im += pv[m][u] * ts64[k];
                }
                part += re * re + im * im;
            }
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (lane == 0 && part != 0.0) atomicAdd(&lam64, part);
            __syncthreads();
            if (lam64 < lh) a += mult;
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) ranks[grp] = a;
}

}  // namespace

// Host copy of the per-slice basis computation (used by the CPU tests of the eigensolver).
extern "C" void htsvd_internal_slice_basis(const unsigned long long* mom, int C, int which, int f, double* out) {
    double R[PS][PS][2], work[4 * PS2];
    slice_basis(mom, C, which, f, work, R);
    for (int a = 0; a < PS2; ++a) {
        out[2 * a] = R[a / PS][a % PS][0];
        out[2 * a + 1] = R[a / PS][a % PS][1];
    }
}

// Internal hooks for device-side checks of the moments and the basis solve.
extern "C" int htsvd_internal_moments(const uint8_t* d_img, int H, int W, int C, int stride,
                                      unsigned long long* d_mom) {
    Geo g = make_geo(H, W, C, stride, 8, 2);
    if (launch_moments(d_img, g, d_mom, 0) != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}
extern "C" int htsvd_internal_basis(const unsigned long long* d_mom, int C, double* d_b64, float* d_b32) {
    if (launch_basis(d_mom, C, d_b64, d_b32, 0) != cudaSuccess) return 1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : 1;
}

cudaError_t launch_moments(const uint8_t* img, const Geo& g, unsigned long long* d_mom, cudaStream_t s) {
    const int n = g.ngroups();
    const int blocks = (n + MOM_CHUNK - 1) / MOM_CHUNK;
    cudaError_t e = cudaMemsetAsync(d_mom, 0, sizeof(unsigned long long) * 2 * PS2 * g.C * g.C, s);
    if (e != cudaSuccess) return e;
    if (g.C == 3) moments_kernel<3><<<blocks, 256, 0, s>>>(img, g, d_mom);
    else moments_kernel<1><<<blocks, 256, 0, s>>>(img, g, d_mom);
    return cudaGetLastError();
}

int moments_chunks(const Geo& g) { return (g.ngroups() + MOM_CHUNK - 1) / MOM_CHUNK; }

cudaError_t launch_moments_batch(int C, const BMArgs* d_args, unsigned long long* const* d_moms, const int* d_prefix,
                                 int nimg, int grid, cudaStream_t s) {
    if (C == 3) moments_batch_kernel<3><<<grid, 256, 0, s>>>(d_args, d_moms, d_prefix, nimg);
    else moments_batch_kernel<1><<<grid, 256, 0, s>>>(d_args, d_moms, d_prefix, nimg);
    return cudaGetLastError();
}

cudaError_t launch_basis_batch(int C, const FilterArgs* d_fargs, unsigned long long* const* d_moms, int nimg,
                               cudaStream_t s) {
    basis_batch_kernel<<<nimg * 2 * (C / 2 + 1), 32, 0, s>>>(d_fargs, d_moms, C);
    return cudaGetLastError();
}

cudaError_t launch_moments_from_full(const unsigned long long* d_M, int C, unsigned long long* d_mom, cudaStream_t s) {
    const int ne = 2 * PS2 * C * C;
    if (C == 3) moments_from_full_kernel<3><<<(ne + 255) / 256, 256, 0, s>>>(d_M, d_mom);
    else moments_from_full_kernel<1><<<(ne + 255) / 256, 256, 0, s>>>(d_M, d_mom);
    return cudaGetLastError();
}

cudaError_t launch_full_moment(const uint8_t* img, const Geo& g, unsigned long long* d_M, unsigned long long* d_s,
                               cudaStream_t s) {
    const int d = PS2 * g.C;
    cudaError_t e = cudaMemsetAsync(d_M, 0, sizeof(unsigned long long) * d * d, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_s, 0, sizeof(unsigned long long) * d, s);
    if (e != cudaSuccess) return e;
    const int n = g.ngroups();
    const int nt = (d + 63) / 64;
    const int ntiles = nt * (nt + 1) / 2;                       // tiles on and below the diagonal
    // chunks of whole staging batches, about four CTAs per SM in total
    int nchunk = (4 * device_sm_count() + ntiles - 1) / ntiles;
    const int nbatch = (n + FM_BATCH - 1) / FM_BATCH;
    if (nchunk > nbatch) nchunk = nbatch;
    int chunk = (nbatch + nchunk - 1) / nchunk * FM_BATCH;
    if (chunk > FM_CHUNK_MAX) chunk = FM_CHUNK_MAX;
    dim3 grid((n + chunk - 1) / chunk, ntiles);
    if (g.C == 3) full_moment_kernel<3><<<grid, 256, 0, s>>>(img, g, chunk, d_M, d_s);
    else full_moment_kernel<1><<<grid, 256, 0, s>>>(img, g, chunk, d_M, d_s);
    return cudaGetLastError();
}

cudaError_t launch_cube_moments(const uint8_t* img, const Geo& g, unsigned long long* d_mom, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(d_mom, 0, sizeof(unsigned long long) * 2 * PS2 * g.C * g.C, s);
    if (e != cudaSuccess) return e;
    const int ntile = (PS * g.C + CM_T - 1) / CM_T;
    dim3 grid(2 * (ntile * (ntile + 1) / 2), (g.ngroups() + CM_CHUNK - 1) / CM_CHUNK);
    cube_moments_kernel<<<grid, 256, 0, s>>>(img, g, ntile, d_mom);
    return cudaGetLastError();
}

cudaError_t launch_basis(const unsigned long long* d_mom, int C, double* d_basis64, float* d_basis32, cudaStream_t s,
                         double* d_gap) {
    basis_kernel<<<2 * (C / 2 + 1), 32, 0, s>>>(d_mom, C, d_basis64, d_basis32, d_gap);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const float* x, int64_t n, uint8_t* q, cudaStream_t s) {
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    quantize_kernel<<<blocks, 256, 0, s>>>(x, n, q);
    return cudaGetLastError();
}

cudaError_t launch_group_rank(const uint8_t* img, const Geo& g, const int32_t* idx, int ngroups, int32_t* ranks,
                              cudaStream_t s) {
    if (ngroups <= 0) return cudaSuccess;
    group_rank_kernel<<<ngroups, 256, 0, s>>>(img, g, idx, ranks);
    return cudaGetLastError();
}

}  // namespace htsvd

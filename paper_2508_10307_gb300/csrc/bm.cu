// Block matching (grouping, Alg. 1 Step 1; Sec. III-A, Eq. (GCP distance)).
//
// One CTA per tile of references; the match planes of the tile's union of search windows
// are staged in shared memory. One warp per reference. Each lane scores 4 horizontally
// adjacent candidates (8 lanes cover a window row of up to 32 candidates, 4 rows per step;
// wider windows use 16 lanes per row, 2 rows per step):
//  - byte planes (gray, G, or R, G, B in full mode): 4 pixels per instruction with
//    __vabsdiffu4 and __dp4a on words funnel-shifted to the candidate's alignment;
//  - the R+G+B plane of the "average" branch (values up to 765): FP32 differences and
//    squares summed two rows at a time (each partial sum < 2^24, so exact) and converted to
//    int32 before the final sum.
// Both give the exact integer SSD. Keys (SSD << 32 | y*W + x) are merged into a warp-wide
// sorted list (lane l holds the l-th smallest), so ties break by the lowest linear index.
// Slot 0 of every group is the reference itself.
#include "kernels.h"

namespace htsvd {

namespace {

constexpr int BM_THREADS = 256;
constexpr int BM_PAD = 16;          // zero bytes after each staged byte row (funnel-shift over-read)

struct Region {
    int y0, x0, h, w;
};

__device__ inline Region bm_region(const BMArgs& a, int iy0, int iy1, int ix0, int ix1) {
    const Geo& g = a.g;
    Region r;
    int ry0 = ref_pos(iy0 * a.rstep, g.s, g.H), ry1 = ref_pos(iy1 * a.rstep, g.s, g.H);
    int rx0 = ref_pos(ix0 * a.rstep, g.s, g.W), rx1 = ref_pos(ix1 * a.rstep, g.s, g.W);
    r.y0 = win_start(ry0, g.npy, g.win);
    r.x0 = win_start(rx0, g.npx, g.win);
    r.h = win_start(ry1, g.npy, g.win) + g.wny + PS - 1 - r.y0;
    r.w = win_start(rx1, g.npx, g.win) + g.wnx + PS - 1 - r.x0;
    return r;
}

__host__ __device__ inline int byte_planes(int mode, int C) {
    if (C == 1) return 1;
    return mode == MM_FULL ? 3 : 1;       // gray | G (green and GCP) | R, G, B (full)
}
__host__ __device__ inline int bytes_pitch(int w) { return ((w + BM_PAD) + 3) & ~3; }

// Bytes [u, u + 4) of the 16-byte little-endian window w0..w3, u in [0, 7].
__device__ __forceinline__ uint32_t window4(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, int u) {
    const uint32_t lo = u < 4 ? w0 : w1;
    const uint32_t mi = u < 4 ? w1 : w2;
    return __funnelshift_r(lo, mi, 8 * (u & 3));
    (void)w3;
}

// Bitonic sort of one key per lane, ascending across the warp.
__device__ __forceinline__ unsigned long long warp_sort_asc(unsigned long long v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
        }
    return v;
}

// Merges the key of every lane into the warp's sorted list (lane l: l-th smallest; the
// K-1 smallest keys seen so far are in lanes 0..K-2). Few passing keys are inserted one by
// one; many are sorted and merged with the list in one bitonic pass.
__device__ __forceinline__ void merge_keys(unsigned long long key, unsigned long long& list, int K, int lane) {
    unsigned long long thr = __shfl_sync(0xffffffffu, list, K - 2);
    unsigned pass = __ballot_sync(0xffffffffu, key < thr);
    if (__popc(pass) > 4) {
        const unsigned long long b = warp_sort_asc(key, lane);
        const unsigned long long br = __shfl_sync(0xffffffffu, b, 31 - lane);
        unsigned long long v = br < list ? br : list;     // bitonic: the 32 smallest of both lists
#pragma unroll
        for (int j = 16; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
            v = ((lane & j) == 0) ? (o < v ? o : v) : (o > v ? o : v);
        }
        list = v;
        return;
    }
    while (pass) {
        const int src = __ffs(pass) - 1;
        pass &= pass - 1;
        const unsigned long long kk = __shfl_sync(0xffffffffu, key, src);
        thr = __shfl_sync(0xffffffffu, list, K - 2);
        if (kk < thr) {
            const unsigned gt = __ballot_sync(0xffffffffu, list > kk);
            const int pos = __ffs(gt) - 1;
            const unsigned long long prev = __shfl_up_sync(0xffffffffu, list, 1);
            if (lane == pos) list = kk;
            else if (lane > pos) list = prev;
        }
    }
}

// Grouping of one tile (by, bx) of references; bsm: bm_smem_bytes(a) of shared memory.
__device__ __forceinline__ void bm_tile(const BMArgs& a, int by, int bx, unsigned char* bsm) {
    const Geo& g = a.g;
    const int iy0 = by * a.TRy, ix0 = bx * a.TRx;
    const int iy1 = min(iy0 + a.TRy, a.nry_s) - 1, ix1 = min(ix0 + a.TRx, a.nrx_s) - 1;
    const Region R = bm_region(a, iy0, iy1, ix0, ix1);
    const int nb = byte_planes(a.mode, g.C);
    const int P8 = bytes_pitch(R.w);
    const bool gcp = g.C == 3 && a.mode == MM_GCP;
    uint8_t* bp = bsm;                                              // nb byte planes [R.h][P8]
    float* sp = reinterpret_cast<float*>(bsm + (((size_t)nb * R.h * P8 + 15) & ~(size_t)15));   // R+G+B plane

    // Stage the planes of the region (byte rows zero-padded).
    for (int t = threadIdx.x; t < R.h * P8; t += BM_THREADS) {
        const int r = t / P8, c = t - r * P8;
        if (c < R.w) {
            const uint8_t* px = a.img + ((size_t)(R.y0 + r) * g.W + (R.x0 + c)) * g.C;
            if (g.C == 1) {
                bp[t] = px[0];
            } else if (a.mode == MM_FULL) {
                bp[t] = px[0];
                bp[(size_t)R.h * P8 + t] = px[1];
                bp[(size_t)2 * R.h * P8 + t] = px[2];
            } else {
                bp[t] = px[1];
                if (gcp) sp[r * R.w + c] = (float)((int)px[0] + (int)px[1] + (int)px[2]);
            }
        } else {
            for (int p = 0; p < nb; ++p) bp[(size_t)p * R.h * P8 + t] = 0;
        }
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // lane -> (window row within the step, candidate quad): 8 quads (32 columns) per row for windows up to
    // 32 wide, else 16 quads (64 columns) per row
    const int qpr = g.wnx > 32 ? 16 : 8;
    const int rps = 32 / qpr;
    const int sub = lane / qpr, q = lane % qpr;
    const int tw = ix1 - ix0 + 1;
    const int nt = (iy1 - iy0 + 1) * tw;
    const int K = g.K;
    for (int t = warp; t < nt; t += BM_THREADS / 32) {
        const int iy = iy0 + t / tw, ix = ix0 + t % tw;
        const int ry = ref_pos(iy * a.rstep, g.s, g.H), rx = ref_pos(ix * a.rstep, g.s, g.W);
        const int wy0 = win_start(ry, g.npy, g.win), wx0 = win_start(rx, g.npx, g.win);

        // Plane choice (Eq. GCP distance on the reference patch).
        bool green = true;
        if (gcp) {
            int r2 = 0, g2 = 0, b2 = 0;
            for (int pi = lane; pi < PS2; pi += 32) {
                const uint8_t* px = a.img + ((size_t)(ry + pi / PS) * g.W + rx + pi % PS) * 3;
                const int rr = px[0], gg = px[1], bb = px[2];
                r2 += rr * rr;
                g2 += gg * gg;
                b2 += bb * bb;
            }
            r2 = __reduce_add_sync(0xffffffffu, r2);
            g2 = __reduce_add_sync(0xffffffffu, g2);
            b2 = __reduce_add_sync(0xffffffffu, b2);
            const double lhs = a.gamma2 * (double)g2;
            green = (lhs >= (double)r2) && (lhs >= (double)b2);
        }

        unsigned long long list = ~0ull;       // lane l: l-th smallest key so far
        const int cx0 = 4 * q;
        const bool quad_ok = cx0 < g.wnx;
        if (green) {
            // reference rows as two words per plane and row
            uint32_t rw[3][PS][2];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                if (p >= nb) break;
                const uint8_t* pl = bp + (size_t)p * R.h * P8;
#pragma unroll
                for (int i = 0; i < PS; ++i) {
                    const int bo = (ry - R.y0 + i) * P8 + (rx - R.x0);
                    const uint32_t* wp = reinterpret_cast<const uint32_t*>(pl + (bo & ~3));
                    const int u = bo & 3;
                    const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2];
                    rw[p][i][0] = __funnelshift_r(w0, w1, 8 * u);
                    rw[p][i][1] = __funnelshift_r(w1, w2, 8 * u);
                }
            }
            for (int ybase = 0; ybase < g.wny; ybase += rps) {
                const int cy = ybase + sub;
                uint32_t acc[4] = {0u, 0u, 0u, 0u};
                const bool ok = quad_ok && cy < g.wny;
                if (ok) {
#pragma unroll
                    for (int p = 0; p < 3; ++p) {
                        if (p >= nb) break;
                        const uint8_t* pl = bp + (size_t)p * R.h * P8;
#pragma unroll
                        for (int i = 0; i < PS; ++i) {
                            const int bo = (wy0 + cy - R.y0 + i) * P8 + (wx0 - R.x0) + cx0;
                            const uint32_t* wp = reinterpret_cast<const uint32_t*>(pl + (bo & ~3));
                            const int sh = bo & 3;
                            const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2], w3 = wp[3];
#pragma unroll
                            for (int s = 0; s < 4; ++s) {
                                const int u = sh + s;
                                const uint32_t lo = window4(w0, w1, w2, w3, u);
                                const uint32_t hi = window4(w1, w2, w3, w3, u);
                                const uint32_t d0 = __vabsdiffu4(lo, rw[p][i][0]);
                                const uint32_t d1 = __vabsdiffu4(hi, rw[p][i][1]);
                                acc[s] = __dp4a(d0, d0, acc[s]);
                                acc[s] = __dp4a(d1, d1, acc[s]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    unsigned long long key = ~0ull;
                    const int cx = cx0 + s;
                    if (ok && cx < g.wnx) {
                        const int py = wy0 + cy, px = wx0 + cx;
                        if (py != ry || px != rx)
                            key = ((unsigned long long)acc[s] << 32) | (unsigned)(py * g.W + px);
                    }
                    merge_keys(key, list, K, lane);
                }
            }
        } else {
            // R+G+B plane: exact integer SSD via FP32 partial sums of two rows
            float rv[PS][PS];
#pragma unroll
            for (int i = 0; i < PS; ++i)
#pragma unroll
                for (int j = 0; j < PS; ++j) rv[i][j] = sp[(ry - R.y0 + i) * R.w + (rx - R.x0) + j];
            for (int ybase = 0; ybase < g.wny; ybase += rps) {
                const int cy = ybase + sub;
                int acc[4] = {0, 0, 0, 0};
                const bool ok = quad_ok && cy < g.wny;
                if (ok) {
                    // columns cx0 .. cx0 + 10 of the rows; clamp reads of candidates beyond the window
                    const int maxc = R.w - 1 - (wx0 - R.x0);
#pragma unroll
                    for (int i2 = 0; i2 < PS; i2 += 2) {
                        float part[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int ii = 0; ii < 2; ++ii) {
                            const int i = i2 + ii;
                            const float* row = sp + (wy0 + cy - R.y0 + i) * R.w + (wx0 - R.x0);
                            float v[PS + 3];
#pragma unroll
                            for (int c = 0; c < PS + 3; ++c) v[c] = row[min(cx0 + c, maxc)];
#pragma unroll
                            for (int s = 0; s < 4; ++s)
#pragma unroll
                                for (int j = 0; j < PS; ++j) {
                                    const float d = v[s + j] - rv[i][j];
                                    part[s] = fmaf(d, d, part[s]);
                                }
                        }
#pragma unroll
                        for (int s = 0; s < 4; ++s) acc[s] += __float2int_rn(part[s]);
                    }
                }
#pragma unroll
                for (int s = 0; s < 4; ++s) {
                    unsigned long long key = ~0ull;
                    const int cx = cx0 + s;
                    if (ok && cx < g.wnx) {
                        const int py = wy0 + cy, px = wx0 + cx;
                        if (py != ry || px != rx)
                            key = ((unsigned long long)(unsigned)acc[s] << 32) | (unsigned)(py * g.W + px);
                    }
                    merge_keys(key, list, K, lane);
                }
            }
        }
        int32_t* out = a.idx + (size_t)(iy * a.nrx_s + ix) * K;
        if (lane == 0) out[0] = ry * g.W + rx;
        if (lane < K - 1) out[1 + lane] = (int32_t)(unsigned)(list & 0xffffffffull);
    }
}

__global__ void __launch_bounds__(BM_THREADS, 2) block_match_kernel(BMArgs a) {
    extern __shared__ __align__(16) unsigned char bsm[];
    bm_tile(a, blockIdx.y, blockIdx.x, bsm);
}

// Persistent form over the tiles of many images: work item w -> image by prefix[], then tile.
__global__ void __launch_bounds__(BM_THREADS, 2) block_match_batch_kernel(const BMArgs* __restrict__ args,
                                                                          const int* __restrict__ prefix, int nimg,
                                                                          int* __restrict__ counter) {
    extern __shared__ __align__(16) unsigned char bsm[];
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
        const BMArgs& a = args[lo];
        const int t = w - prefix[lo];
        const int ntx = (a.nrx_s + a.TRx - 1) / a.TRx;
        bm_tile(a, t / ntx, t % ntx, bsm);
    }
}

}  // namespace

size_t bm_smem_bytes(const BMArgs& a) {
    const Geo& g = a.g;
    // Largest region over tiles: reference span of a tile plus the window plus ps - 1.
    int hy = (a.TRy - 1) * a.rstep * g.s + g.wny + PS - 1;
    int hx = (a.TRx - 1) * a.rstep * g.s + g.wnx + PS - 1;
    if (hy > g.H) hy = g.H;
    if (hx > g.W) hx = g.W;
    const size_t bytes = (size_t)byte_planes(a.mode, g.C) * hy * bytes_pitch(hx);
    const bool gcp = g.C == 3 && a.mode == MM_GCP;
    return ((bytes + 15) & ~(size_t)15) + (gcp ? (size_t)hy * hx * sizeof(float) : 0);
}

int bm_tiles(const BMArgs& a) {
    return ((a.nrx_s + a.TRx - 1) / a.TRx) * ((a.nry_s + a.TRy - 1) / a.TRy);
}

cudaError_t launch_block_match_batch(const BMArgs* d_args, const int* d_prefix, int nimg, size_t smem, int grid,
                                     int* d_counter, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(block_match_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    block_match_batch_kernel<<<grid, BM_THREADS, smem, s>>>(d_args, d_prefix, nimg, d_counter);
    return cudaGetLastError();
}

cudaError_t launch_block_match(const BMArgs& a, cudaStream_t s) {
    size_t smem = bm_smem_bytes(a);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(block_match_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((a.nrx_s + a.TRx - 1) / a.TRx, (a.nry_s + a.TRy - 1) / a.TRy);
    block_match_kernel<<<grid, BM_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace htsvd

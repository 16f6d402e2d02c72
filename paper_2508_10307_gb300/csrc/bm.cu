// Block matching (grouping, Alg. 1 Step 1; Sec. III-A, Eq. (GCP distance)).
//
// One CTA per tile of references. The match planes of the tile's union of search
// windows are staged in shared memory as uint16 (G or gray plane, R+G+B plane, or the
// three channels). One warp per reference: exact int32 SSD of every candidate, keys
// (SSD << 32 | y*W + x) kept in a warp-wide sorted list (lane l holds the l-th smallest),
// so ties break by the lowest linear index. Slot 0 is the reference itself.
#include "kernels.h"

namespace htsvd {

namespace {

constexpr int BM_THREADS = 256;

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

__device__ __forceinline__ int nplanes_of(int mode, int C) {
    if (C == 1) return 1;
    if (mode == MM_GCP) return 2;
    if (mode == MM_FULL) return 3;
    return 1;
}

__global__ void __launch_bounds__(BM_THREADS) block_match_kernel(BMArgs a) {
    extern __shared__ uint16_t sm[];
    const Geo& g = a.g;
    const int iy0 = blockIdx.y * a.TRy, ix0 = blockIdx.x * a.TRx;
    const int iy1 = min(iy0 + a.TRy, a.nry_s) - 1, ix1 = min(ix0 + a.TRx, a.nrx_s) - 1;
    const Region R = bm_region(a, iy0, iy1, ix0, ix1);
    const int np = nplanes_of(a.mode, g.C);
    const int plane = R.h * R.w;

    // Stage the planes of the region.
    for (int t = threadIdx.x; t < plane; t += BM_THREADS) {
        int r = t / R.w, c = t - r * R.w;
        const uint8_t* px = a.img + ((size_t)(R.y0 + r) * g.W + (R.x0 + c)) * g.C;
        if (g.C == 1) {
            sm[t] = px[0];
        } else if (a.mode == MM_GCP) {
            sm[t] = px[1];
            sm[plane + t] = (uint16_t)(px[0] + px[1] + px[2]);
        } else if (a.mode == MM_FULL) {
            sm[t] = px[0];
            sm[plane + t] = px[1];
            sm[2 * plane + t] = px[2];
        } else {
            sm[t] = px[1];
        }
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tw = ix1 - ix0 + 1;
    const int nt = (iy1 - iy0 + 1) * tw;
    const int K = g.K;
    for (int q = warp; q < nt; q += BM_THREADS / 32) {
        const int iy = iy0 + q / tw, ix = ix0 + q % tw;
        const int ry = ref_pos(iy * a.rstep, g.s, g.H), rx = ref_pos(ix * a.rstep, g.s, g.W);
        const int wy0 = win_start(ry, g.npy, g.win), wx0 = win_start(rx, g.npx, g.win);

        // Plane choice (Eq. GCP distance on the reference patch).
        int pl0 = 0;
        if (g.C == 3 && a.mode == MM_GCP) {
            int r2 = 0, g2 = 0, b2 = 0;
            for (int pi = lane; pi < PS2; pi += 32) {
                const uint8_t* px = a.img + ((size_t)(ry + pi / PS) * g.W + rx + pi % PS) * 3;
                int rr = px[0], gg = px[1], bb = px[2];
                r2 += rr * rr; g2 += gg * gg; b2 += bb * bb;
            }
            r2 = __reduce_add_sync(0xffffffffu, r2);
            g2 = __reduce_add_sync(0xffffffffu, g2);
            b2 = __reduce_add_sync(0xffffffffu, b2);
            const double lhs = a.gamma2 * (double)g2;
            const bool green = (lhs >= (double)r2) && (lhs >= (double)b2);
            pl0 = green ? 0 : 1;
        }
        const uint16_t* P = sm + pl0 * plane;
        int refv[PS2];
        {
            const uint16_t* rp = P + (ry - R.y0) * R.w + (rx - R.x0);
#pragma unroll
            for (int i = 0; i < PS; ++i)
#pragma unroll
                for (int j = 0; j < PS; ++j) refv[i * PS + j] = rp[i * R.w + j];
        }
        const bool full = (g.C == 3 && a.mode == MM_FULL);

        unsigned long long list = ~0ull;       // lane l: l-th smallest key so far
        const int ncand = g.wny * g.wnx;
        for (int base = 0; base < ncand; base += 32) {
            const int c = base + lane;
            unsigned long long key = ~0ull;
            if (c < ncand) {
                const int cy = c / g.wnx, cx = c - cy * g.wnx;
                const int py = wy0 + cy, px = wx0 + cx;
                if (py != ry || px != rx) {
                    const uint16_t* cp = P + (py - R.y0) * R.w + (px - R.x0);
                    int acc = 0;
#pragma unroll
                    for (int i = 0; i < PS; ++i)
#pragma unroll
                        for (int j = 0; j < PS; ++j) {
                            int d = refv[i * PS + j] - (int)cp[i * R.w + j];
                            acc += d * d;
                        }
                    if (full) {
                        for (int pp = 1; pp < 3; ++pp) {
                            const uint16_t* Pp = sm + pp * plane;
                            const uint16_t* rp = Pp + (ry - R.y0) * R.w + (rx - R.x0);
                            const uint16_t* cq = Pp + (py - R.y0) * R.w + (px - R.x0);
                            for (int i = 0; i < PS; ++i)
                                for (int j = 0; j < PS; ++j) {
                                    int d = (int)rp[i * R.w + j] - (int)cq[i * R.w + j];
                                    acc += d * d;
                                }
                        }
                    }
                    key = ((unsigned long long)(unsigned)acc << 32) | (unsigned)(py * g.W + px);
                }
            }
            unsigned long long thr = __shfl_sync(0xffffffffu, list, K - 2);
            unsigned pass = __ballot_sync(0xffffffffu, key < thr);
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
        int32_t* out = a.idx + (size_t)(iy * a.nrx_s + ix) * K;
        if (lane == 0) out[0] = ry * g.W + rx;
        if (lane < K - 1) out[1 + lane] = (int32_t)(unsigned)(list & 0xffffffffull);
    }
}

}  // namespace

size_t bm_smem_bytes(const BMArgs& a) {
    const Geo& g = a.g;
    int np = (g.C == 1) ? 1 : (a.mode == MM_GCP ? 2 : (a.mode == MM_FULL ? 3 : 1));
    // Largest region over tiles: reference span of a tile plus the window plus ps - 1.
    int hy = (a.TRy - 1) * a.rstep * g.s + g.wny + PS - 1;
    int hx = (a.TRx - 1) * a.rstep * g.s + g.wnx + PS - 1;
    if (hy > g.H) hy = g.H;
    if (hx > g.W) hx = g.W;
    return (size_t)np * hy * hx * sizeof(uint16_t);
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

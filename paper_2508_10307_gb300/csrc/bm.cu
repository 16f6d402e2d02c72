// Block matching (grouping, Alg. 1 Step 1; Sec. III-A, Eq. (GCP distance)).
//
// One CTA per tile of references; the match planes of the tile's union of search windows
// are staged in shared memory, together with the 8x8 box sums of their squares at every
// candidate position (S_vv). One warp per reference. The exact integer SSD of a candidate v
// against the reference r is
//     SSD = S_vv(v) - 2 <v, r> + S_vv(r),
// so per candidate only the cross term <v, r> is accumulated:
//  - byte planes (gray, G, or R, G, B in full mode): __dp4a on words shifted to the
//    candidate's alignment (4 pixels per instruction);
//  - the R+G+B plane of the "average" branch (values up to 765): FP32 products summed two
//    rows at a time (each partial sum < 2^24, so exact) and converted to int32.
// Lane layout: lane (g, q) owns the candidate columns 4q .. 4q+3 of a strip of R = 4 consecutive
// candidate rows; each staged image row is loaded once and used for every candidate row of the
// strip it overlaps (reference row i = image row - candidate row).
// Keys (SSD << 32 | y*W + x) below the warp's current threshold (the (K-1)-th smallest key
// merged so far) are appended to a per-warp buffer; 32 buffered keys at a time are sorted and
// merged into the warp-wide sorted list (lane l holds the l-th smallest). Ties therefore break
// by the lowest linear index. Slot 0 of every group is the reference itself.
#include "kernels.h"

namespace htsvd {

namespace {

constexpr int BM_THREADS = 256;
constexpr int BM_WARPS = BM_THREADS / 32;
constexpr int BM_PAD = 16;          // zero bytes after each staged byte row (shifted-word over-read)
constexpr int BM_BUF = 64;          // per-warp key buffer (< 32 left after a merge + 32 appended)
constexpr int BM_FR = 4;            // candidate rows per strip on the R+G+B plane
constexpr unsigned FULL = 0xffffffffu;

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
    return mode == MM_FULL ? C : 1;       // gray | G (green and GCP) | every channel or band (full)
}
__host__ __device__ inline bool uses_sum_plane(int mode, int C) { return C == 3 && mode == MM_GCP; }
__host__ __device__ inline int bytes_pitch(int w) { return ((w + BM_PAD) + 3) & ~3; }

// Shared-memory layout of a region of h x w pixels (h, w >= ps) staged from nfr frames: each
// section holds one block per frame, the blocks sz_* bytes apart.
struct BmLayout {
    size_t bytes, fplane, svv, warp, total;
    size_t sz_bytes, sz_fplane, sz_svv;
};
__host__ __device__ inline size_t a16(size_t o) { return (o + 15) & ~(size_t)15; }
__host__ __device__ inline BmLayout bm_layout(int h, int w, int nb, bool sum_plane, int nfr = 1) {
    BmLayout L;
    L.sz_bytes = a16((size_t)nb * h * bytes_pitch(w));                                  // nb byte planes [h][pitch]
    L.sz_fplane = sum_plane ? a16(sizeof(float) * h * w) : 0;                          // R+G+B plane [h][w]
    L.sz_svv = a16(sizeof(int) * (sum_plane ? 2 : 1) * (size_t)(h - PS + 1) * (w - PS + 1));   // S_vv [h-7][w-7]
    size_t o = 0;
    L.bytes = o;
    o += nfr * L.sz_bytes;
    L.fplane = o;
    o += nfr * L.sz_fplane;
    L.svv = o;
    o += nfr * L.sz_svv;
    L.warp = o;
    o += (size_t)BM_WARPS * (BM_BUF * sizeof(unsigned long long) + PS2 * sizeof(float));
    L.total = o;
    return L;
}

// Bitonic sort of one key per lane, ascending across the warp.
__device__ __forceinline__ unsigned long long warp_sort_asc(unsigned long long v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(FULL, v, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            v = keep_min ? (o < v ? o : v) : (o > v ? o : v);
        }
    return v;
}

// Top-(K-1) selection state of one warp: the sorted list (lane l: l-th smallest key merged so
// far), its (K-1)-th key as the admission threshold, and the buffer of admitted keys.
struct Select {
    unsigned long long list, thr;
    unsigned long long* buf;
    int cnt;
};

struct MergeOut {
    unsigned long long list, thr;
    int cnt;
};

// Merges the first min(cnt, 32) buffered keys into the list and moves the rest down. Kept out
// of line: it runs a few times per reference, while its call sites are many (one per offered
// register), and inlining it everywhere overflows the instruction cache.
__device__ __noinline__ MergeOut sel_merge_fn(unsigned long long list, unsigned long long* buf, int cnt, int K,
                                              int lane) {
    __syncwarp();
    const int n = cnt < 32 ? cnt : 32;
    const unsigned long long k = lane < n ? buf[lane] : ~0ull;
    const unsigned long long b = warp_sort_asc(k, lane);
    const unsigned long long br = __shfl_sync(FULL, b, 31 - lane);
    unsigned long long v = br < list ? br : list;           // bitonic: the 32 smallest of both lists
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const unsigned long long o = __shfl_xor_sync(FULL, v, j);
        v = ((lane & j) == 0) ? (o < v ? o : v) : (o > v ? o : v);
    }
    MergeOut m;
    m.list = v;
    m.thr = __shfl_sync(FULL, v, K - 2);
    const int rest = cnt - n;
    unsigned long long t = 0;
    if (lane < rest) t = buf[32 + lane];
    __syncwarp();
    if (lane < rest) buf[lane] = t;
    __syncwarp();
    m.cnt = rest;
    return m;
}

__device__ __forceinline__ void sel_merge(Select& S, int K, int lane) {
    const MergeOut m = sel_merge_fn(S.list, S.buf, S.cnt, K, lane);
    S.list = m.list;
    S.thr = m.thr;
    S.cnt = m.cnt;
}

// Offers one key per lane: keys below the threshold are appended to the buffer.
__device__ __forceinline__ void sel_offer(Select& S, unsigned long long key, int K, int lane) {
    const bool p = key < S.thr;
    const unsigned pass = __ballot_sync(FULL, p);
    if (!pass) return;
    if (p) S.buf[S.cnt + __popc(pass & ((1u << lane) - 1u))] = key;
    S.cnt += __popc(pass);
    if (S.cnt >= 32) sel_merge(S, K, lane);
}

// Per-reference geometry shared by both distance paths.
struct RefCtx {
    int ry, rx, wy0, wx0;
    int oy, ox;            // window origin in region coordinates
    int wv;                // S_vv pitch (candidate positions per region row)
};

__device__ __forceinline__ unsigned long long make_key(int ssd, int py, int px, int W, unsigned koff) {
    return ((unsigned long long)(unsigned)ssd << 32) | (koff + (unsigned)(py * W + px));
}

// Byte planes: cross terms of the candidates of the lane's strips, keys offered per strip.
// bp, svv: the candidate frame's byte planes and box sums; rbp, srr: the reference frame's planes
// and the reference's own box sum; koff: index offset of the candidate frame; self: the candidate
// frame is the reference frame (its reference position is not a candidate).
template <int R, int NB>
__device__ __forceinline__ void match_bytes(const BMArgs& a, const Region& Rg, const uint8_t* bp,
                                            const uint8_t* rbp, int P8, const int* svv, int srr,
                                            const RefCtx& c, Select& S, int lane, unsigned koff, bool self) {
    const Geo& g = a.g;
    const int qpr = (g.wnx + 3) / 4, G = 32 / qpr;
    const int sg = lane / qpr, q = lane - sg * qpr;
    const bool active = sg < G;
    const int cx0 = 4 * q;
    // reference rows: two words per plane and row
    uint32_t rw[NB][PS][2];
#pragma unroll
    for (int p = 0; p < NB; ++p) {
        const uint8_t* pl = rbp + (size_t)p * Rg.h * P8;
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const int bo = (c.ry - Rg.y0 + i) * P8 + (c.rx - Rg.x0);
            const uint32_t* wp = reinterpret_cast<const uint32_t*>(pl + (bo & ~3));
            const int u = 8 * (bo & 3);
            const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2];
            rw[p][i][0] = __funnelshift_r(w0, w1, u);
            rw[p][i][1] = __funnelshift_r(w1, w2, u);
        }
    }
    const int sh = 8 * (c.ox & 3);                            // byte offset of every candidate word in a row
    const int last_row = g.wny + PS - 2;                      // last window row any valid candidate reads
    // warp-uniform chunk count (every lane offers the same number of keys); idle lanes and strips
    // past the window offer none
    const int nch = (g.wny + G * R - 1) / (G * R);
    for (int ch = 0; ch < nch; ++ch) {
        const int cy0 = (ch * G + sg) * R;
        const bool run = active && cy0 < g.wny;
        uint32_t acc[R][4];
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int s = 0; s < 4; ++s) acc[k][s] = 0u;
        if (run) {
#pragma unroll
            for (int t = 0; t < R + PS - 1; ++t) {
                const int rr = min(cy0 + t, last_row);
#pragma unroll
                for (int p = 0; p < NB; ++p) {
                    const uint8_t* pl = bp + (size_t)p * Rg.h * P8;
                    const uint32_t* wp =
                        reinterpret_cast<const uint32_t*>(pl + (((c.oy + rr) * P8 + c.ox + cx0) & ~3));
                    const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2], w3 = wp[3];
                    const uint32_t a0 = __funnelshift_r(w0, w1, sh);
                    const uint32_t a1 = __funnelshift_r(w1, w2, sh);
                    const uint32_t a2 = __funnelshift_r(w2, w3, sh);
                    uint32_t lo[4], hi[4];
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        lo[s] = s == 0 ? a0 : __funnelshift_r(a0, a1, 8 * s);
                        hi[s] = s == 0 ? a1 : __funnelshift_r(a1, a2, 8 * s);
                    }
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const int i = t - k;                  // reference row met by candidate row k
                        if (i < 0 || i >= PS) continue;
#pragma unroll
                        for (int s = 0; s < 4; ++s) {
                            acc[k][s] = __dp4a(lo[s], rw[p][i][0], acc[k][s]);
                            acc[k][s] = __dp4a(hi[s], rw[p][i][1], acc[k][s]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int cy = cy0 + k, cx = cx0 + s;
                unsigned long long key = ~0ull;
                if (run && cy < g.wny && cx < g.wnx) {
                    const int py = c.wy0 + cy, px = c.wx0 + cx;
                    if (!self || py != c.ry || px != c.rx)
                        key = make_key(svv[(c.oy + cy) * c.wv + c.ox + cx] + srr - 2 * (int)acc[k][s], py, px, g.W,
                                       koff);
                }
                sel_offer(S, key, g.K, lane);
            }
    }
}

// Many byte planes (the bands of a hyperspectral cube, SSD over all of them): as match_bytes, but
// with the plane loop outermost inside each strip chunk, so that only one plane's reference rows
// are held in registers (the cross terms of all planes add into the same accumulators; every
// partial sum stays below 2^31 for up to 500 planes: 64 x 255^2 per plane).
template <int R>
__device__ __forceinline__ void match_bytes_n(const BMArgs& a, const Region& Rg, const uint8_t* bp,
                                              const uint8_t* rbp, int P8, const int* svv, int srr,
                                              const RefCtx& c, Select& S, int lane, unsigned koff, bool self,
                                              int nb) {
    const Geo& g = a.g;
    const int qpr = (g.wnx + 3) / 4, G = 32 / qpr;
    const int sg = lane / qpr, q = lane - sg * qpr;
    const bool active = sg < G;
    const int cx0 = 4 * q;
    const int sh = 8 * (c.ox & 3);
    const int last_row = g.wny + PS - 2;
    const int nch = (g.wny + G * R - 1) / (G * R);
    for (int ch = 0; ch < nch; ++ch) {
        const int cy0 = (ch * G + sg) * R;
        const bool run = active && cy0 < g.wny;
        uint32_t acc[R][4];
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int s = 0; s < 4; ++s) acc[k][s] = 0u;
        if (run) {
#pragma unroll 1
            for (int p = 0; p < nb; ++p) {
                uint32_t rw[PS][2];
                const uint8_t* rpl = rbp + (size_t)p * Rg.h * P8;
#pragma unroll
                for (int i = 0; i < PS; ++i) {
                    const int bo = (c.ry - Rg.y0 + i) * P8 + (c.rx - Rg.x0);
                    const uint32_t* wp = reinterpret_cast<const uint32_t*>(rpl + (bo & ~3));
                    const int u = 8 * (bo & 3);
                    const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2];
                    rw[i][0] = __funnelshift_r(w0, w1, u);
                    rw[i][1] = __funnelshift_r(w1, w2, u);
                }
                const uint8_t* pl = bp + (size_t)p * Rg.h * P8;
#pragma unroll
                for (int t = 0; t < R + PS - 1; ++t) {
                    const int rr = min(cy0 + t, last_row);
                    const uint32_t* wp =
                        reinterpret_cast<const uint32_t*>(pl + (((c.oy + rr) * P8 + c.ox + cx0) & ~3));
                    const uint32_t w0 = wp[0], w1 = wp[1], w2 = wp[2], w3 = wp[3];
                    const uint32_t a0 = __funnelshift_r(w0, w1, sh);
                    const uint32_t a1 = __funnelshift_r(w1, w2, sh);
                    const uint32_t a2 = __funnelshift_r(w2, w3, sh);
                    uint32_t lo[4], hi[4];
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        lo[s] = s == 0 ? a0 : __funnelshift_r(a0, a1, 8 * s);
                        hi[s] = s == 0 ? a1 : __funnelshift_r(a1, a2, 8 * s);
                    }
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        const int i = t - k;
                        if (i < 0 || i >= PS) continue;
#pragma unroll
                        for (int s = 0; s < 4; ++s) {
                            acc[k][s] = __dp4a(lo[s], rw[i][0], acc[k][s]);
                            acc[k][s] = __dp4a(hi[s], rw[i][1], acc[k][s]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int cy = cy0 + k, cx = cx0 + s;
                unsigned long long key = ~0ull;
                if (run && cy < g.wny && cx < g.wnx) {
                    const int py = c.wy0 + cy, px = c.wx0 + cx;
                    if (!self || py != c.ry || px != c.rx)
                        key = make_key(svv[(c.oy + cy) * c.wv + c.ox + cx] + srr - 2 * (int)acc[k][s], py, px, g.W,
                                       koff);
                }
                sel_offer(S, key, g.K, lane);
            }
    }
}

// R+G+B plane: exact cross terms from FP32 partial sums over two reference rows.
// sp, svv2: the candidate frame's R+G+B plane and box sums; rsp, srr: the reference frame's plane
// and the reference's box sum; koff, self as for the byte planes.
__device__ __forceinline__ void match_sum_plane(const BMArgs& a, const Region& Rg, const float* sp,
                                                const float* rsp, const int* svv2, int srr, float* rvw,
                                                const RefCtx& c, Select& S, int lane, unsigned koff, bool self) {
    const Geo& g = a.g;
    constexpr int R = BM_FR;
    const int qpr = (g.wnx + 3) / 4, G = 32 / qpr;
    const int sg = lane / qpr, q = lane - sg * qpr;
    const bool active = sg < G;
    const int cx0 = 4 * q;
    // the reference patch, for broadcast reads
    __syncwarp();                              // rvw of the previous frame or reference is read
    for (int e = lane; e < PS2; e += 32) rvw[e] = rsp[(c.ry - Rg.y0 + e / PS) * Rg.w + (c.rx - Rg.x0) + e % PS];
    __syncwarp();
    const int last_row = g.wny + PS - 2;
    const int maxc = Rg.w - 1 - c.ox;          // clamp of the columns of idle candidates beyond the window
    const int nch = (g.wny + G * R - 1) / (G * R);           // warp-uniform, as on the byte planes
    for (int ch = 0; ch < nch; ++ch) {
        const int cy0 = (ch * G + sg) * R;
        const bool run = active && cy0 < g.wny;
        int acc[R][4];
        float part[R][4];
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                acc[k][s] = 0;
                part[k][s] = 0.f;
            }
        if (run) {
#pragma unroll
            for (int t = 0; t < R + PS - 1; ++t) {
                const int rr = min(cy0 + t, last_row);
                const float* row = sp + (c.oy + rr) * Rg.w + c.ox;
                float v[PS + 3];
#pragma unroll
                for (int j = 0; j < PS + 3; ++j) v[j] = row[min(cx0 + j, maxc)];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const int i = t - k;
                    if (i < 0 || i >= PS) continue;
                    const float4 r0 = reinterpret_cast<const float4*>(rvw + i * PS)[0];
                    const float4 r1 = reinterpret_cast<const float4*>(rvw + i * PS)[1];
                    const float rv[PS] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
#pragma unroll
                        for (int j = 0; j < PS; ++j) part[k][s] = fmaf(v[s + j], rv[j], part[k][s]);
                        if (i & 1) {
                            acc[k][s] += __float2int_rn(part[k][s]);
                            part[k][s] = 0.f;
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const int cy = cy0 + k, cx = cx0 + s;
                unsigned long long key = ~0ull;
                if (run && cy < g.wny && cx < g.wnx) {
                    const int py = c.wy0 + cy, px = c.wx0 + cx;
                    if (!self || py != c.ry || px != c.rx)
                        key = make_key(svv2[(c.oy + cy) * c.wv + c.ox + cx] + srr - 2 * acc[k][s], py, px, g.W,
                                       koff);
                }
                sel_offer(S, key, g.K, lane);
            }
    }
    __syncwarp();
}

// Grouping of one tile (by, bx) of references; bsm: bm_smem_bytes(a) of shared memory.
// MF: spatio-temporal search over a.nfr frames (a separate instantiation, so that the image
// kernels carry no frame loop).
// CUBE: more than three byte planes (hyperspectral bands), a separate instantiation so that the image
// kernels carry no plane loop.
template <bool MF, bool CUBE = false>
__device__ __forceinline__ void bm_tile(const BMArgs& a, int by, int bx, unsigned char* bsm) {
    const Geo& g = a.g;
    const int iy0 = by * a.TRy, ix0 = bx * a.TRx;
    const int iy1 = min(iy0 + a.TRy, a.nry_s) - 1, ix1 = min(ix0 + a.TRx, a.nrx_s) - 1;
    const Region Rg = bm_region(a, iy0, iy1, ix0, ix1);
    const int nb = byte_planes(a.mode, g.C);
    const bool gcp = uses_sum_plane(a.mode, g.C);
    const int P8 = bytes_pitch(Rg.w);
    const int nfr = MF ? a.nfr : 1;                                  // frames searched
    const BmLayout L = bm_layout(Rg.h, Rg.w, nb, gcp, nfr);
    const int hv = Rg.h - PS + 1, wv = Rg.w - PS + 1;
    // frame slot fs: nb byte planes [h][P8], R+G+B plane [h][w], S_vv [nsv][h-7][w-7]
    auto planes_of = [&](int fs) { return bsm + L.bytes + fs * L.sz_bytes; };
    auto sum_of = [&](int fs) { return reinterpret_cast<float*>(bsm + L.fplane + fs * L.sz_fplane); };
    auto svv_of = [&](int fs) { return reinterpret_cast<int*>(bsm + L.svv + fs * L.sz_svv); };
    const int fsref = MF ? a.fref - a.f0 : 0;                         // slot of the reference frame

    // Stage the planes of the region of every frame (byte rows zero-padded).
    for (int t = threadIdx.x; t < nfr * Rg.h * P8; t += BM_THREADS) {
        const int fs = t / (Rg.h * P8), tt = t - fs * (Rg.h * P8);
        const int r = tt / P8, cc = tt - r * P8;
        uint8_t* bp = planes_of(fs);
        float* sp = sum_of(fs);
        const uint8_t* frame = MF ? a.vid + (size_t)(a.f0 + fs) * a.fstride : a.img;
        const int t_ = tt;
        if (cc < Rg.w) {
            const uint8_t* px = frame + ((size_t)(Rg.y0 + r) * g.W + (Rg.x0 + cc)) * g.C;
            if (g.C == 1) {
                bp[t_] = px[0];
            } else if (a.mode == MM_FULL) {
                for (int p = 0; p < nb; ++p) bp[(size_t)p * Rg.h * P8 + t_] = px[p];
            } else {
                bp[t_] = px[1];
                if (gcp) sp[r * Rg.w + cc] = (float)((int)px[0] + (int)px[1] + (int)px[2]);
            }
        } else {
            for (int p = 0; p < nb; ++p) bp[(size_t)p * Rg.h * P8 + t_] = 0;
        }
    }
    __syncthreads();
    // S_vv: 8x8 box sums of the squared plane values (summed over the byte planes; the R+G+B
    // plane separately). Work item (plane, block of 8 output rows, column x).
    {
        const int nyc = (hv + PS - 1) / PS;
        const int nsv = gcp ? 2 : 1;
        for (int it0 = threadIdx.x; it0 < nfr * nsv * nyc * wv; it0 += BM_THREADS) {
            const int fs = it0 / (nsv * nyc * wv), it = it0 - fs * (nsv * nyc * wv);
            const uint8_t* bp = planes_of(fs);
            const float* sp = sum_of(fs);
            int* svv = svv_of(fs);
            const int pl = it / (nyc * wv);
            const int rem = it - pl * nyc * wv;
            const int yc = rem / wv, x = rem - yc * wv;
            const int y0 = yc * PS;
            int hs[2 * PS - 1];
#pragma unroll
            for (int t = 0; t < 2 * PS - 1; ++t) {
                int v = 0;
                const int r = y0 + t;
                if (r < Rg.h) {
                    if (pl == 0) {
                        for (int p = 0; p < nb; ++p) {
                            const uint8_t* rowp = bp + (size_t)p * Rg.h * P8 + (size_t)r * P8 + x;
#pragma unroll
                            for (int j = 0; j < PS; ++j) v += (int)rowp[j] * (int)rowp[j];
                        }
                    } else {
                        const float* rowp = sp + r * Rg.w + x;
#pragma unroll
                        for (int j = 0; j < PS; ++j) {
                            const int u = (int)rowp[j];
                            v += u * u;
                        }
                    }
                }
                hs[t] = v;
            }
            int* out = svv + (size_t)pl * hv * wv;
#pragma unroll
            for (int o = 0; o < PS; ++o) {
                if (y0 + o < hv) {
                    int sum = 0;
#pragma unroll
                    for (int i = 0; i < PS; ++i) sum += hs[o + i];
                    out[(y0 + o) * wv + x] = sum;
                }
            }
        }
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* wbase = bsm + L.warp + (size_t)warp * (BM_BUF * sizeof(unsigned long long) + PS2 * sizeof(float));
    unsigned long long* buf = reinterpret_cast<unsigned long long*>(wbase);
    float* rvw = reinterpret_cast<float*>(wbase + BM_BUF * sizeof(unsigned long long));
    const int tw = ix1 - ix0 + 1;
    const int nt = (iy1 - iy0 + 1) * tw;
    const int K = g.K;
    for (int t = warp; t < nt; t += BM_WARPS) {
        const int iy = iy0 + t / tw, ix = ix0 + t % tw;
        RefCtx c;
        c.ry = ref_pos(iy * a.rstep, g.s, g.H);
        c.rx = ref_pos(ix * a.rstep, g.s, g.W);
        c.wy0 = win_start(c.ry, g.npy, g.win);
        c.wx0 = win_start(c.rx, g.npx, g.win);
        c.oy = c.wy0 - Rg.y0;
        c.ox = c.wx0 - Rg.x0;
        c.wv = wv;

        // Plane choice (Eq. GCP distance on the reference patch).
        bool green = true;
        if (gcp) {
            int r2 = 0, g2 = 0, b2 = 0;
            for (int pi = lane; pi < PS2; pi += 32) {
                const uint8_t* px = a.img + ((size_t)(c.ry + pi / PS) * g.W + c.rx + pi % PS) * 3;
                const int rr = px[0], gg = px[1], bb = px[2];
                r2 += rr * rr;
                g2 += gg * gg;
                b2 += bb * bb;
            }
            r2 = __reduce_add_sync(FULL, r2);
            g2 = __reduce_add_sync(FULL, g2);
            b2 = __reduce_add_sync(FULL, b2);
            const double lhs = a.gamma2 * (double)g2;
            green = (lhs >= (double)r2) && (lhs >= (double)b2);
        }

        Select S;
        S.list = ~0ull;
        S.thr = ~0ull;
        S.buf = buf;
        S.cnt = 0;
        // the reference patch and its box sums come from the reference frame's slot
        const uint8_t* rbp = planes_of(fsref);
        const float* rsp = sum_of(fsref);
        const int* rsvv = svv_of(fsref);
        const int rsrr = rsvv[(size_t)(green ? 0 : hv * wv) + (c.ry - Rg.y0) * wv + (c.rx - Rg.x0)];
        for (int fs = 0; fs < nfr; ++fs) {
            const unsigned koff = MF ? (unsigned)(a.f0 + fs) * (unsigned)(g.H * g.W) : 0u;
            const bool self = fs == fsref;
            const uint8_t* bp = planes_of(fs);
            const int* svv = svv_of(fs);
            if (!green) {
                match_sum_plane(a, Rg, sum_of(fs), rsp, svv + (size_t)hv * wv, rsrr, rvw, c, S, lane, koff, self);
            } else if constexpr (CUBE) {
                match_bytes_n<4>(a, Rg, bp, rbp, P8, svv, rsrr, c, S, lane, koff, self, nb);
            } else if (nb == 3) {
                match_bytes<4, 3>(a, Rg, bp, rbp, P8, svv, rsrr, c, S, lane, koff, self);
            } else {
                // strips of 4 candidate rows: strips of 8 load fewer rows per product (R + 7 rows for
                // 8 R row pairs), but their fully unrolled body costs more in instruction fetch than
                // it saves (3-5% slower on the 512x512x3 and 3840x2160x3 workloads)
                match_bytes<4, 1>(a, Rg, bp, rbp, P8, svv, rsrr, c, S, lane, koff, self);
            }
        }
        if (S.cnt > 0) sel_merge(S, K, lane);
        int32_t* out = a.idx + (size_t)(iy * a.nrx_s + ix) * K;
        if (lane == 0) out[0] = (MF ? a.fref * g.H * g.W : 0) + c.ry * g.W + c.rx;
        if (lane < K - 1) out[1 + lane] = (int32_t)(unsigned)(S.list & 0xffffffffull);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(BM_THREADS, 2) block_match_kernel(BMArgs a) {
    extern __shared__ __align__(16) unsigned char bsm[];
    bm_tile<false>(a, blockIdx.y, blockIdx.x, bsm);
}

__global__ void __launch_bounds__(BM_THREADS, 2) block_match_cube_kernel(BMArgs a) {
    extern __shared__ __align__(16) unsigned char bsm[];
    bm_tile<false, true>(a, blockIdx.y, blockIdx.x, bsm);
}

__global__ void __launch_bounds__(BM_THREADS, 2) block_match_video_kernel(BMArgs a) {
    extern __shared__ __align__(16) unsigned char bsm[];
    bm_tile<true>(a, blockIdx.y, blockIdx.x, bsm);
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
        bm_tile<false>(a, t / ntx, t % ntx, bsm);
    }
}

constexpr size_t BM_SMEM_TARGET = 100 * 1024;    // leaves room for two CTAs per SM
constexpr size_t BM_SMEM_MAX = 227 * 1024;

}  // namespace

size_t bm_smem_bytes(const BMArgs& a) {
    const Geo& g = a.g;
    // Largest region over tiles: reference span of a tile plus the window plus ps - 1.
    int hy = (a.TRy - 1) * a.rstep * g.s + g.wny + PS - 1;
    int hx = (a.TRx - 1) * a.rstep * g.s + g.wnx + PS - 1;
    if (hy > g.H) hy = g.H;
    if (hx > g.W) hx = g.W;
    return bm_layout(hy, hx, byte_planes(a.mode, g.C), uses_sum_plane(a.mode, g.C), a.nfr > 0 ? a.nfr : 1).total;
}

void bm_fit_tiles(BMArgs& a) {
    while (bm_smem_bytes(a) > BM_SMEM_TARGET && (a.TRx > 1 || a.TRy > 1)) {
        if (a.TRx >= a.TRy) a.TRx = (a.TRx + 1) / 2;
        else a.TRy = (a.TRy + 1) / 2;
    }
}

int bm_tiles(const BMArgs& a) {
    return ((a.nrx_s + a.TRx - 1) / a.TRx) * ((a.nry_s + a.TRy - 1) / a.TRy);
}

cudaError_t launch_block_match_batch(const BMArgs* d_args, const int* d_prefix, int nimg, size_t smem, int grid,
                                     int* d_counter, cudaStream_t s) {
    if (smem > BM_SMEM_MAX) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(block_match_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    block_match_batch_kernel<<<grid, BM_THREADS, smem, s>>>(d_args, d_prefix, nimg, d_counter);
    return cudaGetLastError();
}

cudaError_t launch_block_match(const BMArgs& a, cudaStream_t s) {
    size_t smem = bm_smem_bytes(a);
    if (smem > BM_SMEM_MAX) return cudaErrorInvalidValue;
    if (byte_planes(a.mode, a.g.C) > 3 && a.nfr > 0) return cudaErrorInvalidValue;   // no video cubes
    auto fn = byte_planes(a.mode, a.g.C) > 3 ? block_match_cube_kernel
              : a.nfr > 0                    ? block_match_video_kernel
                                             : block_match_kernel;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((a.nrx_s + a.TRx - 1) / a.TRx, (a.nry_s + a.TRy - 1) / a.TRy);
    fn<<<grid, BM_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace htsvd

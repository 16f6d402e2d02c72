// Shared geometry and small helpers of the CUDA path (device and host).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace htsvd {

constexpr int PS = 8;          // patch edge; the kernels are written for the paper's ps = 8 (Sec. IV-A)
constexpr int PS2 = PS * PS;

// Reference grid {0, s, 2s, ...} U {n - ps} along one axis (row-major order of groups).
__host__ __device__ inline int ref_count(int n, int s) {
    int last = n - PS;
    return last / s + 1 + ((last % s) != 0 ? 1 : 0);
}
__host__ __device__ inline int ref_pos(int i, int s, int n) {
    int v = i * s, last = n - PS;
    return v < last ? v : last;
}
// First candidate top-left position of the search window of a reference at r along one
// axis: the window of `win` positions is shifted to lie inside the npos = n - ps + 1 positions.
__host__ __device__ inline int win_start(int r, int npos, int win) {
    if (npos <= win) return 0;
    int st = r - (win - 1) / 2;
    st = st < 0 ? 0 : st;
    int mx = npos - win;
    return st > mx ? mx : st;
}
__host__ __device__ inline int win_len(int npos, int win) { return npos < win ? npos : win; }

// Geometry of one image under one parameter set.
struct Geo {
    int H, W, C;
    int s, win, K;
    int nry, nrx;        // references per axis
    int npy, npx;        // candidate positions per axis
    int wny, wnx;        // window extent per axis
    __host__ __device__ int ngroups() const { return nry * nrx; }
};

__host__ inline Geo make_geo(int H, int W, int C, int s, int win, int K) {
    Geo g;
    g.H = H; g.W = W; g.C = C; g.s = s; g.win = win; g.K = K;
    g.nry = ref_count(H, s); g.nrx = ref_count(W, s);
    g.npy = H - PS + 1; g.npx = W - PS + 1;
    g.wny = win_len(g.npy, win); g.wnx = win_len(g.npx, win);
    return g;
}

// Footprint [f0, f1) along one axis of a tile of references [t*TR, t*TR+TR): the union of
// the search windows of its references, widened by ps - 1 (every matched patch lies inside).
__host__ __device__ inline void tile_span(int t, int TR, int nref, int s, int n, int npos, int wlen, int win,
                                          int& f0, int& f1) {
    int r0 = t * TR;
    int r1 = r0 + TR - 1;
    if (r1 > nref - 1) r1 = nref - 1;
    f0 = win_start(ref_pos(r0, s, n), npos, win);
    f1 = win_start(ref_pos(r1, s, n), npos, win) + wlen + PS - 1;
}

}  // namespace htsvd

// Host-side parameter resolution and filter tiling shared by the C-ABI entry points
// (api.cu, noalloc.cu), so that every entry point validates the same way and picks the same tiles.
#pragma once
#include <cstdint>

#include "../../include/htsvd.h"
#include "kernels.h"

namespace htsvd {

// Smallest relative gap between consecutive eigenvalues of a basis slice below which the slice's
// eigenvectors are treated as not unique (reading of the eigenvector convention, Sec. III-B.1).
constexpr double kDegenerateGap = 1e-9;

// htsvd_params with the defaults filled in (Sec. IV-A) and checked.
struct Resolved {
    int ps, s, win, K, match_mode, agg_mode, adapt, rank_gamma, tile;
    int strict_basis;          // eigen-gap check requested (strict mode or a gap output)
    double tau_mult, gamma, beta;
};

// Fills r from p (NULL: defaults). INVALID_ARG for negative sizes, a tile edge outside 0..16, K not a
// power of two in [2, 32] or an unknown mode; UNSUPPORTED for ps != 8, K > 32 or a window above 64.
htsvd_status resolve(const htsvd_params* p, int C, Resolved& r);
// Image checks shared by the entry points: C in {1, 3}, H, W >= ps, H W C < 2^31, and a search
// window holding at least K positions.
htsvd_status check_image(int H, int W, int C, const Resolved& r);
// Matching plane of the resolved mode (gray for C = 1).
int resolve_mode(const Resolved& r, int C);

struct FilterTiling {
    int TR, ntx, nty, FHmax, FWmax;
};
// Tile edge of the group filter: a forced edge (1..16) if its shared memory fits a CTA (TR = 0 if
// not), else the largest edge that keeps two CTAs per SM and still yields 8 waves.
FilterTiling choose_filter_tiling(const Geo& g, int in_bytes, int mode, int forced, int nfr = 1);

}  // namespace htsvd

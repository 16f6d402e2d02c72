// C ABI entry points: parameter resolution, workspace, launch sequences.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <chrono>
#include <mutex>
#include <string>
#include <thread>
#include <new>
#include <vector>

#include "../../include/htsvd.h"
#include "kernels.h"
#include "host_plan.h"

namespace htsvd {
bool symmetric_eigenvalues(double* A, int n, double* out);
}

using namespace htsvd;

namespace htsvd {

// ----------------------------------------------------------------------------- parameters

htsvd_status resolve(const htsvd_params* p, int C, Resolved& r) {
    htsvd_params z;
    std::memset(&z, 0, sizeof(z));
    if (!p) p = &z;
    r.ps = p->ps > 0 ? p->ps : 8;
    r.s = p->stride > 0 ? p->stride : 3;
    r.win = p->window > 0 ? p->window : 18;
    r.K = p->K > 0 ? p->K : 32;
    r.match_mode = p->match_mode;
    r.agg_mode = p->agg_mode;
    r.adapt = p->adapt;
    r.gamma = p->gcp_gamma > 0 ? p->gcp_gamma : 1.2;
    r.beta = p->beta > 0 ? p->beta : 1.2;
    r.rank_gamma = p->rank_gamma > 0 ? p->rank_gamma : (13 * r.K + 16) / 32;
    r.tile = p->tile;
    r.strict_basis = p->strict_basis != 0 || p->h_basis_gap_out != nullptr;
    if (p->stride < 0 || p->window < 0 || p->K < 0 || p->ps < 0) return HTSVD_ERR_INVALID_ARG;
    if (p->tile < 0 || p->tile > 16) return HTSVD_ERR_INVALID_ARG;
    if (r.K < 2 || (r.K & (r.K - 1))) return HTSVD_ERR_INVALID_ARG;
    if (r.match_mode < 0 || r.match_mode > 3 || r.agg_mode < 0 || r.agg_mode > 1) return HTSVD_ERR_INVALID_ARG;
    if (r.ps != PS || r.K > 32 || r.win > 64) return HTSVD_ERR_UNSUPPORTED;
    r.tau_mult = p->tau_mult > 0 ? p->tau_mult : std::sqrt(2.0 * std::log((double)C * r.K * r.ps * r.ps));
    return HTSVD_OK;
}

htsvd_status check_image(int H, int W, int C, const Resolved& r) {
    if (C != 1 && C != 3) return HTSVD_ERR_INVALID_ARG;
    if (H < r.ps || W < r.ps) return HTSVD_ERR_INVALID_ARG;
    if ((int64_t)H * W * C >= ((int64_t)1 << 31)) return HTSVD_ERR_UNSUPPORTED;
    Geo g = make_geo(H, W, C, r.s, r.win, r.K);
    if ((int64_t)g.wny * g.wnx < r.K) return HTSVD_ERR_INVALID_ARG;
    return HTSVD_OK;
}

int resolve_mode(const Resolved& r, int C) {
    if (C == 1) return MM_GRAY;
    switch (r.match_mode) {
        case HTSVD_MATCH_FULL: return MM_FULL;
        case HTSVD_MATCH_GREEN: return MM_GREEN;
        default: return MM_GCP;
    }
}

// ----------------------------------------------------------------------------- tiling choices

FilterTiling choose_filter_tiling(const Geo& g, int in_bytes, int mode, int forced, int nfr) {
    // Among the tiles whose shared memory lets two CTAs share an SM (228 KB, 1 KB reserved per
    // CTA): the largest that still gives 8 waves of two CTAs per SM (the last, partial wave then
    // costs little), else the largest with one such wave, else the largest that fits at all. A
    // forced edge is taken as given if its shared memory fits a CTA (TR = 0 returned otherwise).
    const int cands[] = {8, 7, 6, 5, 4, 3, 2, 1};
    const int64_t nsm = device_sm_count();
    FilterTiling fit2{}, fit1{}, wave1{};
    bool have2 = false, have1 = false, havew = false;
    if (forced > 0) {
        FilterTiling t{};
        t.TR = forced;
        t.ntx = (g.nrx + forced - 1) / forced;
        t.nty = (g.nry + forced - 1) / forced;
        t.FHmax = std::min(g.H, (forced - 1) * g.s + g.wny + PS - 1);
        t.FWmax = std::min(g.W, (forced - 1) * g.s + g.wnx + PS - 1);
        FilterArgs fa{};
        fa.g = g;
        fa.FHmax = t.FHmax;
        fa.FWmax = t.FWmax;
        fa.img_is_float = in_bytes == 4;
        fa.mode = mode;
        fa.nfr = nfr;
        if (filter_smem_bytes(fa) > 227 * 1024) t.TR = 0;
        return t;
    }
    for (int TR : cands) {
        FilterTiling t;
        t.TR = TR;
        t.ntx = (g.nrx + TR - 1) / TR;
        t.nty = (g.nry + TR - 1) / TR;
        t.FHmax = std::min(g.H, (TR - 1) * g.s + g.wny + PS - 1);
        t.FWmax = std::min(g.W, (TR - 1) * g.s + g.wnx + PS - 1);
        FilterArgs fa{};
        fa.g = g;
        fa.FHmax = t.FHmax;
        fa.FWmax = t.FWmax;
        fa.img_is_float = in_bytes == 4;
        fa.mode = mode;
        fa.nfr = nfr;
        const size_t smem = filter_smem_bytes(fa);
        if (smem <= 112 * 1024) {
            const int64_t tiles = (int64_t)t.ntx * t.nty;
            if (!have2) fit2 = t, have2 = true;
            if (tiles >= 8 * 2 * nsm) return t;
            if (tiles >= 2 * nsm && !havew) wave1 = t, havew = true;
        } else if (smem <= 200 * 1024 && !have1) {
            fit1 = t, have1 = true;
        }
    }
    return havew ? wave1 : have2 ? fit2 : fit1;
}

}  // namespace htsvd

namespace {

// ----------------------------------------------------------------------------- workspace

enum Slot {
    S_IDX, S_MOM, S_B64, S_B32, S_PART, S_FULLM, S_FULLS, S_RANKS, S_IDX2, S_Q, S_DEN, S_R, S_TMP,
    S_AIN, S_AOUT,                   // S_AIN, S_AOUT: parts of the adaptive image and volume calls
    S_COEF, S_CPN, S_CNRM,           // coefficient cache of htsvd_denoise_tau_sweep
    S_SOUT, S_SGX, S_SIDX, S_SRED,   // htsvd_sure: estimate, adjoint or perturbed image, grouping, sums
    S_GAP,                           // eigen-gaps of the basis slices (strict mode)
    S_WIDX0, S_WIDX1, S_WB64, S_WB32, S_WZ, S_WF, S_WU, S_WGX, S_WG2, S_WRED,   // weight tuning by SURE
    S_CSCR, S_CNUM, S_CDEN,          // hyperspectral cubes: per-CTA Haar slots, numerator, denominator
    S_PROJ,                          // split BF16 basis matrix of htsvd_project_patches
    S_VMOM, S_VB64, S_VNUM, S_VDEN,  // MRI volumes: moments, bases, numerator, denominator
    S_NSLOT
};

struct Workspace {
    int device = -1;
    cudaStream_t stream = nullptr;
    void* buf[S_NSLOT] = {};
    size_t cap[S_NSLOT] = {};
    void* hpin = nullptr;
    size_t hcap = 0;
    cudaStream_t side = nullptr;          // moments + basis run here (highest priority), concurrently with
                                          // block matching
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

std::mutex g_mu;
std::vector<Workspace*> g_ws;

Workspace* workspace_for(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    for (Workspace* w : g_ws)
        if (w->device == dev && w->stream == s) return w;
    Workspace* w = new (std::nothrow) Workspace();
    if (!w) return nullptr;
    w->device = dev;
    w->stream = s;
    g_ws.push_back(w);
    return w;
}

htsvd_status ws_get(Workspace* w, int slot, size_t bytes, void** out) {
    if (bytes == 0) bytes = 16;
    if (w->cap[slot] < bytes) {
        if (w->buf[slot]) {
            cudaFree(w->buf[slot]);
            w->buf[slot] = nullptr;
            w->cap[slot] = 0;
        }
        size_t b = bytes + bytes / 8;
        if (cudaMalloc(&w->buf[slot], b) != cudaSuccess) {
            cudaGetLastError();
            return HTSVD_ERR_OOM;
        }
        w->cap[slot] = b;
    }
    *out = w->buf[slot];
    return HTSVD_OK;
}

// Side stream and fork/join events of a workspace, created on first use.
htsvd_status ws_side(Workspace* w) {
    if (w->side) return HTSVD_OK;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);       // hi: numerically lowest = most urgent
    if (cudaStreamCreateWithPriority(&w->side, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&w->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return HTSVD_ERR_CUDA;
    }
    return HTSVD_OK;
}

htsvd_status ws_host(Workspace* w, size_t bytes, void** out) {
    if (w->hcap < bytes) {
        if (w->hpin) cudaFreeHost(w->hpin);
        w->hpin = nullptr;
        w->hcap = 0;
        if (cudaMallocHost(&w->hpin, bytes) != cudaSuccess) {
            cudaGetLastError();
            return HTSVD_ERR_OOM;
        }
        w->hcap = bytes;
    }
    *out = w->hpin;
    return HTSVD_OK;
}

// ----------------------------------------------------------------------------- kernel timing

struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
    double host_ms;       // >= 0: a host step timed with the wall clock (no events)
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;

// Brackets the launches made in its scope with events on `s` while profiling is enabled.
struct ProfScope {
    ProfRec r{nullptr, nullptr, nullptr, -1.0};
    cudaStream_t s;
    ProfScope(const char* name, cudaStream_t st) : s(st) {
        if (!g_prof_on) return;
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
            cudaGetLastError();
            r.a = r.b = nullptr;
            return;
        }
        r.name = name;
        cudaEventRecord(r.a, s);
    }
    ~ProfScope() {
        if (!r.name) return;
        cudaEventRecord(r.b, s);
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof.push_back(r);
    }
};

// Wall-clock timing of a host step, recorded under `name` while profiling is enabled.
struct HostProfScope {
    const char* name;
    std::chrono::steady_clock::time_point t0;
    explicit HostProfScope(const char* n) : name(g_prof_on ? n : nullptr) {
        if (name) t0 = std::chrono::steady_clock::now();
    }
    ~HostProfScope() {
        if (!name) return;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof.push_back(ProfRec{name, nullptr, nullptr, ms});
    }
};

#define CK(x)                                         \
    do {                                              \
        cudaError_t e_ = (x);                         \
        if (e_ != cudaSuccess) return HTSVD_ERR_CUDA; \
    } while (0)
#define ST(x)                               \
    do {                                    \
        htsvd_status s_ = (x);              \
        if (s_ != HTSVD_OK) return s_;      \
    } while (0)

void choose_bm_tiles(const Geo& g, int rstep, int& TRy, int& TRx) {
    TRy = 4;
    TRx = 8;
    (void)g;
    (void)rstep;
}

// ----------------------------------------------------------------------------- pieces

// Spatio-temporal context of one output frame of a clip: candidate frames f0 .. f0 + nfr - 1 of
// vid (fstride bytes apart), reference frame fref.
struct VideoCtx {
    const uint8_t* vid;
    long long fstride;
    int f0, nfr, fref;
};

htsvd_status run_block_match(const uint8_t* q, const Geo& g, const Resolved& r, int rstep, int32_t* idx,
                             cudaStream_t s, const VideoCtx* vc = nullptr) {
    BMArgs a{};
    a.img = q;
    if (vc) {
        a.vid = vc->vid;
        a.fstride = vc->fstride;
        a.f0 = vc->f0;
        a.nfr = vc->nfr;
        a.fref = vc->fref;
    }
    a.g = g;
    a.mode = resolve_mode(r, g.C);
    a.gamma2 = r.gamma * r.gamma;
    a.rstep = rstep;
    a.nry_s = (g.nry + rstep - 1) / rstep;
    a.nrx_s = (g.nrx + rstep - 1) / rstep;
    choose_bm_tiles(g, rstep, a.TRy, a.TRx);
    bm_fit_tiles(a);
    if (bm_smem_bytes(a) > 227 * 1024) return HTSVD_ERR_UNSUPPORTED;   // e.g. too many frames in reach
    a.idx = idx;
    { ProfScope ps_("block_match", s); CK(launch_block_match(a, s)); }
    return HTSVD_OK;
}

// Noise level from the covariance eigenvalues (host FP64). M, S: uint64 moments on the host.
double sigma_from_moments(const unsigned long long* M, const unsigned long long* S, int d, int64_t n,
                          double* lam_out = nullptr) {
    std::vector<double> A((size_t)d * d), lam(d);
    std::vector<double> mu(d);
    for (int u = 0; u < d; ++u) mu[u] = (double)S[u] / (double)n;
    for (int u = 0; u < d; ++u)          // lower triangle: all the eigensolver reads
        for (int v = 0; v <= u; ++v) A[(size_t)u * d + v] = (double)M[(size_t)u * d + v] / (double)n - mu[u] * mu[v];
    if (!symmetric_eigenvalues(A.data(), d, lam.data())) return -1.0;
    std::sort(lam.begin(), lam.end());
    if (lam_out) std::copy(lam.begin(), lam.end(), lam_out);
    int rstar = 1;
    double sum = 0.0;
    std::vector<double> pref(d + 1, 0.0);
    for (int r = 1; r <= d; ++r) {
        sum += lam[r - 1];
        pref[r] = sum;
        const double mean = sum / r;
        const double med = (r & 1) ? lam[(r - 1) / 2] : 0.5 * (lam[r / 2 - 1] + lam[r / 2]);
        if (mean <= 1.02 * med) rstar = r;
    }
    const double m = pref[rstar] / rstar;
    return std::sqrt(m > 0 ? m : 0.0);
}

// Launches the moments of the quantised image and the basis solve. With fullM (the full second
// moment of the same references, already formed on this stream's predecessors) the row and
// column moments are summed from it instead of re-read from the image.
htsvd_status run_basis(Workspace* w, const uint8_t* q, const Geo& g, double** b64, float** b32, cudaStream_t s,
                       const unsigned long long* fullM = nullptr, double* d_gap = nullptr) {
    void *mom, *p64, *p32;
    ST(ws_get(w, S_MOM, sizeof(unsigned long long) * 2 * PS2 * g.C * g.C, &mom));
    ST(ws_get(w, S_B64, sizeof(double) * 2 * 2 * g.C * PS2, &p64));
    ST(ws_get(w, S_B32, sizeof(float) * 512, &p32));
    if (fullM) {
        ProfScope ps_("moments_from_full", s);
        CK(launch_moments_from_full(fullM, g.C, (unsigned long long*)mom, s));
    } else {
        ProfScope ps_("moments", s);
        CK(launch_moments(q, g, (unsigned long long*)mom, s));
    }
    { ProfScope ps_("basis", s); CK(launch_basis((const unsigned long long*)mom, g.C, (double*)p64, (float*)p32, s, d_gap)); }
    *b64 = (double*)p64;
    *b32 = (float*)p32;
    return HTSVD_OK;
}

// Strict-mode eigen-gap check: waits for the per-slice gaps of the basis solve (queued on s), writes
// the smallest to p->h_basis_gap_out and fails with DEGENERATE_BASIS below kDegenerateGap when
// p->strict_basis is set.
htsvd_status check_basis_gap(const double* d_gap, int C, const htsvd_params* p, cudaStream_t s) {
    const int n = basis_problems(C);
    std::vector<double> h((size_t)n);
    CK(cudaMemcpyAsync(h.data(), d_gap, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double m = h[0];
    for (int i = 1; i < n; ++i) m = std::min(m, h[i]);
    if (p->h_basis_gap_out) *p->h_basis_gap_out = m;
    if (p->strict_basis && !(m >= kDegenerateGap)) return HTSVD_ERR_DEGENERATE_BASIS;
    return HTSVD_OK;
}

// Launches what the estimate needs (full moment, optional sampled grouping and ranks) and
// copies it to pinned host memory; *done is recorded after the copies.
// Host bytes of the estimate's inputs: moment M (d x d), sums S (d), rank votes of the sampled groups.
size_t sigma_host_bytes(const Geo& g) {
    const int d = PS2 * g.C;
    const int ny8 = (g.nry + 7) / 8, nx8 = (g.nrx + 7) / 8;
    return sizeof(unsigned long long) * ((size_t)d * d + d) + sizeof(int32_t) * ny8 * nx8;
}

// Launches what the estimate needs (full moment, optional sampled grouping and ranks) and copies
// it to the pinned host memory at h (sigma_host_bytes(g) bytes).
htsvd_status enqueue_sigma_inputs(Workspace* w, const uint8_t* q, const Geo& g, const Resolved& r, cudaStream_t s,
                                  unsigned long long* h) {
    const int d = PS2 * g.C;
    void *M, *S;
    ST(ws_get(w, S_FULLM, sizeof(unsigned long long) * d * d, &M));
    ST(ws_get(w, S_FULLS, sizeof(unsigned long long) * d, &S));
    { ProfScope ps_("full_moment", s); CK(launch_full_moment(q, g, (unsigned long long*)M, (unsigned long long*)S, s)); }
    const int ny8 = (g.nry + 7) / 8, nx8 = (g.nrx + 7) / 8;
    CK(cudaMemcpyAsync(h, M, sizeof(unsigned long long) * d * d, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h + (size_t)d * d, S, sizeof(unsigned long long) * d, cudaMemcpyDeviceToHost, s));
    if (r.adapt) {
        void *idx2, *ranks;
        ST(ws_get(w, S_IDX2, sizeof(int32_t) * ny8 * nx8 * g.K, &idx2));
        ST(ws_get(w, S_RANKS, sizeof(int32_t) * ny8 * nx8, &ranks));
        ST(run_block_match(q, g, r, 8, (int32_t*)idx2, s));
        { ProfScope ps_("group_rank", s); CK(launch_group_rank(q, g, (const int32_t*)idx2, ny8 * nx8, (int32_t*)ranks, s)); }
        CK(cudaMemcpyAsync(h + (size_t)d * d + d, ranks, sizeof(int32_t) * ny8 * nx8, cudaMemcpyDeviceToHost, s));
    }
    return HTSVD_OK;
}

htsvd_status launch_sigma_inputs(Workspace* w, const uint8_t* q, const Geo& g, const Resolved& r, cudaStream_t s,
                                 void** hbuf) {
    ST(ws_host(w, sigma_host_bytes(g), hbuf));
    return enqueue_sigma_inputs(w, q, g, r, s, (unsigned long long*)*hbuf);
}

htsvd_status finish_sigma(const void* hbuf, const Geo& g, const Resolved& r, double* sigma) {
    const int d = PS2 * g.C;
    const unsigned long long* h = (const unsigned long long*)hbuf;
    double sg;
    {
        HostProfScope hp_("sigma_host");
        sg = sigma_from_moments(h, h + (size_t)d * d, d, (int64_t)g.ngroups());
    }
    if (sg < 0) return HTSVD_ERR_CUDA;
    if (r.adapt) {
        const int ny8 = (g.nry + 7) / 8, nx8 = (g.nrx + 7) / 8;
        const int32_t* ranks = (const int32_t*)(h + (size_t)d * d + d);
        int low = 0, high = 0;
        for (int i = 0; i < ny8 * nx8; ++i) (ranks[i] <= r.rank_gamma ? low : high)++;
        if (low > high) sg /= r.beta;
    }
    *sigma = sg;
    return HTSVD_OK;
}

struct FilterOut {
    float* out;
    float* den_out;
};

// Filter + reduce for the forward pass.
// Coefficient cache of the noisy groups (FM_ANALYZE writes it, FM_SYNTH reads it).
struct CoefCache {
    float* coef;
    float* pn;
    int* nrm;
    int mode;                // FM_ANALYZE or FM_SYNTH
};

htsvd_status run_forward_filter(Workspace* w, const void* img, int is_float, const Geo& g, const Resolved& r,
                                const int32_t* idx, const double* b64, const float* b32, double tau,
                                const float* w_in, const htsvd_params* p, float* d_out, cudaStream_t s,
                                const VideoCtx* vc = nullptr, const CoefCache* cc = nullptr) {
    const int mode = vc ? FM_VIDEO : cc ? cc->mode : FM_FORWARD;
    FilterTiling t = choose_filter_tiling(g, is_float ? 4 : 1, mode, r.tile, vc ? vc->nfr : 1);
    if (t.TR == 0) return HTSVD_ERR_UNSUPPORTED;
    FilterArgs a{};
    a.img = img;
    a.img_is_float = is_float;
    a.g = g;
    a.TR = t.TR;
    a.ntx = t.ntx;
    a.nty = t.nty;
    a.FHmax = t.FHmax;
    a.FWmax = t.FWmax;
    a.idx = idx;
    a.basis32 = b32;
    a.basis64 = b64;
    a.tau64 = tau;
    a.tau32 = (float)tau;
    a.band_rel = kBandRel;
    a.band_abs = (float)(tau * kBandTau) + 1e-6f;
    a.w_in = w_in;
    a.agg_mode = r.agg_mode;
    a.mode = mode;
    if (vc) {
        a.vid = vc->vid;
        a.fstride = vc->fstride;                  // uint8 elements = bytes
        a.f0 = vc->f0;
        a.nfr = vc->nfr;
        a.fref = vc->fref;
    }
    if (cc) {
        a.cache_coef = cc->coef;
        a.cache_pn = cc->pn;
        a.cache_nrm = cc->nrm;
    }
    a.mask_out = p ? p->d_mask_out : nullptr;
    a.weights_out = p ? p->d_weights_out : nullptr;
    a.coef_out = p ? p->d_coef_out : nullptr;
    void* part;
    const int acc = g.C == 3 ? 4 : 2;
    ST(ws_get(w, S_PART, sizeof(float) * (size_t)t.ntx * t.nty * t.FHmax * t.FWmax * acc, &part));
    a.partials = (float*)part;
    if (mode == FM_ANALYZE) {
        ProfScope ps_("filter_analyze", s);
        CK(launch_filter(a, s));
        return HTSVD_OK;
    }
    { ProfScope ps_(mode == FM_SYNTH ? "filter_synth" : "filter", s); CK(launch_filter(a, s)); }
    { ProfScope ps_("reduce", s); CK(launch_reduce((float*)part, g, t.TR, t.ntx, t.nty, t.FHmax, t.FWmax, d_out, nullptr, 0, nullptr, s)); }
    return HTSVD_OK;
}

// Owns the event that marks the estimate's inputs on the host's side of a call; destroyed on
// every return path.
struct HostEvent {
    cudaEvent_t ev = nullptr;
    ~HostEvent() {
        if (ev) cudaEventDestroy(ev);
    }
};

htsvd_status denoise_impl(const void* d_in, int is_float, int H, int W, int C, double sigma, const htsvd_params* p,
                          const float* d_w, float* d_out, int32_t* d_idx_out, cudaStream_t s) {
    if (!d_in || !d_out) return HTSVD_ERR_INVALID_ARG;
    Resolved r;
    ST(resolve(p, C, r));
    ST(check_image(H, W, C, r));
    if (std::isnan(sigma)) return HTSVD_ERR_INVALID_ARG;
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    const Geo g = make_geo(H, W, C, r.s, r.win, r.K);
    const int64_t N = g.ngroups();
    const uint8_t* q = (const uint8_t*)d_in;
    if (is_float) {
        void* qb;
        ST(ws_get(w, S_Q, (size_t)H * W * C, &qb));
        { ProfScope ps_("quantize", s); CK(launch_quantize((const float*)d_in, (int64_t)H * W * C, (uint8_t*)qb, s)); }
        q = (const uint8_t*)qb;
    }
    int32_t* idx = d_idx_out;
    if (!idx) {
        void* ib;
        ST(ws_get(w, S_IDX, sizeof(int32_t) * N * r.K, &ib));
        idx = (int32_t*)ib;
    }
    void* hbuf = nullptr;
    if (sigma < 0) ST(launch_sigma_inputs(w, q, g, r, s, &hbuf));
    HostEvent hev;
    if (sigma < 0) {
        CK(cudaEventCreateWithFlags(&hev.ev, cudaEventDisableTiming));
        CK(cudaEventRecord(hev.ev, s));
    }
    // Grouping and the bases do not depend on sigma: they run while the host finishes the estimate,
    // the bases on the side stream concurrently with block matching (joined before the filter).
    ST(ws_side(w));
    CK(cudaEventRecord(w->ev_fork, s));
    CK(cudaStreamWaitEvent(w->side, w->ev_fork, 0));
    double* b64;
    float* b32;
    void* fullM = nullptr;
    if (sigma < 0) ST(ws_get(w, S_FULLM, sizeof(unsigned long long) * PS2 * C * PS2 * C, &fullM));
    void* gap = nullptr;
    if (r.strict_basis) ST(ws_get(w, S_GAP, sizeof(double) * basis_problems(C), &gap));
    ST(run_basis(w, q, g, &b64, &b32, w->side, (const unsigned long long*)fullM, (double*)gap));
    CK(cudaEventRecord(w->ev_join, w->side));
    ST(run_block_match(q, g, r, 1, idx, s));
    CK(cudaStreamWaitEvent(s, w->ev_join, 0));
    if (p && p->d_basis_out)
        CK(cudaMemcpyAsync(p->d_basis_out, b64, sizeof(double) * 2 * 2 * C * PS2, cudaMemcpyDeviceToDevice, s));
    if (r.strict_basis) ST(check_basis_gap((const double*)gap, C, p, s));
    if (sigma < 0) {
        if (cudaEventSynchronize(hev.ev) != cudaSuccess) return HTSVD_ERR_CUDA;
        ST(finish_sigma(hbuf, g, r, &sigma));
    }
    if (p && p->h_sigma_out) *p->h_sigma_out = sigma;
    const double tau = r.tau_mult * sigma;
    return run_forward_filter(w, is_float ? d_in : (const void*)q, is_float, g, r, idx, b64, b32, tau, d_w, p, d_out,
                              s);
}

// A clip, frame by frame (real-world color video denoising, Sec. IV): output frame t is Alg. 1 on
// frame t (its own sigma, estimated or given, and its own global bases), except that grouping
// searches the spatial window in frames t - T .. t + T and only the patches lying in frame t are
// aggregated into it.
htsvd_status video_impl(const uint8_t* d_vid, int F, int H, int W, int C, int T, double sigma,
                        const htsvd_params* p, float* d_out, int32_t* d_idx_out, double* h_sigmas, cudaStream_t s) {
    if (!d_vid || !d_out || F < 1 || T < 0) return HTSVD_ERR_INVALID_ARG;
    Resolved r;
    ST(resolve(p, C, r));
    ST(check_image(H, W, C, r));
    if (std::isnan(sigma)) return HTSVD_ERR_INVALID_ARG;
    if ((int64_t)F * H * W >= ((int64_t)1 << 31)) return HTSVD_ERR_UNSUPPORTED;   // int32 global indices
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    const Geo g = make_geo(H, W, C, r.s, r.win, r.K);
    const int64_t N = g.ngroups();
    const long long fr = (long long)H * W * C;
    void* ib = nullptr;
    if (!d_idx_out) ST(ws_get(w, S_IDX, sizeof(int32_t) * N * r.K, &ib));
    ST(ws_side(w));
    for (int t = 0; t < F; ++t) {
        int32_t* idx = d_idx_out ? d_idx_out + (size_t)t * N * r.K : (int32_t*)ib;
        const uint8_t* q = d_vid + t * fr;
        double sg = sigma;
        void* hbuf = nullptr;
        HostEvent hev;
        if (sg < 0) {
            ST(launch_sigma_inputs(w, q, g, r, s, &hbuf));
            CK(cudaEventCreateWithFlags(&hev.ev, cudaEventDisableTiming));
            CK(cudaEventRecord(hev.ev, s));
        }
        CK(cudaEventRecord(w->ev_fork, s));
        CK(cudaStreamWaitEvent(w->side, w->ev_fork, 0));
        double* b64;
        float* b32;
        void* fullM = nullptr;
        if (sg < 0) ST(ws_get(w, S_FULLM, sizeof(unsigned long long) * PS2 * C * PS2 * C, &fullM));
        ST(run_basis(w, q, g, &b64, &b32, w->side, (const unsigned long long*)fullM));
        CK(cudaEventRecord(w->ev_join, w->side));
        const int f0 = std::max(0, t - T), f1 = std::min(F - 1, t + T);
        const VideoCtx vc{d_vid, fr, f0, f1 - f0 + 1, t};
        ST(run_block_match(q, g, r, 1, idx, s, &vc));
        CK(cudaStreamWaitEvent(s, w->ev_join, 0));
        if (sg < 0) {
            if (cudaEventSynchronize(hev.ev) != cudaSuccess) return HTSVD_ERR_CUDA;
            ST(finish_sigma(hbuf, g, r, &sg));
        }
        if (h_sigmas) h_sigmas[t] = sg;
        ST(run_forward_filter(w, q, 0, g, r, idx, b64, b32, r.tau_mult * sg, nullptr, nullptr, d_out + t * fr, s,
                              &vc));
    }
    return HTSVD_OK;
}

// A sweep of thresholds over one image with the grouping, bases, sigma and the noisy group
// coefficients computed once and cached (the speed-up of parameter tuning that Sec. III-E
// points to): output i is Alg. 1 at tau = tau_mults[i] * sigma.
htsvd_status sweep_impl(const uint8_t* d_in, int H, int W, int C, double sigma, const double* tau_mults, int n_tau,
                        const htsvd_params* p, float* d_outs, double* h_sigma, cudaStream_t s) {
    if (!d_in || !d_outs || !tau_mults || n_tau < 1) return HTSVD_ERR_INVALID_ARG;
    for (int i = 0; i < n_tau; ++i)
        if (!(tau_mults[i] >= 0.0) || std::isinf(tau_mults[i])) return HTSVD_ERR_INVALID_ARG;
    Resolved r;
    ST(resolve(p, C, r));
    ST(check_image(H, W, C, r));
    if (std::isnan(sigma)) return HTSVD_ERR_INVALID_ARG;
    if (r.K < 8) return HTSVD_ERR_UNSUPPORTED;
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    const Geo g = make_geo(H, W, C, r.s, r.win, r.K);
    const int64_t N = g.ngroups();
    void *ib, *cc, *cp, *cn;
    ST(ws_get(w, S_IDX, sizeof(int32_t) * N * r.K, &ib));
    ST(ws_get(w, S_COEF, sizeof(float) * (size_t)N * r.K * PS2 * C, &cc));
    ST(ws_get(w, S_CPN, sizeof(float) * (size_t)N * 32, &cp));
    ST(ws_get(w, S_CNRM, sizeof(int) * (size_t)N, &cn));
    int32_t* idx = (int32_t*)ib;
    void* hbuf = nullptr;
    HostEvent hev;
    if (sigma < 0) {
        ST(launch_sigma_inputs(w, d_in, g, r, s, &hbuf));
        CK(cudaEventCreateWithFlags(&hev.ev, cudaEventDisableTiming));
        CK(cudaEventRecord(hev.ev, s));
    }
    ST(ws_side(w));
    CK(cudaEventRecord(w->ev_fork, s));
    CK(cudaStreamWaitEvent(w->side, w->ev_fork, 0));
    double* b64;
    float* b32;
    void* fullM = nullptr;
    if (sigma < 0) ST(ws_get(w, S_FULLM, sizeof(unsigned long long) * PS2 * C * PS2 * C, &fullM));
    ST(run_basis(w, d_in, g, &b64, &b32, w->side, (const unsigned long long*)fullM));
    CK(cudaEventRecord(w->ev_join, w->side));
    ST(run_block_match(d_in, g, r, 1, idx, s));
    CK(cudaStreamWaitEvent(s, w->ev_join, 0));
    // the noisy coefficients (tau plays no part in the analysis)
    CoefCache cache{(float*)cc, (float*)cp, (int*)cn, FM_ANALYZE};
    ST(run_forward_filter(w, d_in, 0, g, r, idx, b64, b32, 0.0, nullptr, nullptr, nullptr, s, nullptr, &cache));
    if (sigma < 0) {
        if (cudaEventSynchronize(hev.ev) != cudaSuccess) return HTSVD_ERR_CUDA;
        ST(finish_sigma(hbuf, g, r, &sigma));
    }
    if (h_sigma) *h_sigma = sigma;
    cache.mode = FM_SYNTH;
    const size_t img = (size_t)H * W * C;
    for (int i = 0; i < n_tau; ++i)
        ST(run_forward_filter(w, d_in, 0, g, r, idx, b64, b32, tau_mults[i] * sigma, nullptr, nullptr,
                              d_outs + i * img, s, nullptr, &cache));
    return HTSVD_OK;
}

// The VJP's device passes with grouping and bases given (FP64 b64 and packed FP32 b32): the
// denominator D, r = gout / D, and the adjoint filter on r with the masks of x at tau.
htsvd_status vjp_core(Workspace* w, const float* d_x, const Geo& g, const Resolved& r, const int32_t* d_idx,
                      const float* d_w, const double* b64, const float* b32, double tau, const float* d_out,
                      const float* d_grad_out, float* d_grad_x, float* d_grad_w, cudaStream_t s) {
    const int C = g.C;
    const int64_t npix = (int64_t)g.H * g.W;
    void *den, *rimg, *tmp;
    ST(ws_get(w, S_DEN, sizeof(float) * npix, &den));
    ST(ws_get(w, S_R, sizeof(float) * npix * C, &rimg));
    ST(ws_get(w, S_TMP, sizeof(float) * npix * C, &tmp));

    // D = sum_g w_g Scatter_g 1
    FilterTiling td = choose_filter_tiling(g, 4, FM_DENOM, r.tile);
    if (td.TR == 0) return HTSVD_ERR_UNSUPPORTED;
    FilterArgs a{};
    a.img = d_x;
    a.img_is_float = 1;
    a.g = g;
    a.idx = d_idx;
    a.basis32 = b32;
    a.basis64 = b64;
    a.tau64 = tau;
    a.tau32 = (float)tau;
    a.band_rel = kBandRel;
    a.band_abs = (float)(tau * kBandTau) + 1e-6f;
    a.w_in = d_w;
    a.agg_mode = 0;
    a.mode = FM_DENOM;
    a.TR = td.TR;
    a.ntx = td.ntx;
    a.nty = td.nty;
    a.FHmax = td.FHmax;
    a.FWmax = td.FWmax;
    const int acc = C == 3 ? 4 : 2;
    void* part;
    ST(ws_get(w, S_PART, sizeof(float) * (size_t)td.ntx * td.nty * td.FHmax * td.FWmax * acc, &part));
    a.partials = (float*)part;
    { ProfScope ps_("filter", s); CK(launch_filter(a, s)); }
    { ProfScope ps_("reduce", s); CK(launch_reduce((float*)part, g, td.TR, td.ntx, td.nty, td.FHmax, td.FWmax, (float*)tmp, (float*)den, 0,
                     nullptr, s)); }
    { ProfScope ps_("div", s); CK(launch_div(d_grad_out, (const float*)den, npix, C, (float*)rimg, s)); }

    // adjoint filter on r = gout / D with the masks of x
    FilterTiling ta = choose_filter_tiling(g, 4, FM_ADJOINT, r.tile);
    if (ta.TR == 0) return HTSVD_ERR_UNSUPPORTED;
    a.mode = FM_ADJOINT;
    a.TR = ta.TR;
    a.ntx = ta.ntx;
    a.nty = ta.nty;
    a.FHmax = ta.FHmax;
    a.FWmax = ta.FWmax;
    a.r_img = (const float*)rimg;
    a.out_img = d_out;
    a.grad_w = d_grad_w;
    ST(ws_get(w, S_PART, sizeof(float) * (size_t)ta.ntx * ta.nty * ta.FHmax * ta.FWmax * acc, &part));
    a.partials = (float*)part;
    { ProfScope ps_("filter", s); CK(launch_filter(a, s)); }
    { ProfScope ps_("reduce", s); CK(launch_reduce((float*)part, g, ta.TR, ta.ntx, ta.nty, ta.FHmax, ta.FWmax, d_grad_x, nullptr, 1, nullptr, s)); }
    return HTSVD_OK;
}

// SURE of the per-group weights (reading R19). The grouping and the bases of y and of z = y + eps b
// do not depend on w: prepared once, then any number of evaluations.
struct SureW {
    Geo g;
    Resolved r;
    int64_t n = 0, ng = 0;
    double sigma = 0.0, eps = 0.0, tau = 0.0;
    const float* y = nullptr;
    const float* b = nullptr;
    const float* img[2] = {};       // y, z
    int32_t* idx[2] = {};
    double* b64[2] = {};
    float* b32[2] = {};
};

htsvd_status sure_w_prepare(Workspace* w, const float* d_y, int H, int W, int C, double sigma, const float* d_probe,
                            double eps, const htsvd_params* p, SureW& c, cudaStream_t s) {
    if (!d_y || !d_probe) return HTSVD_ERR_INVALID_ARG;
    if (!(sigma > 0) || std::isinf(sigma)) return HTSVD_ERR_INVALID_ARG;
    if (!(eps > 0.0) || !std::isfinite((float)eps) || !((float)eps > 0.0f)) return HTSVD_ERR_INVALID_ARG;
    ST(resolve(p, C, c.r));
    ST(check_image(H, W, C, c.r));
    c.g = make_geo(H, W, C, c.r.s, c.r.win, c.r.K);
    c.n = (int64_t)H * W * C;
    c.ng = c.g.ngroups();
    c.sigma = sigma;
    c.eps = eps;
    c.tau = c.r.tau_mult * sigma;
    c.y = d_y;
    c.b = d_probe;
    void *z, *i0, *i1, *b64, *b32, *qb;
    ST(ws_get(w, S_WZ, sizeof(float) * c.n, &z));
    ST(ws_get(w, S_WIDX0, sizeof(int32_t) * c.ng * c.r.K, &i0));
    ST(ws_get(w, S_WIDX1, sizeof(int32_t) * c.ng * c.r.K, &i1));
    ST(ws_get(w, S_WB64, sizeof(double) * 2 * 2 * 2 * C * PS2, &b64));
    ST(ws_get(w, S_WB32, sizeof(float) * 2 * 512, &b32));
    ST(ws_get(w, S_Q, (size_t)c.n, &qb));
    { ProfScope ps_("perturb", s); CK(launch_perturb(d_y, d_probe, (float)eps, c.n, (float*)z, s)); }
    c.img[0] = d_y;
    c.img[1] = (const float*)z;
    c.idx[0] = (int32_t*)i0;
    c.idx[1] = (int32_t*)i1;
    for (int k = 0; k < 2; ++k) {
        c.b64[k] = (double*)b64 + (size_t)k * 2 * 2 * C * PS2;
        c.b32[k] = (float*)b32 + (size_t)k * 512;
        { ProfScope ps_("quantize", s); CK(launch_quantize(c.img[k], c.n, (uint8_t*)qb, s)); }
        double* p64;
        float* p32;
        ST(run_basis(w, (const uint8_t*)qb, c.g, &p64, &p32, s));
        CK(cudaMemcpyAsync(c.b64[k], p64, sizeof(double) * 2 * 2 * C * PS2, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c.b32[k], p32, sizeof(float) * 512, cudaMemcpyDeviceToDevice, s));
        ST(run_block_match((const uint8_t*)qb, c.g, c.r, 1, c.idx[k], s));
    }
    return HTSVD_OK;
}

// SURE(w) to *h_sure (HOST; synchronises s) and its gradient to d_grad_w.
htsvd_status sure_w_eval(Workspace* w, const SureW& c, const float* d_w, double* h_sure, float* d_grad_w,
                         cudaStream_t s) {
    void *f, *u, *gx, *g2, *red;
    ST(ws_get(w, S_WF, sizeof(float) * c.n, &f));
    ST(ws_get(w, S_WU, sizeof(float) * c.n, &u));
    ST(ws_get(w, S_WGX, sizeof(float) * c.n, &gx));
    ST(ws_get(w, S_WG2, sizeof(float) * c.ng, &g2));
    ST(ws_get(w, S_WRED, sizeof(double) * (sure_scratch_doubles() + 4), &red));
    double* scratch = (double*)red;
    double* terms = scratch + sure_scratch_doubles();   // |f_y - y|^2, b.f_y, |f_z - z|^2, b.f_z
    // beta = 2 sigma^2 / (n eps): the divergence's weight in SURE
    const double beta = 2.0 * c.sigma * c.sigma / ((double)c.n * c.eps);
    for (int k = 0; k < 2; ++k) {
        ST(run_forward_filter(w, c.img[k], 1, c.g, c.r, c.idx[k], c.b64[k], c.b32[k], c.tau, d_w, nullptr, (float*)f,
                              s));
        { ProfScope ps_("sure_terms", s);
          CK(launch_sure_terms((const float*)f, c.img[k], c.b, (const float*)f, c.n, scratch, terms + 2 * k, s)); }
        // cotangents: (2/n)(f_y - y) - beta b at y, beta b at z
        { ProfScope ps_("cotangent", s);
          CK(launch_sure_cotangent((const float*)f, c.img[k], c.b, k == 0 ? (float)(2.0 / (double)c.n) : 0.f,
                                   k == 0 ? (float)beta : -(float)beta, c.n, (float*)u, s)); }
        ST(vjp_core(w, c.img[k], c.g, c.r, c.idx[k], d_w, c.b64[k], c.b32[k], c.tau, (const float*)f,
                    (const float*)u, (float*)gx, k == 0 ? d_grad_w : (float*)g2, s));
    }
    { ProfScope ps_("add", s); CK(launch_add((const float*)g2, d_grad_w, c.ng, s)); }
    double h[4];
    CK(cudaMemcpyAsync(h, terms, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *h_sure = h[0] / (double)c.n - c.sigma * c.sigma + beta * (h[3] - h[1]);
    return HTSVD_OK;
}

}  // namespace

// ============================================================================= C ABI

extern "C" {

int32_t htsvd_internal_sampled_ranks(const uint8_t* d_img, int32_t H, int32_t W, int32_t C, const htsvd_params* p,
                                     int32_t* h_ranks, int32_t max_ranks) {
    Resolved r;
    if (!d_img || !h_ranks || resolve(p, C, r) != HTSVD_OK || check_image(H, W, C, r) != HTSVD_OK) return -1;
    const Geo g = make_geo(H, W, C, r.s, r.win, r.K);
    const int ny8 = (g.nry + 7) / 8, nx8 = (g.nrx + 7) / 8, n = ny8 * nx8;
    if (n > max_ranks) return -1;
    Workspace* w = workspace_for(nullptr);
    if (!w) return -1;
    void *idx2, *ranks;
    if (ws_get(w, S_IDX2, sizeof(int32_t) * n * g.K, &idx2) != HTSVD_OK ||
        ws_get(w, S_RANKS, sizeof(int32_t) * n, &ranks) != HTSVD_OK)
        return -1;
    if (run_block_match(d_img, g, r, 8, (int32_t*)idx2, nullptr) != HTSVD_OK) return -1;
    if (launch_group_rank(d_img, g, (const int32_t*)idx2, n, (int32_t*)ranks, nullptr) != cudaSuccess) return -1;
    if (cudaMemcpy(h_ranks, ranks, sizeof(int32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return n;
}

int32_t htsvd_internal_filter_tile(int32_t H, int32_t W, int32_t C, const htsvd_params* p) {
    Resolved r;
    if (resolve(p, C, r) != HTSVD_OK || check_image(H, W, C, r) != HTSVD_OK) return -1;
    return choose_filter_tiling(make_geo(H, W, C, r.s, r.win, r.K), 1, FM_FORWARD, r.tile).TR;
}

double htsvd_internal_sigma_from_moments(const unsigned long long* M, const unsigned long long* S, int d, int64_t n,
                                         double* lam) {
    if (!M || !S || d < 1 || n < 1) return -1.0;
    return sigma_from_moments(M, S, d, n, lam);
}

htsvd_status htsvd_denoise(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, double sigma,
                           const htsvd_params* p, float* d_out, int32_t* d_idx_out, cudaStream_t stream) {
    return denoise_impl(d_noisy, 0, H, W, C, sigma, p, nullptr, d_out, d_idx_out, stream);
}

htsvd_status htsvd_denoise_video(const uint8_t* d_video, int32_t F, int32_t H, int32_t W, int32_t C, int32_t T,
                                 double sigma, const htsvd_params* p, float* d_out, int32_t* d_idx_out,
                                 double* h_sigmas, cudaStream_t stream) {
    return video_impl(d_video, F, H, W, C, T, sigma, p, d_out, d_idx_out, h_sigmas, stream);
}

htsvd_status htsvd_denoise_tau_sweep(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, double sigma,
                                     const double* h_tau_mults, int32_t n_tau, const htsvd_params* p,
                                     float* d_outs, double* h_sigma, cudaStream_t stream) {
    return sweep_impl(d_noisy, H, W, C, sigma, h_tau_mults, n_tau, p, d_outs, h_sigma, stream);
}

htsvd_status htsvd_denoise_f32(const float* d_x, int32_t H, int32_t W, int32_t C, double sigma,
                               const htsvd_params* p, const float* d_w, float* d_out, int32_t* d_idx_out,
                               cudaStream_t stream) {
    return denoise_impl(d_x, 1, H, W, C, sigma, p, d_w, d_out, d_idx_out, stream);
}

htsvd_status htsvd_estimate_sigma(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, const htsvd_params* p,
                                  double* h_sigma, cudaStream_t stream) {
    if (!d_noisy || !h_sigma) return HTSVD_ERR_INVALID_ARG;
    Resolved r;
    ST(resolve(p, C, r));
    ST(check_image(H, W, C, r));
    Workspace* w = workspace_for(stream);
    if (!w) return HTSVD_ERR_OOM;
    const Geo g = make_geo(H, W, C, r.s, r.win, r.K);
    void* hbuf;
    ST(launch_sigma_inputs(w, d_noisy, g, r, stream, &hbuf));
    CK(cudaStreamSynchronize(stream));
    return finish_sigma(hbuf, g, r, h_sigma);
}

htsvd_status htsvd_denoise_adaptive(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, int32_t sub_h,
                                    int32_t sub_w, const htsvd_params* p, float* d_out, double* h_sigmas,
                                    cudaStream_t s) {
    if (!d_noisy || !d_out || sub_h < 1 || sub_w < 1) return HTSVD_ERR_INVALID_ARG;
    Resolved r;
    ST(resolve(p, C, r));
    ST(check_image(H, W, C, r));
    // subimage bounds per axis: t = max(1, n / n_sub) parts, boundaries floor(i n / t)
    auto bounds = [](int n, int sub) {
        const int t = std::max(1, n / sub);
        std::vector<int> b(t + 1);
        for (int i = 0; i <= t; ++i) b[i] = (int)(((int64_t)i * n) / t);
        return b;
    };
    const std::vector<int> by = bounds(H, sub_h), bx = bounds(W, sub_w);
    const int ny = (int)by.size() - 1, nx = (int)bx.size() - 1, n = ny * nx;
    struct Tile {
        int y0, x0, h, w;
        Geo g;
        size_t in_off, out_off, h_off;
    };
    std::vector<Tile> tiles(n);
    size_t in_bytes = 0, out_bytes = 0, h_bytes = 0;
    for (int t = 0; t < n; ++t) {
        Tile& T = tiles[t];
        T.y0 = by[t / nx];
        T.x0 = bx[t % nx];
        T.h = by[t / nx + 1] - T.y0;
        T.w = bx[t % nx + 1] - T.x0;
        ST(check_image(T.h, T.w, C, r));
        T.g = make_geo(T.h, T.w, C, r.s, r.win, r.K);
        T.in_off = in_bytes;
        T.out_off = out_bytes;
        T.h_off = h_bytes;
        in_bytes += ((size_t)T.h * T.w * C + 255) & ~(size_t)255;
        out_bytes += (sizeof(float) * T.h * T.w * C + 255) & ~(size_t)255;
        h_bytes += (sigma_host_bytes(T.g) + 15) & ~(size_t)15;
    }
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    void *vin, *vout, *vh;
    ST(ws_get(w, S_AIN, in_bytes, &vin));
    ST(ws_get(w, S_AOUT, out_bytes, &vout));
    ST(ws_host(w, h_bytes, &vh));
    uint8_t* tin = (uint8_t*)vin;
    unsigned char* tout = (unsigned char*)vout;
    unsigned char* hb = (unsigned char*)vh;
    // Step 1 (Alg. 2): copy each subimage out and launch the inputs of its noise estimate
    for (const Tile& T : tiles) {
        CK(cudaMemcpy2DAsync(tin + T.in_off, (size_t)T.w * C, d_noisy + ((size_t)T.y0 * W + T.x0) * C, (size_t)W * C,
                             (size_t)T.w * C, T.h, cudaMemcpyDeviceToDevice, s));
        ST(enqueue_sigma_inputs(w, tin + T.in_off, T.g, r, s, (unsigned long long*)(hb + T.h_off)));
    }
    CK(cudaStreamSynchronize(s));
    // host eigenvalue problems of the subimages are independent: a few threads share them
    std::vector<double> sig(n, 0.0);
    std::vector<htsvd_status> st(n, HTSVD_OK);
    {
        const unsigned hw = std::thread::hardware_concurrency();
        const int nth = std::max(1, std::min(n, (int)std::min(8u, hw > 1 ? hw / 2 : 1u)));
        auto work = [&](int k) {
            for (int t = k; t < n; t += nth) st[t] = finish_sigma(hb + tiles[t].h_off, tiles[t].g, r, &sig[t]);
        };
        std::vector<std::thread> th;
        try {
            for (int k = 1; k < nth; ++k) th.emplace_back(work, k);
        } catch (...) {
        }
        work(0);
        for (int k = 1; k < nth; ++k)
            if (k - 1 >= (int)th.size()) work(k);
        for (auto& x : th) x.join();
    }
    for (int t = 0; t < n; ++t) ST(st[t]);
    if (h_sigmas)
        for (int t = 0; t < n; ++t) h_sigmas[t] = sig[t];
    // Step 2: all subimages in one batched pass, each at its own sigma; then back into place
    std::vector<htsvd_image> imgs(n);
    for (int t = 0; t < n; ++t) {
        imgs[t].d_in = tin + tiles[t].in_off;
        imgs[t].H = tiles[t].h;
        imgs[t].W = tiles[t].w;
        imgs[t].C = C;
        imgs[t].sigma = sig[t];
        imgs[t].d_out = (float*)(tout + tiles[t].out_off);
    }
    ST(htsvd_denoise_batch(imgs.data(), n, p, s));
    for (const Tile& T : tiles)
        CK(cudaMemcpy2DAsync(d_out + ((size_t)T.y0 * W + T.x0) * C, sizeof(float) * W * C, tout + T.out_off,
                             sizeof(float) * T.w * C, sizeof(float) * T.w * C, T.h, cudaMemcpyDeviceToDevice, s));
    return HTSVD_OK;
}

htsvd_status htsvd_denoise_vjp(const float* d_x, int32_t H, int32_t W, int32_t C, double sigma,
                               const htsvd_params* p, const int32_t* d_idx, const float* d_w, const float* d_out,
                               const float* d_grad_out, float* d_grad_x, float* d_grad_w, cudaStream_t s) {
    if (!d_x || !d_idx || !d_out || !d_grad_out || !d_grad_x) return HTSVD_ERR_INVALID_ARG;
    if (!(sigma >= 0)) return HTSVD_ERR_INVALID_ARG;
    Resolved r;
    ST(resolve(p, C, r));
    ST(check_image(H, W, C, r));
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    const Geo g = make_geo(H, W, C, r.s, r.win, r.K);
    const int64_t npix = (int64_t)H * W;
    void* qb;
    ST(ws_get(w, S_Q, (size_t)npix * C, &qb));
    { ProfScope ps_("quantize", s); CK(launch_quantize(d_x, npix * C, (uint8_t*)qb, s)); }
    double* b64;
    float* b32;
    ST(run_basis(w, (const uint8_t*)qb, g, &b64, &b32, s));
    return vjp_core(w, d_x, g, r, d_idx, d_w, b64, b32, r.tau_mult * sigma, d_out, d_grad_out, d_grad_x, d_grad_w,
                    s);
}

htsvd_status htsvd_sure(const float* d_y, int32_t H, int32_t W, int32_t C, double sigma, const double* h_tau_mults,
                        int32_t n_tau, const float* d_probe, double eps, const htsvd_params* p, double* h_sure,
                        cudaStream_t s) {
    if (!d_y || !d_probe || !h_tau_mults || !h_sure || n_tau < 1) return HTSVD_ERR_INVALID_ARG;
    if (!(sigma > 0) || std::isinf(sigma)) return HTSVD_ERR_INVALID_ARG;
    if (!(eps >= 0.0) || (eps > 0.0 && !(std::isfinite((float)eps) && (float)eps > 0.0f))) return HTSVD_ERR_INVALID_ARG;
    for (int i = 0; i < n_tau; ++i)
        if (!(h_tau_mults[i] > 0.0) || std::isinf(h_tau_mults[i])) return HTSVD_ERR_INVALID_ARG;
    Resolved r;
    ST(resolve(p, C, r));
    ST(check_image(H, W, C, r));
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    const int64_t n = (int64_t)H * W * C;
    const Geo g = make_geo(H, W, C, r.s, r.win, r.K);
    const bool fd = eps > 0.0;
    void *out, *gx, *idx, *red;
    ST(ws_get(w, S_SOUT, sizeof(float) * n, &out));
    ST(ws_get(w, S_SGX, sizeof(float) * n, &gx));     // J^T b (eps = 0) or the perturbed image z (eps > 0)
    ST(ws_get(w, S_SIDX, sizeof(int32_t) * g.ngroups() * r.K, &idx));
    ST(ws_get(w, S_SRED, sizeof(double) * (sure_scratch_doubles() + 4 * (size_t)n_tau), &red));
    double* scratch = (double*)red;
    double* terms = scratch + sure_scratch_doubles();   // per multiplier: |f - y|^2, b.g, then b.f(z) (fd)
    htsvd_params pm;
    if (p) pm = *p;
    else std::memset(&pm, 0, sizeof(pm));
    pm.h_sigma_out = nullptr;
    pm.d_mask_out = nullptr;
    pm.d_weights_out = nullptr;
    pm.d_basis_out = nullptr;
    pm.d_coef_out = nullptr;
    std::vector<Resolved> rs((size_t)n_tau);
    for (int i = 0; i < n_tau; ++i) {
        pm.tau_mult = h_tau_mults[i];
        ST(resolve(&pm, C, rs[i]));
    }
    void* qb;
    ST(ws_get(w, S_Q, (size_t)n, &qb));
    // Pass 0 denoises y at every multiplier; with eps > 0 pass 1 denoises z = y + eps b. Each pass
    // groups and solves the bases of its own rounded image once, shared by every multiplier.
    const int passes = fd ? 2 : 1;
    for (int pass = 0; pass < passes; ++pass) {
        const float* img = d_y;
        if (pass == 1) {
            ProfScope ps_("perturb", s);
            CK(launch_perturb(d_y, d_probe, (float)eps, n, (float*)gx, s));
            img = (const float*)gx;
        }
        { ProfScope ps_("quantize", s); CK(launch_quantize(img, n, (uint8_t*)qb, s)); }
        double* b64;
        float* b32;
        ST(run_basis(w, (const uint8_t*)qb, g, &b64, &b32, s));
        ST(run_block_match((const uint8_t*)qb, g, r, 1, (int32_t*)idx, s));
        for (int i = 0; i < n_tau; ++i) {
            const Resolved& ri = rs[i];
            const double tau = ri.tau_mult * sigma;
            ST(run_forward_filter(w, img, 1, g, ri, (const int32_t*)idx, b64, b32, tau, nullptr, nullptr,
                                  (float*)out, s));
            const float* gv = (const float*)out;        // fd: b.f(y) in pass 0, b.f(z) in pass 1
            if (!fd) {
                // J^T b through the frozen-mask adjoint
                ST(vjp_core(w, d_y, g, ri, (const int32_t*)idx, nullptr, b64, b32, tau, (const float*)out, d_probe,
                            (float*)gx, nullptr, s));
                gv = (const float*)gx;
            }
            ProfScope ps_("sure_terms", s);
            CK(launch_sure_terms((const float*)out, img, d_probe, gv, n, scratch, terms + 4 * i + 2 * pass, s));
        }
    }
    std::vector<double> h(4 * (size_t)n_tau);
    CK(cudaMemcpyAsync(h.data(), terms, sizeof(double) * 4 * n_tau, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < n_tau; ++i) {
        const double* t = &h[4 * (size_t)i];
        const double div = fd ? (t[3] - t[1]) / eps : t[1];
        h_sure[i] = t[0] / (double)n - sigma * sigma + 2.0 * sigma * sigma / (double)n * div;
    }
    return HTSVD_OK;
}

htsvd_status htsvd_sure_weights(const float* d_y, int32_t H, int32_t W, int32_t C, double sigma, const float* d_w,
                                const float* d_probe, double eps, const htsvd_params* p, double* h_sure,
                                float* d_grad_w, cudaStream_t s) {
    if (!d_w || !h_sure || !d_grad_w) return HTSVD_ERR_INVALID_ARG;
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    SureW c;
    ST(sure_w_prepare(w, d_y, H, W, C, sigma, d_probe, eps, p, c, s));
    return sure_w_eval(w, c, d_w, h_sure, d_grad_w, s);
}

htsvd_status htsvd_tune_weights(const float* d_y, int32_t H, int32_t W, int32_t C, double sigma, const float* d_probe,
                                double eps, int32_t n_steps, double step, const htsvd_params* p, float* d_w,
                                double* h_sure, cudaStream_t s) {
    if (!d_w || !h_sure || n_steps < 0 || !(step > 0.0) || !std::isfinite((float)step)) return HTSVD_ERR_INVALID_ARG;
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    SureW c;
    ST(sure_w_prepare(w, d_y, H, W, C, sigma, d_probe, eps, p, c, s));
    void *gw, *mx;
    ST(ws_get(w, S_SGX, sizeof(float) * c.ng, &gw));
    ST(ws_get(w, S_SIDX, sizeof(unsigned), &mx));
    for (int it = 0; it <= n_steps; ++it) {
        ST(sure_w_eval(w, c, d_w, &h_sure[it], (float*)gw, s));
        if (it == n_steps) break;
        ProfScope ps_("eg_update", s);
        CK(launch_eg_update(d_w, (const float*)gw, c.ng, (float)step, (unsigned*)mx, s));
    }
    return HTSVD_OK;
}

htsvd_status htsvd_denoise_cube(const uint8_t* d_cube, int32_t H, int32_t W, int32_t N, double sigma,
                                const htsvd_params* p, float* d_out, int32_t* d_idx_out, cudaStream_t s) {
    if (!d_cube || !d_out || !(sigma >= 0) || std::isinf(sigma)) return HTSVD_ERR_INVALID_ARG;
    if (N < 2 || N > 64) return HTSVD_ERR_INVALID_ARG;
    Resolved r;
    ST(resolve(p, N, r));
    if (r.match_mode != HTSVD_MATCH_AUTO && r.match_mode != HTSVD_MATCH_FULL) return HTSVD_ERR_INVALID_ARG;
    if (H < r.ps || W < r.ps) return HTSVD_ERR_INVALID_ARG;
    if ((int64_t)H * W * N >= ((int64_t)1 << 31)) return HTSVD_ERR_UNSUPPORTED;
    const Geo g = make_geo(H, W, N, r.s, r.win, r.K);
    if ((int64_t)g.wny * g.wnx < r.K) return HTSVD_ERR_INVALID_ARG;
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    const int64_t ng = g.ngroups();
    int32_t* idx = d_idx_out;
    if (!idx) {
        void* ib;
        ST(ws_get(w, S_IDX, sizeof(int32_t) * ng * r.K, &ib));
        idx = (int32_t*)ib;
    }
    void *mom, *p64, *p32, *gap = nullptr, *scr, *num, *den;
    ST(ws_get(w, S_MOM, sizeof(unsigned long long) * 2 * PS2 * N * N, &mom));
    ST(ws_get(w, S_B64, sizeof(double) * 2 * 2 * N * PS2, &p64));
    ST(ws_get(w, S_B32, sizeof(float) * basis32_floats(N), &p32));
    if (r.strict_basis) ST(ws_get(w, S_GAP, sizeof(double) * basis_problems(N), &gap));
    const int grid = cube_grid(N, r.K, ng);
    ST(ws_get(w, S_CSCR, sizeof(float) * (size_t)grid * r.K * PS2 * N, &scr));
    ST(ws_get(w, S_CNUM, sizeof(float) * (size_t)H * W * N, &num));
    ST(ws_get(w, S_CDEN, sizeof(float) * (size_t)H * W, &den));
    if (cube_smem_bytes(N, r.K) > 227 * 1024) return HTSVD_ERR_UNSUPPORTED;
    // grouping: SSD over all bands (reading of the paper's silence on matching for cubes)
    BMArgs ba{};
    ba.img = d_cube;
    ba.g = g;
    ba.mode = MM_FULL;
    ba.gamma2 = r.gamma * r.gamma;
    ba.rstep = 1;
    ba.nry_s = g.nry;
    ba.nrx_s = g.nrx;
    choose_bm_tiles(g, 1, ba.TRy, ba.TRx);
    bm_fit_tiles(ba);
    if (bm_smem_bytes(ba) > 227 * 1024) return HTSVD_ERR_UNSUPPORTED;
    ba.idx = idx;
    { ProfScope ps_("block_match", s); CK(launch_block_match(ba, s)); }
    { ProfScope ps_("moments", s); CK(launch_cube_moments(d_cube, g, (unsigned long long*)mom, s)); }
    { ProfScope ps_("basis", s);
      CK(launch_basis((const unsigned long long*)mom, N, (double*)p64, (float*)p32, s, (double*)gap)); }
    if (p && p->d_basis_out)
        CK(cudaMemcpyAsync(p->d_basis_out, p64, sizeof(double) * 2 * 2 * N * PS2, cudaMemcpyDeviceToDevice, s));
    if (r.strict_basis) ST(check_basis_gap((const double*)gap, N, p, s));
    if (p && p->h_sigma_out) *p->h_sigma_out = sigma;
    const double tau = r.tau_mult * sigma;
    CubeArgs a{};
    a.img = d_cube;
    a.g = g;
    a.idx = idx;
    a.basis32 = (const float*)p32;
    a.basis64 = (const double*)p64;
    a.tau32 = (float)tau;
    a.tau64 = tau;
    a.band_rel = kBandRelCube;
    a.band_abs = (float)(tau * kBandTau) + 1e-6f;
    a.w_in = nullptr;
    a.agg_mode = r.agg_mode;
    a.scratch = (float*)scr;
    a.num = (float*)num;
    a.den = (float*)den;
    a.out = d_out;
    a.mask_out = p ? p->d_mask_out : nullptr;
    a.weights_out = p ? p->d_weights_out : nullptr;
    a.coef_out = p ? p->d_coef_out : nullptr;
    { ProfScope ps_("cube_filter", s); CK(launch_cube_filter(a, grid, s)); }
    return HTSVD_OK;
}

htsvd_status htsvd_denoise_volume(const uint8_t* d_vol, int32_t D, int32_t H, int32_t W, double sigma,
                                  const htsvd_params* p, float* d_out, int32_t* d_idx_out, cudaStream_t s) {
    if (!d_vol || !d_out || std::isnan(sigma) || std::isinf(sigma)) return HTSVD_ERR_INVALID_ARG;
    if ((uintptr_t)d_vol & 3) return HTSVD_ERR_INVALID_ARG;
    htsvd_params z;
    std::memset(&z, 0, sizeof(z));
    const htsvd_params& q = p ? *p : z;
    const int ps = q.ps > 0 ? q.ps : 4, stride = q.stride > 0 ? q.stride : 2;
    const int win = q.window > 0 ? q.window : 5, K = q.K > 0 ? q.K : 32;
    if (ps != 4) return HTSVD_ERR_UNSUPPORTED;
    if (K < 2 || K > 32 || (K & (K - 1)) != 0 || win < 1 || win > volume_max_window()) return HTSVD_ERR_INVALID_ARG;
    if (q.match_mode != HTSVD_MATCH_AUTO && q.match_mode != HTSVD_MATCH_FULL) return HTSVD_ERR_INVALID_ARG;
    if (q.agg_mode != HTSVD_AGG_UNIFORM && q.agg_mode != HTSVD_AGG_SPARSITY) return HTSVD_ERR_INVALID_ARG;
    if (D < ps || H < ps || W < ps) return HTSVD_ERR_INVALID_ARG;
    if ((int64_t)D * H * W >= ((int64_t)1 << 31)) return HTSVD_ERR_UNSUPPORTED;
    const VolGeo g = make_vol_geo(D, H, W, stride, win, K);
    if ((int64_t)g.wnz * g.wny * g.wnx < K) return HTSVD_ERR_INVALID_ARG;
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    const int64_t ng = (int64_t)g.nrz * g.nry * g.nrx;
    const int64_t nvox = (int64_t)D * H * W;
    int32_t* idx = d_idx_out;
    if (!idx) {
        void* ib;
        ST(ws_get(w, S_IDX, sizeof(int32_t) * ng * K, &ib));
        idx = (int32_t*)ib;
    }
    void *mom, *b64, *num, *den, *hbuf;
    ST(ws_get(w, S_VMOM, sizeof(unsigned long long) * 512, &mom));
    ST(ws_get(w, S_VB64, sizeof(double) * 256, &b64));
    ST(ws_get(w, S_VNUM, sizeof(float) * nvox, &num));
    ST(ws_get(w, S_VDEN, sizeof(float) * nvox, &den));
    const bool estimate = sigma < 0;
    const size_t fm_words = estimate ? 64 * 64 + 64 : 0;
    ST(ws_host(w, sizeof(unsigned long long) * (512 + fm_words) + sizeof(double) * 256, &hbuf));
    ST(ws_side(w));
    unsigned long long* hmom = (unsigned long long*)hbuf;
    unsigned long long* hfm = hmom + 512;
    double* hb64 = (double*)(hfm + fm_words);
    // moments first (and the full moment when sigma is estimated), their copy to the host, then the
    // grouping runs while the host solves the bases and the noise level
    { ProfScope ps_("volume_moments", s); CK(launch_volume_moments(d_vol, g, (unsigned long long*)mom, s)); }
    CK(cudaMemcpyAsync(hmom, mom, sizeof(unsigned long long) * 512, cudaMemcpyDeviceToHost, s));
    if (estimate) {
        void* fm;
        ST(ws_get(w, S_FULLM, sizeof(unsigned long long) * fm_words, &fm));
        unsigned long long* dM = (unsigned long long*)fm;
        { ProfScope ps_("volume_full_moment", s); CK(launch_volume_full_moment(d_vol, g, dM, dM + 64 * 64, s)); }
        CK(cudaMemcpyAsync(hfm, dM, sizeof(unsigned long long) * fm_words, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventRecord(w->ev_join, s));
    { ProfScope ps_("block_match_volume", s); CK(launch_block_match_volume(d_vol, g, idx, s)); }
    CK(cudaEventSynchronize(w->ev_join));
    double gap;
    { HostProfScope hp_("volume_bases_host"); gap = volume_bases_host(hmom, hb64); }
    if (estimate) {
        HostProfScope hp_("volume_sigma_host");
        sigma = sigma_from_moments(hfm, hfm + 64 * 64, 64, ng);
        if (!(sigma >= 0)) return HTSVD_ERR_CUDA;
    }
    if (p && p->h_basis_gap_out) *p->h_basis_gap_out = gap;
    if (q.strict_basis && !(gap >= kDegenerateGap)) return HTSVD_ERR_DEGENERATE_BASIS;
    CK(cudaMemcpyAsync(b64, hb64, sizeof(double) * 256, cudaMemcpyHostToDevice, s));
    if (p && p->d_basis_out)
        CK(cudaMemcpyAsync(p->d_basis_out, b64, sizeof(double) * 256, cudaMemcpyDeviceToDevice, s));
    if (p && p->h_sigma_out) *p->h_sigma_out = sigma;
    const double tau_mult = q.tau_mult > 0 ? q.tau_mult : std::sqrt(2.0 * std::log((double)ps * K * ps * ps));
    const double tau = tau_mult * sigma;
    VolFilterArgs a{};
    a.vol = d_vol;
    a.g = g;
    a.idx = idx;
    a.basis64 = (const double*)b64;
    a.tau32 = (float)tau;
    a.tau64 = tau;
    a.band_rel = kBandRel;
    a.band_abs = (float)(tau * kBandTau) + 1e-6f;
    a.w_in = nullptr;
    a.agg_mode = q.agg_mode;
    a.num = (float*)num;
    a.den = (float*)den;
    a.mask_out = p ? p->d_mask_out : nullptr;
    a.weights_out = p ? p->d_weights_out : nullptr;
    CK(cudaMemsetAsync(num, 0, sizeof(float) * nvox, s));
    CK(cudaMemsetAsync(den, 0, sizeof(float) * nvox, s));
    { ProfScope ps_("volume_filter", s); CK(launch_volume_filter(a, s)); }
    { ProfScope ps_("volume_finalize", s); CK(launch_volume_finalize((const float*)num, (const float*)den, nvox, d_out, s)); }
    return HTSVD_OK;
}

// One 3-D box of a uint8 or float volume moved between a whole volume and a packed sub-volume.
static cudaError_t copy_box(void* dst, size_t dst_pitch, size_t dst_rows, const void* src, size_t src_pitch,
                            size_t src_rows, size_t row_bytes, size_t rows, size_t slabs, cudaStream_t s) {
    cudaMemcpy3DParms m;
    std::memset(&m, 0, sizeof(m));
    m.srcPtr = make_cudaPitchedPtr(const_cast<void*>(src), src_pitch, row_bytes, src_rows);
    m.dstPtr = make_cudaPitchedPtr(dst, dst_pitch, row_bytes, dst_rows);
    m.extent = make_cudaExtent(row_bytes, rows, slabs);
    m.kind = cudaMemcpyDeviceToDevice;
    return cudaMemcpy3DAsync(&m, s);
}

htsvd_status htsvd_denoise_volume_adaptive(const uint8_t* d_vol, int32_t D, int32_t H, int32_t W, int32_t sub_d,
                                           int32_t sub_h, int32_t sub_w, const htsvd_params* p, float* d_out,
                                           double* h_sigmas, cudaStream_t s) {
    if (!d_vol || !d_out || sub_d < 1 || sub_h < 1 || sub_w < 1 || D < 1 || H < 1 || W < 1)
        return HTSVD_ERR_INVALID_ARG;
    if ((int64_t)D * H * W >= ((int64_t)1 << 31)) return HTSVD_ERR_UNSUPPORTED;
    // each axis cut as the subimage axes of Alg. 2: t = max(1, n / n_sub) parts, boundaries floor(i n / t)
    auto bounds = [](int n, int sub) {
        const int t = std::max(1, n / sub);
        std::vector<int> b(t + 1);
        for (int i = 0; i <= t; ++i) b[i] = (int)(((int64_t)i * n) / t);
        return b;
    };
    const std::vector<int> bz = bounds(D, sub_d), by = bounds(H, sub_h), bx = bounds(W, sub_w);
    const int nz = (int)bz.size() - 1, ny = (int)by.size() - 1, nx = (int)bx.size() - 1;
    const int n = nz * ny * nx;
    struct Box {
        int z0, y0, x0, d, h, w;
        size_t in_off, out_off;
    };
    std::vector<Box> boxes(n);
    size_t in_bytes = 0, out_bytes = 0;
    for (int t = 0; t < n; ++t) {
        Box& B = boxes[t];
        const int iz = t / (ny * nx), iy = (t / nx) % ny, ix = t % nx;
        B.z0 = bz[iz];
        B.y0 = by[iy];
        B.x0 = bx[ix];
        B.d = bz[iz + 1] - B.z0;
        B.h = by[iy + 1] - B.y0;
        B.w = bx[ix + 1] - B.x0;
        B.in_off = in_bytes;
        B.out_off = out_bytes;
        in_bytes += ((size_t)B.d * B.h * B.w + 255) & ~(size_t)255;
        out_bytes += (sizeof(float) * B.d * B.h * B.w + 255) & ~(size_t)255;
    }
    // every part passes the checks of htsvd_denoise_volume before any device work, so a bad part
    // size leaves d_out untouched
    {
        htsvd_params z;
        std::memset(&z, 0, sizeof(z));
        const htsvd_params& c = p ? *p : z;
        const int ps = c.ps > 0 ? c.ps : 4, stride = c.stride > 0 ? c.stride : 2;
        const int win = c.window > 0 ? c.window : 5, K = c.K > 0 ? c.K : 32;
        if (ps != 4) return HTSVD_ERR_UNSUPPORTED;
        if (K < 2 || K > 32 || (K & (K - 1)) != 0 || win < 1 || win > volume_max_window()) return HTSVD_ERR_INVALID_ARG;
        if (c.match_mode != HTSVD_MATCH_AUTO && c.match_mode != HTSVD_MATCH_FULL) return HTSVD_ERR_INVALID_ARG;
        if (c.agg_mode != HTSVD_AGG_UNIFORM && c.agg_mode != HTSVD_AGG_SPARSITY) return HTSVD_ERR_INVALID_ARG;
        for (const Box& B : boxes) {
            if (B.d < ps || B.h < ps || B.w < ps) return HTSVD_ERR_INVALID_ARG;
            const VolGeo g = make_vol_geo(B.d, B.h, B.w, stride, win, K);
            if ((int64_t)g.wnz * g.wny * g.wnx < K) return HTSVD_ERR_INVALID_ARG;
        }
    }
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    void *vin, *vout;
    ST(ws_get(w, S_AIN, in_bytes, &vin));
    ST(ws_get(w, S_AOUT, out_bytes, &vout));
    uint8_t* tin = (uint8_t*)vin;
    unsigned char* tout = (unsigned char*)vout;
    htsvd_params q;
    if (p) q = *p;
    else std::memset(&q, 0, sizeof(q));
    // per-volume outputs have no meaning for the parts; each part reports only its noise level
    q.d_basis_out = nullptr;
    q.d_mask_out = nullptr;
    q.d_weights_out = nullptr;
    q.h_basis_gap_out = nullptr;
    for (int t = 0; t < n; ++t) {
        const Box& B = boxes[t];
        CK(copy_box(tin + B.in_off, B.w, B.h, d_vol + ((size_t)B.z0 * H + B.y0) * W + B.x0, W, H, B.w, B.h, B.d, s));
        double sg = -1.0;
        q.h_sigma_out = &sg;
        // Step 1 (Alg. 2): the part's noise level by the eigenvalue rule; Step 2: Alg. 1 at that level
        ST(htsvd_denoise_volume(tin + B.in_off, B.d, B.h, B.w, -1.0, &q, (float*)(tout + B.out_off), nullptr, s));
        if (h_sigmas) h_sigmas[t] = sg;
        CK(copy_box(d_out + ((size_t)B.z0 * H + B.y0) * W + B.x0, sizeof(float) * W, H, tout + B.out_off,
                    sizeof(float) * B.w, B.h, sizeof(float) * B.w, B.h, B.d, s));
    }
    return HTSVD_OK;
}

static htsvd_status check_projection(const uint8_t* d_img, int32_t H, int32_t W, int32_t C, const int32_t* d_pos,
                                     int64_t n, const double* d_basis, const float* d_coef) {
    if (C != 1 && C != 3) return HTSVD_ERR_INVALID_ARG;
    if (H < PS || W < PS || n < 0) return HTSVD_ERR_INVALID_ARG;
    if ((int64_t)H * W * C >= ((int64_t)1 << 31)) return HTSVD_ERR_UNSUPPORTED;
    if (n == 0) return HTSVD_OK;
    if (!d_img || !d_basis || !d_coef) return HTSVD_ERR_INVALID_ARG;
    if (!d_pos && n != (int64_t)(H - PS + 1) * (W - PS + 1)) return HTSVD_ERR_INVALID_ARG;
    if (((uintptr_t)d_img & 3) || ((uintptr_t)d_coef & 15)) return HTSVD_ERR_INVALID_ARG;
    return HTSVD_OK;
}

htsvd_status htsvd_project_patches(const uint8_t* d_img, int32_t H, int32_t W, int32_t C, const int32_t* d_pos,
                                   int64_t n, const double* d_basis, float* d_coef, int32_t* d_flag, cudaStream_t s) {
    ST(check_projection(d_img, H, W, C, d_pos, n, d_basis, d_coef));
    if (n == 0) return HTSVD_OK;
    Workspace* w = workspace_for(s);
    if (!w) return HTSVD_ERR_OOM;
    void* pieces;
    ST(ws_get(w, S_PROJ, project_pieces_bytes(C), &pieces));
    { ProfScope ps_("project_split", s); CK(launch_project_split(d_basis, C, pieces, s)); }
    { ProfScope ps_("project_tc", s);
      CK(launch_project_tc(d_img, H, W, C, d_pos, n, pieces, d_coef, (int*)d_flag, s)); }
    return HTSVD_OK;
}

htsvd_status htsvd_internal_project_simt(const uint8_t* d_img, int32_t H, int32_t W, int32_t C, const int32_t* d_pos,
                                         int64_t n, const double* d_basis, float* d_coef, cudaStream_t s) {
    ST(check_projection(d_img, H, W, C, d_pos, n, d_basis, d_coef));
    if (n == 0) return HTSVD_OK;
    { ProfScope ps_("project_simt", s); CK(launch_project_simt(d_img, H, W, C, d_pos, n, d_basis, d_coef, s)); }
    return HTSVD_OK;
}

int64_t htsvd_num_groups(int32_t H, int32_t W, const htsvd_params* p) {
    Resolved r;
    if (resolve(p, 1, r) != HTSVD_OK) return -1;
    if (H < r.ps || W < r.ps) return -1;
    return (int64_t)ref_count(H, r.s) * ref_count(W, r.s);
}

const char* htsvd_status_string(htsvd_status s) {
    switch (s) {
        case HTSVD_OK: return "ok";
        case HTSVD_ERR_INVALID_ARG: return "invalid argument";
        case HTSVD_ERR_UNSUPPORTED: return "unsupported configuration";
        case HTSVD_ERR_CUDA: return "CUDA error";
        case HTSVD_ERR_OOM: return "out of memory";
        case HTSVD_ERR_TIMEOUT: return "device wait timed out";
        case HTSVD_ERR_DEGENERATE_BASIS: return "degenerate basis: two eigenvalues of a basis slice coincide";
    }
    return "unknown status";
}

htsvd_status htsvd_profile_enable(int32_t enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = enable != 0;
    return HTSVD_OK;
}

int32_t htsvd_profile_collect(int32_t max_kernels, char* names, int32_t name_len, int64_t* launches,
                              double* total_ms) {
    std::vector<ProfRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        recs.swap(g_prof);
    }
    std::vector<std::string> nm;
    std::vector<int64_t> cnt;
    std::vector<double> tot;
    int32_t status = 0;
    for (const ProfRec& r : recs) {
        float ms = 0.f;
        if (r.host_ms >= 0) {
            ms = (float)r.host_ms;
        } else {
            if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
                cudaGetLastError();
                status = -1;
            }
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        size_t i = 0;
        while (i < nm.size() && nm[i] != r.name) ++i;
        if (i == nm.size()) {
            nm.push_back(r.name);
            cnt.push_back(0);
            tot.push_back(0.0);
        }
        cnt[i] += 1;
        tot[i] += ms;
    }
    if (status < 0) return -1;
    const int32_t n = (int32_t)nm.size() < max_kernels ? (int32_t)nm.size() : max_kernels;
    for (int32_t i = 0; i < n; ++i) {
        if (names && name_len > 0) {
            std::strncpy(names + (size_t)i * name_len, nm[i].c_str(), name_len - 1);
            names[(size_t)i * name_len + name_len - 1] = 0;
        }
        if (launches) launches[i] = cnt[i];
        if (total_ms) total_ms[i] = tot[i];
    }
    return n;
}

htsvd_status htsvd_release_workspace(void) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HTSVD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_ws.begin(); it != g_ws.end();) {
        Workspace* w = *it;
        if (w->device == dev) {
            for (int i = 0; i < S_NSLOT; ++i)
                if (w->buf[i]) cudaFree(w->buf[i]);
            if (w->hpin) cudaFreeHost(w->hpin);
            if (w->side) cudaStreamDestroy(w->side);
            if (w->ev_fork) cudaEventDestroy(w->ev_fork);
            if (w->ev_join) cudaEventDestroy(w->ev_join);
            delete w;
            it = g_ws.erase(it);
        } else {
            ++it;
        }
    }
    return HTSVD_OK;
}

}  // extern "C"

// htsvd_denoise_batch: many images of any sizes in one persistent launch per phase.
//
// Each phase (moments, bases, grouping, filter, reduction) is one kernel whose CTAs pull
// (image, tile) work items from a queue spanning every image (an atomic counter, or a
// grid-stride walk for the uniform phases). The whole launch sequence, with the bases on a
// forked stream concurrent with grouping, is captured once into a CUDA graph and replayed
// for the same batch. Filter and grouping tile shapes come from an autotuner that times the
// candidate shapes on the first batch of a given shape signature. No kernel waits on
// another CTA, so no phase can stall on a device-side wait.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/htsvd.h"
#include "kernels.h"

using namespace htsvd;

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Tuning {
    int TR = 8;          // filter tile edge
    int bmy = 4, bmx = 8; // grouping tile
};

struct Plan {
    int n = 0, C = 0, K = 0;
    std::vector<BMArgs> bm;
    std::vector<FilterArgs> fa;
    std::vector<unsigned long long*> mom;
    std::vector<float*> outs;
    std::vector<int> p_bm, p_mom, p_f, p_red;   // prefix sums of work items (n + 1)
    size_t smem_bm = 0, smem_f = 0;
    size_t dev_bytes = 0;                       // per-image temporaries
    size_t mom_bytes = 0;
};

// Device-side copies of a plan (descriptors and prefix arrays) and its graph.
struct BatchCache {
    int device = -1;
    cudaStream_t stream = nullptr;
    std::vector<unsigned char> key;
    void* dev = nullptr;            // temporaries of all images
    size_t dev_cap = 0;
    void* desc = nullptr;           // device descriptors
    size_t desc_cap = 0;
    void* hdesc = nullptr;          // pinned host copy (source of the captured memcpy)
    size_t hdesc_cap = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;     // the sequence is captured here (the caller's stream may be the legacy one)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

std::mutex g_bmu;
std::vector<BatchCache*> g_caches;
std::map<std::tuple<int, int, int, int, int, int>, Tuning> g_tuned;   // (C, K, s, win, ps, size bucket)

BatchCache* cache_for(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    for (BatchCache* c : g_caches)
        if (c->device == dev && c->stream == s) return c;
    BatchCache* c = new BatchCache();
    c->device = dev;
    c->stream = s;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return nullptr;
    }
    g_caches.push_back(c);
    return c;
}

htsvd_status grow(void** p, size_t* cap, size_t bytes, bool pinned) {
    if (*cap >= bytes) return HTSVD_OK;
    if (*p) (pinned ? cudaFreeHost(*p) : cudaFree(*p));
    *p = nullptr;
    *cap = 0;
    const size_t b = bytes + bytes / 8 + 256;
    if ((pinned ? cudaMallocHost(p, b) : cudaMalloc(p, b)) != cudaSuccess) {
        cudaGetLastError();
        return HTSVD_ERR_OOM;
    }
    *cap = b;
    return HTSVD_OK;
}

// Builds the per-image descriptors for a tuning; pointers are offsets from base (nullptr: sizes only).
htsvd_status make_plan(const htsvd_image* imgs, int n, const htsvd_params* p, const Tuning& t, unsigned char* base,
                       Plan& P) {
    htsvd_params z;
    std::memset(&z, 0, sizeof(z));
    if (!p) p = &z;
    const int s = p->stride > 0 ? p->stride : 3, win = p->window > 0 ? p->window : 18;
    const int K = p->K > 0 ? p->K : 32, ps = p->ps > 0 ? p->ps : 8;
    if (p->ps < 0 || p->stride < 0 || p->window < 0 || p->K < 0) return HTSVD_ERR_INVALID_ARG;
    if (K < 2 || (K & (K - 1))) return HTSVD_ERR_INVALID_ARG;
    if (p->match_mode < 0 || p->match_mode > 3 || p->agg_mode < 0 || p->agg_mode > 1) return HTSVD_ERR_INVALID_ARG;
    if (ps != PS || K > 32 || win > 64) return HTSVD_ERR_UNSUPPORTED;
    const double gamma = p->gcp_gamma > 0 ? p->gcp_gamma : 1.2;
    P = Plan();
    P.n = n;
    P.K = K;
    P.C = imgs[0].C;
    P.p_bm.assign(n + 1, 0);
    P.p_mom.assign(n + 1, 0);
    P.p_f.assign(n + 1, 0);
    P.p_red.assign(n + 1, 0);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const htsvd_image& im = imgs[i];
        if (!im.d_in || !im.d_out || !(im.sigma >= 0) || im.C != P.C || (im.C != 1 && im.C != 3) || im.H < PS ||
            im.W < PS)
            return HTSVD_ERR_INVALID_ARG;
        const Geo g = make_geo(im.H, im.W, im.C, s, win, K);
        if ((int64_t)g.wny * g.wnx < K) return HTSVD_ERR_INVALID_ARG;
        const double mult = p->tau_mult > 0 ? p->tau_mult : std::sqrt(2.0 * std::log((double)im.C * K * PS * PS));
        const double tau = mult * im.sigma;
        BMArgs b{};
        b.img = im.d_in;
        b.g = g;
        b.mode = im.C == 1 ? MM_GRAY
                           : (p->match_mode == HTSVD_MATCH_FULL ? MM_FULL
                                                                : p->match_mode == HTSVD_MATCH_GREEN ? MM_GREEN : MM_GCP);
        b.gamma2 = gamma * gamma;
        b.rstep = 1;
        b.nry_s = g.nry;
        b.nrx_s = g.nrx;
        b.TRy = t.bmy;
        b.TRx = t.bmx;
        bm_fit_tiles(b);
        FilterArgs f{};
        f.img = im.d_in;
        f.img_is_float = 0;
        f.g = g;
        f.TR = t.TR;
        f.ntx = (g.nrx + t.TR - 1) / t.TR;
        f.nty = (g.nry + t.TR - 1) / t.TR;
        f.FHmax = std::min(g.H, (t.TR - 1) * s + g.wny + PS - 1);
        f.FWmax = std::min(g.W, (t.TR - 1) * s + g.wnx + PS - 1);
        f.mode = FM_FORWARD;
        f.tau64 = tau;
        f.tau32 = (float)tau;
        f.band_rel = kBandRel;
        f.band_abs = (float)(tau * kBandTau) + 1e-6f;
        f.agg_mode = p->agg_mode;
        const int acc = im.C == 3 ? 4 : 2;
        const size_t b_idx = a256(sizeof(int32_t) * (size_t)g.ngroups() * K);
        const size_t b_mom = a256(sizeof(unsigned long long) * 2 * PS2 * im.C * im.C);
        const size_t b_b64 = a256(sizeof(double) * 2 * 2 * im.C * PS2);
        const size_t b_b32 = a256(sizeof(float) * 512);
        const size_t b_part = a256(sizeof(float) * (size_t)f.ntx * f.nty * f.FHmax * f.FWmax * acc);
        // moments first (one memset clears every image's accumulators)
        unsigned long long* mom = base ? reinterpret_cast<unsigned long long*>(base + P.mom_bytes) : nullptr;
        P.mom_bytes += b_mom;
        b.idx = base ? reinterpret_cast<int32_t*>(base + off) : nullptr;
        if (base && im.d_idx_out) b.idx = im.d_idx_out;          // the caller's buffer holds the grouping
        f.idx = b.idx;
        f.basis64 = base ? reinterpret_cast<double*>(base + off + b_idx) : nullptr;
        f.basis32 = base ? reinterpret_cast<float*>(base + off + b_idx + b_b64) : nullptr;
        f.partials = base ? reinterpret_cast<float*>(base + off + b_idx + b_b64 + b_b32) : nullptr;
        off += b_idx + b_b64 + b_b32 + b_part;
        P.bm.push_back(b);
        P.fa.push_back(f);
        P.mom.push_back(mom);
        P.outs.push_back(im.d_out);
        P.p_bm[i + 1] = P.p_bm[i] + bm_tiles(b);
        P.p_mom[i + 1] = P.p_mom[i] + moments_chunks(g);
        P.p_f[i + 1] = P.p_f[i] + f.ntx * f.nty;
        P.p_red[i + 1] = P.p_red[i] + (int)(((int64_t)g.H * g.W + 255) / 256);
        P.smem_bm = std::max(P.smem_bm, bm_smem_bytes(b));
        P.smem_f = std::max(P.smem_f, filter_smem_bytes(f));
    }
    // the per-image blocks follow the moment accumulators
    P.mom_bytes = a256(P.mom_bytes);
    if (base) {
        for (int i = 0; i < n; ++i) {
            auto sh = [&](auto* q) { return reinterpret_cast<decltype(q)>(reinterpret_cast<unsigned char*>(q) + P.mom_bytes); };
            if (!imgs[i].d_idx_out) P.bm[i].idx = sh(P.bm[i].idx);
            P.fa[i].idx = P.bm[i].idx;
            P.fa[i].basis64 = sh(const_cast<double*>(P.fa[i].basis64));
            P.fa[i].basis32 = sh(const_cast<float*>(P.fa[i].basis32));
            P.fa[i].partials = sh(P.fa[i].partials);
        }
    }
    P.dev_bytes = P.mom_bytes + off;
    if (P.smem_f > 227 * 1024 || P.smem_bm > 227 * 1024) return HTSVD_ERR_UNSUPPORTED;
    return HTSVD_OK;
}

// Layout of the device descriptor block: BMArgs[n], FilterArgs[n], mom*[n], out*[n], 4 prefix arrays, 2 counters.
struct DescLayout {
    size_t bm, fa, mom, outs, pbm, pmom, pf, pred, ctr, total;
};
DescLayout desc_layout(int n) {
    DescLayout L;
    size_t o = 0;
    L.bm = o; o = a256(o + sizeof(BMArgs) * n);
    L.fa = o; o = a256(o + sizeof(FilterArgs) * n);
    L.mom = o; o = a256(o + sizeof(void*) * n);
    L.outs = o; o = a256(o + sizeof(void*) * n);
    L.pbm = o; o = a256(o + sizeof(int) * (n + 1));
    L.pmom = o; o = a256(o + sizeof(int) * (n + 1));
    L.pf = o; o = a256(o + sizeof(int) * (n + 1));
    L.pred = o; o = a256(o + sizeof(int) * (n + 1));
    L.ctr = o; o = a256(o + sizeof(int) * 2);
    L.total = o;
    return L;
}

void fill_desc(const Plan& P, unsigned char* h) {
    const DescLayout L = desc_layout(P.n);
    std::memset(h, 0, L.total);
    std::memcpy(h + L.bm, P.bm.data(), sizeof(BMArgs) * P.n);
    std::memcpy(h + L.fa, P.fa.data(), sizeof(FilterArgs) * P.n);
    std::memcpy(h + L.mom, P.mom.data(), sizeof(void*) * P.n);
    std::memcpy(h + L.outs, P.outs.data(), sizeof(void*) * P.n);
    std::memcpy(h + L.pbm, P.p_bm.data(), sizeof(int) * (P.n + 1));
    std::memcpy(h + L.pmom, P.p_mom.data(), sizeof(int) * (P.n + 1));
    std::memcpy(h + L.pf, P.p_f.data(), sizeof(int) * (P.n + 1));
    std::memcpy(h + L.pred, P.p_red.data(), sizeof(int) * (P.n + 1));
}

#define BCK(x)                                        \
    do {                                              \
        if ((x) != cudaSuccess) return HTSVD_ERR_CUDA; \
    } while (0)

// The launch sequence of one batch (phase order; bases forked onto the side stream).
htsvd_status enqueue(BatchCache* c, const Plan& P, cudaStream_t s, int phase_mask = 0x1f) {
    const DescLayout L = desc_layout(P.n);
    unsigned char* d = static_cast<unsigned char*>(c->desc);
    const BMArgs* dbm = reinterpret_cast<const BMArgs*>(d + L.bm);
    const FilterArgs* dfa = reinterpret_cast<const FilterArgs*>(d + L.fa);
    unsigned long long* const* dmom = reinterpret_cast<unsigned long long* const*>(d + L.mom);
    float* const* douts = reinterpret_cast<float* const*>(d + L.outs);
    const int* pbm = reinterpret_cast<const int*>(d + L.pbm);
    const int* pmom = reinterpret_cast<const int*>(d + L.pmom);
    const int* pf = reinterpret_cast<const int*>(d + L.pf);
    const int* pred = reinterpret_cast<const int*>(d + L.pred);
    int* ctr = reinterpret_cast<int*>(d + L.ctr);
    BCK(cudaMemcpyAsync(d, c->hdesc, L.total, cudaMemcpyHostToDevice, s));
    BCK(cudaMemsetAsync(c->dev, 0, P.mom_bytes, s));
    const int nsm = device_sm_count();
    BCK(cudaEventRecord(c->ev_fork, s));
    BCK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    if (phase_mask & 1) BCK(launch_moments_batch(P.C, dbm, dmom, pmom, P.n, std::min(P.p_mom[P.n], nsm * 8), c->side));
    if (phase_mask & 2) BCK(launch_basis_batch(P.C, dfa, dmom, P.n, c->side));
    BCK(cudaEventRecord(c->ev_join, c->side));
    if (phase_mask & 4)
        BCK(launch_block_match_batch(dbm, pbm, P.n, P.smem_bm, std::min(P.p_bm[P.n], nsm * 2), ctr, s));
    BCK(cudaStreamWaitEvent(s, c->ev_join, 0));
    if (phase_mask & 8)
        BCK(launch_filter_batch(P.K, P.C, dfa, pf, P.n, P.smem_f, std::min(P.p_f[P.n], nsm * 2), ctr + 1, s));
    if (phase_mask & 16) BCK(launch_reduce_batch(P.C, dfa, douts, pred, P.n, std::min(P.p_red[P.n], nsm * 16), s));
    return HTSVD_OK;
}

htsvd_status prepare(BatchCache* c, const htsvd_image* imgs, int n, const htsvd_params* p, const Tuning& t, Plan& P) {
    htsvd_status st = make_plan(imgs, n, p, t, nullptr, P);
    if (st != HTSVD_OK) return st;
    if ((st = grow(&c->dev, &c->dev_cap, P.dev_bytes, false)) != HTSVD_OK) return st;
    const DescLayout L = desc_layout(n);
    if ((st = grow(&c->desc, &c->desc_cap, L.total, false)) != HTSVD_OK) return st;
    if ((st = grow(&c->hdesc, &c->hdesc_cap, L.total, true)) != HTSVD_OK) return st;
    if ((st = make_plan(imgs, n, p, t, static_cast<unsigned char*>(c->dev), P)) != HTSVD_OK) return st;
    fill_desc(P, static_cast<unsigned char*>(c->hdesc));
    return HTSVD_OK;
}

// Times phases 3 (grouping) and 4 (filter) for candidate tile shapes and keeps the fastest.
Tuning autotune(BatchCache* c, const htsvd_image* imgs, int n, const htsvd_params* p, cudaStream_t s) {
    Tuning best;
    float best_bm = 1e30f, best_f = 1e30f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return best;
    }
    // five filter tile edges; the three grouping tile shapes are tried alongside the first three
    const int trs[] = {5, 4, 6, 8, 7};
    const int bms[][2] = {{4, 8}, {2, 16}, {8, 8}};
    for (int ti = 0; ti < 5; ++ti) {
        Tuning t;
        t.TR = trs[ti];
        t.bmy = bms[ti % 3][0];
        t.bmx = bms[ti % 3][1];
        Plan P;
        if (prepare(c, imgs, n, p, t, P) != HTSVD_OK) continue;
        // bases and grouping first (the filter needs both), then time grouping and filter separately
        if (enqueue(c, P, s, 0x3) != HTSVD_OK) continue;
        float ms = 0.f;
        cudaEventRecord(e0, s);
        if (enqueue(c, P, s, 0x4) != HTSVD_OK) continue;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_bm) {
            best_bm = ms;
            best.bmy = t.bmy;
            best.bmx = t.bmx;
        }
        cudaEventRecord(e0, s);
        if (enqueue(c, P, s, 0x8) != HTSVD_OK) continue;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_f) {
            best_f = ms;
            best.TR = t.TR;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return best;
}

std::vector<unsigned char> batch_key(const htsvd_image* imgs, int n, const htsvd_params* p) {
    std::vector<unsigned char> k(sizeof(htsvd_image) * n + sizeof(htsvd_params) + sizeof(int));
    std::memcpy(k.data(), &n, sizeof(int));
    std::memcpy(k.data() + sizeof(int), imgs, sizeof(htsvd_image) * n);
    htsvd_params z;
    std::memset(&z, 0, sizeof(z));
    if (p) {
        z = *p;
        z.h_sigma_out = nullptr;
        z.d_mask_out = nullptr;
        z.d_weights_out = nullptr;
        z.d_basis_out = nullptr;
        z.d_coef_out = nullptr;
    }
    std::memcpy(k.data() + sizeof(int) + sizeof(htsvd_image) * n, &z, sizeof(z));
    return k;
}

}  // namespace

extern "C" htsvd_status htsvd_denoise_batch(const htsvd_image* imgs, int32_t n, const htsvd_params* p,
                                            cudaStream_t s) {
    if (n < 0 || (n > 0 && !imgs)) return HTSVD_ERR_INVALID_ARG;
    if (n == 0) return HTSVD_OK;
    {   // validate before any device work
        Plan P;
        htsvd_status st = make_plan(imgs, n, p, Tuning(), nullptr, P);
        if (st != HTSVD_OK) return st;
    }
    std::lock_guard<std::mutex> lk(g_bmu);
    BatchCache* c = cache_for(s);
    if (!c) return HTSVD_ERR_CUDA;
    std::vector<unsigned char> key = batch_key(imgs, n, p);
    if (c->exec && key == c->key) {
        BCK(cudaGraphLaunch(c->exec, s));
        return HTSVD_OK;
    }
    // tile shapes: tuned once per (C, K, stride, window, size bucket)
    const int s_ = p && p->stride > 0 ? p->stride : 3, w_ = p && p->window > 0 ? p->window : 18;
    const int K_ = p && p->K > 0 ? p->K : 32;
    int64_t px = 0;
    for (int i = 0; i < n; ++i) px += (int64_t)imgs[i].H * imgs[i].W;
    const int bucket = (int)std::log2((double)std::max<int64_t>(px, 1));
    const auto tk = std::make_tuple(imgs[0].C, K_, s_, w_, 8, bucket);
    Tuning t;
    auto it = g_tuned.find(tk);
    if (it != g_tuned.end()) {
        t = it->second;
    } else if (p && p->tile > 0) {
        t.TR = p->tile;
    } else {
        t = autotune(c, imgs, n, p, s);
        g_tuned[tk] = t;
    }
    // a previous batch's graph may still read the buffers that are about to be rewritten
    BCK(cudaStreamSynchronize(s));
    Plan P;
    htsvd_status st = prepare(c, imgs, n, p, t, P);
    if (st != HTSVD_OK) return st;
    if (c->exec) {
        cudaGraphExecDestroy(c->exec);
        c->exec = nullptr;
    }
    // capture the sequence and replay it
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        st = enqueue(c, P, c->cap);
        ce = cudaStreamEndCapture(c->cap, &graph);
    }
    if (st != HTSVD_OK || ce != cudaSuccess) {
        // the stream cannot be captured (e.g. it is itself being captured by the caller): run eagerly
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        c->key.clear();
        return enqueue(c, P, s);
    }
    ce = cudaGraphInstantiate(&c->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        c->exec = nullptr;
        cudaGetLastError();
        return HTSVD_ERR_CUDA;
    }
    c->key = key;
    BCK(cudaGraphLaunch(c->exec, s));
    return HTSVD_OK;
}

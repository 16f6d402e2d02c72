// htsvd_denoise_noalloc: the plain denoiser for callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc/cudaFree while they run: a host
// application whose own caching allocator has reserved the device memory (a library
// allocating behind it can fail or fragment that pool), and latency-bound processing
// loops in which the implicit device synchronisation of cudaFree would stall other
// streams. This entry point runs the same kernels as htsvd_denoise, with the same parameter
// checks and the same filter tiles (so the same output), but takes every temporary buffer
// (match indices, moments, bases, eigen-gaps, tile partials) from one fixed array in device
// memory that the library declares statically; it calls no allocator at all.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/htsvd.h"
#include "../../include/htsvd_internal.h"
#include "host_plan.h"
#include "kernels.h"

using namespace htsvd;

namespace {

// Every device that loads the library holds this array until the process exits.
constexpr size_t kScratchBytes = (size_t)HTSVD_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device.
htsvd_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HTSVD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HTSVD_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return HTSVD_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carve-up of the scratch array for one call (byte offsets), from the resolved parameters.
struct Carve {
    Geo g;
    FilterTiling t;
    size_t o_idx, o_mom, o_b64, o_b32, o_gap, o_part, total;
};

htsvd_status plan(int H, int W, int C, const htsvd_params* p, Resolved& r, Carve& c) {
    htsvd_status st = resolve(p, C, r);
    if (st != HTSVD_OK) return st;
    if ((st = check_image(H, W, C, r)) != HTSVD_OK) return st;
    c.g = make_geo(H, W, C, r.s, r.win, r.K);
    auto carve = [&](const FilterTiling& t) {
        const size_t n = (size_t)c.g.ngroups();
        size_t o = 0;
        c.t = t;
        c.o_idx = o; o += align256(sizeof(int32_t) * n * r.K);
        c.o_mom = o; o += align256(sizeof(unsigned long long) * 2 * PS2 * C * C);
        c.o_b64 = o; o += align256(sizeof(double) * 2 * 2 * C * PS2);
        c.o_b32 = o; o += align256(sizeof(float) * 512);
        c.o_gap = o; o += align256(sizeof(double) * basis_problems(C));
        c.o_part = o; o += align256(sizeof(float) * (size_t)t.ntx * t.nty * t.FHmax * t.FWmax * (C == 3 ? 4 : 2));
        c.total = o;
    };
    // the tiles of htsvd_denoise; if their partials do not fit the array (and no edge is forced), the
    // largest edge whose shared memory fits a CTA (fewest overlapping footprints, smallest partials)
    const FilterTiling t = choose_filter_tiling(c.g, 1, FM_FORWARD, r.tile);
    if (t.TR == 0) return HTSVD_ERR_UNSUPPORTED;
    carve(t);
    if (c.total > kScratchBytes && r.tile == 0) {
        for (int e = 16; e > t.TR; --e) {
            const FilterTiling te = choose_filter_tiling(c.g, 1, FM_FORWARD, e);
            if (te.TR == 0) continue;
            carve(te);
            break;
        }
    }
    return HTSVD_OK;
}

}  // namespace

extern "C" int64_t htsvd_internal_noalloc_bytes(int32_t H, int32_t W, int32_t C, const htsvd_params* p) {
    Resolved r;
    Carve c;
    if (plan(H, W, C, p, r, c) != HTSVD_OK) return -1;
    return (int64_t)c.total;
}

extern "C" htsvd_status htsvd_denoise_noalloc(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, double sigma,
                                              const htsvd_params* p, float* d_out, cudaStream_t stream) {
    if (!d_noisy || !d_out || !(sigma >= 0) || std::isinf(sigma)) return HTSVD_ERR_INVALID_ARG;
    Resolved r;
    Carve c;
    htsvd_status st = plan(H, W, C, p, r, c);
    if (st != HTSVD_OK) return st;
    // Sizes beyond the array are rejected before any device work.
    if (c.total > kScratchBytes) return HTSVD_ERR_INVALID_ARG;

    void* base = nullptr;
    if ((st = scratch_address(&base)) != HTSVD_OK) return st;
    unsigned char* q = static_cast<unsigned char*>(base);
    int32_t* idx = reinterpret_cast<int32_t*>(q + c.o_idx);
    unsigned long long* mom = reinterpret_cast<unsigned long long*>(q + c.o_mom);
    double* b64 = reinterpret_cast<double*>(q + c.o_b64);
    float* b32 = reinterpret_cast<float*>(q + c.o_b32);
    double* gap = reinterpret_cast<double*>(q + c.o_gap);
    float* part = reinterpret_cast<float*>(q + c.o_part);
    const Geo& g = c.g;

    BMArgs ba{};
    ba.img = d_noisy;
    ba.g = g;
    ba.mode = resolve_mode(r, C);
    ba.gamma2 = r.gamma * r.gamma;
    ba.rstep = 1;
    ba.nry_s = g.nry;
    ba.nrx_s = g.nrx;
    ba.TRy = 4;
    ba.TRx = 8;
    bm_fit_tiles(ba);
    if (bm_smem_bytes(ba) > 227 * 1024) return HTSVD_ERR_UNSUPPORTED;
    ba.idx = idx;
    if (launch_block_match(ba, stream) != cudaSuccess) return HTSVD_ERR_CUDA;
    // launch_moments clears the moment accumulators (left over from the previous call) first.
    if (launch_moments(d_noisy, g, mom, stream) != cudaSuccess) return HTSVD_ERR_CUDA;
    if (launch_basis(mom, C, b64, b32, stream, r.strict_basis ? gap : nullptr) != cudaSuccess) return HTSVD_ERR_CUDA;
    if (p && p->d_basis_out &&
        cudaMemcpyAsync(p->d_basis_out, b64, sizeof(double) * 2 * 2 * C * PS2, cudaMemcpyDeviceToDevice, stream) !=
            cudaSuccess)
        return HTSVD_ERR_CUDA;
    if (r.strict_basis) {
        // the gaps go to a host array on the stack (pageable memory: the copy completes before it returns)
        double h[8];                              // C is 1 or 3 here: at most 4 problems
        const int n = basis_problems(C);
        if (cudaMemcpyAsync(h, gap, sizeof(double) * n, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
            return HTSVD_ERR_CUDA;
        double m = h[0];
        for (int i = 1; i < n; ++i) m = m < h[i] ? m : h[i];
        if (p->h_basis_gap_out) *p->h_basis_gap_out = m;
        if (p->strict_basis && !(m >= kDegenerateGap)) return HTSVD_ERR_DEGENERATE_BASIS;
    }
    if (p && p->h_sigma_out) *p->h_sigma_out = sigma;

    const double tau = r.tau_mult * sigma;
    FilterArgs fa{};
    fa.img = d_noisy;
    fa.img_is_float = 0;
    fa.g = g;
    fa.TR = c.t.TR;
    fa.ntx = c.t.ntx;
    fa.nty = c.t.nty;
    fa.FHmax = c.t.FHmax;
    fa.FWmax = c.t.FWmax;
    fa.idx = idx;
    fa.basis32 = b32;
    fa.basis64 = b64;
    fa.tau64 = tau;
    fa.tau32 = (float)tau;
    fa.band_rel = kBandRel;
    fa.band_abs = (float)(tau * kBandTau) + 1e-6f;
    fa.w_in = nullptr;
    fa.agg_mode = r.agg_mode;
    fa.partials = part;
    fa.mode = FM_FORWARD;
    fa.mask_out = p ? p->d_mask_out : nullptr;
    fa.weights_out = p ? p->d_weights_out : nullptr;
    fa.coef_out = p ? p->d_coef_out : nullptr;
    if (launch_filter(fa, stream) != cudaSuccess) return HTSVD_ERR_CUDA;
    if (launch_reduce(part, g, c.t.TR, c.t.ntx, c.t.nty, c.t.FHmax, c.t.FWmax, d_out, nullptr, 0, nullptr, stream) !=
        cudaSuccess)
        return HTSVD_ERR_CUDA;
    return HTSVD_OK;
}

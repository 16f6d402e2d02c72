// htsvd_denoise_noalloc: the plain denoiser for callers that must not allocate device memory.
//
// Some callers cannot let a library call cudaMalloc/cudaFree while they run: a host
// application whose own caching allocator has reserved the device memory (a library
// allocating behind it can fail or fragment that pool), and latency-bound processing
// loops in which the implicit device synchronisation of cudaFree would stall other
// streams. This entry point runs the same kernels as htsvd_denoise but takes every
// temporary buffer (match indices, moments, bases, tile partials) from one fixed array
// in device memory that the library declares statically; it calls no allocator at all.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/htsvd.h"
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

}  // namespace

extern "C" htsvd_status htsvd_denoise_noalloc(const uint8_t* d_noisy, int32_t H, int32_t W, int32_t C, double sigma,
                                              const htsvd_params* p, float* d_out, cudaStream_t stream) {
    if (!d_noisy || !d_out || !(sigma >= 0)) return HTSVD_ERR_INVALID_ARG;
    htsvd_params z;
    std::memset(&z, 0, sizeof(z));
    if (!p) p = &z;
    const int ps = p->ps > 0 ? p->ps : 8, s = p->stride > 0 ? p->stride : 3;
    const int win = p->window > 0 ? p->window : 18, K = p->K > 0 ? p->K : 32;
    if (p->ps < 0 || p->stride < 0 || p->window < 0 || p->K < 0) return HTSVD_ERR_INVALID_ARG;
    if (K < 2 || (K & (K - 1)) || (C != 1 && C != 3) || H < ps || W < ps) return HTSVD_ERR_INVALID_ARG;
    if (p->match_mode < 0 || p->match_mode > 3 || p->agg_mode < 0 || p->agg_mode > 1) return HTSVD_ERR_INVALID_ARG;
    if (ps != PS || K > 32 || win > 64) return HTSVD_ERR_UNSUPPORTED;
    const Geo g = make_geo(H, W, C, s, win, K);
    if ((int64_t)g.wny * g.wnx < K) return HTSVD_ERR_INVALID_ARG;
    const double gamma = p->gcp_gamma > 0 ? p->gcp_gamma : 1.2;
    const double mult = p->tau_mult > 0 ? p->tau_mult : std::sqrt(2.0 * std::log((double)C * K * ps * ps));
    const double tau = mult * sigma;

    // Tile edge for the filter: the largest of these whose shared memory fits.
    const int cands[] = {8, 6, 4, 2, 1};
    FilterArgs fa{};
    int TR = 1;
    for (int c : cands) {
        fa.g = g;
        fa.FHmax = (c - 1) * s + g.wny + PS - 1 < H ? (c - 1) * s + g.wny + PS - 1 : H;
        fa.FWmax = (c - 1) * s + g.wnx + PS - 1 < W ? (c - 1) * s + g.wnx + PS - 1 : W;
        fa.img_is_float = 0;
        fa.mode = FM_FORWARD;
        if (filter_smem_bytes(fa) <= 200 * 1024) {
            TR = c;
            break;
        }
    }
    const int ntx = (g.nrx + TR - 1) / TR, nty = (g.nry + TR - 1) / TR;
    const int acc = C == 3 ? 4 : 2;

    // Carve the scratch array; sizes beyond it are rejected before any device work.
    const size_t n = (size_t)g.ngroups();
    const size_t b_idx = align256(sizeof(int32_t) * n * K);
    const size_t b_mom = align256(sizeof(unsigned long long) * 2 * PS2 * C * C);
    const size_t b_b64 = align256(sizeof(double) * 2 * 2 * C * PS2);
    const size_t b_b32 = align256(sizeof(float) * 512);
    const size_t b_part = align256(sizeof(float) * (size_t)ntx * nty * fa.FHmax * fa.FWmax * acc);
    if (b_idx + b_mom + b_b64 + b_b32 + b_part > kScratchBytes) return HTSVD_ERR_INVALID_ARG;

    void* base = nullptr;
    htsvd_status st = scratch_address(&base);
    if (st != HTSVD_OK) return st;
    unsigned char* q = static_cast<unsigned char*>(base);
    int32_t* idx = reinterpret_cast<int32_t*>(q);
    unsigned long long* mom = reinterpret_cast<unsigned long long*>(q + b_idx);
    double* b64 = reinterpret_cast<double*>(q + b_idx + b_mom);
    float* b32 = reinterpret_cast<float*>(q + b_idx + b_mom + b_b64);
    float* part = reinterpret_cast<float*>(q + b_idx + b_mom + b_b64 + b_b32);

    BMArgs ba{};
    ba.img = d_noisy;
    ba.g = g;
    ba.mode = C == 1 ? MM_GRAY : (p->match_mode == HTSVD_MATCH_FULL ? MM_FULL
                                  : p->match_mode == HTSVD_MATCH_GREEN ? MM_GREEN : MM_GCP);
    ba.gamma2 = gamma * gamma;
    ba.rstep = 1;
    ba.nry_s = g.nry;
    ba.nrx_s = g.nrx;
    ba.TRy = 4;
    ba.TRx = 8;
    bm_fit_tiles(ba);
    ba.idx = idx;
    if (launch_block_match(ba, stream) != cudaSuccess) return HTSVD_ERR_CUDA;
    // launch_moments clears the moment accumulators (left over from the previous call) first.
    if (launch_moments(d_noisy, g, mom, stream) != cudaSuccess) return HTSVD_ERR_CUDA;
    if (launch_basis(mom, C, b64, b32, stream) != cudaSuccess) return HTSVD_ERR_CUDA;

    fa.img = d_noisy;
    fa.img_is_float = 0;
    fa.g = g;
    fa.TR = TR;
    fa.ntx = ntx;
    fa.nty = nty;
    fa.idx = idx;
    fa.basis32 = b32;
    fa.basis64 = b64;
    fa.tau64 = tau;
    fa.tau32 = (float)tau;
    fa.band_rel = kBandRel;
    fa.band_abs = (float)(tau * kBandTau) + 1e-6f;
    fa.w_in = nullptr;
    fa.agg_mode = p->agg_mode;
    fa.partials = part;
    fa.mode = FM_FORWARD;
    if (launch_filter(fa, stream) != cudaSuccess) return HTSVD_ERR_CUDA;
    if (launch_reduce(part, g, TR, ntx, nty, fa.FHmax, fa.FWmax, d_out, nullptr, 0, nullptr, stream) != cudaSuccess)
        return HTSVD_ERR_CUDA;
    return HTSVD_OK;
}

// Issue-rate probe of the arithmetic pipes the path is bound by: FP32 FMA (the group filter) and the
// integer multiply-add and 4-way byte dot product (block matching). Every thread runs 8 independent
// dependency chains of one instruction kind for a fixed number of iterations; each CTA records its SM
// and its start and end clock, so the rate is counted in operations per SM clock, independent of the
// clock frequency. The loops are bounded and nothing waits on another thread.
#include <cstdint>
#include <vector>

#include "../../include/htsvd_internal.h"
#include "kernels.h"

namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeCtasPerSm = 2;

__device__ __forceinline__ unsigned smid() {
    unsigned r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) alu_probe_kernel(int iters, float fm, float fa, int im, int ia,
                                                                  unsigned long long* rec, float* sink) {
    float f[8];
    int v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        f[k] = 1.0f + 1e-3f * (threadIdx.x + k);
        v[k] = (int)threadIdx.x * 7 + k;
    }
    __syncthreads();
    const unsigned long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if constexpr (OP == 0) f[k] = fmaf(f[k], fm, fa);
                else if constexpr (OP == 1) v[k] = v[k] * im + ia;
                else v[k] = __dp4a(v[k], im, v[k]);
            }
    }
    __syncthreads();
    const unsigned long long t1 = clock64();
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc += f[k] + (float)v[k];
    if (acc == 12345.678f) sink[threadIdx.x] = acc;      // keeps the chains live; never true in practice
    if (threadIdx.x == 0) {
        rec[3 * blockIdx.x] = smid();
        rec[3 * blockIdx.x + 1] = t0;
        rec[3 * blockIdx.x + 2] = t1;
    }
}

}  // namespace

extern "C" double htsvd_internal_alu_probe(int32_t op, int32_t iters) {
    if (op < 0 || op > 2 || iters < 1 || iters > (1 << 20)) return -1.0;
    const int nsm = htsvd::device_sm_count();
    const int grid = kProbeCtasPerSm * nsm;
    unsigned long long* rec = nullptr;
    float* sink = nullptr;
    if (cudaMalloc(&rec, sizeof(unsigned long long) * 3 * grid) != cudaSuccess ||
        cudaMalloc(&sink, sizeof(float) * kProbeThreads) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(rec);
        return -1.0;
    }
    if (op == 0) alu_probe_kernel<0><<<grid, kProbeThreads>>>(iters, 0.999f, 1e-4f, 0x01010101, 3, rec, sink);
    else if (op == 1) alu_probe_kernel<1><<<grid, kProbeThreads>>>(iters, 0.999f, 1e-4f, 0x01010101, 3, rec, sink);
    else alu_probe_kernel<2><<<grid, kProbeThreads>>>(iters, 0.999f, 1e-4f, 0x01010101, 3, rec, sink);
    std::vector<unsigned long long> h(3 * (size_t)grid);
    const bool ok = cudaGetLastError() == cudaSuccess &&
                    cudaMemcpy(h.data(), rec, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost) ==
                        cudaSuccess;
    cudaFree(rec);
    cudaFree(sink);
    if (!ok) return -1.0;
    // per SM: operations of its CTAs over the span from the first start to the last end
    std::vector<unsigned long long> lo(1024, ~0ull), hi(1024, 0);
    std::vector<int> cnt(1024, 0);
    for (int b = 0; b < grid; ++b) {
        const unsigned s = (unsigned)h[3 * b];
        if (s >= 1024) return -1.0;
        lo[s] = h[3 * b + 1] < lo[s] ? h[3 * b + 1] : lo[s];
        hi[s] = h[3 * b + 2] > hi[s] ? h[3 * b + 2] : hi[s];
        cnt[s] += 1;
    }
    const double ops_per_cta = (double)kProbeThreads * iters * 32.0;
    double sum = 0.0;
    int nused = 0;
    for (int s = 0; s < 1024; ++s)
        if (cnt[s] > 0 && hi[s] > lo[s]) {
            sum += ops_per_cta * cnt[s] / (double)(hi[s] - lo[s]);
            ++nused;
        }
    return nused ? sum / nused : -1.0;
}

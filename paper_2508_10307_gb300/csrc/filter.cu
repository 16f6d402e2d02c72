// Dispatch of the group filter, the deterministic reduction of tile partials, and the small kernels
// of the SURE path (perturbed image, FP64 sums).
#include "filter_impl.cuh"

namespace htsvd {

namespace {

template <int K, int C>
cudaError_t dispatch_mode(const FilterArgs& a, cudaStream_t s) {
    switch (a.mode) {
        case FM_FORWARD:
            return a.img_is_float ? launch_filter_t<K, C, float, FM_FORWARD>(a, s)
                                  : launch_filter_t<K, C, uint8_t, FM_FORWARD>(a, s);
        case FM_DENOM:
            return launch_filter_t<K, C, float, FM_DENOM>(a, s);
        case FM_ADJOINT:
            return a.img_is_float ? launch_filter_t<K, C, float, FM_ADJOINT>(a, s) : cudaErrorInvalidValue;
        case FM_VIDEO:
            return a.img_is_float || a.nfr < 1 ? cudaErrorInvalidValue : launch_filter_t<K, C, uint8_t, FM_VIDEO>(a, s);
        case FM_ANALYZE:
        case FM_SYNTH:
            if constexpr (K >= 8) {
                if (a.img_is_float) return cudaErrorInvalidValue;
                return a.mode == FM_ANALYZE ? launch_filter_t<K, C, uint8_t, FM_ANALYZE>(a, s)
                                            : launch_filter_t<K, C, uint8_t, FM_SYNTH>(a, s);
            }
            return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

template <int C>
cudaError_t dispatch_k(const FilterArgs& a, cudaStream_t s) {
    switch (a.g.K) {
        case 2: return dispatch_mode<2, C>(a, s);
        case 4: return dispatch_mode<4, C>(a, s);
        case 8: return dispatch_mode<8, C>(a, s);
        case 16: return dispatch_mode<16, C>(a, s);
        case 32: return dispatch_mode<32, C>(a, s);
    }
    return cudaErrorInvalidValue;
}

// First tile (along one axis) whose footprint ends after p, and last tile whose footprint starts at or before p.
__device__ inline void covering_tiles(int p, int nt, int TR, int nref, int s, int n, int npos, int wlen, int win,
                                      int& lo, int& hi) {
    int a = 0, b = nt - 1;
    while (a < b) {           // smallest t with f1(t) > p
        int m = (a + b) >> 1, f0, f1;
        tile_span(m, TR, nref, s, n, npos, wlen, win, f0, f1);
        if (f1 > p) b = m;
        else a = m + 1;
    }
    lo = a;
    a = 0;
    b = nt - 1;
    while (a < b) {           // largest t with f0(t) <= p
        int m = (a + b + 1) >> 1, f0, f1;
        tile_span(m, TR, nref, s, n, npos, wlen, win, f0, f1);
        if (f0 <= p) a = m;
        else b = m - 1;
    }
    hi = a;
}

// Sum of the tile partials covering pixel p (deterministic tile order), then out = num / den.
template <int C>
__device__ __forceinline__ void reduce_pixel(int64_t p, const float* __restrict__ partials, const Geo& g, int TR,
                                             int ntx, int nty, int FHmax, int FWmax, float* __restrict__ out,
                                             float* __restrict__ den_out, int num_only,
                                             const float* __restrict__ den_in) {
    constexpr int ACC = (C == 3) ? 4 : 2;
    {
        const int y = (int)(p / g.W), x = (int)(p - (int64_t)y * g.W);
        int ylo, yhi, xlo, xhi;
        covering_tiles(y, nty, TR, g.nry, g.s, g.H, g.npy, g.wny, g.win, ylo, yhi);
        covering_tiles(x, ntx, TR, g.nrx, g.s, g.W, g.npx, g.wnx, g.win, xlo, xhi);
        float v[ACC];
#pragma unroll
        for (int c = 0; c < ACC; ++c) v[c] = 0.f;
        for (int ty = ylo; ty <= yhi; ++ty) {
            int fy0, fy1;
            tile_span(ty, TR, g.nry, g.s, g.H, g.npy, g.wny, g.win, fy0, fy1);
            for (int tx = xlo; tx <= xhi; ++tx) {
                int fx0, fx1;
                tile_span(tx, TR, g.nrx, g.s, g.W, g.npx, g.wnx, g.win, fx0, fx1);
                const float* src = partials + (((size_t)(ty * ntx + tx) * FHmax + (y - fy0)) * FWmax + (x - fx0)) * ACC;
                if constexpr (C == 3) {
                    const float4 q = *reinterpret_cast<const float4*>(src);
                    v[0] += q.x; v[1] += q.y; v[2] += q.z; v[3] += q.w;
                } else {
                    const float2 q = *reinterpret_cast<const float2*>(src);
                    v[0] += q.x; v[1] += q.y;
                }
            }
        }
        const float den = den_in ? den_in[p] : v[C];
#pragma unroll
        for (int c = 0; c < C; ++c) out[p * C + c] = num_only ? v[c] : v[c] / den;
        if (den_out) den_out[p] = v[C];
    }
}

template <int C>
__global__ void reduce_kernel(const float* __restrict__ partials, Geo g, int TR, int ntx, int nty, int FHmax,
                              int FWmax, float* __restrict__ out, float* __restrict__ den_out, int num_only,
                              const float* __restrict__ den_in) {
    const int64_t npix = (int64_t)g.H * g.W;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x)
        reduce_pixel<C>(p, partials, g, TR, ntx, nty, FHmax, FWmax, out, den_out, num_only, den_in);
}

// Batch form: pixel blocks of 256 of all images; block w -> image by prefix[] (in blocks).
template <int C>
__global__ void reduce_batch_kernel(const FilterArgs* __restrict__ args, float* const* __restrict__ outs,
                                    const int* __restrict__ prefix, int nimg) {
    const int total = prefix[nimg];
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        int lo = 0, hi = nimg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= w) lo = mid;
            else hi = mid - 1;
        }
        const FilterArgs& a = args[lo];
        const int64_t p = (int64_t)(w - prefix[lo]) * 256 + threadIdx.x;
        if (p < (int64_t)a.g.H * a.g.W)
            reduce_pixel<C>(p, a.partials, a.g, a.TR, a.ntx, a.nty, a.FHmax, a.FWmax, outs[lo], nullptr, 0, nullptr);
    }
}

template <int K, int C>
cudaError_t launch_filter_batch_t(const FilterArgs* d_args, const int* d_prefix, int nimg, size_t smem, int grid,
                                  int* d_counter, cudaStream_t s) {
    auto fn = filter_batch_kernel<K, C>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    fn<<<grid, FT_THREADS, smem, s>>>(d_args, d_prefix, nimg, d_counter);
    return cudaGetLastError();
}

__global__ void div_kernel(const float* __restrict__ gout, const float* __restrict__ den, int64_t npix, int C,
                           float* __restrict__ r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix * C; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = gout[i] / den[i / C];
}

// SURE terms: block b sums (out - x)^2 and probe * g over a strided range in FP64, then a tree in
// shared memory; part[2b], part[2b+1]. Fixed order, so the result is reproducible.
constexpr int SURE_THREADS = 256;
constexpr int SURE_BLOCKS = 304;

__global__ void __launch_bounds__(SURE_THREADS) sure_terms_kernel(const float* __restrict__ out,
                                                                  const float* __restrict__ x,
                                                                  const float* __restrict__ b,
                                                                  const float* __restrict__ g, int64_t n,
                                                                  double* __restrict__ part) {
    __shared__ double s1[SURE_THREADS], s2[SURE_THREADS];
    double a1 = 0.0, a2 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)SURE_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * SURE_THREADS) {
        const double d = (double)out[i] - (double)x[i];
        a1 += d * d;
        a2 += (double)b[i] * (double)g[i];
    }
    s1[threadIdx.x] = a1;
    s2[threadIdx.x] = a2;
    __syncthreads();
    for (int h = SURE_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s1[threadIdx.x] += s1[threadIdx.x + h];
            s2[threadIdx.x] += s2[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

__global__ void sure_sum_kernel(const double* __restrict__ part, int nb, double* __restrict__ res) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a1 = 0.0, a2 = 0.0;
        for (int i = 0; i < nb; ++i) {
            a1 += part[2 * i];
            a2 += part[2 * i + 1];
        }
        res[0] = a1;
        res[1] = a2;
    }
}

// z = y + eps b in float32 with each operation rounded once (no contraction into an FMA), so the
// perturbed image is the one a host forms with IEEE single arithmetic.
__global__ void perturb_kernel(const float* __restrict__ y, const float* __restrict__ b, float eps, int64_t n,
                               float* __restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = __fadd_rn(y[i], __fmul_rn(eps, b[i]));
}

// Cotangent of SURE(w) at one of its two images: u = alpha (f - x) - beta b.
__global__ void sure_cotangent_kernel(const float* __restrict__ f, const float* __restrict__ x,
                                      const float* __restrict__ b, float alpha, float beta, int64_t n,
                                      float* __restrict__ u) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = alpha * (f[i] - x[i]) - beta * b[i];
}

__global__ void add_kernel(const float* __restrict__ a, float* __restrict__ acc, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[i] += a[i];
}

// max |g| as the bits of a non-negative float (their integer order is the float order); *res is
// zeroed by the launcher.
__global__ void absmax_kernel(const float* __restrict__ g, int64_t n, unsigned* __restrict__ res) {
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(g[i]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(res, __float_as_uint(m));
}

// w <- w exp(-step g / max|g|) (nothing when g vanishes).
__global__ void eg_update_kernel(float* __restrict__ w, const float* __restrict__ g, int64_t n, float step,
                                 const unsigned* __restrict__ gmax) {
    const float m = __uint_as_float(*gmax);
    if (!(m > 0.f)) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        w[i] *= expf(-step * g[i] / m);
}

int elementwise_blocks(int64_t n) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > device_sm_count() * 8) blocks = device_sm_count() * 8;
    return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace

cudaError_t launch_sure_cotangent(const float* f, const float* x, const float* b, float alpha, float beta, int64_t n,
                                  float* u, cudaStream_t s) {
    sure_cotangent_kernel<<<elementwise_blocks(n), 256, 0, s>>>(f, x, b, alpha, beta, n, u);
    return cudaGetLastError();
}

cudaError_t launch_add(const float* a, float* acc, int64_t n, cudaStream_t s) {
    add_kernel<<<elementwise_blocks(n), 256, 0, s>>>(a, acc, n);
    return cudaGetLastError();
}

cudaError_t launch_eg_update(float* w, const float* g, int64_t n, float step, unsigned* scratch, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    absmax_kernel<<<elementwise_blocks(n), 256, 0, s>>>(g, n, scratch);
    eg_update_kernel<<<elementwise_blocks(n), 256, 0, s>>>(w, g, n, step, scratch);
    return cudaGetLastError();
}

size_t sure_scratch_doubles() { return 2 * (size_t)SURE_BLOCKS; }

int device_sm_count() {
    constexpr int kMaxDev = 64;
    static int cached[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return 1;
    }
    if (cached[dev] <= 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            return 1;
        }
        cached[dev] = n;          // benign race: every writer stores the same value
    }
    return cached[dev];
}

cudaError_t launch_perturb(const float* y, const float* b, float eps, int64_t n, float* z, cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    if (blocks > device_sm_count() * 8) blocks = device_sm_count() * 8;
    if (blocks < 1) blocks = 1;
    perturb_kernel<<<(int)blocks, 256, 0, s>>>(y, b, eps, n, z);
    return cudaGetLastError();
}

cudaError_t launch_sure_terms(const float* out, const float* x, const float* b, const float* g, int64_t n,
                              double* scratch, double* res, cudaStream_t s) {
    sure_terms_kernel<<<SURE_BLOCKS, SURE_THREADS, 0, s>>>(out, x, b, g, n, scratch);
    sure_sum_kernel<<<1, 32, 0, s>>>(scratch, SURE_BLOCKS, res);
    return cudaGetLastError();
}

size_t filter_smem_bytes(const FilterArgs& a) {
    const int inb = a.img_is_float ? 4 : 1;
    if (a.mode == FM_FORWARD || a.mode == FM_VIDEO || a.mode == FM_ANALYZE || a.mode == FM_SYNTH) {
        const int nfr = a.mode == FM_VIDEO && a.nfr > 0 ? a.nfr : 1;
        return a.g.C == 3 ? f_layout_fwd<32, 3>(a.FHmax, a.FWmax, inb, nfr).total
                          : f_layout_fwd<32, 1>(a.FHmax, a.FWmax, inb, nfr).total;
    }
    if (a.g.C == 3) return f_layout<32, 3>(a.FHmax, a.FWmax, inb, a.mode).total;
    return f_layout<32, 1>(a.FHmax, a.FWmax, inb, a.mode).total;
}

cudaError_t launch_filter(const FilterArgs& a, cudaStream_t s) {
    return a.g.C == 3 ? dispatch_k<3>(a, s) : dispatch_k<1>(a, s);
}

cudaError_t launch_reduce(const float* partials, const Geo& g, int TR, int ntx, int nty, int FHmax, int FWmax,
                          float* out, float* den_out, int num_only, const float* den_in, cudaStream_t s) {
    const int64_t npix = (int64_t)g.H * g.W;
    int blocks = (int)((npix + 255) / 256);
    if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
    if (g.C == 3)
        reduce_kernel<3><<<blocks, 256, 0, s>>>(partials, g, TR, ntx, nty, FHmax, FWmax, out, den_out, num_only, den_in);
    else
        reduce_kernel<1><<<blocks, 256, 0, s>>>(partials, g, TR, ntx, nty, FHmax, FWmax, out, den_out, num_only, den_in);
    return cudaGetLastError();
}

cudaError_t launch_filter_batch(int K, int C, const FilterArgs* d_args, const int* d_prefix, int nimg, size_t smem,
                                int grid, int* d_counter, cudaStream_t s) {
    if (C == 3) {
        switch (K) {
            case 2: return launch_filter_batch_t<2, 3>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
            case 4: return launch_filter_batch_t<4, 3>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
            case 8: return launch_filter_batch_t<8, 3>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
            case 16: return launch_filter_batch_t<16, 3>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
            case 32: return launch_filter_batch_t<32, 3>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
        }
    } else {
        switch (K) {
            case 2: return launch_filter_batch_t<2, 1>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
            case 4: return launch_filter_batch_t<4, 1>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
            case 8: return launch_filter_batch_t<8, 1>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
            case 16: return launch_filter_batch_t<16, 1>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
            case 32: return launch_filter_batch_t<32, 1>(d_args, d_prefix, nimg, smem, grid, d_counter, s);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_reduce_batch(int C, const FilterArgs* d_args, float* const* d_outs, const int* d_prefix, int nimg,
                                int grid, cudaStream_t s) {
    if (C == 3) reduce_batch_kernel<3><<<grid, 256, 0, s>>>(d_args, d_outs, d_prefix, nimg);
    else reduce_batch_kernel<1><<<grid, 256, 0, s>>>(d_args, d_outs, d_prefix, nimg);
    return cudaGetLastError();
}

cudaError_t launch_div(const float* gout, const float* den, int64_t npix, int C, float* r, cudaStream_t s) {
    int blocks = (int)((npix * C + 255) / 256);
    if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
    div_kernel<<<blocks, 256, 0, s>>>(gout, den, npix, C, r);
    return cudaGetLastError();
}

}  // namespace htsvd

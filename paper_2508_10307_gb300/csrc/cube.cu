// Alg. 1 on hyperspectral cubes (Sec. III-E, extension to other imaging; Sec. IV, real-world HSI
// denoising): a patch is a ps x ps x N tube and the t-SVD runs along the band mode, with N Fourier
// slices instead of the three of an RGB image.
//
// The group tensor of a cube (K x 64 x N floats: 254 KB at K = 32, N = 31) does not fit a CTA's
// shared memory, so the filter runs over the group one Haar slot at a time. The Haar transform
// along the group mode and the per-patch t-SVD projection commute, so each slot is formed directly
// from the uint8 patches in its Haar support (exact integer sums and differences), projected
//   band DFT -> per slice f: U_f^H X_f V_f -> inverse band DFT,
// thresholded (FP32; FP64 inside a guard band proportional to the slot's own norm), and, if it keeps a
// coefficient, inverted on the
// kept basis rows only; the 8 x 8 x N spatial slot goes to a per-CTA scratch in global memory that
// stays in L2 (K slots per CTA). After the last slot the CTA runs the Haar synthesis per fibre from
// that scratch and adds every estimated patch into the numerator and denominator planes with float
// atomics (the per-CTA footprint accumulator of the image filter would need (W + 7)^2 x (N + 1)
// floats). The summation order of the atomics varies between runs, so outputs agree to rounding,
// not bit for bit.
#include "filter_impl.cuh"

namespace htsvd {

namespace {

constexpr int CB_THREADS = 256;

struct CubeLayout {
    int bas, tw, tw64, xr, fa, fb, sc, pos, misc, pixnz, total;   // byte offsets
};
__host__ __device__ inline CubeLayout cube_layout(int C, int K) {
    const int nf = C / 2 + 1;
    CubeLayout L;
    int o = 0;
    L.bas = o; o += 4 * (2 * nf * 2 * PS2);        // U, V slices f = 0 .. C/2: [which][f][re, im][a][i]
    L.tw = o; o += 4 * (2 * C);                     // cos, sin of 2 pi k / C
    o = (o + 7) & ~7;
    L.tw64 = o; o += 8 * (2 * C);                   // the same in FP64 (guard-band recomputation)
    L.xr = o; o += 4 * (PS2 * C);                   // raw Haar slot, [pixel][band]
    L.fa = o; o += 4 * (nf * PS2 * 2);              // Fourier slices [f][pixel][re, im]
    L.fb = o; o += 4 * (nf * PS2 * 2);
    L.sc = o; o += 4 * (PS2 * C);                   // real coefficients of the slot [pixel][band]
    L.pos = o; o += 4 * (2 * K);
    L.misc = o; o += 4 * 16;
    L.pixnz = o; o += 4 * PS2;
    L.total = o;
    return L;
}

// Haar row m of the unnormalised in-place transform: support [k0, k0 + L), first half added, second
// half subtracted (all added for m = 0), coefficient stored in slot sl (as haar_for_each).
template <int K>
__device__ __forceinline__ void haar_row(int m, int& k0, int& L, int& half, int& sl) {
    if (m == 0) {
        k0 = 0; L = K; half = K; sl = 0;
        return;
    }
    const int l = 31 - __clz(m), mm = m - (1 << l);
    L = K >> l;
    k0 = mm * L;
    half = L / 2;
    sl = (2 * mm + 1) * (K >> (l + 1));
}

template <int K>
__global__ void __launch_bounds__(CB_THREADS) cube_filter_kernel(CubeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Geo& g = a.g;
    const int C = g.C, nf = C / 2 + 1, NE = PS2 * C;
    const CubeLayout Ly = cube_layout(C, K);
    float* bas = reinterpret_cast<float*>(smem + Ly.bas);
    float* twc = reinterpret_cast<float*>(smem + Ly.tw);
    float* tws = twc + C;
    double* t64c = reinterpret_cast<double*>(smem + Ly.tw64);
    double* t64s = t64c + C;
    float* xr = reinterpret_cast<float*>(smem + Ly.xr);
    float* fa = reinterpret_cast<float*>(smem + Ly.fa);
    float* fb = reinterpret_cast<float*>(smem + Ly.fb);
    float* sc = reinterpret_cast<float*>(smem + Ly.sc);
    int* pos = reinterpret_cast<int*>(smem + Ly.pos);
    int* misc = reinterpret_cast<int*>(smem + Ly.misc);      // 0 kept in group, 1 kept in slot, 2 row mask,
                                                              // 5, 6 squared slot norms (float, by slot parity)
    int* pixnz = reinterpret_cast<int*>(smem + Ly.pixnz);
    const int tid = threadIdx.x, lane = tid & 31;
    float* scratch = a.scratch + (size_t)blockIdx.x * K * NE;
    const uint8_t* img = a.img;
    const int nbw = (K * NE + 31) / 32;

    for (int t = tid; t < 2 * nf * 2 * PS2; t += CB_THREADS) bas[t] = a.basis32[t];
    for (int t = tid; t < C; t += CB_THREADS) {
        float sn, cs;
        sincospif(2.f * (float)t / (float)C, &sn, &cs);
        twc[t] = cs;
        tws[t] = sn;
        double sd, cd;
        sincospi(2.0 * t / C, &sd, &cd);
        t64c[t] = cd;
        t64s[t] = sd;
    }
    auto U = [&](int f, int ri, int a_, int i) { return bas[((0 * nf + f) * 2 + ri) * PS2 + a_ * PS + i]; };
    auto V = [&](int f, int ri, int b_, int j) { return bas[((1 * nf + f) * 2 + ri) * PS2 + b_ * PS + j]; };

    for (int grp = blockIdx.x; grp < g.ngroups(); grp += gridDim.x) {
        __syncthreads();
        if (tid < K) {
            // a caller-given index outside the image is clamped so that no access leaves it
            const int v = a.idx[(size_t)grp * K + tid];
            const int y = v / g.W, x = v - y * g.W;
            pos[2 * tid] = min(max(y, 0), g.H - PS);
            pos[2 * tid + 1] = min(max(x, 0), g.W - PS);
        }
        if (tid < 16) misc[tid] = 0;
        if (a.mask_out)
            for (int t = tid; t < nbw; t += CB_THREADS) a.mask_out[(size_t)grp * nbw + t] = 0u;
        __syncthreads();
        for (int m = 0; m < K; ++m) {
            int k0, L, half, sl;
            haar_row<K>(m, k0, L, half, sl);
            // raw slot: integer Haar combination of the support's patches, and its squared norm
            float nq = 0.f;
            for (int e = tid; e < NE; e += CB_THREADS) {
                const int p = e / C, c = e - p * C, pa = p / PS, pb = p - pa * PS;
                int s = 0;
                for (int k = k0; k < k0 + L; ++k) {
                    const int v = img[((size_t)(pos[2 * k] + pa) * g.W + pos[2 * k + 1] + pb) * C + c];
                    s += (k - k0 < half) ? v : -v;
                }
                xr[e] = (float)s;
                nq = fmaf((float)s, (float)s, nq);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) nq += __shfl_xor_sync(0xffffffffu, nq, off);
            if (tid == 0) { misc[1] = 0; misc[2] = 0; }
            if (tid < PS2) pixnz[tid] = 0;
            if (lane == 0) atomicAdd(reinterpret_cast<float*>(&misc[5 + (m & 1)]), nq);
            __syncthreads();
            // band DFT: X_f[p] = sum_c x[p][c] w^{fc}, w = exp(-2 pi i / C)
            for (int t = tid; t < nf * PS2; t += CB_THREADS) {
                const int f = t / PS2, p = t - f * PS2;
                float re = 0.f, im = 0.f;
                for (int c = 0, k = 0; c < C; ++c, k = (k + f >= C) ? k + f - C : k + f) {
                    const float x = xr[p * C + c];
                    re = fmaf(x, twc[k], re);
                    im = fmaf(-x, tws[k], im);
                }
                fa[2 * t] = re;
                fa[2 * t + 1] = im;
            }
            __syncthreads();
            // Y_f[i][b] = sum_a conj(U_f[a][i]) X_f[a][b]
            for (int t = tid; t < nf * PS2; t += CB_THREADS) {
                const int f = t / PS2, i = (t / PS) % PS, b = t % PS;
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int a_ = 0; a_ < PS; ++a_) {
                    const float ur = U(f, 0, a_, i), ui = U(f, 1, a_, i);
                    const float xr_ = fa[2 * (f * PS2 + a_ * PS + b)], xi = fa[2 * (f * PS2 + a_ * PS + b) + 1];
                    re = fmaf(ur, xr_, fmaf(ui, xi, re));
                    im = fmaf(ur, xi, fmaf(-ui, xr_, im));
                }
                fb[2 * t] = re;
                fb[2 * t + 1] = im;
            }
            __syncthreads();
            // S_f[i][j] = sum_b Y_f[i][b] V_f[b][j]
            for (int t = tid; t < nf * PS2; t += CB_THREADS) {
                const int f = t / PS2, i = (t / PS) % PS, j = t % PS;
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int b = 0; b < PS; ++b) {
                    const float vr = V(f, 0, b, j), vi = V(f, 1, b, j);
                    const float yr = fb[2 * (f * PS2 + i * PS + b)], yi = fb[2 * (f * PS2 + i * PS + b) + 1];
                    re = fmaf(yr, vr, fmaf(-yi, vi, re));
                    im = fmaf(yr, vi, fmaf(yi, vr, im));
                }
                fa[2 * t] = re;
                fa[2 * t + 1] = im;
            }
            __syncthreads();
            // inverse band DFT (real result): S[p][c] = (1/C) sum_f S_f[p] w^{-fc}, slices C - f = conj(f)
            for (int e = tid; e < NE; e += CB_THREADS) {
                const int p = e / C, c = e - p * C;
                float s = fa[2 * p];
                for (int f = 1, k = c; 2 * f < C; ++f, k = (k + c >= C) ? k + c - C : k + c) {
                    const float re = fa[2 * (f * PS2 + p)], im = fa[2 * (f * PS2 + p) + 1];
                    s = fmaf(2.f * re, twc[k], fmaf(-2.f * im, tws[k], s));
                }
                if ((C & 1) == 0) s = fmaf(fa[2 * ((C / 2) * PS2 + p)], (c & 1) ? -1.f : 1.f, s);
                sc[e] = s / (float)C;
            }
            __syncthreads();
            // threshold (the unnormalised slot carries sqrt(L)); kept values scaled by 1/L for the
            // unnormalised synthesis. Entries inside the guard band are decided again in FP64 by the
            // warp that met them.
            {
                // The FP32 error of a slot's coefficients is bounded by a multiple of the slot's own
                // norm (its transform is orthonormal up to the unnormalised Haar factor), so the band
                // is band_rel x ||slot||_F, plus the rounding of tau.
                const float r = sqrtf((float)L), tl = a.tau32 * r;
                const float dl = a.band_rel * sqrtf(__int_as_float(misc[5 + (m & 1)])) + a.band_abs * r;
                const int iters = (NE + CB_THREADS - 1) / CB_THREADS;
                for (int it = 0; it < iters; ++it) {
                    const int e = it * CB_THREADS + tid;
                    const bool valid = e < NE;
                    const float v = valid ? sc[e] : 0.f;
                    if (valid && a.coef_out) a.coef_out[((size_t)grp * K + m) * NE + e] = v / r;
                    const float d = fabsf(v) - tl;
                    const bool band = valid && fabsf(d) <= dl;
                    bool keep = valid && !band && d >= 0.f;
                    unsigned bal = __ballot_sync(0xffffffffu, band);
                    while (bal) {                       // warp-uniform
                        const int l = __ffs(bal) - 1;
                        bal &= bal - 1;
                        const int eb = __shfl_sync(0xffffffffu, e, l);
                        const int pb = eb / C, cb = eb - pb * C, ib = pb / PS, jb = pb - ib * PS;
                        // FP64: P_f = sum_{pixels} conj(U_f[a][ib]) V_f[b][jb] X_f[a][b], X_f the band DFT
                        // of the raw slot (exact integers); S = (1/C) sum_f w^{-f cb} P_f, slices C - f
                        // being the conjugates of f. Lane l takes pixels l and l + 32.
                        double acc = 0.0;
                        for (int f = 0; 2 * f <= C; ++f) {
                            double pr = 0.0, pi = 0.0;
                            for (int q = lane; q < PS2; q += 32) {
                                const int qa = q / PS, qb = q - qa * PS;
                                double xre = 0.0, xim = 0.0;
                                for (int cp = 0, k = 0; cp < C; ++cp, k = (k + f >= C) ? k + f - C : k + f) {
                                    const double x = (double)xr[q * C + cp];
                                    xre = fma(x, t64c[k], xre);
                                    xim = fma(-x, t64s[k], xim);
                                }
                                const double* u = a.basis64 + 2 * (((size_t)0 * C + f) * PS2 + qa * PS + ib);
                                const double* vv = a.basis64 + 2 * (((size_t)1 * C + f) * PS2 + qb * PS + jb);
                                const double cr = u[0] * vv[0] + u[1] * vv[1];      // conj(u) v
                                const double ci = u[0] * vv[1] - u[1] * vv[0];
                                pr += cr * xre - ci * xim;
                                pi += cr * xim + ci * xre;
                            }
#pragma unroll
                            for (int off = 16; off > 0; off >>= 1) {
                                pr += __shfl_xor_sync(0xffffffffu, pr, off);
                                pi += __shfl_xor_sync(0xffffffffu, pi, off);
                            }
                            const int k2 = (int)(((long long)f * cb) % C);
                            const double wgt = (f == 0 || 2 * f == C) ? 1.0 : 2.0;
                            acc += wgt * (t64c[k2] * pr - t64s[k2] * pi);  // Re(w^{-f cb} P_f)
                        }
                        if (lane == l) keep = fabs(acc / (double)C) >= a.tau64 * sqrt((double)L);
                    }
                    if (valid) {
                        sc[e] = keep ? v * (1.f / (float)L) : 0.f;
                        if (keep) {
                            const int p = e / C;
                            pixnz[p] = 1;
                            atomicOr(&misc[2], 1 << (p / PS));
                            if (a.mask_out) {
                                const size_t bit = (size_t)m * NE + e;
                                atomicOr(&a.mask_out[(size_t)grp * nbw + bit / 32], 1u << (bit % 32));
                            }
                        }
                    }
                    const int wk = __reduce_add_sync(0xffffffffu, keep ? 1 : 0);
                    if (lane == 0 && wk) atomicAdd(&misc[1], wk);
                }
                if (tid == 0) misc[5 + ((m + 1) & 1)] = 0;      // the next slot's norm accumulator
            }
            __syncthreads();
            float* dst = scratch + (size_t)sl * NE;
            if (misc[1] == 0) {
                for (int e = tid; e < NE; e += CB_THREADS) dst[e] = 0.f;
                continue;                               // no barrier needed: the next slot's first writes
            }                                           // (xr, misc, pixnz) are after a barrier below
            if (tid == 0) misc[0] += misc[1];
            const int rows = misc[2];
            // inverse: band DFT of the kept coefficients (pixels without one stay zero)
            for (int t = tid; t < nf * PS2; t += CB_THREADS) {
                const int f = t / PS2, p = t - f * PS2;
                float re = 0.f, im = 0.f;
                if (pixnz[p])
                    for (int c = 0, k = 0; c < C; ++c, k = (k + f >= C) ? k + f - C : k + f) {
                        const float x = sc[p * C + c];
                        re = fmaf(x, twc[k], re);
                        im = fmaf(-x, tws[k], im);
                    }
                fa[2 * t] = re;
                fa[2 * t + 1] = im;
            }
            __syncthreads();
            // Z_f[i][b] = sum_j T_f[i][j] conj(V_f[b][j]) on the kept rows
            for (int t = tid; t < nf * PS2; t += CB_THREADS) {
                const int f = t / PS2, i = (t / PS) % PS, b = t % PS;
                float re = 0.f, im = 0.f;
                if ((rows >> i) & 1)
#pragma unroll
                    for (int j = 0; j < PS; ++j) {
                        const float vr = V(f, 0, b, j), vi = V(f, 1, b, j);
                        const float tr = fa[2 * (f * PS2 + i * PS + j)], ti = fa[2 * (f * PS2 + i * PS + j) + 1];
                        re = fmaf(tr, vr, fmaf(ti, vi, re));
                        im = fmaf(ti, vr, fmaf(-tr, vi, im));
                    }
                fb[2 * t] = re;
                fb[2 * t + 1] = im;
            }
            __syncthreads();
            // G_f[a][b] = sum_i U_f[a][i] Z_f[i][b] over the kept rows
            for (int t = tid; t < nf * PS2; t += CB_THREADS) {
                const int f = t / PS2, a_ = (t / PS) % PS, b = t % PS;
                float re = 0.f, im = 0.f;
                for (int r = rows; r; r &= r - 1) {
                    const int i = __ffs(r) - 1;
                    const float ur = U(f, 0, a_, i), ui = U(f, 1, a_, i);
                    const float zr = fb[2 * (f * PS2 + i * PS + b)], zi = fb[2 * (f * PS2 + i * PS + b) + 1];
                    re = fmaf(ur, zr, fmaf(-ui, zi, re));
                    im = fmaf(ur, zi, fmaf(ui, zr, im));
                }
                fa[2 * t] = re;
                fa[2 * t + 1] = im;
            }
            __syncthreads();
            // inverse band DFT -> spatial slot in the scratch
            for (int e = tid; e < NE; e += CB_THREADS) {
                const int p = e / C, c = e - p * C;
                float s = fa[2 * p];
                for (int f = 1, k = c; 2 * f < C; ++f, k = (k + c >= C) ? k + c - C : k + c) {
                    const float re = fa[2 * (f * PS2 + p)], im = fa[2 * (f * PS2 + p) + 1];
                    s = fmaf(2.f * re, twc[k], fmaf(-2.f * im, tws[k], s));
                }
                if ((C & 1) == 0) s = fmaf(fa[2 * ((C / 2) * PS2 + p)], (c & 1) ? -1.f : 1.f, s);
                dst[e] = s / (float)C;
            }
            __syncthreads();
        }
        __syncthreads();
        // weight of the group, then Haar synthesis per fibre and aggregation
        float wg = 1.f;
        if (a.w_in) wg = a.w_in[grp];
        else if (a.agg_mode == 1) wg = 1.f / (float)max(1, misc[0]);
        if (tid == 0 && a.weights_out) a.weights_out[grp] = wg;
        for (int e = tid; e < NE; e += CB_THREADS) {
            float v[K];
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = scratch[(size_t)k * NE + e];
            haar_inv_sum<K>(v);
            const int p = e / C, c = e - p * C, pa = p / PS, pb = p - pa * PS;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const size_t pix = (size_t)(pos[2 * k] + pa) * g.W + pos[2 * k + 1] + pb;
                atomicAdd(&a.num[pix * C + c], wg * v[k]);
                if (c == 0) atomicAdd(&a.den[pix], wg);
            }
        }
    }
}

__global__ void cube_finalize_kernel(const float* __restrict__ num, const float* __restrict__ den, int64_t npix,
                                     int C, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix * C; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = num[i] / den[i / C];
}

template <int K>
cudaError_t launch_cube_t(const CubeArgs& a, int grid, cudaStream_t s) {
    const int smem = cube_layout(a.g.C, K).total;
    auto fn = cube_filter_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, CB_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t cube_smem_bytes(int C, int K) { return (size_t)cube_layout(C, K).total; }

int cube_grid(int C, int K, int64_t ngroups) {
    const size_t smem = cube_smem_bytes(C, K);
    int per_sm = (int)((227 * 1024) / (smem + 1024));
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    const int64_t grid = (int64_t)per_sm * device_sm_count();
    return (int)(grid < ngroups ? grid : ngroups);
}

cudaError_t launch_cube_filter(const CubeArgs& a, int grid, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.num, 0, sizeof(float) * (size_t)a.g.H * a.g.W * a.g.C, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.den, 0, sizeof(float) * (size_t)a.g.H * a.g.W, s);
    if (e != cudaSuccess) return e;
    switch (a.g.K) {
        case 2: e = launch_cube_t<2>(a, grid, s); break;
        case 4: e = launch_cube_t<4>(a, grid, s); break;
        case 8: e = launch_cube_t<8>(a, grid, s); break;
        case 16: e = launch_cube_t<16>(a, grid, s); break;
        case 32: e = launch_cube_t<32>(a, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int64_t n = (int64_t)a.g.H * a.g.W * a.g.C;
    int blocks = (int)((n + 255) / 256);
    if (blocks > device_sm_count() * 16) blocks = device_sm_count() * 16;
    cube_finalize_kernel<<<blocks, 256, 0, s>>>(a.num, a.den, (int64_t)a.g.H * a.g.W, a.g.C, a.out);
    return cudaGetLastError();
}

}  // namespace htsvd

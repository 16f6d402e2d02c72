// Batched forward projection of patches onto the global t-SVD bases (Sec. III-B.2, Eq. (forward
// transform) without the Haar step along the group mode): for every patch P (8 x 8 x C uint8),
// S = U^T * P * V, i.e. per channel-Fourier slice f: S_f = U_f^H P_f V_f, then the inverse DFT
// along the channel mode (Sec. II-C, Def. T-product; the FFT along mode 3).
//
// Two kernels compute the same 64 C coefficients per patch:
//
// * project_tc_kernel: the map P -> S is one real (64 C) x (64 C) matrix T (real because slices
//   f and C - f are conjugate), so a batch of patches is a dense contraction S = P T^T on the
//   fifth-generation tensor cores (tcgen05.mma, kind::f16, FP32 accumulation in tensor memory).
//   The patch bytes are exact in FP16; T (scaled by 2^14) is split into two FP16 pieces
//   T = T_hi + T_lo (T_lo the rounding of what T_hi leaves: 22 significant bits), so two products
//   per K step give an FP32-level result. The pieces of all of T would take 2 x 72 KB of shared
//   memory at C = 3 beside the A tiles, so each CTA holds the pieces of one half of the
//   coefficients (N = 32 C) and the grid runs both halves; the A tile (128 patches x 64 C FP16,
//   gathered from the image by 16 warps) is double-buffered, the accumulator is double-buffered in
//   tensor memory, and one thread issues the MMAs of tile t while the CTA loads the image words of
//   tile t + 1 and reads tile t - 1 out of tensor memory.
// * project_simt_kernel: the structured per-slice form in FP32 on the CUDA cores (channel DFT,
//   U_f^H X_f on patch columns, (.) V_f on patch rows, inverse channel DFT), the form the group
//   filter uses, for comparison.
//
// Coefficient order of both: n = (i * 8 + j) * C + c (basis row i, basis column j, channel c),
// patch input order k = (a * 8 + b) * C + c (image row a, column b, channel c of the patch).
#include <cuda_fp16.h>
#include <cstdint>

#include "kernels.h"

namespace htsvd {
namespace {

constexpr int kProjThreads = 256;           // structured FP32 kernel
constexpr int kTcThreads = 512;             // tensor-core kernel: 16 warps gather, one thread issues the MMAs
constexpr int kTileM = 128;                 // patches per MMA tile (TMEM lanes)
constexpr int kPieces = 2;                  // FP16 pieces of the basis matrix
constexpr float kSplitScale = 16384.0f;     // 2^14: the matrix is split after this scaling, undone on output

template <int C>
struct ProjDims {
    static constexpr int D = 64 * C;                      // inputs per patch = coefficients per patch
    static constexpr int NH = D / 2;                      // coefficients per CTA (one half)
    static constexpr int KCH = D / 8;                     // 8-element K chunks (core-matrix columns)
    static constexpr int KSTEPS = D / 16;                 // MMAs per piece (K = 16 each)
    // bytes between K-adjacent core matrices of A: a plane of 128 rows of 16 bytes plus 64 bytes, so that
    // the gather's stores into the three planes of a patch row fall in two halves of the banks
    static constexpr int LBO_A = kTileM * 16 + 64;
    static constexpr int LBO_B = NH * 16;                 // ... of B
    static constexpr int A_BYTES = KCH * LBO_A;
    static constexpr int B_PIECE = NH * D * 2;
    static constexpr int ACC_COLS = C == 3 ? 128 : 32;   // TMEM column stride of the two accumulators
    static constexpr int TMEM_COLS = 2 * ACC_COLS;       // power of two >= 32
    static constexpr int POS_OFF = 2 * A_BYTES + kPieces * B_PIECE;   // [2][128] int32 patch byte offsets
    static constexpr int BAR_OFF = POS_OFF + 2 * kTileM * 4;    // two mbarriers, then the TMEM slot
    static constexpr int SMEM = BAR_OFF + 32;
    // every-position batches: the eight image rows of a tile staged as words (their first byte shifted
    // by up to 3), SW words per row
    static constexpr int SW = (((kTileM + PS - 1) * C + 6) / 4 + 3) & ~3;
    static constexpr int STAGE_OFF = 2 * A_BYTES + kPieces * B_PIECE;
    static constexpr int DBAR_OFF = STAGE_OFF + PS * SW * 4;
    static constexpr int SMEM_DENSE = DBAR_OFF + 32;
};
static_assert(ProjDims<3>::SMEM <= 232448, "projection tile does not fit shared memory");

// Instruction descriptor of tcgen05.mma kind::f16: D FP32, A and B FP16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle: 8-row x 16-byte core matrices, rows 16 bytes apart;
// lbo = bytes between core matrices adjacent along K, sbo = along M (or N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of `parity` to complete; gives up after about two seconds (false).
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 0; i < (1 << 28); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane, waited for in the same statement.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of the top-left of the patch at linear position p (y * W + x) in an H x W x C image,
// or -1 if the 8 x 8 patch does not lie inside it.
__device__ __forceinline__ int patch_offset(int p, int H, int W, int C) {
    if (p < 0) return -1;
    const int y = p / W, x = p - (p / W) * W;
    if (y > H - PS || x > W - PS) return -1;
    return p * C;
}

// Aligned 32-bit word of the image at byte offset wa; bytes past the end read as zero.
__device__ __forceinline__ uint32_t image_word(const uint8_t* img, long long wa, long long total) {
    if (wa + 4 <= total) return __ldg(reinterpret_cast<const uint32_t*>(img + wa));
    uint32_t v = 0;
    for (int k = 0; k < 4; ++k)
        if (wa + k < total) v |= (uint32_t)img[wa + k] << (8 * k);
    return v;
}


// ------------------------------------------------------------------------------ split basis matrix

// T[n][k] with n = (i, j, co), k = (a, b, ci):  T = Re (1/C) sum_f e^{2 pi i f (co - ci) / C} conj(U_f[a][i]) V_f[b][j]
// in FP64, scaled by 2^14 (|T| <= 1: the pieces stay normal FP16 numbers down to |T| ~ 2^-17, below which
// the dropped part is under 2^-39 absolute), then T_hi = f16(2^14 T), T_lo = f16(2^14 T - T_hi); the
// pair carries 22 significant bits. Written in the shared-memory image of the projection kernel:
// [half][piece][k chunk][n within half][8].
template <int C>
__global__ void split_basis_kernel(const double* __restrict__ b64, __half* __restrict__ out) {
    using Dm = ProjDims<C>;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Dm::D * Dm::D) return;
    const int n = e / Dm::D, k = e - (e / Dm::D) * Dm::D;
    const int co = n % C, j = (n / C) % 8, i = n / (8 * C);
    const int ci = k % C, b = (k / C) % 8, a = k / (8 * C);
    double t = 0.0;
    for (int f = 0; f < C; ++f) {
        const double* U = b64 + 2 * ((size_t)f * 64 + a * 8 + i);                 // U_f[a][i]
        const double* V = b64 + 2 * ((size_t)(C + f) * 64 + b * 8 + j);           // V_f[b][j]
        const double ur = U[0], ui = -U[1];                                        // conj(U_f[a][i])
        const double pr = ur * V[0] - ui * V[1], pi = ur * V[1] + ui * V[0];
        double sn = 0.0, cs = 1.0;
        const int d = ((co - ci) * f) % C;
        if (d != 0) sincospi(2.0 * d / C, &sn, &cs);
        t += pr * cs - pi * sn;                                                    // Re(phase * product)
    }
    t = t / C * kSplitScale;
    const __half hi = __float2half_rn((float)t);
    const __half lo = __float2half_rn((float)(t - (double)__half2float(hi)));
    const int h = n / Dm::NH, r = n % Dm::NH;
    out[((((size_t)h * kPieces + 0) * Dm::KCH + k / 8) * Dm::NH + r) * 8 + (k % 8)] = hi;
    out[((((size_t)h * kPieces + 1) * Dm::KCH + k / 8) * Dm::NH + r) * 8 + (k % 8)] = lo;
}

// ------------------------------------------------------------------------------ tensor-core kernel

// FP16 pair (b0 + 1024, b1 + 1024) from two bytes of w (exact: 1024 + b has 11 significant bits),
// then minus 1024: the bytes as FP16, also exact.
__device__ __forceinline__ uint32_t f16x2_of_bytes(uint32_t w, uint32_t sel) {
    const uint32_t biased = __byte_perm(w, 0x00006400u, sel);
    __half2 h = *reinterpret_cast<const __half2*>(&biased);
    h = __hsub2(h, __half2(__ushort_as_half(0x6400), __ushort_as_half(0x6400)));
    return *reinterpret_cast<const uint32_t*>(&h);
}

// One tile's share of the gather for this lane. Groups of 8 lanes take one patch row at a time:
// lanes 0 .. 2C - 1 each convert 4 bytes of the row (8 C bytes), lane 2C loads the word after the row
// for the byte shift. Lane group g covers patches g and 64 + g of the tile, rows 0..7 (16 words).
struct GatherRegs {
    int o[2];            // byte offsets of the two patches (-1: none)
    uint32_t w[16];      // word of pass p: patch p & 1, row p >> 1
};

template <int C>
__device__ __forceinline__ void gather_fetch(const uint8_t* __restrict__ img, int total, int rowbytes,
                                             const int32_t* __restrict__ pos, long long n, int H, int W,
                                             long long tile, int g, int l, GatherRegs& R) {
    constexpr int NW = 2 * C;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const long long P = tile * kTileM + h * 64 + g;
        R.o[h] = P < n ? patch_offset(__ldg(pos + P), H, W, C) : -1;
    }
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        const int op = R.o[p & 1];
        R.w[p] = 0;
        if (op >= 0 && l <= NW) {
            const int wa = ((op + (p >> 1) * rowbytes) & ~3) + 4 * l;       // < H W C < 2^31
            R.w[p] = wa + 4 <= total ? __ldg(reinterpret_cast<const uint32_t*>(img + wa))
                                     : image_word(img, wa, total);
        }
    }
}

// Converts the fetched words into the A stage (no-swizzle K-major: plane k chunk, row patch, 8 FP16).
template <int C>
__device__ __forceinline__ void gather_store(const GatherRegs& R, int rowbytes, int g, int l, uint8_t* sa) {
    using Dm = ProjDims<C>;
    constexpr int NW = 2 * C;
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        const uint32_t wn = __shfl_down_sync(0xffffffffu, R.w[p], 1, 8);
        const int op = R.o[p & 1], a = p >> 1, m = ((p & 1) << 6) | g;
        if (l < NW) {
            uint2 v = make_uint2(0u, 0u);
            if (op >= 0) {
                const uint32_t bytes = __funnelshift_r(R.w[p], wn, ((op + a * rowbytes) & 3) * 8);
                v.x = f16x2_of_bytes(bytes, 0x5150u);
                v.y = f16x2_of_bytes(bytes, 0x5352u);
            }
            *reinterpret_cast<uint2*>(sa + (a * C + (l >> 1)) * Dm::LBO_A + m * 16 + (l & 1) * 8) = v;
        }
    }
}

// The MMAs of one tile: D[128 x N] = A[128 x K] B^T summed over the pieces (smallest first),
// committed to the tile's mbarrier. Issued by one thread.
template <int C>
__device__ __forceinline__ void issue_tile_mmas(uint32_t a0, uint32_t b0, uint32_t d, uint32_t bar) {
    using Dm = ProjDims<C>;
    constexpr uint32_t kIdesc = idesc_f16(kTileM, Dm::NH);
    uint32_t acc = 0;
#pragma unroll 1
    for (int p = kPieces - 1; p >= 0; --p) {
#pragma unroll
        for (int s = 0; s < Dm::KSTEPS; ++s) {
            const uint64_t ad = smem_desc(a0 + s * 2 * Dm::LBO_A, Dm::LBO_A, 128);
            const uint64_t bd = smem_desc(b0 + p * Dm::B_PIECE + s * 2 * Dm::LBO_B, Dm::LBO_B, 128);
            mma_f16(d, ad, bd, kIdesc, acc);
            acc = 1;
        }
    }
    mma_commit(bar);
}

// Copies this thread's share of a tile's accumulator (TMEM lanes 32 (warp % 4) .., NH / 4 columns
// from (warp / 4) NH / 4) to row `row` of the output (nothing if row < 0; NaN if !valid).
template <int C>
__device__ __forceinline__ void read_out_tile(uint32_t tacc, int warp, long long row, bool valid, int half,
                                              float* __restrict__ coef) {
    using Dm = ProjDims<C>;
    const int q = warp & 3;
    const int cb = (warp >> 2) * (Dm::NH / 4);
    const uint32_t ta = tacc + ((uint32_t)(q * 32) << 16) + cb;
    float* dst = coef + row * Dm::D + half * Dm::NH + cb;
    constexpr float unscale = 1.0f / kSplitScale;
#pragma unroll
    for (int c = 0; c < Dm::NH / 4; c += 8) {
        float v[8];
        tmem_ld8(ta + c, v);
        if (row >= 0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = valid ? v[i] * unscale : __int_as_float(0x7fc00000);
            *reinterpret_cast<float4*>(dst + c) = make_float4(v[0], v[1], v[2], v[3]);
            *reinterpret_cast<float4*>(dst + c + 4) = make_float4(v[4], v[5], v[6], v[7]);
        }
    }
}

template <int C>
__global__ void __launch_bounds__(kTcThreads, 1)
project_tc_kernel(const uint8_t* __restrict__ img, int H, int W, const int32_t* __restrict__ pos, long long n,
                  const uint4* __restrict__ pieces, float* __restrict__ coef, int* __restrict__ flag) {
    using Dm = ProjDims<C>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + 2 * Dm::A_BYTES;
    int* sOff = reinterpret_cast<int*>(smem + Dm::POS_OFF);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Dm::BAR_OFF);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Dm::BAR_OFF + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = tid >> 3, l = tid & 7;
    const int half = blockIdx.x & 1;
    const long long stride = gridDim.x >> 1;
    const long long ntiles = (n + kTileM - 1) / kTileM;
    const long long total = (long long)H * W * C;
    const int rowbytes = W * C;

    {   // this half's pieces of T, one contiguous block in the kernel's smem layout
        const uint4* src = pieces + (size_t)half * (kPieces * Dm::B_PIECE / 16);
        uint4* dst = reinterpret_cast<uint4*>(sB);
        for (int i = tid; i < kPieces * Dm::B_PIECE / 16; i += kTcThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(Dm::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // Software pipeline: the image words of tile t + 2 stride are loaded into the register set that
    // tile t was just stored from, so every load has a whole iteration (the MMAs of tile t and the
    // read-out of tile t - stride) to arrive.
    GatherRegs RA, RB;
    const long long t0 = blockIdx.x >> 1;
    const int totali = (int)total;
    if (t0 < ntiles) gather_fetch<C>(img, totali, rowbytes, pos, n, H, W, t0, g, l, RA);
    if (t0 + stride < ntiles) gather_fetch<C>(img, totali, rowbytes, pos, n, H, W, t0 + stride, g, l, RB);
    bool ok = true;
    long long it = 0;
    long long t = t0;
    auto step = [&](GatherRegs& R) -> bool {
        const bool have = t < ntiles;        // uniform over the CTA
        const int b = (int)(it & 1);
        if (have) {
            gather_store<C>(R, rowbytes, g, l, sA + b * Dm::A_BYTES);
            if (l == 0) {
                sOff[b * kTileM + g] = R.o[0];
                sOff[b * kTileM + 64 + g] = R.o[1];
            }
            fence_async_smem();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (have && tid == 0)
            issue_tile_mmas<C>(smem_u32(sA + b * Dm::A_BYTES), smem_u32(sB), tmem + b * Dm::ACC_COLS,
                               smem_u32(&bars[b]));
        if (t + 2 * stride < ntiles) gather_fetch<C>(img, totali, rowbytes, pos, n, H, W, t + 2 * stride, g, l, R);
        if (it > 0) {   // read out tile t - stride (buffer b ^ 1)
            const int pb = b ^ 1;
            const int m = (warp & 3) * 32 + lane;
            const long long P = (t - stride) * kTileM + m;
            // read before the barrier: once every thread has passed it, the next tile's offsets may
            // overwrite this buffer
            const bool valid = sOff[pb * kTileM + m] >= 0;
            const bool done = mbar_wait_bounded(smem_u32(&bars[pb]), (uint32_t)(((it - 1) >> 1) & 1));
            ok = __syncthreads_and(done) != 0;
            if (!ok) return false;
            tc_fence_after();
            read_out_tile<C>(tmem + pb * Dm::ACC_COLS, warp, P < n ? P : -1, valid, half, coef);
        }
        tc_fence_before();
        if (!have) return false;
        t += stride;
        ++it;
        return true;
    };
    while (step(RA) && step(RB)) {
    }
    tc_fence_before();
    if (!ok) {
        // a read-out wait ran out: report it, and give the tile issued last the same bounded wait before
        // the tensor memory is released
        if (tid == 0 && flag) atomicOr(flag, 1);
        if ((blockIdx.x >> 1) + it * stride < ntiles)
            mbar_wait_bounded(smem_u32(&bars[it & 1]), (uint32_t)((it >> 1) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Dm::TMEM_COLS)
                     : "memory");
    }
}

// Every patch position of the image, row-major over the (H - 7) x (W - 7) grid of top-left corners
// (an im2col batch): a tile is 128 consecutive positions of one grid row, so the eight image rows it
// covers hold all its bytes; each thread loads two words of them, coalesced, for the next tile while
// the current one is multiplied, and the A tile is built from the staged rows in shared memory.
template <int C>
__global__ void __launch_bounds__(kTcThreads, 1)
project_tc_dense_kernel(const uint8_t* __restrict__ img, int H, int W, const uint4* __restrict__ pieces,
                        float* __restrict__ coef, int* __restrict__ flag) {
    using Dm = ProjDims<C>;
    constexpr int NW = 2 * C;
    constexpr int SW = Dm::SW;
    static_assert(PS * SW <= 2 * kTcThreads, "two staged words per thread");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + 2 * Dm::A_BYTES;
    uint32_t* sS = reinterpret_cast<uint32_t*>(smem + Dm::STAGE_OFF);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Dm::DBAR_OFF);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Dm::DBAR_OFF + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = tid >> 3, l = tid & 7;
    const int half = blockIdx.x & 1;
    const long long stride = gridDim.x >> 1;
    const int npx = W - PS + 1, npy = H - PS + 1;
    const int tpr = (npx + kTileM - 1) / kTileM;                 // tiles per row of positions
    const long long ntiles = (long long)npy * tpr;
    const int rowbytes = W * C;
    const long long total = (long long)H * rowbytes;

    {
        const uint4* src = pieces + (size_t)half * (kPieces * Dm::B_PIECE / 16);
        uint4* dst = reinterpret_cast<uint4*>(sB);
        for (int i = tid; i < kPieces * Dm::B_PIECE / 16; i += kTcThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(Dm::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // word w of staged row a of tile tt: the image word at ((y + a) W + x0) C rounded down to 4, + 4 w
    auto fetch = [&](long long tt, uint32_t (&wd)[2]) {
        const int y = (int)(tt / tpr), x0 = (int)(tt % tpr) * kTileM;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int idx = tid + h * kTcThreads;
            wd[h] = 0;
            if (idx < PS * SW) {
                const int a = idx / SW, w = idx - (idx / SW) * SW;
                const long long base = ((long long)(y + a) * rowbytes + (long long)x0 * C) & ~3ll;
                wd[h] = image_word(img, base + 4 * w, total);
            }
        }
    };
    uint32_t wd[2];
    const long long t0 = blockIdx.x >> 1;
    if (t0 < ntiles) fetch(t0, wd);
    bool ok = true;
    long long it = 0;
    for (long long t = t0;; t += stride, ++it) {
        const bool have = t < ntiles;        // uniform over the CTA
        const int b = (int)(it & 1);
        if (have) {
            if (tid < PS * SW) sS[tid] = wd[0];
            if (tid + kTcThreads < PS * SW) sS[tid + kTcThreads] = wd[1];
        }
        __syncthreads();
        if (have) {
            const int y = (int)(t / tpr), x0 = (int)(t % tpr) * kTileM;
            const int cnt = min(kTileM, npx - x0);
            uint8_t* sa = sA + b * Dm::A_BYTES;
#pragma unroll 4
            for (int p = 0; p < 16; ++p) {                // pass p: patch row p / 2 of patches g, 64 + g
                const int a = p >> 1, m = ((p & 1) << 6) | g;
                if (l < NW) {
                    uint2 v = make_uint2(0u, 0u);
                    if (m < cnt) {
                        const int bo = (int)(((long long)(y + a) * rowbytes + (long long)x0 * C) & 3) + m * C + 4 * l;
                        const uint32_t* row = sS + a * SW + (bo >> 2);
                        const uint32_t bytes = __funnelshift_r(row[0], row[1], (bo & 3) * 8);
                        v.x = f16x2_of_bytes(bytes, 0x5150u);
                        v.y = f16x2_of_bytes(bytes, 0x5352u);
                    }
                    *reinterpret_cast<uint2*>(sa + (a * C + (l >> 1)) * Dm::LBO_A + m * 16 + (l & 1) * 8) = v;
                }
            }
            fence_async_smem();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (have && tid == 0)
            issue_tile_mmas<C>(smem_u32(sA + b * Dm::A_BYTES), smem_u32(sB), tmem + b * Dm::ACC_COLS,
                               smem_u32(&bars[b]));
        if (t + stride < ntiles) fetch(t + stride, wd);
        if (it > 0) {   // read out tile t - stride (buffer b ^ 1)
            const int pb = b ^ 1;
            const long long tp = t - stride;
            const int y = (int)(tp / tpr), x0 = (int)(tp % tpr) * kTileM;
            const int m = (warp & 3) * 32 + lane;
            const long long row = m < min(kTileM, npx - x0) ? (long long)y * npx + x0 + m : -1;
            const bool done = mbar_wait_bounded(smem_u32(&bars[pb]), (uint32_t)(((it - 1) >> 1) & 1));
            ok = __syncthreads_and(done) != 0;
            if (!ok) break;
            tc_fence_after();
            read_out_tile<C>(tmem + pb * Dm::ACC_COLS, warp, row, true, half, coef);
        }
        tc_fence_before();
        if (!have) break;
    }
    tc_fence_before();
    if (!ok) {
        if (tid == 0 && flag) atomicOr(flag, 1);
        if ((blockIdx.x >> 1) + it * stride < ntiles)
            mbar_wait_bounded(smem_u32(&bars[it & 1]), (uint32_t)((it >> 1) & 1));
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Dm::TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------------------ structured FP32 kernel

constexpr int kSimtPatches = 32;     // patches per CTA round: 8 lanes each, 4 per warp

// One CTA round: 32 patches staged as bytes, then lane l of a patch computes column l of
// Y_f = U_f^H X_f (X_f the channel DFT of the patch), then row l of Z_f = Y_f V_f and the inverse
// channel DFT of that row, written as 8 C contiguous coefficients.
template <int C>
__global__ void __launch_bounds__(kProjThreads)
project_simt_kernel(const uint8_t* __restrict__ img, int H, int W, const int32_t* __restrict__ pos, long long n,
                    const double* __restrict__ b64, float* __restrict__ coef) {
    constexpr int NF = C / 2 + 1;                       // slices computed (slice C - f is the conjugate of f)
    __shared__ float sU[NF][2][64], sV[NF][2][64];      // [slice][re, im][a * 8 + i]
    __shared__ uint32_t sP[kSimtPatches][2 * C * PS];   // patch bytes, row a at words 2C a ..
    // Y_f[i][b] of patch pl at sY[pl * PSTR + (2 f + re/im) * 72 + i * 9 + b]: the row pad 9 and the patch
    // stride (a multiple of 32 plus 8) keep both the column writes and the row reads free of bank conflicts.
    constexpr int PSTR = NF * 2 * 72 + 8;
    __shared__ float sY[kSimtPatches * PSTR];
    __shared__ int sOk[kSimtPatches];
    const int tid = threadIdx.x;
    for (int e = tid; e < NF * 64; e += kProjThreads) {
        const int f = e / 64, ai = e % 64;
        sU[f][0][ai] = (float)b64[2 * ((size_t)f * 64 + ai)];
        sU[f][1][ai] = (float)b64[2 * ((size_t)f * 64 + ai) + 1];
        sV[f][0][ai] = (float)b64[2 * ((size_t)(C + f) * 64 + ai)];
        sV[f][1][ai] = (float)b64[2 * ((size_t)(C + f) * 64 + ai) + 1];
    }
    const long long total = (long long)H * W * C;
    const int rowbytes = W * C;
    const int pl = tid >> 3, l = tid & 7;               // patch of the round, lane within the patch
    for (long long base = (long long)blockIdx.x * kSimtPatches; base < n; base += (long long)gridDim.x * kSimtPatches) {
        __syncthreads();
        {   // stage row l of patch pl: 2C words from the 2C + 1 aligned words that cover it
            const long long P = base + pl;
            const int o = P < n ? patch_offset(pos ? pos[P] : (int)(P / (W - PS + 1)) * W + (int)(P % (W - PS + 1)), H, W, C)
                                : -1;
            if (l == 0) sOk[pl] = o >= 0 ? 1 : 0;
            const long long ob = (long long)(o >= 0 ? o : 0) + (long long)l * rowbytes;
            const int sh = (int)(ob & 3) * 8;
            uint32_t prev = o >= 0 ? image_word(img, ob & ~3ll, total) : 0u;
#pragma unroll
            for (int wdx = 0; wdx < 2 * C; ++wdx) {
                const uint32_t nxt = o >= 0 ? image_word(img, (ob & ~3ll) + 4 * (wdx + 1), total) : 0u;
                sP[pl][2 * C * l + wdx] = __funnelshift_r(prev, nxt, sh);
                prev = nxt;
            }
        }
        __syncthreads();
        {   // column b = l: channel DFT of the column, then Y_f[:, b] = U_f^H X_f[:, b]
            const uint8_t* pb = reinterpret_cast<const uint8_t*>(sP[pl]);
            float x0[PS], xr[PS], xi[PS];
#pragma unroll
            for (int a = 0; a < PS; ++a) {
                const uint8_t* px = pb + (a * PS + l) * C;
                if (C == 1) {
                    x0[a] = (float)px[0];
                } else {
                    const float r = px[0], g = px[1], bl = px[2];
                    x0[a] = r + g + bl;
                    xr[a] = r - 0.5f * (g + bl);
                    xi[a] = 0.8660254037844386f * (bl - g);      // sqrt(3)/2 (B - G)
                }
            }
#pragma unroll
            for (int i = 0; i < PS; ++i) {
                float y0 = 0.f;
#pragma unroll
                for (int a = 0; a < PS; ++a) y0 = fmaf(sU[0][0][a * 8 + i], x0[a], y0);
                sY[pl * PSTR + i * 9 + l] = y0;
                if (C == 3) {
                    float yr = 0.f, yi = 0.f;
#pragma unroll
                    for (int a = 0; a < PS; ++a) {
                        const float ur = sU[1][0][a * 8 + i], ui = sU[1][1][a * 8 + i];
                        yr = fmaf(ur, xr[a], fmaf(ui, xi[a], yr));      // conj(u) x
                        yi = fmaf(ur, xi[a], fmaf(-ui, xr[a], yi));
                    }
                    sY[pl * PSTR + 2 * 72 + i * 9 + l] = yr;
                    sY[pl * PSTR + 3 * 72 + i * 9 + l] = yi;
                }
            }
        }
        __syncthreads();
        {   // row i = l: Z_f[i, :] = Y_f[i, :] V_f, inverse channel DFT, 8 C coefficients
            const long long P = base + pl;
            float z0[PS], zr[PS], zi[PS];
#pragma unroll
            for (int j = 0; j < PS; ++j) {
                float s0 = 0.f;
#pragma unroll
                for (int b = 0; b < PS; ++b) s0 = fmaf(sY[pl * PSTR + l * 9 + b], sV[0][0][b * 8 + j], s0);
                z0[j] = s0;
                if (C == 3) {
                    float sr = 0.f, si = 0.f;
#pragma unroll
                    for (int b = 0; b < PS; ++b) {
                        const float yr = sY[pl * PSTR + 2 * 72 + l * 9 + b], yi = sY[pl * PSTR + 3 * 72 + l * 9 + b];
                        const float vr = sV[1][0][b * 8 + j], vi = sV[1][1][b * 8 + j];
                        sr = fmaf(yr, vr, fmaf(-yi, vi, sr));
                        si = fmaf(yr, vi, fmaf(yi, vr, si));
                    }
                    zr[j] = sr;
                    zi[j] = si;
                }
            }
            if (P < n) {
                float* dst = coef + P * (64 * C) + l * 8 * C;
                const bool ok = sOk[pl] != 0;
                const float nan = __int_as_float(0x7fc00000);
                if (C == 1) {
#pragma unroll
                    for (int j = 0; j < PS; j += 4)
                        *reinterpret_cast<float4*>(dst + j) =
                            ok ? make_float4(z0[j], z0[j + 1], z0[j + 2], z0[j + 3]) : make_float4(nan, nan, nan, nan);
                } else {
                    float o[24];
                    constexpr float third = 1.0f / 3.0f, s3 = 1.7320508075688772f;
#pragma unroll
                    for (int j = 0; j < PS; ++j) {
                        o[3 * j + 0] = (z0[j] + 2.f * zr[j]) * third;
                        o[3 * j + 1] = (z0[j] - zr[j] - s3 * zi[j]) * third;
                        o[3 * j + 2] = (z0[j] - zr[j] + s3 * zi[j]) * third;
                    }
#pragma unroll
                    for (int q = 0; q < 24; q += 4)
                        *reinterpret_cast<float4*>(dst + q) =
                            ok ? make_float4(o[q], o[q + 1], o[q + 2], o[q + 3]) : make_float4(nan, nan, nan, nan);
                }
            }
        }
    }
}

}  // namespace

size_t project_pieces_bytes(int C) {
    return C == 3 ? (size_t)2 * kPieces * ProjDims<3>::B_PIECE : (size_t)2 * kPieces * ProjDims<1>::B_PIECE;
}

cudaError_t launch_project_split(const double* d_b64, int C, void* d_pieces, cudaStream_t s) {
    const int D = 64 * C, nth = 256, nbl = (D * D + nth - 1) / nth;
    if (C == 3) split_basis_kernel<3><<<nbl, nth, 0, s>>>(d_b64, static_cast<__half*>(d_pieces));
    else split_basis_kernel<1><<<nbl, nth, 0, s>>>(d_b64, static_cast<__half*>(d_pieces));
    return cudaGetLastError();
}

template <int C>
static cudaError_t launch_tc_c(const uint8_t* img, int H, int W, const int32_t* pos, long long n, const void* pieces,
                               float* coef, int* flag, cudaStream_t s) {
    using Dm = ProjDims<C>;
    static int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(project_tc_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, Dm::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(project_tc_dense_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     Dm::SMEM_DENSE);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    const int half_grid = device_sm_count() / 2 > 0 ? device_sm_count() / 2 : 1;
    const long long ntiles = pos ? (n + kTileM - 1) / kTileM
                                 : (long long)(H - PS + 1) * ((W - PS + 1 + kTileM - 1) / kTileM);
    const int g = (int)(ntiles < half_grid ? ntiles : half_grid);
    if (pos)
        project_tc_kernel<C><<<2 * g, kTcThreads, Dm::SMEM, s>>>(img, H, W, pos, n, static_cast<const uint4*>(pieces),
                                                                  coef, flag);
    else
        project_tc_dense_kernel<C><<<2 * g, kTcThreads, Dm::SMEM_DENSE, s>>>(img, H, W,
                                                                             static_cast<const uint4*>(pieces), coef, flag);
    return cudaGetLastError();
}

cudaError_t launch_project_tc(const uint8_t* img, int H, int W, int C, const int32_t* pos, long long n,
                              const void* d_pieces, float* coef, int* flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    return C == 3 ? launch_tc_c<3>(img, H, W, pos, n, d_pieces, coef, flag, s)
                  : launch_tc_c<1>(img, H, W, pos, n, d_pieces, coef, flag, s);
}

cudaError_t launch_project_simt(const uint8_t* img, int H, int W, int C, const int32_t* pos, long long n,
                                const double* d_b64, float* coef, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long rounds = (n + kSimtPatches - 1) / kSimtPatches;
    const long long cap = (long long)device_sm_count() * 8;
    const int g = (int)(rounds < cap ? rounds : cap);
    if (C == 3) project_simt_kernel<3><<<g, kProjThreads, 0, s>>>(img, H, W, pos, n, d_b64, coef);
    else project_simt_kernel<1><<<g, kProjThreads, 0, s>>>(img, H, W, pos, n, d_b64, coef);
    return cudaGetLastError();
}

}  // namespace htsvd

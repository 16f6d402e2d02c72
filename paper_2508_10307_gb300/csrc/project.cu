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
//   coefficients (N = 32 C) and the grid runs both halves. Warp-specialised: eleven warps gather
//   128-patch A tiles (FP16) into a two-stage ring, one thread issues the MMAs into one of two TMEM
//   accumulators, four warps read the accumulators out; mbarriers hand the stages and accumulators
//   over. Batches are a list of positions or every position of the image (row-major corners).
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
    static constexpr int BAR_OFF = POS_OFF + 2 * kTileM * 4;    // eight mbarriers, the TMEM slot, the abort word
    static constexpr int SMEM = BAR_OFF + 80;
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

// Waits for the phase of `parity` of an mbarrier, giving up when the CTA's abort word is set or after
// about two seconds (then it sets the abort word). Returns false on giving up.
__device__ bool mbar_wait_or_abort(uint32_t bar, uint32_t parity, volatile int* abort_word) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int i = 0; i < (1 << 28); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_word) return false;
        if (global_ns() - t0 > 2000000000ull) break;
    }
    *abort_word = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// The MMAs of one tile: D[128 x N] = A[128 x K] B^T summed over the pieces (smallest first). Issued by
// one thread; the caller commits.
template <int C>
__device__ __forceinline__ void issue_tile_mmas(uint32_t a0, uint32_t b0, uint32_t d) {
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
}

// Byte offset of patch m of tile t (-1: none) and its output row (-1: none). DENSE: tile t is positions
// x0 .. x0 + 127 of row y of the (H - 7) x (W - 7) corner grid; otherwise patches t * 128 + m of pos.
template <int C, bool DENSE>
__device__ __forceinline__ int tile_patch(long long t, int m, const int32_t* __restrict__ pos, long long n, int H,
                                          int W, int tpr, long long& row) {
    if (DENSE) {
        const int npx = W - PS + 1;
        const int y = (int)(t / tpr), x = (int)(t % tpr) * kTileM + m;
        if (x >= npx) { row = -1; return -1; }
        row = (long long)y * npx + x;
        return (y * W + x) * C;
    }
    const long long P = t * kTileM + m;
    if (P >= n) { row = -1; return -1; }
    row = P;
    return patch_offset(__ldg(pos + P), H, W, C);
}

// Warp-specialised projection (one CTA per SM, 16 warps, each CTA one half of the coefficients):
//   warps 5..15 gather: patch bytes of tile i -> FP16 A stage i % 2 (one task = 8 bytes of a patch row
//     -> 16 bytes of a core-matrix row), then arrive on full[i % 2];
//   warp 4, one thread: waits full[s] and the accumulator's release, issues the tile's MMAs into TMEM
//     accumulator i % 2, commits to empty[s] (the stage may be refilled) and accfull[b];
//   warps 0..3 (TMEM lane quarters 0..3): wait accfull[b], read the accumulator out, release it.
// Every wait is bounded; a wait that runs out sets the CTA's abort word, which ends every role.
template <int C, bool DENSE>
__global__ void __launch_bounds__(kTcThreads, 1)
project_tc_kernel(const uint8_t* __restrict__ img, int H, int W, const int32_t* __restrict__ pos, long long n,
                  const uint4* __restrict__ pieces, float* __restrict__ coef, int* __restrict__ flag) {
    using Dm = ProjDims<C>;
    constexpr int kProdWarp0 = 5;
    constexpr int kProdThreads = kTcThreads - kProdWarp0 * 32;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + 2 * Dm::A_BYTES;
    int* sOff = reinterpret_cast<int*>(smem + Dm::POS_OFF);                  // [2][128] patch byte offsets
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Dm::BAR_OFF);        // full[2] empty[2] accfull[2] accempty[2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Dm::BAR_OFF + 64);
    volatile int* abort_word = reinterpret_cast<volatile int*>(smem + Dm::BAR_OFF + 68);
    volatile int* issued = reinterpret_cast<volatile int*>(smem + Dm::BAR_OFF + 72);   // tiles the MMA thread issued
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int half = blockIdx.x & 1;
    const long long stride = gridDim.x >> 1;
    const int tpr = (W - PS + 1 + kTileM - 1) / kTileM;
    const long long ntiles = DENSE ? (long long)(H - PS + 1) * tpr : (n + kTileM - 1) / kTileM;
    const int rowbytes = W * C;
    const int total = H * rowbytes;

    {   // this half's pieces of T, one contiguous block in the kernel's smem layout
        const uint4* src = pieces + (size_t)half * (kPieces * Dm::B_PIECE / 16);
        uint4* dst = reinterpret_cast<uint4*>(sB);
        for (int i = tid; i < kPieces * Dm::B_PIECE / 16; i += kTcThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&bars[s]), kProdThreads);          // full: every gather thread
            mbar_init(smem_u32(&bars[2 + s]), 1);                 // empty: the MMA commit
            mbar_init(smem_u32(&bars[4 + s]), 1);                 // accfull: the MMA commit
            mbar_init(smem_u32(&bars[6 + s]), 128);               // accempty: every read-out thread
        }
        *abort_word = 0;
        *issued = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) {
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
    const long long t0 = blockIdx.x >> 1;

    if (warp >= kProdWarp0) {
        // ---- gather
        const int pt = tid - kProdWarp0 * 32;
        long long row;
        long long i = 0;
        for (long long t = t0; t < ntiles; t += stride, ++i) {
            const int s = (int)(i & 1);
            const bool free_ = i < 2 || mbar_wait_or_abort(smem_u32(&bars[2 + s]), (uint32_t)(((i >> 1) & 1) ^ 1),
                                                          abort_word);
            if (free_ && pt < kTileM) sOff[s * kTileM + pt] = tile_patch<C, DENSE>(t, pt, pos, n, H, W, tpr, row);
            // every gather thread passes this barrier, and all of them leave together if any wait ran out
            uint32_t all_free;
            asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
                         "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
                         : "=r"(all_free)
                         : "r"((uint32_t)free_), "n"(kProdThreads)
                         : "memory");
            if (!all_free) break;
            uint8_t* sa = sA + s * Dm::A_BYTES;
            // every load of this thread's tasks first (three aligned words per task), then the
            // conversions and stores, so that all of them are in flight together
            constexpr int NTASK = kTileM * PS * C;
            constexpr int NT = (NTASK + kProdThreads - 1) / kProdThreads;
            uint32_t wv[NT][3];
            int sh[NT];
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int task = pt + j * kProdThreads;
                wv[j][0] = wv[j][1] = wv[j][2] = 0u;
                sh[j] = -1;
                if (task < NTASK) {
                    const int m = task & (kTileM - 1), r = task >> 7;
                    const int a = r / C, c = r - (r / C) * C;
                    const int o = sOff[s * kTileM + m];
                    if (o >= 0) {
                        const int off = o + a * rowbytes + 8 * c, al = off & ~3;
                        if (al + 12 <= total) {
                            const uint32_t* p = reinterpret_cast<const uint32_t*>(img + al);
                            wv[j][0] = __ldg(p);
                            wv[j][1] = __ldg(p + 1);
                            wv[j][2] = __ldg(p + 2);
                        } else {
                            wv[j][0] = image_word(img, al, total);
                            wv[j][1] = image_word(img, al + 4, total);
                            wv[j][2] = image_word(img, al + 8, total);
                        }
                        sh[j] = (off & 3) * 8;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int task = pt + j * kProdThreads;
                if (task < NTASK) {
                    const int m = task & (kTileM - 1), r = task >> 7;
                    const int a = r / C, c = r - (r / C) * C;
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (sh[j] >= 0) {
                        const uint32_t lo = __funnelshift_r(wv[j][0], wv[j][1], sh[j]);
                        const uint32_t hi = __funnelshift_r(wv[j][1], wv[j][2], sh[j]);
                        v = make_uint4(f16x2_of_bytes(lo, 0x5150u), f16x2_of_bytes(lo, 0x5352u),
                                       f16x2_of_bytes(hi, 0x5150u), f16x2_of_bytes(hi, 0x5352u));
                    }
                    *reinterpret_cast<uint4*>(sa + (a * C + c) * Dm::LBO_A + m * 16) = v;
                }
            }
            fence_async_smem();
            mbar_arrive(smem_u32(&bars[s]));
            // the offsets of this stage are read again only by the next use of the stage, after
            // empty[s]; the gather threads pass the named barrier before rewriting them
        }
    } else if (warp == 4) {
        // ---- MMA issue
        if (lane == 0) {
            long long i = 0;
            for (long long t = t0; t < ntiles; t += stride, ++i) {
                const int s = (int)(i & 1);
                const uint32_t ph = (uint32_t)((i >> 1) & 1);
                if (!mbar_wait_or_abort(smem_u32(&bars[s]), ph, abort_word)) break;
                if (i >= 2 && !mbar_wait_or_abort(smem_u32(&bars[6 + s]), ph ^ 1u, abort_word)) break;
                tc_fence_after();
                issue_tile_mmas<C>(smem_u32(sA + s * Dm::A_BYTES), smem_u32(sB), tmem + s * Dm::ACC_COLS);
                mma_commit(smem_u32(&bars[2 + s]));
                mma_commit(smem_u32(&bars[4 + s]));
            }
            *issued = (int)i;
        }
        __syncwarp();
    } else {
        // ---- read-out: warp w holds TMEM lanes 32 w .. 32 w + 31 = patches of the tile
        const int m = warp * 32 + lane;
        constexpr float unscale = 1.0f / kSplitScale;
        long long i = 0;
        for (long long t = t0; t < ntiles; t += stride, ++i) {
            const int b = (int)(i & 1);
            long long row;
            const int o = tile_patch<C, DENSE>(t, m, pos, n, H, W, tpr, row);
            const bool got = mbar_wait_or_abort(smem_u32(&bars[4 + b]), (uint32_t)((i >> 1) & 1), abort_word);
            if (__any_sync(0xffffffffu, !got)) break;
            tc_fence_after();
            const uint32_t ta = tmem + b * Dm::ACC_COLS + ((uint32_t)(warp * 32) << 16);
            float* dst = coef + row * Dm::D + half * Dm::NH;
#pragma unroll 4
            for (int c = 0; c < Dm::NH; c += 8) {
                float v[8];
                tmem_ld8(ta + c, v);
                if (row >= 0) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) v[q] = o >= 0 ? v[q] * unscale : __int_as_float(0x7fc00000);
                    *reinterpret_cast<float4*>(dst + c) = make_float4(v[0], v[1], v[2], v[3]);
                    *reinterpret_cast<float4*>(dst + c + 4) = make_float4(v[4], v[5], v[6], v[7]);
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(&bars[6 + b]));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_word) {
        // a wait ran out: report it, and let the MMAs issued last finish (they complete in order; the
        // wait is bounded) before the tensor memory is released
        if (warp == 4 && lane == 0) {
            if (flag) atomicOr(flag, 1);
            const int last = *issued - 1;
            if (last >= 0) mbar_wait_bounded(smem_u32(&bars[4 + (last & 1)]), (uint32_t)((last >> 1) & 1));
        }
        __syncthreads();
    }
    if (warp == 4) {
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
        e = cudaFuncSetAttribute(project_tc_kernel<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, Dm::SMEM);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(project_tc_kernel<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, Dm::SMEM);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    const int half_grid = device_sm_count() / 2 > 0 ? device_sm_count() / 2 : 1;
    const long long ntiles = pos ? (n + kTileM - 1) / kTileM
                                 : (long long)(H - PS + 1) * ((W - PS + 1 + kTileM - 1) / kTileM);
    const int g = (int)(ntiles < half_grid ? ntiles : half_grid);
    const uint4* pc = static_cast<const uint4*>(pieces);
    if (pos) project_tc_kernel<C, false><<<2 * g, kTcThreads, Dm::SMEM, s>>>(img, H, W, pos, n, pc, coef, flag);
    else project_tc_kernel<C, true><<<2 * g, kTcThreads, Dm::SMEM, s>>>(img, H, W, pos, n, pc, coef, flag);
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

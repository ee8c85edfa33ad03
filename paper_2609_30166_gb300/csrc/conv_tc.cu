// conv_tc.cu -- 3x3x3 convolution (stride 1, zero "same" padding) as an
// implicit GEMM on the 5th-generation tensor cores (tcgen05, sm_103a), for
// the learned warm start (a 3D U-Net).  BF16 operands, FP32 accumulation in
// tensor memory (TMEM).  The paper has no such operator; it motivates learned
// components combined with the physics operators (Sec. 5).
//
// One kernel computes C[M][N] = sum_k A[M][k] B[N][k] tile by tile:
//   * M tile 128 (one UMMA row block, cta_group::1), N tile = BN in {16..128},
//     K staged 64 elements (one 128-byte row per operand row) at a time;
//   * operands are gathered from global memory by the CTA's 128 threads
//     (implicit im2col, so no TMA tiled box fits them) and written straight
//     into the 128-byte-swizzled K-major shared-memory layout the UMMA
//     descriptors describe; for FWD with channel counts that are multiples
//     of 8 by asynchronous 16-byte copies (conv_fwd_async_kernel), otherwise
//     by loads and stores; the gather of chunk c+1 overlaps the MMAs of
//     chunk c;
//   * one thread issues four tcgen05.mma (K = 16 each) per chunk and commits
//     them to the stage's mbarrier; the accumulator tile lives in TMEM and is
//     read back with tcgen05.ld by the four warps (one row per thread) for
//     the epilogue.
// Three operand layouts use it:
//   FWD   A = im2col(x)[m][(tap, ci)], B = w[co][(tap, ci)], C -> y[m][co]
//         (+ bias, optional ReLU);  m runs over N*D*H*W output voxels (NDHWC).
//   DGRAD the same with dy as input and the flipped, transposed weights
//         w'[ci][(tap, co)] (prepared by the caller): dx = conv(dy, w').
//   WGRAD A = im2col(x)^T[(tap, ci)][m], B = dy^T[co][m]: K runs over voxels,
//         split across CTAs, partial tiles added to dw[co][(tap, ci)] (FP32).
// Every wait on an mbarrier is bounded; on expiry the kernel records an error
// in the status word, releases its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "ctrex.h"

namespace {

#ifndef CTREX_CONV_BRICK
#define CTREX_CONV_BRICK 1
#endif

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int STAGES = 2;
constexpr int THREADS = 128;
constexpr long long WAIT_LIMIT = 1LL << 26;

enum Op { OP_FWD = 0, OP_WGRAD = 1 };

struct ConvShape {
    int nb, d, h, w;   // batch and spatial size (NDHWC)
    int cin, cout;     // channels of the conv input / output (for WGRAD: of x and dy)
    int relu;          // FWD epilogue
    long long m_total; // GEMM M (FWD: voxels) / rows of A (WGRAD: 27 * cin)
    int n_total;       // GEMM N (FWD: cout; WGRAD: cout)
    long long k_total; // GEMM K (FWD: 27 * cin; WGRAD: voxels)
    long long k_per_cta;  // WGRAD split-K range per CTA (multiple of BK)
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of
// 8 rows x 16 bytes stored contiguously; lbo = byte stride between core
// matrices along K, sbo = byte stride between 8-row groups along M (or N).
__device__ __forceinline__ uint64_t sdesc_none(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Bounded wait for the given phase parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    const uint32_t a = smem_addr(bar);
    for (long long i = 0; i < WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id, bool accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(id), "r"((uint32_t)accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared; src_bytes 0 writes zeros.
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of 16-byte chunk j of row r in a 128B-swizzled K-major tile.
__device__ __forceinline__ uint32_t swz(int r, int j) { return (uint32_t)(r * 128 + ((j ^ (r & 7)) << 4)); }

// FWD epilogue of 16 accumulator columns of one output voxel (row): bias,
// optional ReLU, channels c .. c+15 of y[row] (those below n_total).
__device__ __forceinline__ void store16_fwd(const float v[16], const float *__restrict__ bias, void *__restrict__ out,
                                            int out_bf16, const ConvShape &S, long long row, int c)
{
    float y[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int co = c + i;
        y[i] = v[i] + ((bias && co < S.n_total) ? bias[co] : 0.0f);
        if (S.relu) y[i] = fmaxf(y[i], 0.0f);
    }
    const long long o = row * S.n_total + c;
    if ((S.n_total & 15) == 0) {  // 16 whole channels, 16-byte aligned
        if (out_bf16) {
            uint32_t pk[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(y[2 * i], y[2 * i + 1]);
                pk[i] = *reinterpret_cast<const uint32_t *>(&h2);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(out) + o);
            dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        } else {
            float4 *dst = reinterpret_cast<float4 *>(static_cast<float *>(out) + o);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = make_float4(y[4 * i], y[4 * i + 1], y[4 * i + 2], y[4 * i + 3]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if (c + i >= S.n_total) continue;
            if (out_bf16)
                static_cast<__nv_bfloat16 *>(out)[o + i] = __float2bfloat16_rn(y[i]);
            else
                static_cast<float *>(out)[o + i] = y[i];
        }
    }
}

// -------- operand loaders (write one BK-wide chunk of a tile into smem) ----

// A for FWD: row r <-> voxel m0 + r (coordinates decoded once per CTA by the
// caller into rc = {n, z, y, x}, n < 0 for rows past the end); columns
// k = (tap, ci), tap = kz*9 + ky*3 + kx.
__device__ __forceinline__ void load_im2col_rows(const __nv_bfloat16 *__restrict__ x, const ConvShape &S,
                                                 const int4 rc, long long k0, uint8_t *tile)
{
    const int r = threadIdx.x;
    const bool mrow = rc.x >= 0;
    const int cin = S.cin;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const long long kb = k0 + 8 * j;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (mrow && (cin & 7) == 0) {
            const int tap = (int)(kb / cin), ci = (int)(kb - (long long)tap * cin);
            if (tap < 27) {
                const int zz = rc.y + tap / 9 - 1, yy = rc.z + (tap / 3) % 3 - 1, xs = rc.w + tap % 3 - 1;
                if ((unsigned)zz < (unsigned)S.d && (unsigned)yy < (unsigned)S.h && (unsigned)xs < (unsigned)S.w)
                    v = __ldg(reinterpret_cast<const uint4 *>(
                        x + ((((long long)rc.x * S.d + zz) * S.h + yy) * S.w + xs) * cin + ci));
            }
        } else if (mrow) {
            __nv_bfloat16 e[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                e[q] = __float2bfloat16_rn(0.0f);
                const long long k = kb + q;
                const int tap = (int)(k / cin), ci = (int)(k - (long long)tap * cin);
                if (tap < 27) {
                    const int zz = rc.y + tap / 9 - 1, yy = rc.z + (tap / 3) % 3 - 1, xs = rc.w + tap % 3 - 1;
                    if ((unsigned)zz < (unsigned)S.d && (unsigned)yy < (unsigned)S.h && (unsigned)xs < (unsigned)S.w)
                        e[q] = x[((((long long)rc.x * S.d + zz) * S.h + yy) * S.w + xs) * cin + ci];
                }
            }
            v = *reinterpret_cast<const uint4 *>(e);
        }
        *reinterpret_cast<uint4 *>(tile + swz(r, j)) = v;
    }
}

// The same A chunk with asynchronous copies (channel counts that are
// multiples of 8: every 16-byte chunk is one tap's eight channels).
__device__ __forceinline__ void load_im2col_rows_async(const __nv_bfloat16 *__restrict__ x, const ConvShape &S,
                                                       const int4 rc, long long k0, uint8_t *tile)
{
    const int r = threadIdx.x;
    const int cin = S.cin;
    // (tap, channel) of the chunk's first column, then stepped by 8 channels
    int tap = (int)k0 / cin, ci = (int)k0 - tap * cin;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const __nv_bfloat16 *src = x;
        int bytes = 0;
        if (rc.x >= 0 && tap < 27) {
            const int tz = tap / 9, ty = (tap - 9 * tz) / 3, tx = tap - 9 * tz - 3 * ty;
            const int zz = rc.y + tz - 1, yy = rc.z + ty - 1, xs = rc.w + tx - 1;
            if ((unsigned)zz < (unsigned)S.d && (unsigned)yy < (unsigned)S.h && (unsigned)xs < (unsigned)S.w) {
                src = x + ((((long long)rc.x * S.d + zz) * S.h + yy) * S.w + xs) * cin + ci;
                bytes = 16;
            }
        }
        cp_async16(tile + swz(r, j), src, bytes);
        ci += 8;
        if (ci >= cin) {
            ci -= cin;
            ++tap;
        }
    }
}

// B chunk with asynchronous copies (K a multiple of 8).
template <int BN>
__device__ __forceinline__ void load_rows_kmajor_async(const __nv_bfloat16 *__restrict__ w, long long ktot,
                                                       int nrows, int n0, long long k0, uint8_t *tile)
{
    for (int i = threadIdx.x; i < BN * 8; i += THREADS) {
        const int r = i >> 3, j = i & 7;
        const long long kb = k0 + 8 * j;
        const int row = n0 + r;
        const bool in = row < nrows && kb + 8 <= ktot;
        cp_async16(tile + swz(r, j), in ? w + (long long)row * ktot + kb : w, in ? 16 : 0);
    }
}

// B for FWD: rows n0 .. n0+BN of a row-major [N][K] matrix (K = ktot).
template <int BN>
__device__ __forceinline__ void load_rows_kmajor(const __nv_bfloat16 *__restrict__ w, long long ktot, int nrows,
                                                 int n0, long long k0, uint8_t *tile)
{
    for (int i = threadIdx.x; i < BN * 8; i += THREADS) {
        const int r = i >> 3, j = i & 7;
        const long long kb = k0 + 8 * j;
        const int row = n0 + r;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (row < nrows) {
            const __nv_bfloat16 *src = w + (long long)row * ktot + kb;
            if ((ktot & 7) == 0 && kb + 8 <= ktot) {
                v = __ldg(reinterpret_cast<const uint4 *>(src));
            } else {
                __nv_bfloat16 e[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) e[q] = (kb + q < ktot) ? src[q] : __float2bfloat16_rn(0.0f);
                v = *reinterpret_cast<const uint4 *>(e);
            }
        }
        *reinterpret_cast<uint4 *>(tile + swz(r, j)) = v;
    }
}

// Transposes an 8x8 block of BF16 held as 8 rows of 16 bytes (in[v] = eight
// channels of voxel v) into out[c] = channel c of the eight voxels.
__device__ __forceinline__ void transpose8x8(const uint4 in[8], uint4 out[8])
{
    const uint32_t *w = reinterpret_cast<const uint32_t *>(in);  // w[4 v + c / 2]
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t sel = (c & 1) ? 0x7632u : 0x5410u;
        uint32_t o[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) o[p] = __byte_perm(w[4 * (2 * p) + c / 2], w[4 * (2 * p + 1) + c / 2], sel);
        out[c] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

// Decodes voxel m (x fastest) of the NDHWC grid.
__device__ __forceinline__ void decode_voxel(const ConvShape &S, long long m, int &n, int &z, int &y, int &x)
{
    long long u = m;
    x = (int)(u % S.w);
    u /= S.w;
    y = (int)(u % S.h);
    u /= S.h;
    z = (int)(u % S.d);
    n = (int)(u / S.d);
}

// WGRAD operands (K = voxels, both stored channels-last): each 8 x 8 block of
// (8 rows = channels) x (8 voxels) is read as eight 16-byte channel vectors,
// one per voxel, and transposed in registers into the K-major tile.
//   A: rows (tap, ci) = q0 + r, value x[voxel + offset(tap)][ci];
//   B: rows co = n0 + r,        value dy[voxel][co].
// Channel counts must be multiples of 8 (the caller checks).
template <bool IS_A, int ROWS>
__device__ __forceinline__ void load_kvoxel_blocks(const __nv_bfloat16 *__restrict__ src, const ConvShape &S,
                                                   long long row0, long long k0, uint8_t *tile)
{
    constexpr int NBLK = (ROWS / 8) * 8;  // (row groups) x (8 voxel groups of the 64-voxel chunk)
    const int ch = IS_A ? S.cin : S.cout;
    for (int b = threadIdx.x; b < NBLK; b += THREADS) {
        const int rg = b >> 3, vg = b & 7;
        const long long q = row0 + 8 * rg;  // first row of the group
        int tap = 0, c0 = 0;
        bool rows_ok;
        if (IS_A) {
            rows_ok = q < 27LL * ch;
            tap = rows_ok ? (int)(q / ch) : 0;
            c0 = rows_ok ? (int)(q - (long long)tap * ch) : 0;
        } else {
            rows_ok = q < ch;
            c0 = (int)q;
        }
        const int dz = tap / 9 - 1, dyy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        uint4 in[8];
        // the group's eight voxels are consecutive: decode the first, then step
        const long long mg = k0 + 8 * vg;
        int n = 0, z = 0, y = 0, x = 0;
        if (mg < S.k_total) decode_voxel(S, mg, n, z, y, x);
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            in[t] = make_uint4(0u, 0u, 0u, 0u);
            if (rows_ok && mg + t < S.k_total) {
                const int zz = IS_A ? z + dz : z, yy = IS_A ? y + dyy : y, xx = IS_A ? x + dx : x;
                if ((unsigned)zz < (unsigned)S.d && (unsigned)yy < (unsigned)S.h && (unsigned)xx < (unsigned)S.w)
                    in[t] = __ldg(reinterpret_cast<const uint4 *>(
                        src + ((((long long)n * S.d + zz) * S.h + yy) * S.w + xx) * ch + c0));
            }
            if (++x == S.w) {  // next voxel in x-fastest order
                x = 0;
                if (++y == S.h) {
                    y = 0;
                    if (++z == S.d) {
                        z = 0;
                        ++n;
                    }
                }
            }
        }
        uint4 out[8];
        transpose8x8(in, out);
#pragma unroll
        for (int c = 0; c < 8; ++c) *reinterpret_cast<uint4 *>(tile + swz(8 * rg + c, vg)) = out[c];
    }
}

// ------------------------------- the kernel --------------------------------

template <int OP, int BN>
__global__ void __launch_bounds__(THREADS) conv_tc_kernel(const __nv_bfloat16 *__restrict__ a_src,
                                                          const __nv_bfloat16 *__restrict__ b_src,
                                                          const float *__restrict__ bias, void *__restrict__ out,
                                                          int out_bf16, ConvShape S, int *__restrict__ status)
{
    constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128;
    constexpr int TMEM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : 128);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;                         // STAGES x A_BYTES
    uint8_t *sB = smem + STAGES * A_BYTES;      // STAGES x B_BYTES
    __shared__ uint64_t bars[STAGES];
    __shared__ uint32_t tmem_base_s;
    __shared__ int failed_s;

    const int warp = threadIdx.x >> 5;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    long long k_begin = 0, k_end = S.k_total;
    if (OP == OP_WGRAD) {
        k_begin = (long long)blockIdx.z * S.k_per_cta;
        k_end = k_begin + S.k_per_cta < S.k_total ? k_begin + S.k_per_cta : S.k_total;
    }
    const int nk = (int)((k_end - k_begin + BK - 1) / BK);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed_s = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base_s;
    constexpr uint32_t ID = idesc(BN);

    int4 rc = make_int4(-1, 0, 0, 0);  // FWD: this thread's output voxel (n, z, y, x)
    if (OP == OP_FWD) {
        const long long m = m0 + threadIdx.x;
        if (m < S.m_total) {
            long long t = m;
            rc.w = (int)(t % S.w);
            t /= S.w;
            rc.z = (int)(t % S.h);
            t /= S.h;
            rc.y = (int)(t % S.d);
            rc.x = (int)(t / S.d);
        }
    }
    bool ok = true;
    int committed = -1;
    for (int c = 0; c < nk; ++c) {
        const int s = c % STAGES;
        if (c >= STAGES) {
            // the MMAs that read this stage two chunks ago must be done
            if (!mbar_wait(&bars[s], (unsigned)((c / STAGES - 1) & 1))) ok = false;
        }
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        const long long k0 = k_begin + (long long)c * BK;
        if (OP == OP_FWD) {
            load_im2col_rows(a_src, S, rc, k0, sA + s * A_BYTES);
            load_rows_kmajor<BN>(b_src, S.k_total, S.n_total, n0, k0, sB + s * B_BYTES);
        } else {
            load_kvoxel_blocks<true, BM>(a_src, S, m0, k0, sA + s * A_BYTES);
            load_kvoxel_blocks<false, BN>(b_src, S, n0, k0, sB + s * B_BYTES);
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_after_sync();
            const uint32_t a_base = smem_addr(sA + s * A_BYTES), b_base = smem_addr(sB + s * B_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                umma_bf16(tmem, sdesc(a_base + 32 * kk), sdesc(b_base + 32 * kk), ID, c > 0 || kk > 0);
            umma_commit(&bars[s]);
        }
        committed = c;
    }
    if (ok && nk > 0) {
        const int last = nk - 1;
        if (!mbar_wait(&bars[last % STAGES], (unsigned)((last / STAGES) & 1))) ok = false;
    }
    ok = __syncthreads_and(ok);
    tc_after_sync();
    if (ok && nk > 0) {
        // epilogue: thread (warp w, lane l) owns accumulator row 32 w + l
        const long long row = m0 + threadIdx.x;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(lane_addr + (uint32_t)c0, v);
            if (row >= S.m_total) continue;
            if (OP == OP_FWD) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int co = n0 + c0 + i;
                    if (co >= S.n_total) continue;
                    float y = v[i] + (bias ? bias[co] : 0.0f);
                    if (S.relu) y = fmaxf(y, 0.0f);
                    const long long o = row * S.n_total + co;
                    if (out_bf16)
                        static_cast<__nv_bfloat16 *>(out)[o] = __float2bfloat16_rn(y);
                    else
                        static_cast<float *>(out)[o] = y;
                }
            } else {
                // row = (tap, ci); dw[co][(tap, ci)] += partial
                const long long q = row;
                const long long kq = 27LL * S.cin;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int co = n0 + c0 + i;
                    if (co < S.cout && q < kq) atomicAdd(static_cast<float *>(out) + co * kq + q, v[i]);
                }
            }
        }
    } else if (nk > 0) {
        // a wait expired: record it, and give the MMAs already committed a
        // bounded chance to finish before the tensor memory is released
        if (threadIdx.x == 0) {
            atomicExch(status, 1);
            if (committed >= 0) mbar_wait(&bars[committed % STAGES], (unsigned)((committed / STAGES) & 1));
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// FWD with channel counts that are multiples of 8: the A (im2col) and B
// (weight) chunks arrive by asynchronous copies, ST stages deep, so the
// gathers of ST - 1 chunks are in flight while the tensor cores work.  Stage
// s is refilled only after the MMAs that read it (committed to bars[s]) are
// done.
template <int BN, int ST>
__global__ void __launch_bounds__(THREADS) conv_fwd_async_kernel(const __nv_bfloat16 *__restrict__ x,
                                                                 const __nv_bfloat16 *__restrict__ w,
                                                                 const float *__restrict__ bias, void *__restrict__ out,
                                                                 int out_bf16, ConvShape S, int *__restrict__ status)
{
    constexpr int A_BYTES = BM * 128, B_BYTES = BN * 128;
    constexpr int TMEM_COLS = BN <= 32 ? 32 : (BN <= 64 ? 64 : 128);
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *sA = smem;                 // ST x A_BYTES
    uint8_t *sB = smem + ST * A_BYTES;  // ST x B_BYTES
    __shared__ uint64_t bars[ST];
    __shared__ uint32_t tmem_base_s;

    const int warp = threadIdx.x >> 5;
    const long long m0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    const int nk = (int)((S.k_total + BK - 1) / BK);
    if (threadIdx.x == 0) {
        for (int i = 0; i < ST; ++i) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base_s;
    constexpr uint32_t ID = idesc(BN);
    int4 rc = make_int4(-1, 0, 0, 0);  // this thread's output voxel (n, z, y, x)
    {
        const long long m = m0 + threadIdx.x;
        if (m < S.m_total) {
            long long t = m;
            rc.w = (int)(t % S.w);
            t /= S.w;
            rc.z = (int)(t % S.h);
            t /= S.h;
            rc.y = (int)(t % S.d);
            rc.x = (int)(t / S.d);
        }
    }
    auto issue = [&](int c) {
        const int st = c % ST;
        load_im2col_rows_async(x, S, rc, (long long)c * BK, sA + st * A_BYTES);
        load_rows_kmajor_async<BN>(w, S.k_total, S.n_total, n0, (long long)c * BK, sB + st * B_BYTES);
    };
    // prologue: chunks 0 .. ST-2 in flight (one commit group each, empty past the end)
#pragma unroll
    for (int c = 0; c < ST - 1; ++c) {
        if (c < nk) issue(c);
        cp_async_commit();
    }
    bool ok = true;
    int committed = -1;
    for (int c = 0; c < nk; ++c) {
        const int st = c % ST;
        cp_async_wait<ST - 2>();  // this thread's copies of chunk c have landed
        fence_async_smem();
        tc_before_sync();
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (threadIdx.x == 0) {
            tc_after_sync();
            const uint32_t a_base = smem_addr(sA + st * A_BYTES), b_base = smem_addr(sB + st * B_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                umma_bf16(tmem, sdesc(a_base + 32 * kk), sdesc(b_base + 32 * kk), ID, c > 0 || kk > 0);
            umma_commit(&bars[st]);
        }
        committed = c;
        // refill the stage chunk c - 1 used with chunk c + ST - 1
        const int c2 = c + ST - 1;
        if (c2 < nk) {
            if (c2 >= ST && !mbar_wait(&bars[c2 % ST], (unsigned)((c2 / ST - 1) & 1))) ok = false;
            if (ok) issue(c2);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (ok && nk > 0) {
        const int last = nk - 1;
        if (!mbar_wait(&bars[last % ST], (unsigned)((last / ST) & 1))) ok = false;
    }
    ok = __syncthreads_and(ok);
    tc_after_sync();
    if (ok && nk > 0) {
        // epilogue: thread (warp w, lane l) owns accumulator row 32 w + l
        const long long row = m0 + threadIdx.x;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tmem_ld16(lane_addr + (uint32_t)c0, v);
            if (row >= S.m_total || n0 + c0 >= S.n_total) continue;
            store16_fwd(v, bias, out, out_bf16, S, row, n0 + c0);
        }
    } else if (nk > 0) {
        if (threadIdx.x == 0) {
            atomicExch(status, 1);
            if (committed >= 0) mbar_wait(&bars[committed % ST], (unsigned)((committed / ST) & 1));
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// FWD with the input staged once per tile as a "brick" (channel counts that
// are multiples of 16).  The output tile is 16 rows (y) x 8 NT voxels (x) of
// one (n, z) plane; NT accumulators of 128 rows (8 x 16) sit side by side in
// TMEM.  A pipeline step stages, for 16 input channels and one of the three
// input planes z - 1, z, z + 1 (dz), the plane's (8 NT + 2) x 18 window of
// the input (zero outside the volume) in the non-swizzled K-major layout --
// position p of channel block b at b * NP * 16 + p * 16 bytes -- and the nine
// taps' weights of that plane and channel range.  The A operand of tap
// (dy, dx) for accumulator t is then the brick itself, shifted by
// dy * RW + dx + 8 t positions: MMA row m = 8 g + i reads position
// (g + dy) * RW + 8 t + i + dx, so the 8-row groups are RW positions apart
// (SBO) and the two 8-channel halves of K one block apart (LBO).  Each input
// element is copied into shared memory about (RW * 18 * 3) / (128 NT) times
// instead of 27 times as in the im2col form.
template <int BN, int NT, int ST>
__global__ void __launch_bounds__(THREADS) conv_fwd_brick_kernel(const __nv_bfloat16 *__restrict__ x,
                                                                 const __nv_bfloat16 *__restrict__ w,
                                                                 const float *__restrict__ bias, void *__restrict__ out,
                                                                 int out_bf16, ConvShape S, int *__restrict__ status)
{
    constexpr int RW = 8 * NT + 2;                // brick row length (positions)
    constexpr int NP = RW * 18;                   // positions of one plane's window
    constexpr int A_BYTES = NP * 32;              // two 8-channel blocks
    constexpr int B_BYTES = 9 * 2 * BN * 16;      // nine taps x two 8-channel blocks x BN rows
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    constexpr int ACC = NT * BN;
    constexpr int TMEM_COLS = ACC <= 32 ? 32 : (ACC <= 64 ? 64 : (ACC <= 128 ? 128 : 256));
    static_assert(ACC <= 256, "accumulator columns");
    static_assert(A_BYTES % 16 == 0 && B_BYTES % 16 == 0, "16-byte stage layout");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t bars[ST];
    __shared__ uint32_t tmem_base_s;

    const int warp = threadIdx.x >> 5;
    // tile -> (n, z, y0, x0)
    const int tiles_x = (S.w + 8 * NT - 1) / (8 * NT), tiles_y = (S.h + 15) / 16;
    long long t = blockIdx.x;
    const int tx = (int)(t % tiles_x);
    t /= tiles_x;
    const int ty = (int)(t % tiles_y);
    t /= tiles_y;
    const int z = (int)(t % S.d), nb = (int)(t / S.d);
    const int x0 = tx * 8 * NT, y0 = ty * 16;
    const int n0 = blockIdx.y * BN;
    const int cin = S.cin;
    const long long wrow = 27LL * cin;
    const int nk = 3 * (cin >> 4);
    if (threadIdx.x == 0) {
        for (int i = 0; i < ST; ++i) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base_s;
    constexpr uint32_t ID = idesc(BN);
    // step s: channels 16 (s / 3) .. + 16 of input plane z + s % 3 - 1
    auto issue = [&](int s) {
        uint8_t *sA = smem + (s % ST) * STAGE_BYTES, *sB = sA + A_BYTES;
        const int c16 = (s / 3) << 4, dz = s % 3;
        const int zz = z + dz - 1;
        const bool zin = (unsigned)zz < (unsigned)S.d;
        const __nv_bfloat16 *plane = x + ((long long)nb * S.d + zz) * S.h * S.w * cin + c16;
        for (int i = threadIdx.x; i < 2 * NP; i += THREADS) {
            const int b = i >= NP, p = i - b * NP;
            const int py = p / RW, px = p - py * RW;
            const int yy = y0 + py - 1, xx = x0 + px - 1;
            const bool in = zin && (unsigned)yy < (unsigned)S.h && (unsigned)xx < (unsigned)S.w;
            cp_async16(sA + i * 16, in ? plane + ((long long)yy * S.w + xx) * cin + 8 * b : x, in ? 16 : 0);
        }
        for (int i = threadIdx.x; i < 18 * BN; i += THREADS) {
            const int r = i % BN, jb = i / BN;  // jb = 2 * tap-in-plane + channel block
            const int co = n0 + r;
            const bool in = co < S.n_total;
            const __nv_bfloat16 *src = w + co * wrow + (long long)(9 * dz + (jb >> 1)) * cin + c16 + 8 * (jb & 1);
            cp_async16(sB + i * 16, in ? src : w, in ? 16 : 0);
        }
    };
#pragma unroll
    for (int c = 0; c < ST - 1; ++c) {
        if (c < nk) issue(c);
        cp_async_commit();
    }
    bool ok = true;
    int committed = -1;
    for (int c = 0; c < nk; ++c) {
        const int st = c % ST;
        cp_async_wait<ST - 2>();
        fence_async_smem();
        tc_before_sync();
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (threadIdx.x == 0) {
            tc_after_sync();
            const uint32_t a_base = smem_addr(smem + st * STAGE_BYTES), b_base = a_base + A_BYTES;
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const int dy = j / 3, dx = j - 3 * (j / 3);
                const uint64_t bd = sdesc_none(b_base + (uint32_t)(j * 2 * BN * 16), (uint32_t)(BN * 16), 128u);
#pragma unroll
                for (int q = 0; q < NT; ++q) {
                    const uint64_t ad =
                        sdesc_none(a_base + (uint32_t)((dy * RW + dx + 8 * q) * 16), (uint32_t)(NP * 16), (uint32_t)(RW * 16));
                    umma_bf16(tmem + (uint32_t)(q * BN), ad, bd, ID, c > 0 || j > 0);
                }
            }
            umma_commit(&bars[st]);
        }
        committed = c;
        const int c2 = c + ST - 1;
        if (c2 < nk) {
            if (c2 >= ST && !mbar_wait(&bars[c2 % ST], (unsigned)((c2 / ST - 1) & 1))) ok = false;
            if (ok) issue(c2);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (ok && nk > 0) {
        const int last = nk - 1;
        if (!mbar_wait(&bars[last % ST], (unsigned)((last / ST) & 1))) ok = false;
    }
    ok = __syncthreads_and(ok);
    tc_after_sync();
    if (ok && nk > 0) {
        // thread (warp w, lane l) owns accumulator row m = 32 w + l of every
        // accumulator: voxel (y0 + m / 8, x0 + 8 q + m % 8)
        const int m = threadIdx.x;
        const int y = y0 + (m >> 3);
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int q = 0; q < NT; ++q) {
            const int xo = x0 + 8 * q + (m & 7);
            const bool in = y < S.h && xo < S.w;
            const long long row = (((long long)nb * S.d + z) * S.h + y) * S.w + xo;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(lane_addr + (uint32_t)(q * BN + c0), v);
                if (!in || n0 + c0 >= S.n_total) continue;
                store16_fwd(v, bias, out, out_bf16, S, row, n0 + c0);
            }
        }
    } else if (nk > 0) {
        if (threadIdx.x == 0) {
            atomicExch(status, 1);
            if (committed >= 0) mbar_wait(&bars[committed % ST], (unsigned)((committed / ST) & 1));
        }
    }
    tc_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Brick-staged FWD launch: 4 stages for narrow N tiles, 3 for wide ones
// (shared memory per stage grows with BN).
template <int BN, int NT>
cudaError_t launch_brick(const __nv_bfloat16 *x, const __nv_bfloat16 *w, const float *bias, void *out, int out_bf16,
                         const ConvShape &S, int *status, cudaStream_t stream)
{
    constexpr int ST = BN <= 32 ? 4 : 3;
    constexpr int RW = 8 * NT + 2, NP = RW * 18;
    const int smem = ST * (NP * 32 + 9 * 2 * BN * 16) + 1024;
    cudaError_t e = cudaFuncSetAttribute(conv_fwd_brick_kernel<BN, NT, ST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)S.nb * S.d * ((S.h + 15) / 16) * ((S.w + 8 * NT - 1) / (8 * NT));
    if (tiles > 0x7FFFFFFFLL) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)tiles, (unsigned)((S.n_total + BN - 1) / BN), 1);
    conv_fwd_brick_kernel<BN, NT, ST><<<grid, THREADS, smem, stream>>>(x, w, bias, out, out_bf16, S, status);
    return cudaGetLastError();
}

template <int OP, int BN>
cudaError_t launch_bn(const __nv_bfloat16 *a, const __nv_bfloat16 *b, const float *bias, void *out, int out_bf16,
                      const ConvShape &S, int *status, cudaStream_t stream)
{
    if (OP == OP_FWD && (S.cin & 15) == 0 && CTREX_CONV_BRICK) {
        // tiles 16 x 16 (NT = 2) unless the volume is at most 8 wide
        if (S.w > 8) return launch_brick<BN, 2>(a, b, bias, out, out_bf16, S, status, stream);
        return launch_brick<BN, 1>(a, b, bias, out, out_bf16, S, status, stream);
    }
    if (OP == OP_FWD && (S.cin & 7) == 0) {
        // 2 stages for tiles up to 64 wide (more CTAs per SM beat a deeper
        // prefetch there), 3 for wider ones: measured on the U-Net's layers
        constexpr int ST = BN <= 64 ? 2 : 3;
        const int smem = ST * (BM * 128 + BN * 128) + 1024;
        cudaError_t e = cudaFuncSetAttribute(conv_fwd_async_kernel<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        const dim3 grid((unsigned)((S.m_total + BM - 1) / BM), (unsigned)((S.n_total + BN - 1) / BN), 1);
        conv_fwd_async_kernel<BN, ST><<<grid, THREADS, smem, stream>>>(a, b, bias, out, out_bf16, S, status);
        return cudaGetLastError();
    }
    const int smem = STAGES * (BM * 128 + BN * 128) + 1024;
    cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<OP, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((S.m_total + BM - 1) / BM), (unsigned)((S.n_total + BN - 1) / BN), 1);
    if (OP == OP_WGRAD) grid.z = (unsigned)((S.k_total + S.k_per_cta - 1) / S.k_per_cta);
    conv_tc_kernel<OP, BN><<<grid, THREADS, smem, stream>>>(a, b, bias, out, out_bf16, S, status);
    return cudaGetLastError();
}

template <int OP>
cudaError_t launch_op(int bn, const __nv_bfloat16 *a, const __nv_bfloat16 *b, const float *bias, void *out,
                      int out_bf16, const ConvShape &S, int *status, cudaStream_t stream)
{
    switch (bn) {
    case 16: return launch_bn<OP, 16>(a, b, bias, out, out_bf16, S, status, stream);
    case 32: return launch_bn<OP, 32>(a, b, bias, out, out_bf16, S, status, stream);
    case 48: return launch_bn<OP, 48>(a, b, bias, out, out_bf16, S, status, stream);
    case 64: return launch_bn<OP, 64>(a, b, bias, out, out_bf16, S, status, stream);
    case 96: return launch_bn<OP, 96>(a, b, bias, out, out_bf16, S, status, stream);
    default: return launch_bn<OP, 128>(a, b, bias, out, out_bf16, S, status, stream);
    }
}

// N tile: the smallest supported width covering n (multiples of 16), else 128.
int pick_bn(int n)
{
    const int opts[] = {16, 32, 48, 64, 96, 128};
    for (int o : opts)
        if (n <= o) return o;
    return 128;
}

bool shape_ok(int nb, int d, int h, int w, int cin, int cout)
{
    return nb >= 1 && d >= 1 && h >= 1 && w >= 1 && cin >= 1 && cout >= 1 && cin <= 4096 && cout <= 4096 &&
           (long long)nb * d * h * w <= (1LL << 40);
}

}  // namespace

extern "C" {

int ctrex_conv3d_fwd(const void *x, const void *w, const float *bias, void *y, int y_dtype, int nb, int d, int h,
                     int wd, int cin, int cout, int relu, int *status, void *stream)
{
    if (!x || !w || !y || !status) return CTREX_E_ARG;
    if (y_dtype != CTREX_F32 && y_dtype != CTREX_BF16) return CTREX_E_DTYPE;
    if (!shape_ok(nb, d, h, wd, cin, cout)) return CTREX_E_SHAPE;
    ConvShape S{};
    S.nb = nb;
    S.d = d;
    S.h = h;
    S.w = wd;
    S.cin = cin;
    S.cout = cout;
    S.relu = relu ? 1 : 0;
    S.m_total = (long long)nb * d * h * wd;
    S.n_total = cout;
    S.k_total = 27LL * cin;
    S.k_per_cta = S.k_total;
    const int bn = pick_bn(cout);
    cudaError_t e = launch_op<OP_FWD>(bn, static_cast<const __nv_bfloat16 *>(x), static_cast<const __nv_bfloat16 *>(w),
                                      bias, y, y_dtype == CTREX_BF16, S, status, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CTREX_OK : CTREX_E_CUDA;
}

int ctrex_conv3d_wgrad(const void *x, const void *dy, float *dw, int nb, int d, int h, int wd, int cin, int cout,
                       int *status, void *stream)
{
    if (!x || !dy || !dw || !status) return CTREX_E_ARG;
    if (!shape_ok(nb, d, h, wd, cin, cout) || (cin & 7) || (cout & 7)) return CTREX_E_SHAPE;
    ConvShape S{};
    S.nb = nb;
    S.d = d;
    S.h = h;
    S.w = wd;
    S.cin = cin;
    S.cout = cout;
    S.m_total = 27LL * cin;
    S.n_total = cout;
    S.k_total = (long long)nb * d * h * wd;
    // split K so that the grid fills the GPU about twice
    const long long mt = (S.m_total + BM - 1) / BM;
    long long splits = (2 * 152 + mt - 1) / mt;
    long long per = (S.k_total + splits - 1) / splits;
    per = ((per + BK - 1) / BK) * BK;
    if (per < BK) per = BK;
    S.k_per_cta = per;
    const int bn = pick_bn(cout);
    cudaError_t e = launch_op<OP_WGRAD>(bn, static_cast<const __nv_bfloat16 *>(x),
                                        static_cast<const __nv_bfloat16 *>(dy), nullptr, dw, 0, S, status,
                                        static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CTREX_OK : CTREX_E_CUDA;
}

}  // extern "C"

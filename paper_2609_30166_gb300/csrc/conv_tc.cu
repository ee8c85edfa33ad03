// conv_tc.cu -- 3x3x3 convolution (stride 1, zero "same" padding) as an
// implicit GEMM on the 5th-generation tensor cores (tcgen05, sm_103a), for
// the learned warm start (a 3D U-Net).  BF16 operands, FP32 accumulation in
// tensor memory (TMEM).  The paper has no such operator; it motivates learned
// components combined with the physics operators (Sec. 5).
//
// The tcgen05 kernels compute C[M][N] = sum_k A[M][k] B[N][k] with
// tcgen05.mma (kind::f16, M = 128, cta_group::1), accumulators in TMEM read
// back with tcgen05.ld for the epilogue.  Two families, and one more kernel:
//   * brick kernels (channel counts that are multiples of 16): TMA stages the
//     input window a tile's taps reach once ("brick") and every tap's operand
//     is the brick at a shifted descriptor start address, so no im2col is
//     formed; persistent and warp-specialised (a TMA producer warp, an MMA
//     warp, epilogue warps):
//       conv_fwd_tma_kernel     forward and input gradient,
//       conv_fwd_kx_kernel      the same for at most 16 output channels,
//                               kx taps folded into N, planes reused along z,
//       conv_wgrad_tma_kernel   weight gradient (MN-major operands, K = voxels);
//   * im2col kernels (other channel counts, and the fallback when no tensor
//     map can be made): the CTA's 128 threads gather implicit-im2col chunks
//     of 64 K elements into 128-byte-swizzled K-major tiles (16-byte cp.async
//     copies for multiples of 8 channels: conv_fwd_async_kernel; loads and
//     stores otherwise: conv_tc_kernel), one thread issues four MMAs per
//     chunk;
//   * conv_wgrad_c16_kernel: the weight gradient of layers with 16 output
//     channels on mma.sync (m16n8k16, M = the 16 output channels, no padded
//     rows; tcgen05 has no M below 64).
// Operand layouts:
//   FWD   A = im2col(x)[m][(tap, ci)], B = w[co][(tap, ci)], C -> y[m][co]
//         (+ bias, optional ReLU);  m runs over N*D*H*W output voxels (NDHWC).
//   DGRAD the same with dy as input and the flipped, transposed weights
//         w'[ci][(tap, co)] (prepared by the caller): dx = conv(dy, w').
//   WGRAD dw[co][(tap, ci)] = sum over voxels of dy[m][co] x[m + off(tap)][ci]
//         (FP32, partial sums added with atomics).
// Every wait on an mbarrier is bounded; on expiry the kernel records an error
// in the status word, drains what it issued (bounded), releases its TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ctrex.h"

namespace {

#ifndef CTREX_CONV_TMA
#define CTREX_CONV_TMA 1
#endif
#ifndef CTREX_CONV_FILL
#define CTREX_CONV_FILL 1
#endif
// Layers of at most 16 output channels through conv_fwd_kx_kernel (1), its
// input windows 32-byte swizzled with 16 channels per TMA box (1) or two
// 8-channel blocks (0).
#ifndef CTREX_CONV_KX
#define CTREX_CONV_KX 1
#endif
#ifndef CTREX_CONV_KX_SW32
#define CTREX_CONV_KX_SW32 1
#endif
#ifndef CTREX_CONV_WG_CHUNK
#define CTREX_CONV_WG_CHUNK 32
#endif



constexpr int BM = 128;
constexpr int BK = 64;
constexpr int STAGES = 2;
constexpr int THREADS = 128;
constexpr long long WAIT_LIMIT = 1LL << 26;
// Polls of the epilogue's accumulator waits in the persistent kernels.  The
// default is WAIT_LIMIT; a build with a tiny value makes those waits expire
// on purpose, which is how the abort and drain path is tested (every other
// wait keeps WAIT_LIMIT).
#ifndef CTREX_CONV_EPI_WAIT_LIMIT
#define CTREX_CONV_EPI_WAIT_LIMIT (1LL << 26)
#endif
constexpr long long EPI_WAIT_LIMIT = CTREX_CONV_EPI_WAIT_LIMIT;

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

// Shared-memory matrix descriptor, K-major with 32-byte swizzle: rows of 32
// bytes (K = 16 BF16), 8-row atoms of 256 bytes whose two 16-byte chunks
// are exchanged in rows 4..7 (address bit 4 ^= bit 7, as the TMA writes a
// box with CU_TENSOR_MAP_SWIZZLE_32B); sbo = byte stride between 8-row
// groups; the start address must sit on an atom (256-byte) boundary.
__device__ __forceinline__ uint64_t sdesc_sw32(uint32_t saddr, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)6 << 61;
    return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major,
// N = n, M = m (64 or 128).
__host__ __device__ constexpr uint32_t idesc(int n, int m = BM)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
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

// Columns [0, 48) of this thread's TMEM lane at ta and [0, 32) at tb (80
// FP32 values): five 16-column loads, one wait.
__device__ __forceinline__ void tmem_ld48_32(uint32_t ta, uint32_t tb, float a[48], float b[32])
{
    uint32_t r[80];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%80];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%81];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%82];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%83];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%64,%65,%66,%67,%68,%69,%70,%71,%72,%73,%74,%75,%76,%77,%78,%79}, [%84];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63]),
          "=r"(r[64]), "=r"(r[65]), "=r"(r[66]), "=r"(r[67]), "=r"(r[68]), "=r"(r[69]), "=r"(r[70]), "=r"(r[71]),
          "=r"(r[72]), "=r"(r[73]), "=r"(r[74]), "=r"(r[75]), "=r"(r[76]), "=r"(r[77]), "=r"(r[78]), "=r"(r[79])
        : "r"(ta), "r"(ta + 16u), "r"(ta + 32u), "r"(tb), "r"(tb + 16u)
        : "memory");
#pragma unroll
    for (int i = 0; i < 48; ++i) a[i] = __uint_as_float(r[i]);
#pragma unroll
    for (int i = 0; i < 32; ++i) b[i] = __uint_as_float(r[48 + i]);
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

// ---------------------------------------------------------------------------
// Persistent, warp-specialised FWD with the input staged as "bricks" by TMA
// (channel counts that are multiples of 16).
// Tiles: 16 rows (y) x 8 NT voxels (x) of one (n, z) plane; NT accumulators
// of 128 rows (8 x 16) sit side by side in TMEM.  A pipeline step stages, for
// 16 input channels and one of the three input planes z - 1, z, z + 1 (dz),
// the plane's (8 NT + 2) x 18 window (zero outside the volume) in the
// non-swizzled K-major layout -- position p of 8-channel block b at
// b * A_BLK + p * 16 bytes -- plus, unless the filter is resident, the nine
// taps' weights of that plane and channel range.  The A operand of tap
// (dy, dx) for accumulator t is the window itself, shifted by
// dy * RW + dx + 8 t positions: MMA row m = 8 g + i reads position
// (g + dy) * RW + 8 t + i + dx, so the 8-row groups are RW positions apart
// (SBO) and the two 8-channel halves of K one block apart (LBO).  Each input
// element is copied into shared memory about (RW * 18 * 3) / (128 NT) times
// instead of 27 times as in the im2col form.  Roles:
//   * warp 0 streams the steps of all the CTA's tiles through an ST-deep
//     ring with cp.async.bulk.tensor: per step two 5D boxes of the input
//     (8 channels x RW x 18 positions of one plane; the tensor map zero-fills
//     the halo outside the volume, including planes outside the batch item)
//     and, unless resident, 18 2D boxes of the weights (8 channels x BN rows
//     per tap and channel block), completing on the stage's mbarrier;
//   * warp 1 issues the MMAs of each step and commits them to the stage's
//     "empty" barrier, and a tile's last commit to the accumulator's "full"
//     barrier; two accumulators alternate in TMEM, so the MMAs of tile i + 1
//     overlap the epilogue of tile i;
//   * four epilogue warps (2..5; warp w reads TMEM lanes 32 (w % 4) ..)
//     drain an accumulator, store it and release it.
// The producer and MMA loops run warp-wide with one elected lane issuing,
// so that descriptors and coordinates stay warp-uniform.  Every wait is
// bounded; on expiry a thread raises the shared abort flag, which ends the
// other roles' waits, and the CTA drains its own copies and MMAs (bounded)
// before it frees TMEM.
constexpr int TMA_THREADS = 192;

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// One lane of the warp (all lanes converged): 1 there, 0 elsewhere.
__device__ __forceinline__ uint32_t elect_one()
{
    uint32_t p;
    asm volatile("{\n .reg .pred e;\n elect.sync _|e, 0xffffffff;\n selp.u32 %0, 1, 0, e;\n}\n" : "=r"(p));
    return p;
}
// Variants issued only by the lane whose `leader` is nonzero, so that the
// surrounding loop stays warp-uniform.
__device__ __forceinline__ void expect_tx_p(uint32_t leader, uint64_t *bar, uint32_t bytes)
{
    asm volatile("{\n .reg .pred e;\n setp.ne.b32 e, %0, 0;\n @e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%1], %2;\n}\n" ::"r"(
                     leader),
                 "r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_5d_p(uint32_t leader, uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                              int c2, int c3, int c4, uint64_t *bar)
{
    asm volatile(
        "{\n .reg .pred e;\n setp.ne.b32 e, %0, 0;\n"
        " @e cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%1], [%2, {%3, %4, %5, "
        "%6, %7}], [%8];\n}\n" ::"r"(leader),
        "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_2d_p(uint32_t leader, uint32_t dst, const CUtensorMap *map, int c0, int c1,
                                              uint64_t *bar)
{
    asm volatile(
        "{\n .reg .pred e;\n setp.ne.b32 e, %0, 0;\n"
        " @e cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%1], [%2, {%3, %4}], "
        "[%5];\n}\n" ::"r"(leader),
        "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void umma_bf16_p(uint32_t leader, uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t id,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p, e;\n setp.ne.b32 p, %4, 0;\n setp.ne.b32 e, %5, 0;\n"
        " @e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(id), "r"(accumulate), "r"(leader));
}
__device__ __forceinline__ void umma_commit_p(uint32_t leader, uint64_t *bar)
{
    asm volatile(
        "{\n .reg .pred e;\n setp.ne.b32 e, %0, 0;\n"
        " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%1];\n}\n" ::"r"(leader),
        "r"(smem_addr(bar))
        : "memory");
}
// Warp-wide bounded wait (every lane returns the same answer); with an abort
// flag it also gives up once another role raised it, and raises it itself on
// expiry.  limit: polls before it gives up.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t *bar, unsigned parity, volatile int *abort_flag,
                                               long long limit = WAIT_LIMIT)
{
    for (long long i = 0; i < limit; ++i) {
        if (__any_sync(0xffffffffu, mbar_test(bar, parity))) return true;
        if (abort_flag && (i & 255) == 255 && __any_sync(0xffffffffu, *abort_flag != 0)) return false;
    }
    if (abort_flag) *abort_flag = 1;
    return false;
}

// Warp-wide bounded wait for two phases that are usually complete already:
// one poll of both with non-blocking tests (their latencies overlap: each
// poll costs some hundred cycles on a busy SM), then blocking waits for any
// that is not.
__device__ __forceinline__ bool mbar_wait2_warp(uint64_t *b1, unsigned p1, uint64_t *b2, unsigned p2,
                                                volatile int *abort_flag)
{
    uint32_t d1, d2;
    asm volatile(
        "{\n .reg .pred a, b;\n mbarrier.test_wait.parity.shared::cta.b64 a, [%2], %3;\n"
        " mbarrier.test_wait.parity.shared::cta.b64 b, [%4], %5;\n selp.u32 %0, 1, 0, a;\n selp.u32 %1, 1, 0, b;\n}\n"
        : "=r"(d1), "=r"(d2)
        : "r"(smem_addr(b1)), "r"(p1), "r"(smem_addr(b2)), "r"(p2)
        : "memory");
    const uint32_t dd = __reduce_or_sync(0xffffffffu, d1 | (d2 << 1));
    if (!(dd & 1u) && !mbar_wait_warp(b1, p1, abort_flag)) return false;
    if (!(dd & 2u) && !mbar_wait_warp(b2, p2, abort_flag)) return false;
    return true;
}

// Shared-memory plan of the TMA kernel (bytes; every TMA destination
// 128-byte aligned, every stage 1024-byte aligned).  RESW: the whole filter
// of the (single) N tile stays resident, loaded once per CTA (W_MAX bytes at
// most), and the ring carries only the input windows.
template <int BN, int NT, bool RESW>
struct TmaPlan {
    static constexpr int RW = 8 * NT + 2;
    static constexpr int NP = RW * 18;
    static constexpr int A_BLK = (NP * 16 + 127) / 128 * 128;  // one 8-channel block of the window
    static constexpr int B_BLK = BN * 16;                       // one tap's 8-channel block of BN rows
    static constexpr int W_MAX = 112 * 1024;                    // resident filter budget
    static constexpr int W_BYTES = RESW ? W_MAX : 0;
    static constexpr int STAGE = (2 * A_BLK + (RESW ? 0 : 18 * B_BLK) + 1023) / 1024 * 1024;
    static constexpr uint32_t TX = 2u * NP * 16 + (RESW ? 0u : 18u * B_BLK);  // bytes the TMA writes per step
    static constexpr int ACC = NT * BN;  // columns of one accumulator
    static constexpr int TMEM_COLS = 2 * ACC <= 32 ? 32 : (2 * ACC <= 64 ? 64 : (2 * ACC <= 128 ? 128 : (2 * ACC <= 256 ? 256 : 512)));
    static constexpr int RING = 200 * 1024 - W_BYTES;
    static constexpr int ST = RING / STAGE < 8 ? RING / STAGE : 8;
    static constexpr int SMEM = W_BYTES + ST * STAGE + 1024;
    static_assert(2 * ACC <= 512, "two accumulators must fit in TMEM");
    static_assert(ST >= 2, "at least two stages");
    static_assert(B_BLK % 128 == 0 && W_BYTES % 1024 == 0, "aligned weight boxes");
};

template <int BN, int NT, bool RESW>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    conv_fwd_tma_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw,
                        const float *__restrict__ bias, void *__restrict__ out, int out_bf16, ConvShape S,
                        int *__restrict__ status)
{
    using PL = TmaPlan<BN, NT, RESW>;
    constexpr int ST = PL::ST, RW = PL::RW;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *wres = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *smem = wres + PL::W_BYTES;  // the ring
    __shared__ uint64_t full[ST], empty[ST], acc_full[2], acc_empty[2], drain, wbar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_x = (S.w + 8 * NT - 1) / (8 * NT), tiles_y = (S.h + 15) / 16;
    const int n_tiles = (S.n_total + BN - 1) / BN;  // 1 with RESW
    const long long items = (long long)S.nb * S.d * tiles_y * tiles_x * n_tiles;
    const int nk = 3 * (S.cin >> 4);
    if (threadIdx.x == 0) {
        for (int i = 0; i < ST; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 128);
        }
        mbar_init(&drain, 1);
        mbar_init(&wbar, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmw)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                     "r"(PL::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base_s;
    volatile int *abort_flag = &abort_s;
    // item -> (n, z, y0, x0, n0)
    auto decode = [&](long long it, int &nb, int &z, int &y0, int &x0, int &n0) {
        const int nt = (int)(it % n_tiles);
        long long t = it / n_tiles;
        const int tx = (int)(t % tiles_x);
        t /= tiles_x;
        const int ty = (int)(t % tiles_y);
        t /= tiles_y;
        z = (int)(t % S.d);
        nb = (int)(t / S.d);
        x0 = tx * 8 * NT;
        y0 = ty * 16;
        n0 = nt * BN;
    };

    long long fills = 0;  // producer: copies issued (stage fills)
    bool mmas = false;    // MMA warp: any MMA issued
    if (warp == 0) {
        // producer warp: the loop runs warp-wide (uniform descriptors and
        // coordinates); one elected lane issues each copy
        const uint32_t leader = elect_one();
        long long fill = 0;
        bool ok = true;
        if (RESW) {
            // the whole filter: block (tap t, channel block kb) of BN rows at
            // (t * cin / 8 + kb) * B_BLK
            const int kbs = S.cin >> 3;
            expect_tx_p(leader, &wbar, (uint32_t)(27 * kbs * PL::B_BLK));
            const uint32_t wb = smem_addr(wres);
            for (int t = 0; t < 27; ++t)
                for (int kb = 0; kb < kbs; ++kb)
                    tma_load_2d_p(leader, wb + (uint32_t)((t * kbs + kb) * PL::B_BLK), &tmw, t * S.cin + 8 * kb, 0,
                                  &wbar);
        }
        for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
            int nb, z, y0, x0, n0;
            decode(it, nb, z, y0, x0, n0);
            for (int s = 0; s < nk; ++s, ++fill) {
                const int st = (int)(fill % ST);
                if (fill >= ST && !mbar_wait_warp(&empty[st], (unsigned)(((fill / ST) - 1) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                const int c16 = (s / 3) << 4, dz = s % 3;
                const uint32_t a = smem_addr(smem + st * PL::STAGE), b = a + 2 * PL::A_BLK;
                expect_tx_p(leader, &full[st], PL::TX);
                tma_load_5d_p(leader, a, &tmx, c16, x0 - 1, y0 - 1, z + dz - 1, nb, &full[st]);
                tma_load_5d_p(leader, a + PL::A_BLK, &tmx, c16 + 8, x0 - 1, y0 - 1, z + dz - 1, nb, &full[st]);
                if (!RESW) {
#pragma unroll
                    for (int j = 0; j < 9; ++j)
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            tma_load_2d_p(leader, b + (uint32_t)((2 * j + h) * PL::B_BLK), &tmw,
                                          (9 * dz + j) * S.cin + c16 + 8 * h, n0, &full[st]);
                }
            }
        }
        if (!ok && lane == 0) atomicExch(status, 1);
        fills = fill;
    } else if (warp == 1) {
        // MMA warp: the loop runs warp-wide; one elected lane issues the MMAs
        // and commits
        const uint32_t leader = elect_one();
        constexpr uint32_t ID = idesc(BN);
        long long fill = 0;
        int tile_i = 0;
        bool ok = !RESW || mbar_wait_warp(&wbar, 0u, abort_flag), issued = false;
        const int kbs = S.cin >> 3;
        for (long long it = blockIdx.x; it < items && ok; it += gridDim.x, ++tile_i) {
            const int acc = tile_i & 1;
            if (tile_i >= 2 && !mbar_wait_warp(&acc_empty[acc], (unsigned)(((tile_i >> 1) - 1) & 1), abort_flag)) {
                ok = false;
                break;
            }
            tc_after_sync();
            const uint32_t d = tmem + (uint32_t)(acc * PL::ACC);
            for (int s = 0; s < nk; ++s, ++fill) {
                const int st = (int)(fill % ST);
                if (!mbar_wait_warp(&full[st], (unsigned)((fill / ST) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc_after_sync();
                const uint32_t a_base = smem_addr(smem + st * PL::STAGE);
                // weights of tap (dz, j), channel blocks 2c and 2c + 1
                const uint32_t b_base = RESW ? smem_addr(wres) + (uint32_t)((9 * (s % 3) * kbs + 2 * (s / 3)) * PL::B_BLK)
                                             : a_base + 2 * PL::A_BLK;
                const uint32_t b_tap = RESW ? (uint32_t)(kbs * PL::B_BLK) : (uint32_t)(2 * PL::B_BLK);
                // descriptors are affine in the start address (16-byte units in
                // the low field, far from overflowing it): one base per operand,
                // a constant offset per tap
                const uint64_t a0 = sdesc_none(a_base, (uint32_t)PL::A_BLK, (uint32_t)(RW * 16));
                const uint64_t b0 = sdesc_none(b_base, (uint32_t)PL::B_BLK, 128u);
                const uint64_t b_step = b_tap >> 4;
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    const int dy = j / 3, dx = j - 3 * (j / 3);
                    const uint64_t bd = b0 + (uint64_t)j * b_step;
#pragma unroll
                    for (int q = 0; q < NT; ++q)
                        umma_bf16_p(leader, d + (uint32_t)(q * BN), a0 + (uint64_t)(dy * RW + dx + 8 * q), bd, ID,
                                    (s > 0 || j > 0) ? 1u : 0u);
                }
                umma_commit_p(leader, &empty[st]);
                issued = true;
            }
            if (ok) umma_commit_p(leader, &acc_full[acc]);
        }
        if (!ok && lane == 0) atomicExch(status, 1);
        mmas = issued;
    } else {
        // epilogue warps 2..5: accumulator rows 32 (warp % 4) + lane
        const int quarter = warp & 3;
        const int m = 32 * quarter + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
        int tile_i = 0;
        for (long long it = blockIdx.x; it < items; it += gridDim.x, ++tile_i) {
            const int acc = tile_i & 1;
            if (!mbar_wait_warp(&acc_full[acc], (unsigned)((tile_i >> 1) & 1), abort_flag, EPI_WAIT_LIMIT)) {
                if (lane == 0) atomicExch(status, 1);
                break;
            }
            tc_after_sync();
            int nb, z, y0, x0, n0;
            decode(it, nb, z, y0, x0, n0);
            const int y = y0 + (m >> 3);
#pragma unroll 1
            for (int q = 0; q < NT; ++q) {
                const int xo = x0 + 8 * q + (m & 7);
                const bool in = y < S.h && xo < S.w;
                const long long row = (((long long)nb * S.d + z) * S.h + y) * S.w + xo;
#pragma unroll 1
                for (int c0 = 0; c0 < BN; c0 += 16) {
                    float v[16];
                    tmem_ld16(lane_base + (uint32_t)(acc * PL::ACC + q * BN + c0), v);
                    if (!in || n0 + c0 >= S.n_total) continue;
                    store16_fwd(v, bias, out, out_bf16, S, row, n0 + c0);
                }
            }
            tc_before_sync();
            mbar_arrive(&acc_empty[acc]);
        }
    }
    tc_before_sync();
    __syncthreads();
    // Every role has left its loop, so the abort flag is final.  If a role
    // gave up, the others may have stopped waiting for work still in flight:
    // the producer waits for the last fill of every stage and the filter (the
    // earlier fills of a stage completed before it was refilled), and the MMA
    // warp for every MMA its elected lane issued, before the CTA releases
    // TMEM and its shared memory.  All these waits are bounded.
    if (*abort_flag) {
        if (warp == 0) {
            for (long long f = fills - 1; f >= 0 && f >= fills - ST; --f)
                mbar_wait_warp(&full[f % ST], (unsigned)((f / ST) & 1), nullptr);
            if (RESW) mbar_wait_warp(&wbar, 0u, nullptr);
        } else if (warp == 1 && mmas) {
            // elect.sync picks the same lane for the same member mask, so
            // this commit comes from the lane that issued the MMAs (the
            // leader is not carried out of the loop: keeping it live there
            // cost the issue loop about 40 %)
            umma_commit_p(elect_one(), &drain);
            mbar_wait_warp(&drain, 0u, nullptr);
        }
    }
    if (warp == 1) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PL::TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Forward (and input gradient) of layers with at most 16 output channels and
// a multiple of 16 input channels: the kx taps folded into N, input planes
// reused along z.
//   * N = 48 = (kx, co): one MMA of 128 x 48 x 16 multiplies 8 window columns
//     x 16 rows by the filter rows (kx, co) of one (kz, ky) and 16 input
//     channels, so that the accumulator holds, per window column c,
//     E_kx[c] = sum over kz, ky, ci of w[co][kz][ky][kx][ci] x[..., c][ci];
//     the epilogue forms y[i] = E_0[i] + E_1[i + 1] + E_2[i + 2] with warp
//     shuffles.  A tile of 8 NT output columns x 16 rows needs NG = NT + 1
//     column groups (8 NG >= 8 NT + 2): 9 NG MMAs per 16 input channels
//     instead of 27 NT.
//   * A CTA runs items of ZC consecutive output planes of one (n, y, x)
//     column.  The windows of the input planes z0 - 1 .. z0 + ZC stream
//     through a ring of P plane slots (a slot holds the cin / 16 windows of
//     one plane), so each plane is loaded once per item rather than once per
//     kz tap, and tile z reads the slots of planes z - 1, z and z + 1.  A
//     slot is released when the last tile that reads it has its MMAs done.
//   * The filter is resident: block (tap t, 8-channel block kb) of 16 rows
//     at ((t / 3) * cin / 8 + kb) * 3 + t % 3, so that the 48 rows (kx, co)
//     of one (kz, ky) and channel block are contiguous, 16 bytes apart.
//   * A window (16 channels of 18 rows x 8 NG columns, 6 more than the taps
//     reach) is one TMA box of 32-byte rows, 32-byte swizzled; every MMA's
//     A operand then starts on a 256-byte swizzle atom (columns come in
//     groups of 8, rows are 8 NG positions long).  The extra columns land
//     in accumulator lanes that the epilogue never uses.  (Without the
//     swizzle: two boxes of 8 channels, 16-byte rows.)
//   * The MMA warp polls once per tile: the plane that tile adds and the
//     release of its accumulator together (a poll costs a few hundred
//     cycles on the busy SM, and four of them took a quarter of the time).
// Measured on 128^3 x 2 (16 output channels): 16 -> 16 0.184 ms with the
// 27 NT scheme, 0.102 ms here; 32 -> 16 0.327 -> 0.176; 48 -> 16 0.474 ->
// 0.279.
template <int NT>
struct KxPlan {
    static constexpr bool SW = CTREX_CONV_KX_SW32;  // 32-byte swizzled windows
    static constexpr int NG = NT + 1;       // MMA column groups
    static constexpr int RW = 8 * NG;       // window columns loaded (8 NT + 2 used)
    static constexpr int NP = RW * 18;      // window positions
    static constexpr int NW = 48;           // MMA N
    static constexpr int A_BLK = NP * 16;   // one 8-channel block (a multiple of 128 bytes)
    static constexpr int WIN = 2 * A_BLK;   // one window of 16 channels
    static constexpr uint32_t WIN_TX = 2u * NP * 16;  // bytes the TMA writes per window
    static constexpr int B_BLK = 16 * 16;             // one tap's 8-channel block of 16 rows
    static constexpr int ACC = NG * NW;               // columns of one accumulator
    static constexpr int TMEM_COLS = 2 * ACC <= 128 ? 128 : (2 * ACC <= 256 ? 256 : 512);
    static_assert(2 * ACC <= 512, "two accumulators must fit in TMEM");
    static_assert(A_BLK % 128 == 0, "128-byte aligned window rows");
};

struct KxArgs {
    int cb;       // 16-channel blocks of the input (cin / 16)
    int zc;       // output planes per item
    int w_bytes;  // bytes reserved for the resident filter (multiple of 1024)
};

template <int NT, int P>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    conv_fwd_kx_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmw,
                       const float *__restrict__ bias, void *__restrict__ out, int out_bf16, ConvShape S, KxArgs G,
                       int *__restrict__ status)
{
    using PL = KxPlan<NT>;
    constexpr int RW = PL::RW;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *wres = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *ring = wres + G.w_bytes;
    __shared__ uint64_t full[P], empty[P], acc_full[2], acc_empty[2], drain, wbar;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int CB = G.cb, ZC = G.zc;
    const int tiles_x = (S.w + 8 * NT - 1) / (8 * NT), tiles_y = (S.h + 15) / 16, zchunks = (S.d + ZC - 1) / ZC;
    const long long items = (long long)S.nb * zchunks * tiles_y * tiles_x;
    const int kbs = S.cin >> 3;
    if (threadIdx.x == 0) {
        for (int i = 0; i < P; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 128);
        }
        mbar_init(&drain, 1);
        mbar_init(&wbar, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmw)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                     "r"(PL::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base_s;
    volatile int *abort_flag = &abort_s;
    // item -> (n, first output plane z0, planes nz, y0, x0); x fastest, so
    // that CTAs running at the same time read neighbouring windows
    auto decode = [&](long long it, int &nb, int &z0, int &nz, int &y0, int &x0) {
        const int tx = (int)(it % tiles_x);
        long long t = it / tiles_x;
        const int ty = (int)(t % tiles_y);
        t /= tiles_y;
        z0 = (int)(t % zchunks) * ZC;
        nb = (int)(t / zchunks);
        nz = S.d - z0 < ZC ? S.d - z0 : ZC;
        x0 = tx * 8 * NT;
        y0 = ty * 16;
    };

    long long fills = 0;  // producer: plane fills issued
    bool mmas = false;    // MMA warp: any MMA issued
    if (warp == 0) {
        // producer warp: warp-wide loop, one elected lane issues each copy
        const uint32_t leader = elect_one();
        long long fill = 0;
        bool ok = true;
        expect_tx_p(leader, &wbar, (uint32_t)(27 * kbs * PL::B_BLK));
        const uint32_t wb = smem_addr(wres);
        for (int t = 0; t < 27; ++t)
            for (int kb = 0; kb < kbs; ++kb)
                tma_load_2d_p(leader, wb + (uint32_t)((((t / 3) * kbs + kb) * 3 + t % 3) * PL::B_BLK), &tmw,
                              t * S.cin + 8 * kb, 0, &wbar);
        for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
            int nb, z0, nz, y0, x0;
            decode(it, nb, z0, nz, y0, x0);
            // planes z0 - 1 .. z0 + nz (outside the volume: zero-filled)
            for (int pz = z0 - 1; pz <= z0 + nz; ++pz, ++fill) {
                const int sl = (int)(fill % P);
                if (fill >= P && !mbar_wait_warp(&empty[sl], (unsigned)(((fill / P) - 1) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                const uint32_t base = smem_addr(ring) + (uint32_t)(sl * CB * PL::WIN);
                expect_tx_p(leader, &full[sl], (uint32_t)CB * PL::WIN_TX);
                for (int c = 0; c < CB; ++c) {
                    const uint32_t a = base + (uint32_t)(c * PL::WIN);
                    if (PL::SW) {
                        tma_load_5d_p(leader, a, &tmx, 16 * c, x0 - 1, y0 - 1, pz, nb, &full[sl]);
                    } else {
                        tma_load_5d_p(leader, a, &tmx, 16 * c, x0 - 1, y0 - 1, pz, nb, &full[sl]);
                        tma_load_5d_p(leader, a + PL::A_BLK, &tmx, 16 * c + 8, x0 - 1, y0 - 1, pz, nb, &full[sl]);
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicExch(status, 1);
        fills = fill;
    } else if (warp == 1) {
        // MMA warp: warp-wide loop, one elected lane issues the MMAs and
        // commits
        const uint32_t leader = elect_one();
        constexpr uint32_t ID = idesc(PL::NW);
        long long fill = 0;  // plane fill of the current item's first plane
        int tile_i = 0;
        bool ok = mbar_wait_warp(&wbar, 0u, abort_flag), issued = false;
        const uint32_t wb = smem_addr(wres), rb = smem_addr(ring);
        const uint64_t b_dy = (uint64_t)((3 * kbs * PL::B_BLK) >> 4);
        for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
            int nb, z0, nz, y0, x0;
            decode(it, nb, z0, nz, y0, x0);
            for (int k = 0; k < nz; ++k, ++tile_i) {
                const int acc = tile_i & 1;
                // planes z - 1, z, z + 1 of output plane z = z0 + k: the
                // first two were waited for by the item's earlier tiles
                // (they stay until released below), except at its start
                for (int dz = 0; k == 0 && dz < 2 && ok; ++dz) {
                    const long long f = fill + dz;
                    ok = mbar_wait_warp(&full[f % P], (unsigned)((f / P) & 1), abort_flag);
                }
                const long long f2 = fill + k + 2;
                if (ok && tile_i >= 2)
                    ok = mbar_wait2_warp(&acc_empty[acc], (unsigned)(((tile_i >> 1) - 1) & 1), &full[f2 % P],
                                         (unsigned)((f2 / P) & 1), abort_flag);
                else if (ok)
                    ok = mbar_wait_warp(&full[f2 % P], (unsigned)((f2 / P) & 1), abort_flag);
                if (!ok) break;
                tc_after_sync();
                const uint32_t d = tmem + (uint32_t)(acc * PL::ACC);
                for (int dz = 0; dz < 3; ++dz) {
                    const uint32_t slot = rb + (uint32_t)(((fill + k + dz) % P) * CB * PL::WIN);
                    for (int c = 0; c < CB; ++c) {
                        // A: the window, rows = 8 columns x 16 rows, 8-row
                        // groups one window row apart, channel blocks A_BLK
                        // apart; B: rows (kx, co) of (kz, ky) = (dz, dy),
                        // channel blocks 2c and 2c + 1, 3 B_BLK apart
                        const uint64_t a0 = PL::SW ? sdesc_sw32(slot + (uint32_t)(c * PL::WIN), (uint32_t)(RW * 32))
                                                   : sdesc_none(slot + (uint32_t)(c * PL::WIN), (uint32_t)PL::A_BLK,
                                                                (uint32_t)(RW * 16));
                        constexpr int AU = PL::SW ? 2 : 1;  // 16-byte units per window position
                        const uint64_t b0 = sdesc_none(wb + (uint32_t)((9 * dz * kbs + 6 * c) * PL::B_BLK),
                                                       (uint32_t)(3 * PL::B_BLK), 128u);
#pragma unroll
                        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                            for (int q = 0; q < PL::NG; ++q)
                                umma_bf16_p(leader, d + (uint32_t)(q * PL::NW), a0 + (uint64_t)(AU * (dy * RW + 8 * q)),
                                            b0 + (uint64_t)dy * b_dy, ID, (dz > 0 || c > 0 || dy > 0) ? 1u : 0u);
                    }
                }
                issued = true;
                // plane z - 1 is not read again
                umma_commit_p(leader, &empty[(fill + k) % P]);
                umma_commit_p(leader, &acc_full[acc]);
            }
            if (!ok) break;
            // the item's last two planes
            umma_commit_p(leader, &empty[(fill + nz) % P]);
            umma_commit_p(leader, &empty[(fill + nz + 1) % P]);
            fill += nz + 2;
        }
        if (!ok && lane == 0) atomicExch(status, 1);
        mmas = issued;
    } else {
        // epilogue warps 2..5: accumulator rows 32 (warp % 4) + lane, row
        // m = 8 (window row) + column within the group
        const int quarter = warp & 3;
        const int m = 32 * quarter + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
        // column i + 1 (i + 2) is the next lane of the same 8-lane group or,
        // past the group's end, one of the first lanes of group q + 1: each
        // lane offers the value that the lane asking for it needs
        const int cc = lane & 7;
        const int src1 = cc < 7 ? lane + 1 : lane - 7, src2 = cc < 6 ? lane + 2 : lane - 6;
        int tile_i = 0;
        bool ok = true;
        for (long long it = blockIdx.x; it < items && ok; it += gridDim.x) {
            int nb, z0, nz, y0, x0;
            decode(it, nb, z0, nz, y0, x0);
            for (int k = 0; k < nz; ++k, ++tile_i) {
                const int acc = tile_i & 1;
                if (!mbar_wait_warp(&acc_full[acc], (unsigned)((tile_i >> 1) & 1), abort_flag, EPI_WAIT_LIMIT)) {
                    if (lane == 0) atomicExch(status, 1);
                    ok = false;
                    break;
                }
                tc_after_sync();
                const int y = y0 + (m >> 3);
#pragma unroll 1
                for (int q = 0; q < NT; ++q) {
                    const int xo = x0 + 8 * q + cc;
                    // E_kx of group q (48 columns) and E_1, E_2 of group
                    // q + 1 (32 columns)
                    const uint32_t col = lane_base + (uint32_t)(acc * PL::ACC + q * PL::NW);
                    float e[48], en[32], v[16];
                    tmem_ld48_32(col, col + PL::NW + 16, e, en);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        v[i] = e[i] + __shfl_sync(0xffffffffu, cc == 0 ? en[i] : e[16 + i], src1) +
                               __shfl_sync(0xffffffffu, cc < 2 ? en[16 + i] : e[32 + i], src2);
                    if (y < S.h && xo < S.w)
                        store16_fwd(v, bias, out, out_bf16, S, (((long long)nb * S.d + z0 + k) * S.h + y) * S.w + xo,
                                    0);
                }
                tc_before_sync();
                mbar_arrive(&acc_empty[acc]);
            }
        }
    }
    tc_before_sync();
    __syncthreads();
    // as in conv_fwd_tma_kernel: once a role gave up, the producer waits for
    // the last fill of every slot and the filter, the MMA warp for its MMAs
    // (bounded waits), before TMEM and shared memory are released
    if (*abort_flag) {
        if (warp == 0) {
            for (long long f = fills - 1; f >= 0 && f >= fills - P; --f)
                mbar_wait_warp(&full[f % P], (unsigned)((f / P) & 1), nullptr);
            mbar_wait_warp(&wbar, 0u, nullptr);
        } else if (warp == 1 && mmas) {
            umma_commit_p(elect_one(), &drain);  // the lane that issued the MMAs (same member mask)
            mbar_wait_warp(&drain, 0u, nullptr);
        }
    }
    if (warp == 1) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PL::TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient with the brick scheme (cin a multiple of 16, cout of 8):
//   dW[co][tap][ci] = sum_p dy[p][co] x[p + off(tap)][ci].
// A job is (co tile of 128, ci chunk of CN, input plane offset dz); a CTA
// runs one job over a contiguous range of 16 x 16 position tiles and keeps
// the nine taps' D_tap[co][ci] (128 lanes x 9 CN columns) in TMEM across the
// whole range, adding them to dW (FP32 atomics) once at the end.
// Operands are MN-major (channels contiguous, K = voxels), non-swizzled: a
// core matrix is 8 voxels x 8 channels, 128 contiguous bytes; SBO = stride
// between 8-channel blocks, LBO = stride between 8-voxel groups (confirmed
// by an in-bounds descriptor probe).  Per tile and stage:
//   * dy rows as [row g][co block][16 voxels] x 16 B (one TMA box through a
//     map whose dimensions are (8 channels, x, co block, y, plane)); the MMA
//     of row g reads A = dy^T at g * CB * 256 with SBO 256, LBO 128: K = the
//     row's 16 voxels, M = 128 co, or 64 when cout <= 64 (rows past cout
//     read other rows' data and land in accumulator lanes that are never
//     stored; the region is padded so that they stay inside it);
//   * the input window of plane z + dz - 1 for the CN channels, three
//     times, shifted by kx = 0, 1, 2 voxels: copy kx holds rows y0 - 1 ..
//     y0 + 16 and columns x0 + kx - 1 .. + 15 as [kx][8-channel block][18
//     rows][16 voxels] x 16 B.  The blocks (kx, channel block) are then
//     equally spaced, so one MMA with N = 3 CN (SBO = the block stride,
//     LBO 128) takes the three kx taps of row ky at once: B starts at
//     row g + ky of every copy.
// 16 rows x 3 ky = 48 MMAs of 128 x 3 CN x 16 per tile; tap (ky, kx) lands
// in TMEM columns (3 ky + kx) CN .. + CN.
template <int CN>
struct WgPlan {
    static constexpr int COPY = 18 * 16 * 16;  // one 8-channel block of a window copy: 18 rows x 16 voxels x 16 B
    static constexpr int X_BYTES = 3 * (CN / 8) * COPY;
    static constexpr uint32_t X_TX = X_BYTES;  // the boxes fill the copies exactly
    static constexpr int NK = 3 * CN;           // N of one MMA: the three kx taps x CN channels
    static constexpr int TMEM_COLS = 9 * CN <= 256 ? 256 : 512;
    static_assert(9 * CN <= 512 && NK <= 256 && NK % 16 == 0, "TMEM columns and MMA shape");
};

struct WgArgs {
    int cb;          // 8-channel co blocks loaded per tile (min(16, cout / 8))
    int dy_region;   // bytes of the dy part of a stage (with the padding)
    int stage;       // bytes of a stage
    int st;          // ring depth (<= WG_MAX_ST)
    int splits;      // position-tile ranges per job (gridDim.x)
    long long tiles; // 16 x 16 position tiles
};
constexpr int WG_MAX_ST = 8;
constexpr long long WG_CHUNK = CTREX_CONV_WG_CHUNK;  // tiles per CTA at most (see the launcher)

template <int CN, bool M64>
__global__ void __launch_bounds__(TMA_THREADS, 1)
    conv_wgrad_tma_kernel(const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmdy,
                          float *__restrict__ dw, ConvShape S, WgArgs G, int *__restrict__ status)
{
    using PL = WgPlan<CN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full[WG_MAX_ST], empty[WG_MAX_ST], done, drain;
    __shared__ uint32_t tmem_base_s;
    __shared__ int abort_s;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ST = G.st;
    // job -> (co tile, ci chunk, dz); split -> tile range
    const int chunks = S.cin / CN;
    const int dz = blockIdx.y % 3;
    const int ci0 = (int)((blockIdx.y / 3) % chunks) * CN;
    const int co0 = (int)(blockIdx.y / 3 / chunks) * 128;
    const long long t_begin = G.tiles * blockIdx.x / G.splits, t_end = G.tiles * (blockIdx.x + 1) / G.splits;
    const int tiles_x = (S.w + 15) / 16, tiles_y = (S.h + 15) / 16;
    if (threadIdx.x == 0) {
        for (int i = 0; i < ST; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&done, 1);
        mbar_init(&drain, 1);
        abort_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmdy)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base_s)),
                     "r"(PL::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = tmem_base_s;
    volatile int *abort_flag = &abort_s;
    const bool any = t_end > t_begin;

    long long fills = 0;  // producer: stage fills issued
    bool mmas = false;    // MMA warp: any MMA issued
    if (warp == 0 && any) {
        const uint32_t leader = elect_one();
        const uint32_t tx = (uint32_t)(4096 * G.cb) + PL::X_TX;
        long long i = 0;
        bool ok = true;
        for (long long t = t_begin; t < t_end; ++t, ++i) {
            const int st = (int)(i % ST);
            if (i >= ST && !mbar_wait_warp(&empty[st], (unsigned)(((i / ST) - 1) & 1), abort_flag)) {
                ok = false;
                break;
            }
            long long u = t;
            const int x0 = (int)(u % tiles_x) * 16;
            u /= tiles_x;
            const int y0 = (int)(u % tiles_y) * 16;
            u /= tiles_y;
            const int z = (int)(u % S.d), nb = (int)(u / S.d);
            const uint32_t a = smem_addr(smem + (size_t)st * G.stage), b = a + (uint32_t)G.dy_region;
            expect_tx_p(leader, &full[st], tx);
            tma_load_5d_p(leader, a, &tmdy, 0, x0, co0 >> 3, y0, nb * S.d + z, &full[st]);
#pragma unroll
            for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                for (int h = 0; h < CN / 8; ++h)
                    tma_load_5d_p(leader, b + (uint32_t)((kx * (CN / 8) + h) * PL::COPY), &tmx, ci0 + 8 * h, x0 + kx - 1,
                                  y0 - 1, z + dz - 1, nb, &full[st]);
        }
        if (!ok && lane == 0) atomicExch(status, 1);
        fills = i;
    } else if (warp == 1 && any) {
        const uint32_t leader = elect_one();
        // kind::f16, D F32, A and B BF16, both MN-major, N = 3 CN, M = 64 or 128
        constexpr uint32_t ID = idesc(PL::NK, M64 ? 64 : 128) | (1u << 15) | (1u << 16);
        long long i = 0;
        bool ok = true, issued = false;
        const uint32_t row_step = (uint32_t)(G.cb * 256) >> 4;  // descriptor units per dy row
        for (long long t = t_begin; t < t_end; ++t, ++i) {
            const int st = (int)(i % ST);
            if (!mbar_wait_warp(&full[st], (unsigned)((i / ST) & 1), abort_flag)) {
                ok = false;
                break;
            }
            tc_after_sync();
            const uint32_t a_base = smem_addr(smem + (size_t)st * G.stage);
            const uint64_t a0 = sdesc_none(a_base, 128u, 256u);
            const uint64_t b0 = sdesc_none(a_base + (uint32_t)G.dy_region, 128u, (uint32_t)PL::COPY);
#pragma unroll 1
            for (int g = 0; g < 16; ++g) {
                const uint64_t ad = a0 + (uint64_t)(g * row_step);
                const uint32_t acc = (i > 0 || g > 0) ? 1u : 0u;
#pragma unroll
                for (int ky = 0; ky < 3; ++ky)  // row g + ky of every copy: 16 voxels x 16 B
                    umma_bf16_p(leader, tmem + (uint32_t)(ky * PL::NK), ad, b0 + (uint64_t)((g + ky) * 16), ID, acc);
            }
            umma_commit_p(leader, &empty[st]);
            issued = true;
        }
        if (ok) {
            umma_commit_p(leader, &done);
        } else if (lane == 0) {
            atomicExch(status, 1);
        }
        mmas = issued;
    } else if (warp >= 2 && any) {
        // epilogue, once per CTA: accumulator row m = co - co0 sits in TMEM lane
        // m (M = 128) or 32 (m / 16) + m % 16 (M = 64: lanes 16..31 of each
        // quarter hold no row)
        const int quarter = warp & 3;
        const int co = M64 ? (lane < 16 ? co0 + 16 * quarter + lane : S.cout) : co0 + 32 * quarter + lane;
        if (mbar_wait_warp(&done, 0u, abort_flag, EPI_WAIT_LIMIT)) {
            tc_after_sync();
            const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
            const long long krow = 27LL * S.cin;
#pragma unroll 1
            for (int j = 0; j < 9; ++j) {
#pragma unroll 1
                for (int c0 = 0; c0 < CN; c0 += 16) {
                    float v[16];
                    tmem_ld16(lane_base + (uint32_t)(j * CN + c0), v);
                    if (co < S.cout) {
                        float *dst = dw + co * krow + (long long)(9 * dz + j) * S.cin + ci0 + c0;
#pragma unroll
                        for (int q = 0; q < 16; ++q) atomicAdd(dst + q, v[q]);
                    }
                }
            }
        } else if (lane == 0) {
            atomicExch(status, 1);
        }
    }
    tc_before_sync();
    __syncthreads();
    // as in the forward: once a role gave up, the producer's last fills and
    // the MMA warp's MMAs complete (bounded waits) before TMEM and shared
    // memory are released
    if (*abort_flag) {
        if (warp == 0) {
            for (long long f = fills - 1; f >= 0 && f >= fills - ST; --f)
                mbar_wait_warp(&full[f % ST], (unsigned)((f / ST) & 1), nullptr);
        } else if (warp == 1 && mmas) {
            // elect.sync picks the same lane for the same member mask, so
            // this commit comes from the lane that issued the MMAs (the
            // leader is not carried out of the loop: keeping it live there
            // cost the issue loop about 40 %)
            umma_commit_p(elect_one(), &drain);
            mbar_wait_warp(&drain, 0u, nullptr);
        }
    }
    if (warp == 1) {
        tc_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(PL::TMEM_COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient of layers with 16 output channels (the U-Net's first and
// last level): dW[co][tap][ci] = sum_p dy[p][co] x[p + off(tap)][ci].
// With cout = 16 the tcgen05 form above wastes most of each MMA (M is at
// least 64) and re-reads both operands from shared memory for every MMA.
// Here each warp keeps its nine taps' 16 x 16 sums in registers and runs
// mma.m16n8k16 (BF16, FP32 accumulation; M = co, N = ci, K = 16 voxels of an
// output row) with register-resident operands:
//   * a CTA owns a column of the volume -- 16 input channels, one batch item,
//     W16_TH rows x 32 columns -- and walks a range of planes z.  For plane z
//     it needs the input planes z - 1, z, z + 1 over (W16_TH + 2) x 34 voxels
//     (halo included, zero outside the volume) and the dy tile of plane z; the
//     input planes live in a ring of four slots and the dy tiles in two, so
//     each step loads one new input plane and one dy tile (16-byte cp.async)
//     while the previous step computes.  A staged voxel takes 48 bytes (32
//     of data), so the eight rows of an ldmatrix are spread over all banks;
//   * warp (kz, chunk) walks the W16_TH + 2 rows of input plane z + kz - 1 for its
//     16-column chunk: per row it loads the three kx-shifted x operands once
//     (ldmatrix.trans at shifted row addresses -- the shift costs nothing)
//     and the dy row of the same index, keeps the last three dy rows, and
//     issues the 18 MMAs that pair x row y with dy rows y, y - 1, y - 2 (taps
//     ky = 0, 1, 2): each staged operand feeds up to 18 MMAs;
//   * the register sums go to dW (FP32 atomics) every 32 planes and at the
//     end, so no sum chains more than 512 MMA steps (the tensor core's FP32
//     accumulation drifts over long chains).
// Fragment layouts of mma.m16n8k16 (g = lane / 4, t = lane % 4): A (16 x 16,
// row = co, col = voxel k) a0 (g, 2t..2t+1), a1 (g + 8, 2t..), a2 (g, 2t+8..),
// a3 (g + 8, 2t+8..); B (16 x 8, row = voxel k, col = ci) b0 (2t..2t+1, g),
// b1 (2t+8..2t+9, g); D d0, d1 (g, 2t..2t+1), d2, d3 (g + 8, 2t..2t+1).  With
// voxels as the rows of the staged 8 x 8 matrices, ldmatrix.trans hands each
// lane exactly these pairs.
// tile rows: 8 keeps the staging ring at 90 KB, two CTAs per SM (measured
// faster than 16 rows at one CTA per SM: 0.248 vs 0.300 ms on 2 x 128^3, 16 -> 16)
#ifndef CTREX_W16_ROWS
#define CTREX_W16_ROWS 8
#endif
constexpr int W16_TW = 32, W16_TH = CTREX_W16_ROWS;   // tile: columns (two 16-voxel chunks) x rows
constexpr int W16_XR = W16_TH + 2, W16_XC = W16_TW + 2;  // staged input rows / columns (halo)
constexpr int W16_VS = 48;                             // bytes per staged voxel
constexpr int W16_XPLANE = W16_XR * W16_XC * W16_VS;   // 16 320 bytes for 8 rows
constexpr int W16_DYB = W16_TH * W16_TW * W16_VS;      // 12 288
constexpr int W16_SMEM = 4 * W16_XPLANE + 2 * W16_DYB;  // 89 856
constexpr int W16_CTAS = W16_SMEM <= 110 * 1024 ? 2 : 1;  // resident CTAs per SM the budget allows
constexpr int W16_THREADS = 192;                        // 6 warps: plane kz (3) x column chunk (2)
constexpr int W16_FLUSH = 32;                           // planes between flushes of the register sums

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t r[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16_16816(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Issues (no wait) the copies of input plane zz into a ring slot, or of the
// dy tile of plane zz: 16-byte cp.async per half voxel, zeros outside.
__device__ __forceinline__ void w16_stage_plane(const __nv_bfloat16 *__restrict__ x, const ConvShape &S, int nb,
                                                int zz, int y0, int x0, int ci0, uint8_t *slot)
{
    for (int i = threadIdx.x; i < W16_XR * W16_XC * 2; i += W16_THREADS) {
        const int h = i & 1, v = (i >> 1) % W16_XC, row = (i >> 1) / W16_XC;
        const int yy = y0 - 1 + row, xx = x0 - 1 + v;
        const __nv_bfloat16 *src = x;
        int bytes = 0;
        if ((unsigned)zz < (unsigned)S.d && (unsigned)yy < (unsigned)S.h && (unsigned)xx < (unsigned)S.w) {
            src = x + ((((long long)nb * S.d + zz) * S.h + yy) * S.w + xx) * S.cin + ci0 + 8 * h;
            bytes = 16;
        }
        cp_async16(slot + (row * W16_XC + v) * W16_VS + 16 * h, src, bytes);
    }
}

__device__ __forceinline__ void w16_stage_dy(const __nv_bfloat16 *__restrict__ dy, const ConvShape &S, int nb,
                                             int z, int y0, int x0, uint8_t *slot)
{
    for (int i = threadIdx.x; i < W16_TH * W16_TW * 2; i += W16_THREADS) {
        const int h = i & 1, v = (i >> 1) % W16_TW, row = (i >> 1) / W16_TW;
        const int yy = y0 + row, xx = x0 + v;
        const __nv_bfloat16 *src = dy;
        int bytes = 0;
        if (z < S.d && yy < S.h && xx < S.w) {
            src = dy + ((((long long)nb * S.d + z) * S.h + yy) * S.w + xx) * 16 + 8 * h;
            bytes = 16;
        }
        cp_async16(slot + (row * W16_TW + v) * W16_VS + 16 * h, src, bytes);
    }
}

__global__ void __launch_bounds__(W16_THREADS, W16_CTAS)
    conv_wgrad_c16_kernel(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ dy,
                          float *__restrict__ dw, ConvShape S, int segs)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    uint8_t *planes = smem, *dys = smem + 4 * W16_XPLANE;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kz = warp % 3, chunk = warp / 3;
    const int g = lane >> 2, t = lane & 3;
    // CTA -> (column, plane segment); column -> (ci chunk, n, y band, x chunk)
    const int tiles_x = (S.w + W16_TW - 1) / W16_TW, tiles_y = (S.h + W16_TH - 1) / W16_TH;
    long long col = blockIdx.x / segs;
    const int seg = (int)(blockIdx.x % segs);
    const int x0 = (int)(col % tiles_x) * W16_TW;
    col /= tiles_x;
    const int y0 = (int)(col % tiles_y) * W16_TH;
    col /= tiles_y;
    const int nb = (int)(col % S.nb), ci0 = (int)(col / S.nb) * 16;
    const int zb = (int)((long long)S.d * seg / segs), ze = (int)((long long)S.d * (seg + 1) / segs);
    // this lane's ldmatrix row: matrix mi = lane / 8, row r = lane % 8
    const int mi = lane >> 3, r8 = lane & 7;
    // dy (A): matrices (voxels 0-7, co 0-7), (0-7, 8-15), (8-15, 0-7), (8-15, 8-15)
    const uint32_t a_off = (uint32_t)((16 * chunk + 8 * (mi >> 1) + r8) * W16_VS + 16 * (mi & 1));
    // x (B): matrices (voxels 0-7, ci 0-7), (8-15, 0-7), (0-7, 8-15), (8-15, 8-15)
    const uint32_t b_off = (uint32_t)((16 * chunk + 8 * (mi & 1) + r8) * W16_VS + 16 * (mi >> 1));
    float acc[9][2][4];
#pragma unroll
    for (int q = 0; q < 9; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[q][h][e] = 0.0f;
    auto flush = [&]() {
#pragma unroll
        for (int q = 0; q < 9; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int co = g + 8 * (e >> 1), ci = ci0 + 8 * h + 2 * t + (e & 1);
                    const float v = acc[q][h][e];
                    acc[q][h][e] = 0.0f;
                    if (v != 0.0f) atomicAdd(dw + ((long long)co * 27 + kz * 9 + q) * S.cin + ci, v);
                }
    };
    if (zb >= ze) return;  // uniform over the CTA
    // prologue: input planes zb - 1, zb, zb + 1 in slots 0, 1, 2; dy of zb in slot 0
    for (int q = 0; q < 3; ++q) w16_stage_plane(x, S, nb, zb - 1 + q, y0, x0, ci0, planes + q * W16_XPLANE);
    w16_stage_dy(dy, S, nb, zb, y0, x0, dys);
    cp_async_commit();
    for (int z = zb; z < ze; ++z) {
        const int j = z - zb;
        // prefetch: input plane z + 2 into the free slot, dy of z + 1
        if (z + 1 < ze) {
            w16_stage_plane(x, S, nb, z + 2, y0, x0, ci0, planes + ((j + 3) & 3) * W16_XPLANE);
            w16_stage_dy(dy, S, nb, z + 1, y0, x0, dys + ((j + 1) & 1) * W16_DYB);
        }
        cp_async_commit();
        cp_async_wait<1>();  // everything but the prefetch just issued has landed
        __syncthreads();
        const uint32_t xs = smem_addr(planes + ((j + kz) & 3) * W16_XPLANE);  // input plane z + kz - 1
        const uint32_t ds = smem_addr(dys + (j & 1) * W16_DYB);
        uint32_t a0[4] = {0u, 0u, 0u, 0u}, a1[4] = {0u, 0u, 0u, 0u}, a2[4] = {0u, 0u, 0u, 0u};  // dy rows yp, yp-1, yp-2
#pragma unroll 1
        for (int yp = 0; yp < W16_XR; ++yp) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                a2[e] = a1[e];
                a1[e] = a0[e];
            }
            if (yp < W16_TH) ldsm_x4_trans(ds + (uint32_t)(yp * W16_TW * W16_VS) + a_off, a0);
            uint32_t b[3][4];
#pragma unroll
            for (int kx = 0; kx < 3; ++kx)
                ldsm_x4_trans(xs + (uint32_t)((yp * W16_XC + kx) * W16_VS) + b_off, b[kx]);
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                if (yp < W16_TH) {  // ky = 0: output row yp
                    mma_bf16_16816(acc[kx][0], a0, b[kx][0], b[kx][1]);
                    mma_bf16_16816(acc[kx][1], a0, b[kx][2], b[kx][3]);
                }
                if (yp >= 1 && yp <= W16_TH) {  // ky = 1: output row yp - 1
                    mma_bf16_16816(acc[3 + kx][0], a1, b[kx][0], b[kx][1]);
                    mma_bf16_16816(acc[3 + kx][1], a1, b[kx][2], b[kx][3]);
                }
                if (yp >= 2) {  // ky = 2: output row yp - 2
                    mma_bf16_16816(acc[6 + kx][0], a2, b[kx][0], b[kx][1]);
                    mma_bf16_16816(acc[6 + kx][1], a2, b[kx][2], b[kx][3]);
                }
            }
        }
        if ((j + 1) % W16_FLUSH == 0) flush();
        __syncthreads();  // the slots read here are refilled by the next step's prefetch
    }
    cp_async_wait<0>();
    flush();
}

int sm_count();

cudaError_t launch_wgrad_c16(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, float *dw, const ConvShape &S,
                             cudaStream_t stream)
{
    const long long cols = (long long)(S.cin / 16) * S.nb * ((S.h + W16_TH - 1) / W16_TH) *
                           ((S.w + W16_TW - 1) / W16_TW);
    // split the planes so that the grid covers about three waves of resident
    // CTAs, with at least 8 planes per segment
    long long segs = (3LL * W16_CTAS * sm_count() + cols - 1) / cols;
    const long long max_segs = S.d / 8 > 1 ? S.d / 8 : 1;
    if (segs > max_segs) segs = max_segs;
    if (segs < 1) segs = 1;
    const long long grid = cols * segs;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(conv_wgrad_c16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   W16_SMEM + 128);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    conv_wgrad_c16_kernel<<<(unsigned)grid, W16_THREADS, W16_SMEM + 128, stream>>>(x, dy, dw, S, (int)segs);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if the driver does not provide it.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return n;
}

// Persistent TMA brick FWD: one CTA per SM.  Returns cudaErrorNotSupported
// (nothing launched) when the tensor maps cannot be made, so that the
// caller falls back to the im2col kernel.
template <int BN, int NT, bool RESW>
cudaError_t launch_tma(const __nv_bfloat16 *x, const __nv_bfloat16 *w, const float *bias, void *out, int out_bf16,
                       const ConvShape &S, int *status, cudaStream_t stream)
{
    using PL = TmaPlan<BN, NT, RESW>;
    const EncodeTiledFn enc = encode_tiled();
    const int sms = sm_count();
    if (!enc || sms <= 0 || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(w) & 15))
        return cudaErrorNotSupported;
    const uint64_t es = sizeof(__nv_bfloat16);
    CUtensorMap mx, mw;
    {
        const cuuint64_t dims[5] = {(cuuint64_t)S.cin, (cuuint64_t)S.w, (cuuint64_t)S.h, (cuuint64_t)S.d, (cuuint64_t)S.nb};
        const cuuint64_t strides[4] = {S.cin * es, (uint64_t)S.w * S.cin * es, (uint64_t)S.h * S.w * S.cin * es,
                                       (uint64_t)S.d * S.h * S.w * S.cin * es};
        const cuuint32_t box[5] = {8, (cuuint32_t)PL::RW, 18, 1, 1};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(x), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)(27LL * S.cin), (cuuint64_t)S.n_total};
        const cuuint64_t strides[1] = {27ULL * S.cin * es};
        const cuuint32_t box[2] = {8, (cuuint32_t)BN};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(w), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    cudaError_t e =
        cudaFuncSetAttribute(conv_fwd_tma_kernel<BN, NT, RESW>, cudaFuncAttributeMaxDynamicSharedMemorySize, PL::SMEM);
    if (e != cudaSuccess) return e;
    const long long items = (long long)S.nb * S.d * ((S.h + 15) / 16) * ((S.w + 8 * NT - 1) / (8 * NT)) *
                            ((S.n_total + BN - 1) / BN);
    const unsigned grid = (unsigned)(items < sms ? items : sms);
    conv_fwd_tma_kernel<BN, NT, RESW><<<grid, TMA_THREADS, PL::SMEM, stream>>>(mx, mw, bias, out, out_bf16, S, status);
    return cudaGetLastError();
}

// Forward of a layer with at most 16 output channels (conv_fwd_kx_kernel):
// returns cudaErrorNotSupported (nothing launched) when the tensor maps
// cannot be made or the filter and four plane slots do not fit in shared
// memory.
template <int NT, int P>
cudaError_t launch_kx_nt(const __nv_bfloat16 *x, const __nv_bfloat16 *w, const float *bias, void *out, int out_bf16,
                         const ConvShape &S, const KxArgs &G, int *status, cudaStream_t stream)
{
    using PL = KxPlan<NT>;
    const EncodeTiledFn enc = encode_tiled();
    const int sms = sm_count();
    if (!enc || sms <= 0 || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(w) & 15))
        return cudaErrorNotSupported;
    const uint64_t es = sizeof(__nv_bfloat16);
    CUtensorMap mx, mw;
    {
        const cuuint64_t dims[5] = {(cuuint64_t)S.cin, (cuuint64_t)S.w, (cuuint64_t)S.h, (cuuint64_t)S.d, (cuuint64_t)S.nb};
        const cuuint64_t strides[4] = {S.cin * es, (uint64_t)S.w * S.cin * es, (uint64_t)S.h * S.w * S.cin * es,
                                       (uint64_t)S.d * S.h * S.w * S.cin * es};
        // 16 channels (32 bytes, 32-byte swizzle) or 8 channels per box
        const cuuint32_t box[5] = {PL::SW ? 16u : 8u, (cuuint32_t)PL::RW, 18, 1, 1};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(x), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, PL::SW ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    {
        const cuuint64_t dims[2] = {(cuuint64_t)(27LL * S.cin), (cuuint64_t)S.n_total};
        const cuuint64_t strides[1] = {27ULL * S.cin * es};
        const cuuint32_t box[2] = {8, 16};
        const cuuint32_t estr[2] = {1, 1};
        if (enc(&mw, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(w), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    KxArgs A = G;
    // output planes per item: the whole depth, halved while the grid would
    // hold fewer than six items per SM (each item loads nz + 2 planes)
    const long long cols = (long long)S.nb * ((S.h + 15) / 16) * ((S.w + 8 * NT - 1) / (8 * NT));
    int zc = S.d;
    while (zc > 4 && cols * ((S.d + zc - 1) / zc) < 6LL * sms) zc = (zc + 1) / 2;
    A.zc = zc;
    const int smem = A.w_bytes + P * A.cb * PL::WIN + 1024;
    cudaError_t e = cudaFuncSetAttribute(conv_fwd_kx_kernel<NT, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const long long items = cols * ((S.d + zc - 1) / zc);
    const unsigned grid = (unsigned)(items < sms ? items : sms);
    conv_fwd_kx_kernel<NT, P><<<grid, TMA_THREADS, smem, stream>>>(mx, mw, bias, out, out_bf16, S, A, status);
    return cudaGetLastError();
}

// Tile width: 32 columns (NT = 4) when the filter and four plane slots of
// that width fit in shared memory, else 16; 8 for volumes at most 8 wide.
// Plane slots: 8 where they fit, else 4.
cudaError_t launch_kx(const __nv_bfloat16 *x, const __nv_bfloat16 *w, const float *bias, void *out, int out_bf16,
                      const ConvShape &S, int *status, cudaStream_t stream)
{
    constexpr int SMEM_MAX = 227 * 1024 - 1024 - 512;  // dynamic budget: alignment slack, static barriers
    KxArgs G{};
    G.cb = S.cin / 16;
    G.w_bytes = (27 * S.cin * 16 * 2 + 1023) / 1024 * 1024;
    auto fits = [&](int win, int p) { return G.w_bytes + p * G.cb * win <= SMEM_MAX; };
#define CTREX_KX_LAUNCH(NT)                                                                        \
    if (fits(KxPlan<NT>::WIN, 8)) return launch_kx_nt<NT, 8>(x, w, bias, out, out_bf16, S, G, status, stream); \
    if (fits(KxPlan<NT>::WIN, 4)) return launch_kx_nt<NT, 4>(x, w, bias, out, out_bf16, S, G, status, stream);
    if (S.w <= 8) {
        CTREX_KX_LAUNCH(1)
        return cudaErrorNotSupported;
    }
    CTREX_KX_LAUNCH(4)
    CTREX_KX_LAUNCH(2)
#undef CTREX_KX_LAUNCH
    return cudaErrorNotSupported;
}

// Brick weight gradient: returns cudaErrorNotSupported (nothing launched)
// when the tensor maps cannot be made.
template <int CN, bool M64>
cudaError_t launch_wgrad_tma(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, float *dw, const ConvShape &S,
                             int *status, cudaStream_t stream)
{
    using PL = WgPlan<CN>;
    const EncodeTiledFn enc = encode_tiled();
    const int sms = sm_count();
    if (!enc || sms <= 0 || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(dy) & 15))
        return cudaErrorNotSupported;
    const uint64_t es = sizeof(__nv_bfloat16);
    CUtensorMap mx, mdy;
    {
        const cuuint64_t dims[5] = {(cuuint64_t)S.cin, (cuuint64_t)S.w, (cuuint64_t)S.h, (cuuint64_t)S.d, (cuuint64_t)S.nb};
        const cuuint64_t strides[4] = {S.cin * es, (uint64_t)S.w * S.cin * es, (uint64_t)S.h * S.w * S.cin * es,
                                       (uint64_t)S.d * S.h * S.w * S.cin * es};
        const cuuint32_t box[5] = {8, 16, 18, 1, 1};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        if (enc(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(x), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    const int cb = S.cout / 8 < 16 ? S.cout / 8 : 16;
    {
        // (8 channels, x, 8-channel block, y, plane): the box lands as
        // [y][block][x][8 channels]
        const cuuint64_t dims[5] = {8, (cuuint64_t)S.w, (cuuint64_t)(S.cout / 8), (cuuint64_t)S.h,
                                    (cuuint64_t)S.nb * S.d};
        const cuuint64_t strides[4] = {S.cout * es, 16, (uint64_t)S.w * S.cout * es, (uint64_t)S.h * S.w * S.cout * es};
        const cuuint32_t box[5] = {8, 16, (cuuint32_t)cb, 16, 1};
        const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        if (enc(&mdy, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(dy), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorNotSupported;
    }
    WgArgs G{};
    G.cb = cb;
    // rows 0..15 of cb blocks each; row 15's 16 (M = 64: 8) M blocks read up
    // to 15 * cb * 256 + 16 (8) * 256 bytes
    G.dy_region = (256 * (15 * cb + (M64 ? 8 : 16)) + 1023) / 1024 * 1024;
    G.stage = (G.dy_region + PL::X_BYTES + 1023) / 1024 * 1024;
    G.st = (200 * 1024) / G.stage;
    if (G.st > WG_MAX_ST) G.st = WG_MAX_ST;
    if (G.st < 2) return cudaErrorNotSupported;
    const int smem = G.st * G.stage + 1024;
    G.tiles = (long long)S.nb * S.d * ((S.h + 15) / 16) * ((S.w + 15) / 16);
    const long long jobs = (long long)((S.cout + 127) / 128) * (S.cin / CN) * 3;
    if (jobs > 65535) return cudaErrorNotSupported;
    // The tensor core's FP32 accumulation loses about 2^-24 of the partial
    // sum per K step in a long chain (measured: 5e-4 relative after 5.2 k
    // steps of positive terms), so a CTA accumulates at most WG_CHUNK tiles
    // (16 K steps each) in TMEM before its partial sums go to dW with FP32
    // atomics; and at least one CTA per SM.
    // The grid is rounded up to whole waves of one CTA per SM, the tiles
    // spread evenly over them.
    const long long need = (G.tiles + WG_CHUNK - 1) / WG_CHUNK * jobs;
    const long long waves = (need + sms - 1) / sms;
    long long splits = waves * sms / jobs;
    if (splits < 1) splits = 1;
    if (splits > G.tiles) splits = G.tiles;
    if (splits > 0x7FFFFFFFLL) return cudaErrorNotSupported;
    G.splits = (int)splits;
    cudaError_t e =
        cudaFuncSetAttribute(conv_wgrad_tma_kernel<CN, M64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    conv_wgrad_tma_kernel<CN, M64><<<dim3((unsigned)splits, (unsigned)jobs, 1), TMA_THREADS, smem, stream>>>(
        mx, mdy, dw, S, G, status);
    return cudaGetLastError();
}

template <int OP, int BN>
cudaError_t launch_bn(const __nv_bfloat16 *a, const __nv_bfloat16 *b, const float *bias, void *out, int out_bf16,
                      const ConvShape &S, int *status, cudaStream_t stream)
{
    if constexpr (BN == 16) {
        if (OP == OP_FWD && (S.cin & 15) == 0 && CTREX_CONV_TMA && CTREX_CONV_KX) {
            const cudaError_t e = launch_kx(a, b, bias, out, out_bf16, S, status, stream);
            if (e != cudaErrorNotSupported) return e;  // else: the brick kernel below
        }
    }
    if (OP == OP_FWD && (S.cin & 15) == 0 && CTREX_CONV_TMA) {
        // tiles 16 x 16 (NT = 2) unless the volume is at most 8 wide; the
        // filter stays resident when the layer has one N tile and it fits
        const bool resw = S.n_total <= BN && 27LL * S.cin * BN * 2 <= TmaPlan<BN, 2, true>::W_MAX;
        cudaError_t e;
        if (S.w > 8)
            e = resw ? launch_tma<BN, 2, true>(a, b, bias, out, out_bf16, S, status, stream)
                     : launch_tma<BN, 2, false>(a, b, bias, out, out_bf16, S, status, stream);
        else
            e = resw ? launch_tma<BN, 1, true>(a, b, bias, out, out_bf16, S, status, stream)
                     : launch_tma<BN, 1, false>(a, b, bias, out, out_bf16, S, status, stream);
        if (e != cudaErrorNotSupported) return e;  // else: the im2col kernel below
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
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(y)) & 15)
        return CTREX_E_ARG;  // 16-byte copies and stores
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
    int bn = pick_bn(cout);
    if (CTREX_CONV_TMA && CTREX_CONV_FILL && (cin & 15) == 0) {
        // narrower N tiles while the grid would leave SMs idle (deep layers
        // at small spatial sizes); measured: narrowing further, to two CTAs
        // per SM, costs more in brick reloads than it gains
        const int nt = wd > 8 ? 2 : 1;
        const long long tiles = (long long)nb * d * ((h + 15) / 16) * ((wd + 8 * nt - 1) / (8 * nt));
        while (bn > 32 && tiles * ((cout + bn - 1) / bn) < 152) bn = bn > 64 ? 64 : 32;
    }
    cudaError_t e = launch_op<OP_FWD>(bn, static_cast<const __nv_bfloat16 *>(x), static_cast<const __nv_bfloat16 *>(w),
                                      bias, y, y_dtype == CTREX_BF16, S, status, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CTREX_OK : CTREX_E_CUDA;
}

int ctrex_conv3d_wgrad(const void *x, const void *dy, float *dw, int nb, int d, int h, int wd, int cin, int cout,
                       int *status, void *stream)
{
    if (!x || !dy || !dw || !status) return CTREX_E_ARG;
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(dy)) & 15) return CTREX_E_ARG;
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
    // split K so that the grid fills the GPU about twice, and so that no CTA
    // accumulates more than 8192 voxels (512 K steps) in TMEM: the tensor
    // core's FP32 accumulation drifts over long chains
    const long long mt = (S.m_total + BM - 1) / BM;
    long long splits = (2 * 152 + mt - 1) / mt;
    long long per = (S.k_total + splits - 1) / splits;
    if (per > 8192) per = 8192;
    if ((S.k_total + per - 1) / per > 65535) per = (S.k_total + 65534) / 65535;  // grid z limit
    per = ((per + BK - 1) / BK) * BK;
    if (per < BK) per = BK;
    S.k_per_cta = per;
    if (cout == 16 && (cin & 15) == 0) {  // register-blocked MMAs: no padded M
        const cudaError_t e = launch_wgrad_c16(static_cast<const __nv_bfloat16 *>(x),
                                               static_cast<const __nv_bfloat16 *>(dy), dw, S,
                                               static_cast<cudaStream_t>(stream));
        return e == cudaSuccess ? CTREX_OK : CTREX_E_CUDA;
    }
    if (CTREX_CONV_TMA && (cin & 15) == 0) {
        // 32-channel chunks where two ring stages still fit beside the dy
        // rows; M = 64 MMAs (half the dy operand reads) for up to 64 outputs
        const auto *xb = static_cast<const __nv_bfloat16 *>(x);
        const auto *db = static_cast<const __nv_bfloat16 *>(dy);
        const cudaStream_t st = static_cast<cudaStream_t>(stream);
        const bool c32 = (cin & 31) == 0 && cout <= 64, m64 = cout <= 64;
        const cudaError_t e = c32 ? (m64 ? launch_wgrad_tma<32, true>(xb, db, dw, S, status, st)
                                         : launch_wgrad_tma<32, false>(xb, db, dw, S, status, st))
                                  : (m64 ? launch_wgrad_tma<16, true>(xb, db, dw, S, status, st)
                                         : launch_wgrad_tma<16, false>(xb, db, dw, S, status, st));
        if (e != cudaErrorNotSupported) return e == cudaSuccess ? CTREX_OK : CTREX_E_CUDA;
    }
    const int bn = pick_bn(cout);
    cudaError_t e = launch_op<OP_WGRAD>(bn, static_cast<const __nv_bfloat16 *>(x),
                                        static_cast<const __nv_bfloat16 *>(dy), nullptr, dw, 0, S, status,
                                        static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? CTREX_OK : CTREX_E_CUDA;
}

}  // extern "C"

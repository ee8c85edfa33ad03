// fwd_common.cuh -- launch shape and per-pixel epilogue shared by the forward
// kernels: the projected value (and row sum) is stored, or turned into the
// correction R (p - A x) of Eq. (1) term 2 with the residual norms reduced
// per CTA in a fixed order (Sec. 4.1 "Correction kernel").
#pragma once

#include "ctrex_internal.cuh"

namespace ctrex {

constexpr int FWD_TX = 32;  // pixels per CTA along u (one warp)
constexpr int FWD_TY = 4;   // pixels per CTA along v

enum FwdMode { MODE_PROJECT = 0, MODE_CORRECT = 1 };

// Pixel (iu, iv) of list entry k (view `view`; ok = the view index was
// valid).  s_red: shared scratch of 2 x (warps per CTA) floats.  Every
// thread of the CTA must call it (the correction mode synchronises).
template <typename TP, int MODE>
__device__ __forceinline__ void fwd_epilogue(const Grid &G, int k, int view, bool ok, bool in_pix, int iu, int iv,
                                             float val, float rs, TP *__restrict__ out,
                                             float *__restrict__ rowsum_out, const TP *__restrict__ p,
                                             float *__restrict__ partials, int p_by_view,
                                             float (*s_red)[FWD_TX * FWD_TY / 32])
{
    const bool inside = ok && in_pix;
    const size_t pix = ((size_t)k * G.nv + iv) * G.nu + iu;
    if (MODE == MODE_PROJECT) {
        if (in_pix) {  // a skipped (out-of-range) view gets zeros
            Storage<TP>::store(out + pix, val);
            if (rowsum_out) rowsum_out[pix] = rs;
        }
        return;
    } else {
        float e2 = 0.0f, p2 = 0.0f;
        if (in_pix && !ok) Storage<TP>::store(out + pix, 0.0f);
        if (inside) {
            const float pm = Storage<TP>::load(p + (p_by_view ? ((size_t)view * G.nv + iv) * G.nu + iu : pix));
            const float e = pm - val;
            const float Rw = rs > G.eps_R ? 1.0f / rs : 0.0f;
            Storage<TP>::store(out + pix, Rw * e);
            e2 = e * e;
            p2 = pm * pm;
        }
        // warp-shuffle then fixed-order CTA reduction of the residual norms
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            e2 += __shfl_xor_sync(0xffffffffu, e2, off);
            p2 += __shfl_xor_sync(0xffffffffu, p2, off);
        }
        const int lane = threadIdx.x & 31;
        const int warp = (threadIdx.y * FWD_TX + threadIdx.x) >> 5;
        if (lane == 0) {
            s_red[0][warp] = e2;
            s_red[1][warp] = p2;
        }
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            float a = 0.0f, b = 0.0f;
#pragma unroll
            for (int w = 0; w < FWD_TX * FWD_TY / 32; ++w) {
                a += s_red[0][w];
                b += s_red[1][w];
            }
            const size_t bid = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            partials[2 * bid] = a;
            partials[2 * bid + 1] = b;
        }
    }
}

}  // namespace ctrex

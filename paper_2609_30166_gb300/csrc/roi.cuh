// roi.cuh -- multi-resolution ROI projection (Sec. 3.7, the simultaneous
// form; the projector's sampling stage switches volume by ray position):
// a ray clipped to the context grid's box is split at the ROI box into
// context and ROI pieces.  Each piece follows the fixed-step
// truncated-midpoint rule with its own grid's step and samples its own grid
// (zero-padded trilinear interpolation, two gathers per sample from that
// grid's atlas).  Rays are set up in context index coordinates; ROI index
// coordinates are an affine map of them per axis.
#pragma once

#include "atlas.cuh"
#include "ray.cuh"

// Resident CTAs per SM the multi-resolution projector is compiled for,
// through its own kernel entry (two grids' setup needs more registers than
// the static sampler, and the texture path wants warps in flight).
#ifndef CTREX_FWD_ROI_MIN_BLOCKS
#define CTREX_FWD_ROI_MIN_BLOCKS 8
#endif

namespace ctrex {

// Each grid's table holds 1024 slices (16 KB for both, so that the CTAs the
// kernel is compiled for fit in shared memory).
using RoiAtlasSampler = AtlasSamplerT<1024>;

struct RoiSampler {
    RoiAtlasSampler ctx;  // context grid atlas (tile table: first half)
    RoiAtlasSampler roi;  // ROI grid atlas (tile table: second half)
    RoiGPU R;
    static constexpr int TILE_TABLE = 2 * RoiAtlasSampler::TILE_TABLE;
    static constexpr bool CYLINDER = false;
    static constexpr bool JOSEPH = false;
    static constexpr bool ROI = true;
    static constexpr bool DYRECT = false;
    static constexpr int MIN_BLOCKS = CTREX_FWD_ROI_MIN_BLOCKS;  // own kernel entry, CTAs per SM

    __device__ __forceinline__ void bind(float2 *table, int tid, int nthreads)
    {
        ctx.bind(table, tid, nthreads);
        roi.bind(table + RoiAtlasSampler::TILE_TABLE, tid, nthreads);
    }
    // unused: the ROI path integrates piece by piece
    __device__ __forceinline__ float operator()(float, float, float, float &ws) const
    {
        ws = 0.0f;
        return 0.0f;
    }
    __device__ __forceinline__ float interior(float, float, float) const { return 0.0f; }
};

// Samples k of [0, K-1) whose eight taps all lie inside a grid of n voxels
// per axis: g(k) = X + (a + (k + 1/2) h) dg in [eps, n - 1 - eps] on each
// axis (the margin eps is far above the rounding of the positions), with one
// sample of slack at each end.
__device__ __forceinline__ void piece_interior(const float X[3], const float dg[3], float a, float h, int K,
                                               const int n[3], int &ka, int &kb)
{
    const float eps = 1e-2f;
    float lo = 0.0f, hi = (float)(K - 2);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float g0 = fmaf(a + 0.5f * h, dg[ax], X[ax]), sg = h * dg[ax];
        const float l = eps, u = (float)(n[ax] - 1) - eps;
        if (sg != 0.0f) {
            const float inv = 1.0f / sg;
            const float t0 = (l - g0) * inv, t1 = (u - g0) * inv;
            lo = fmaxf(lo, fminf(t0, t1));
            hi = fminf(hi, fmaxf(t0, t1));
        } else if (!(g0 >= l && g0 <= u)) {
            hi = -1.0f;
        }
    }
    ka = min(max((int)ceilf(lo) + 1, 0), K - 1);
    kb = max(min((int)floorf(hi), K - 1), ka);
}

// Truncated-midpoint samples of the piece [a, b] (mm along the ray) of the
// line g(t) = X + t dg in the index coordinates of grid `smp` (n voxels per
// axis), step h (mm); samples with all taps inside take the short path.
__device__ __forceinline__ void roi_piece(const RoiAtlasSampler &smp, const int n[3], const float X[3],
                                          const float dg[3], float a, float b, float h, float &val, float &rs)
{
    if (!(b > a)) return;
    int K = (int)ceilf((b - a) / h);
    if (K < 1) K = 1;
    int ka, kb;
    piece_interior(X, dg, a, h, K, n, ka, kb);
    float acc = 0.0f, wacc = 0.0f;
    auto general = [&](int k) {
        const float t = fmaf((float)k + 0.5f, h, a);
        float ws;
        acc += smp(fmaf(t, dg[0], X[0]), fmaf(t, dg[1], X[1]), fmaf(t, dg[2], X[2]), ws);
        wacc += ws;
    };
    for (int k = 0; k < ka; ++k) general(k);
    for (int k = ka; k < kb; ++k) {
        const float t = fmaf((float)k + 0.5f, h, a);
        acc += smp.interior(fmaf(t, dg[0], X[0]), fmaf(t, dg[1], X[1]), fmaf(t, dg[2], X[2]));
    }
    wacc += (float)(kb - ka);
    for (int k = kb; k < K - 1; ++k) general(k);
    const float a_last = fmaf((float)(K - 1), h, a);
    const float t_last = 0.5f * (a_last + b), w_last = b - a_last;
    float ws;
    const float last = smp(fmaf(t_last, dg[0], X[0]), fmaf(t_last, dg[1], X[1]), fmaf(t_last, dg[2], X[2]), ws);
    val += fmaf(acc, h, w_last * last);
    rs += fmaf(wacc, h, w_last * ws);
}

// Clip of the half line t >= t_min of X + t dg to the box [lo, hi].
__device__ __forceinline__ bool clip_box(const float X[3], const float dg[3], const float lo[3], const float hi[3],
                                         float t_min, float &t0, float &t1)
{
    t0 = t_min;
    t1 = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dg[a] != 0.0f) {
            const float inv = 1.0f / dg[a];
            const float ta = (lo[a] - X[a]) * inv, tb = (hi[a] - X[a]) * inv;
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else if (X[a] < lo[a] || X[a] > hi[a]) {
            return false;
        }
    }
    return t1 > t0;
}

// Line integral and row sum of one ray over both grids; returns the number
// of samples (for the sample count).
template <bool COUNT_ONLY>
__device__ __forceinline__ long long roi_integral(const Grid &G, const RoiSampler &smp, const ViewGPU &V, float u,
                                                  float v, float &val, float &rs)
{
    val = 0.0f;
    rs = 0.0f;
    float X[3], dg[3], len;
    ray_line(G, V, u, v, X, dg, len);
    float t0, t1;
    if (!clip_box(X, dg, G.lo, G.hi, -len, t0, t1)) return 0;
    const RoiGPU &R = smp.R;
    const float hc = G.step_mm, hf = R.step_mm;
    float r0, r1;
    const bool hit = clip_box(X, dg, R.lo, R.hi, t0, r0, r1) && r0 < t1;
    if (hit) r1 = fminf(r1, t1);
    if (COUNT_ONLY) {
        if (!hit) return (long long)max((int)ceilf((t1 - t0) / hc), 1);
        long long n = (long long)max((int)ceilf((r1 - r0) / hf), 1);
        if (r0 > t0) n += max((int)ceilf((r0 - t0) / hc), 1);
        if (t1 > r1) n += max((int)ceilf((t1 - r1) / hc), 1);
        return n;
    }
    const int nc[3] = {G.nx, G.ny, G.nz}, nr[3] = {R.n[0], R.n[1], R.n[2]};
    if (!hit) {
        roi_piece(smp.ctx, nc, X, dg, t0, t1, hc, val, rs);
        return 0;
    }
    // ROI index coordinates: g_roi = g_ctx * sc + oc per axis
    float Xf[3], dgf[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Xf[a] = fmaf(X[a], R.sc[a], R.oc[a]);
        dgf[a] = dg[a] * R.sc[a];
    }
    roi_piece(smp.ctx, nc, X, dg, t0, r0, hc, val, rs);
    roi_piece(smp.roi, nr, Xf, dgf, r0, r1, hf, val, rs);
    roi_piece(smp.ctx, nc, X, dg, r1, t1, hc, val, rs);
    return 0;
}

}  // namespace ctrex

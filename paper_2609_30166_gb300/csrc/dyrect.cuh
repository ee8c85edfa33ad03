// dyrect.cuh -- the event-based 4D model of Sec. 3.3 in the ray-driven
// projector: three fields per voxel, the initial value mu0, the final value
// mu1 and the transition time tau.  A view acquired at time t sees mu0 at
// the voxels with t < tau and mu1 elsewhere, so each trilinear tap picks one
// of the two values by its voxel's tau; the weights and the row sum are
// those of the static projector.  The three fields live in three texture
// atlases of identical tiling (one tile-origin table serves all), and one
// footprint costs three gathers (mu0, mu1, tau) per slice.
// Interior samples first read the smallest and largest transition time of
// their 8^3 brick (taken over the brick and the voxel past each of its upper
// faces, so that it covers every footprint whose lower corner lies in the
// brick): when the view's time is below the smallest every tap takes mu0,
// when it is at or above the largest every tap takes mu1, and the footprint
// costs one gather per slice; the values and the arithmetic are those the
// per-tap choice gives.
#pragma once

#include "atlas.cuh"

// Resident CTAs per SM the event-model projector is compiled for, through
// its own kernel entry (its per-tap choice needs more registers than the
// static sampler, and the texture path wants warps in flight).
#ifndef CTREX_FWD_DYR_MIN_BLOCKS
#define CTREX_FWD_DYR_MIN_BLOCKS 9
#endif

namespace ctrex {

struct DyrectSampler {
    Atlas A0, A1, At;              // mu0, mu1 and tau atlases (same w, h, n, tshift)
    const float *t_view = nullptr;  // device [n_views]: acquisition time of each view
    const float2 *brick = nullptr;  // device [bz][by][bx]: (min, max) transition time of each 8^3 brick
    int bnx = 0, bny = 0;           // bricks along x and y
    float t = 0.0f;                 // time of the view being projected (set per CTA)
    const float2 *tile = nullptr;

    static constexpr int TILE_TABLE = 2048;
    static constexpr bool CYLINDER = false;
    static constexpr bool JOSEPH = false;
    static constexpr bool ROI = false;
    static constexpr bool DYRECT = true;
    static constexpr int MIN_BLOCKS = CTREX_FWD_DYR_MIN_BLOCKS;  // own kernel entry, CTAs per SM

    __device__ __forceinline__ void bind(float2 *table, int tid, int nthreads)
    {
        const int n = min(A0.n, TILE_TABLE);
        for (int s = tid; s < n; s += nthreads)
            table[s] = make_float2((float)((s & ((1 << A0.tshift) - 1)) * A0.w) + 1.0f,
                                   (float)((s >> A0.tshift) * A0.h) + 1.0f);
        __syncthreads();
        tile = table;
    }
    __device__ __forceinline__ void set_view(int view) { t = __ldg(t_view + view); }
    __device__ __forceinline__ float2 origin(int s) const
    {
        if (s < TILE_TABLE) return tile[s];
        return make_float2((float)((s & ((1 << A0.tshift) - 1)) * A0.w) + 1.0f,
                           (float)((s >> A0.tshift) * A0.h) + 1.0f);
    }
    // The four taps of one slice footprint at atlas corner (X, Y), each
    // taken from mu0 or mu1 by its tau.
    __device__ __forceinline__ void quad(float X, float Y, float &c00, float &c10, float &c01, float &c11) const
    {
        float a00, a10, a01, a11, b00, b10, b01, b11, t00, t10, t01, t11;
        atlas_quad_at(A0, X, Y, a00, a10, a01, a11);
        atlas_quad_at(A1, X, Y, b00, b10, b01, b11);
        atlas_quad_at(At, X, Y, t00, t10, t01, t11);
        c00 = t < t00 ? a00 : b00;
        c10 = t < t10 ? a10 : b10;
        c01 = t < t01 ? a01 : b01;
        c11 = t < t11 ? a11 : b11;
    }

    // All eight taps inside the grid.
    __device__ __forceinline__ float interior(float gx, float gy, float gz) const
    {
        const float fx = floorf(gx), fy = floorf(gy), fz = floorf(gz);
        const int iz = (int)fz;
        const float ax = gx - fx, ay = gy - fy, az = gz - fz;
        const float2 o0 = origin(iz), o1 = origin(iz + 1);
        float a00, a10, a01, a11, b00, b10, b01, b11;
        const float2 lh = __ldg(brick + ((iz >> 3) * bny + ((int)fy >> 3)) * bnx + ((int)fx >> 3));
        if (t < lh.x || t >= lh.y) {
            // one field for the whole footprint
            const Atlas &S = t < lh.x ? A0 : A1;
            atlas_quad_at(S, o0.x + fx, o0.y + fy, a00, a10, a01, a11);
            atlas_quad_at(S, o1.x + fx, o1.y + fy, b00, b10, b01, b11);
        } else {
            quad(o0.x + fx, o0.y + fy, a00, a10, a01, a11);
            quad(o1.x + fx, o1.y + fy, b00, b10, b01, b11);
        }
        const float c0 = fmaf(ay, fmaf(ax, a11 - a01, a01) - fmaf(ax, a10 - a00, a00), fmaf(ax, a10 - a00, a00));
        const float c1 = fmaf(ay, fmaf(ax, b11 - b01, b01) - fmaf(ax, b10 - b00, b00), fmaf(ax, b10 - b00, b00));
        return fmaf(az, c1 - c0, c0);
    }

    // Zero-padded trilinear sample (taps outside the grid weigh nothing).
    __device__ __forceinline__ float operator()(float gx, float gy, float gz, float &wsum) const
    {
        const float fx = floorf(gx), fy = floorf(gy), fz = floorf(gz);
        const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
        const float ax = gx - fx, ay = gy - fy, az = gz - fz;
        const float wx0 = ((unsigned)ix < (unsigned)A0.w) ? 1.0f - ax : 0.0f;
        const float wx1 = ((unsigned)(ix + 1) < (unsigned)A0.w) ? ax : 0.0f;
        const float wy0 = ((unsigned)iy < (unsigned)A0.h) ? 1.0f - ay : 0.0f;
        const float wy1 = ((unsigned)(iy + 1) < (unsigned)A0.h) ? ay : 0.0f;
        const float wz0 = ((unsigned)iz < (unsigned)A0.n) ? 1.0f - az : 0.0f;
        const float wz1 = ((unsigned)(iz + 1) < (unsigned)A0.n) ? az : 0.0f;
        const int x0 = min(max(ix, -1), A0.w - 1), y0 = min(max(iy, -1), A0.h - 1);
        const int s0 = min(max(iz, 0), A0.n - 1), s1 = min(max(iz + 1, 0), A0.n - 1);
        const float2 o0 = origin(s0), o1 = origin(s1);
        float a00, a10, a01, a11, b00, b10, b01, b11;
        quad(o0.x + (float)x0, o0.y + (float)y0, a00, a10, a01, a11);
        quad(o1.x + (float)x0, o1.y + (float)y0, b00, b10, b01, b11);
        const float c0 = fmaf(wy0, fmaf(wx0, a00, wx1 * a10), wy1 * fmaf(wx0, a01, wx1 * a11));
        const float c1 = fmaf(wy0, fmaf(wx0, b00, wx1 * b10), wy1 * fmaf(wx0, b01, wx1 * b11));
        wsum = (wx0 + wx1) * (wy0 + wy1) * (wz0 + wz1);
        return fmaf(wz0, c0, wz1 * c1);
    }
};

}  // namespace ctrex

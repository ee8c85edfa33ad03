// ray.cuh -- per-ray set-up, sampling and interpolation shared by the
// ray-driven kernels (forward, fused correction, adjoint, motion gradient).
#pragma once

#include "ctrex_internal.cuh"

namespace ctrex {

// Geometry of one ray in voxel-index coordinates.  Samples k = 0..K-2 sit at
// g0 + k * sg with weight step_mm; the last one at g_last with weight w_last
// (truncated-midpoint rule of the clipped segment, Sec. 4.1 "weighted by
// their path lengths").
struct Ray {
    float g0[3];
    float sg[3];
    float g_last[3];
    float w_last;
    int K;
};

// The line of view parameters V through detector point (u, v): X, a point
// near the volume, and dg, index units per mm along the ray; the source sits
// at t = -len (t in mm from X).
__device__ __forceinline__ void ray_line(const Grid &G, const ViewGPU &V, float u, float v, float X[3], float dg[3],
                                         float &len)
{
    const float du = u - G.uc, dv = v - G.vc;
    float D[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        X[a] = fmaf(dv, V.qv[a], fmaf(du, V.qu[a], V.ref[a]));
        D[a] = fmaf(dv, V.qv[a], fmaf(du, V.qu[a], V.dref[a]));
    }
    const float m0 = D[0] * G.vox[0], m1 = D[1] * G.vox[1], m2 = D[2] * G.vox[2];
    len = sqrtf(fmaf(m0, m0, fmaf(m1, m1, m2 * m2)));
    const float il = 1.0f / len;
    dg[0] = D[0] * il;
    dg[1] = D[1] * il;
    dg[2] = D[2] * il;
}

// Samples of the clipped segment [t0, t1] (truncated-midpoint rule).
__device__ __forceinline__ void finish_ray(const Grid &G, const float X[3], const float dg[3], float t0, float t1,
                                           Ray &R)
{
    const float step = G.step_mm;
    const float L = t1 - t0;
    int K = (int)ceilf(L / step);
    if (K < 1) K = 1;
    const float th = t0 + 0.5f * step;
    const float a_last = fmaf((float)(K - 1), step, t0);
    const float t_last = 0.5f * (a_last + t1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        R.g0[a] = fmaf(th, dg[a], X[a]);
        R.sg[a] = step * dg[a];
        R.g_last[a] = fmaf(t_last, dg[a], X[a]);
    }
    R.w_last = t1 - a_last;
    R.K = K;
}

// Sets up the ray of view parameters V through detector point (u, v).
// Returns false if the half line from the source misses the clip box.  With
// an offset off, the sample positions come out as index coordinates minus
// off (the clip itself is unchanged): for off = the integer grid centre they
// are formed at magnitudes up to n / 2, which halves their rounding.
__device__ __forceinline__ bool setup_ray(const Grid &G, const ViewGPU &V, float u, float v, Ray &R,
                                          const float *off = nullptr)
{
    float X[3], dg[3], len;
    ray_line(G, V, u, v, X, dg, len);
    float t0 = -len, t1 = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dg[a] != 0.0f) {
            const float inv = 1.0f / dg[a];
            const float ta = (G.lo[a] - X[a]) * inv, tb = (G.hi[a] - X[a]) * inv;
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        } else if (X[a] < G.lo[a] || X[a] > G.hi[a]) {
            return false;
        }
    }
    if (!(t1 > t0)) return false;
    if (off) {
        const float Xo[3] = {X[0] - off[0], X[1] - off[1], X[2] - off[2]};
        finish_ray(G, Xo, dg, t0, t1, R);
    } else {
        finish_ray(G, X, dg, t0, t1, R);
    }
    return true;
}

// Samples k of the interior range [ka, kb) have every trilinear tap inside the
// grid: g0 + k sg in [eps, n - 1 - eps] on each axis, with a margin eps far
// above the rounding of the sample positions, so the short path is exact.
__device__ __forceinline__ void interior_range(const Grid &G, const Ray &R, int &ka, int &kb)
{
    const float eps = 1e-2f;
    const int n[3] = {G.nx, G.ny, G.nz};
    float lo = 0.0f, hi = (float)(R.K - 1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float l = eps, h = (float)(n[a] - 1) - eps;
        if (R.sg[a] != 0.0f) {
            const float inv = 1.0f / R.sg[a];
            const float t0 = (l - R.g0[a]) * inv, t1 = (h - R.g0[a]) * inv;
            lo = fmaxf(lo, fminf(t0, t1));
            hi = fminf(hi, fmaxf(t0, t1));
        } else if (!(R.g0[a] >= l && R.g0[a] <= h)) {
            hi = -1.0f;
        }
    }
    ka = (int)ceilf(lo);
    kb = (int)floorf(hi) + 1;
    // keep one sample of rounding slack on each side in the exact path
    ka = min(max(ka + 1, 0), R.K - 1);
    kb = max(min(kb - 1, R.K - 1), ka);
}

// Zero-padded trilinear interpolation at index coordinate g (reading: taps
// outside [0, n-1] contribute nothing).  wsum receives the summed weight of
// the in-range taps (the interpolant of an all-ones volume, for row sums).
template <typename TV>
__device__ __forceinline__ float trilinear(const TV *__restrict__ vol, int nx, int ny, int nz,
                                           float gx, float gy, float gz, float &wsum)
{
    const float fx = floorf(gx), fy = floorf(gy), fz = floorf(gz);
    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    const float ax = gx - fx, ay = gy - fy, az = gz - fz;
    const float wx0 = ((unsigned)ix < (unsigned)nx) ? 1.0f - ax : 0.0f;
    const float wx1 = ((unsigned)(ix + 1) < (unsigned)nx) ? ax : 0.0f;
    const float wy0 = ((unsigned)iy < (unsigned)ny) ? 1.0f - ay : 0.0f;
    const float wy1 = ((unsigned)(iy + 1) < (unsigned)ny) ? ay : 0.0f;
    const float wz0 = ((unsigned)iz < (unsigned)nz) ? 1.0f - az : 0.0f;
    const float wz1 = ((unsigned)(iz + 1) < (unsigned)nz) ? az : 0.0f;
    const int x0 = min(max(ix, 0), nx - 1), x1 = min(max(ix + 1, 0), nx - 1);
    const int y0 = min(max(iy, 0), ny - 1), y1 = min(max(iy + 1, 0), ny - 1);
    const int z0 = min(max(iz, 0), nz - 1), z1 = min(max(iz + 1, 0), nz - 1);
    const TV *r00 = vol + (z0 * ny + y0) * nx;
    const TV *r01 = vol + (z0 * ny + y1) * nx;
    const TV *r10 = vol + (z1 * ny + y0) * nx;
    const TV *r11 = vol + (z1 * ny + y1) * nx;
    const float v000 = Storage<TV>::load(r00 + x0), v001 = Storage<TV>::load(r00 + x1);
    const float v010 = Storage<TV>::load(r01 + x0), v011 = Storage<TV>::load(r01 + x1);
    const float v100 = Storage<TV>::load(r10 + x0), v101 = Storage<TV>::load(r10 + x1);
    const float v110 = Storage<TV>::load(r11 + x0), v111 = Storage<TV>::load(r11 + x1);
    const float c00 = fmaf(wx0, v000, wx1 * v001), c01 = fmaf(wx0, v010, wx1 * v011);
    const float c10 = fmaf(wx0, v100, wx1 * v101), c11 = fmaf(wx0, v110, wx1 * v111);
    const float c0 = fmaf(wy0, c00, wy1 * c01), c1 = fmaf(wy0, c10, wy1 * c11);
    wsum = (wx0 + wx1) * (wy0 + wy1) * (wz0 + wz1);
    return fmaf(wz0, c0, wz1 * c1);
}

// Uniform cubic B-spline weights of control points i0-1 .. i0+2 at fractional
// offset f in [0, 1) (i0 = floor of the spline coordinate), and derivatives.
__device__ __forceinline__ void bspline_weights(float f, float w[4])
{
    const float f2 = f * f, f3 = f2 * f, g = 1.0f - f;
    w[0] = g * g * g * (1.0f / 6.0f);
    w[1] = fmaf(0.5f, f3, fmaf(-1.0f, f2, 2.0f / 3.0f));
    w[2] = fmaf(-0.5f, f3, fmaf(0.5f, f2, fmaf(0.5f, f, 1.0f / 6.0f)));
    w[3] = f3 * (1.0f / 6.0f);
}

__device__ __forceinline__ void bspline_dweights(float f, float d[4])
{
    const float f2 = f * f, g = 1.0f - f;
    d[0] = -0.5f * g * g;
    d[1] = fmaf(1.5f, f2, -2.0f * f);
    d[2] = fmaf(-1.5f, f2, fmaf(1.0f, f, 0.5f));
    d[3] = 0.5f * f2;
}

// Spline coordinate of index coordinate gp along one axis (clamped to [1, 6]);
// i0 in [1, 6], f in [0, 1); `active` is false where the clamp holds.
__device__ __forceinline__ void spline_coord(float gp, float scale, int &i0, float &f, bool &active)
{
    float xi = fmaf(gp + 0.5f, scale, 1.0f);
    active = (xi > 1.0f) && (xi < 6.0f);
    xi = fminf(fmaxf(xi, 1.0f), 6.0f);
    const float fl = floorf(xi);
    i0 = (int)fl;
    f = xi - fl;
}

// Pixel of this thread in a 32 x 4 pixel CTA tile.  Row layout: warp w is
// detector row w of the tile.  Patch layout (the motion kernels): warp w is
// the 8 x 4 pixel patch at columns 8w .. 8w + 7, so a warp's samples lie
// closer together and more often in one spline cell, whose coefficient
// loads are then shared by the warp.
template <bool PATCH>
__device__ __forceinline__ void tile_pixel(int tile_u0, int tile_v0, int &iu, int &iv)
{
    if (PATCH) {
        const int tid = threadIdx.y * 32 + threadIdx.x;
        const int w = tid >> 5, l = tid & 31;
        iu = tile_u0 + 8 * w + (l & 7);
        iv = tile_v0 + (l >> 3);
    } else {
        iu = tile_u0 + threadIdx.x;
        iv = tile_v0 + threadIdx.y;
    }
}

// Shared-memory copy of the [8][8][8][3] B-spline coefficients as float4
// (one vector load each), zero-padded to 9 x 9 x 9: the 4 x 4 x 4 support of
// spline cell i0 (i0 in [1, 6] per axis) spans control points i0 - 1 ..
// i0 + 2, at most 8, so no index needs clamping; a point 8 is reached only
// at spline coordinate 6 exactly, where its weight (cubic piece 3 at
// fraction 0) is zero.  Tap (i, j, k) of the cell is base[k * 81 + j * 9 + i]
// with base = coef_cell(coef, i0): constant offsets from one address.
constexpr int CPAD = 9;
constexpr int NCOEF_PAD = CPAD * CPAD * CPAD;

__device__ __forceinline__ void load_coef_padded(float4 *__restrict__ s, const float *__restrict__ coef_g, int tid,
                                                 int nthreads)
{
    for (int i = tid; i < NCOEF_PAD; i += nthreads) {
        const int cx = i % CPAD, cy = (i / CPAD) % CPAD, cz = i / (CPAD * CPAD);
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (cx < 8 && cy < 8 && cz < 8) {
            const float *c = coef_g + 3 * ((cz * 8 + cy) * 8 + cx);
            v = make_float4(c[0], c[1], c[2], 0.0f);
        }
        s[i] = v;
    }
}

__device__ __forceinline__ const float4 *coef_cell(const float4 *coef, const int i0[3])
{
    return coef + ((i0[2] - 1) * CPAD + (i0[1] - 1)) * CPAD + (i0[0] - 1);
}

// Integer grid centre c = floor((n - 1) / 2) per axis (index coordinates).
__device__ __forceinline__ void grid_centre(const Grid &G, float c[3])
{
    c[0] = (float)((G.nx - 1) >> 1);
    c[1] = (float)((G.ny - 1) >> 1);
    c[2] = (float)((G.nz - 1) >> 1);
}

// Warp of one sample (Sec. 2.2.2 pose, then Sec. 3.1 displacement), in
// coordinates centred on the integer grid centre c: gc = g - c in (g index
// coordinates), yc = y - c out, with y = M g + b + s u(M g + b).  It runs as
// yc = gc + (D gc + bc + s u) with gc = g - c, D = M - I, bc = M c + b - c:
// the bracket is a displacement of a few voxels for a near-identity pose,
// so its roundings are small, and only the last addition rounds at the
// magnitude of the coordinate (up to n / 2).  Since c is an integer, floor
// and fraction of y follow exactly from yc.  coef: the padded shared-memory
// copy of the coefficients in voxels (load_coef_padded), or nullptr.
__device__ __forceinline__ void warp_sample_c(const Grid &G, const MotionGPU &m, const float4 *coef, const float gc[3],
                                              float yc[3])
{
    float c[3];
    grid_centre(G, c);
    float d[3];  // displacement D gc + bc (+ s u below)
#pragma unroll
    for (int r = 0; r < 3; ++r)
        d[r] = fmaf(m.D[3 * r], gc[0], fmaf(m.D[3 * r + 1], gc[1], fmaf(m.D[3 * r + 2], gc[2], m.bc[r])));
    float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
    if (coef != nullptr && m.s != 0.0f) {
        int i0[3];
        float f[3], wx[4], wy[4], wz[4];
        bool act[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) spline_coord(gc[a] + d[a] + c[a], G.spl_scale[a], i0[a], f[a], act[a]);
        bspline_weights(f[0], wx);
        bspline_weights(f[1], wy);
        bspline_weights(f[2], wz);
        const float4 *base = coef_cell(coef, i0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float wyz = wz[k] * wy[j];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float wt = wyz * wx[i];
                    const float4 cf = base[k * CPAD * CPAD + j * CPAD + i];
                    u0 = fmaf(wt, cf.x, u0);
                    u1 = fmaf(wt, cf.y, u1);
                    u2 = fmaf(wt, cf.z, u2);
                }
            }
        }
    }
    yc[0] = gc[0] + fmaf(m.s, u0, d[0]);
    yc[1] = gc[1] + fmaf(m.s, u1, d[1]);
    yc[2] = gc[2] + fmaf(m.s, u2, d[2]);
}

// The same warp in plain index coordinates, as the forward projector uses it:
// y = M g + b + s u(M g + b) formed directly (fewer operations; the forward
// averages the position rounding out along the ray, so it needs no centring).
__device__ __forceinline__ void warp_sample(const Grid &G, const MotionGPU &m, const float4 *coef, const float g[3],
                                            float y[3])
{
    float gp[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        gp[r] = fmaf(m.M[3 * r], g[0], fmaf(m.M[3 * r + 1], g[1], fmaf(m.M[3 * r + 2], g[2], m.b[r])));
    float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
    if (coef != nullptr && m.s != 0.0f) {
        int i0[3];
        float f[3], wx[4], wy[4], wz[4];
        bool act[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) spline_coord(gp[a], G.spl_scale[a], i0[a], f[a], act[a]);
        bspline_weights(f[0], wx);
        bspline_weights(f[1], wy);
        bspline_weights(f[2], wz);
        const float4 *base = coef_cell(coef, i0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float wyz = wz[k] * wy[j];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float wt = wyz * wx[i];
                    const float4 cf = base[k * CPAD * CPAD + j * CPAD + i];
                    u0 = fmaf(wt, cf.x, u0);
                    u1 = fmaf(wt, cf.y, u1);
                    u2 = fmaf(wt, cf.z, u2);
                }
            }
        }
    }
    y[0] = fmaf(m.s, u0, gp[0]);
    y[1] = fmaf(m.s, u1, gp[1]);
    y[2] = fmaf(m.s, u2, gp[2]);
}

}  // namespace ctrex

// cylinder.cuh -- the aligned cylindrical domain (Sec. 3.5; projector and
// backprojector adaptations of Sec. 4.2 / 4.3): bounding-cylinder clip,
// cylinder-frame -> (r, phi, z) index mapping of samples, and the frame
// position of a voxel for the backprojector.
//
// Ray and voxel positions are in the cylinder frame (mm): the context folds
// the domain's rigid pose into the per-view matrices, so a ray arrives in
// frame coordinates and only the coordinate mapping differs from the
// Cartesian kernels.
//
// Volume layout: [N_z][N_phi][N_r] (r fastest), uploaded as z-slice tiles of
// N_r x (N_phi + 1) texels whose last row repeats sector 0, so the two
// sectors of every bilinear footprint (j, j + 1 mod N_phi) sit in one tile.
#pragma once

#include "atlas.cuh"
#include "ray.cuh"

namespace ctrex {

// Clips the line of V through (u, v) to the bounding cylinder r <= R,
// |z| <= Z (frame coordinates) and sets up its samples.  Returns false if
// the half line from the source misses it.
__device__ __forceinline__ bool setup_ray_cyl(const Grid &G, const CylGPU &C, const ViewGPU &V, float u, float v,
                                              Ray &R)
{
    float X[3], dg[3], len;
    ray_line(G, V, u, v, X, dg, len);
    float t0 = -len, t1 = INFINITY;
    // mantle: |X_xy + t dg_xy|^2 <= R^2, i.e. a t^2 + 2 b t + c <= 0
    const float a = fmaf(dg[0], dg[0], dg[1] * dg[1]);
    const float b = fmaf(X[0], dg[0], X[1] * dg[1]);
    const float c = fmaf(X[0], X[0], fmaf(X[1], X[1], -C.R * C.R));
    if (a > 0.0f) {
        const float disc = fmaf(b, b, -a * c);
        if (!(disc > 0.0f)) return false;
        // roots without cancellation: q = -(b + sign(b) sqrt(disc)); t = q / a and c / q
        const float q = -(b + copysignf(sqrtf(disc), b));
        float ta = q / a, tb = (q != 0.0f) ? c / q : -ta;
        if (ta > tb) {
            const float tmp = ta;
            ta = tb;
            tb = tmp;
        }
        t0 = fmaxf(t0, ta);
        t1 = fminf(t1, tb);
    } else if (c > 0.0f) {
        return false;
    }
    // end caps
    if (dg[2] != 0.0f) {
        const float inv = 1.0f / dg[2];
        const float ta = (-C.Z - X[2]) * inv, tb = (C.Z - X[2]) * inv;
        t0 = fmaxf(t0, fminf(ta, tb));
        t1 = fminf(t1, fmaxf(ta, tb));
    } else if (X[2] < -C.Z || X[2] > C.Z) {
        return false;
    }
    if (!(t1 > t0)) return false;
    finish_ray(G, X, dg, t0, t1, R);
    return true;
}

// Angle of (x, y) in [-pi, pi]: octant reduction to z = min/max in [0, 1],
// atan(z) ~ z P(z^2) with P of degree 7 (coefficients fitted by weighted
// least squares at Chebyshev nodes, refined by Lawson passes toward the
// minimax fit: csrc/fit_atan.py; FP32 error below 2e-7 rad), then the octant
// restored.  The quotient uses the hardware reciprocal plus one Newton step.
__device__ __forceinline__ float cyl_angle(float x, float y)
{
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(mx));
    const float z = mx > 0.0f ? mn * (r0 * fmaf(-mx, r0, 2.0f)) : 0.0f;
    const float t = z * z;
    float p = -4.693705589e-03f;
    p = fmaf(p, t, 2.425401658e-02f);
    p = fmaf(p, t, -5.948881805e-02f);
    p = fmaf(p, t, 9.914478660e-02f);
    p = fmaf(p, t, -1.401955634e-01f);
    p = fmaf(p, t, 1.996974051e-01f);
    p = fmaf(p, t, -3.333199322e-01f);
    p = fmaf(p, t, 9.999998808e-01f);
    float a = p * z;
    if (ay > ax) a = 1.57079632679f - a;
    if (x < 0.0f) a = 3.14159265359f - a;
    return copysignf(a, y);
}

// Trilinear interpolation on the cylindrical grid at frame point (qx, qy,
// qz): r clamped at the first ring centre, phi periodic, zero outside in r
// and z.  Two gathers per sample, FP32 weights.
struct CylSampler {
    AtlasSampler base;  // atlas and its per-CTA tile-origin table
    CylGPU C;
    static constexpr int TILE_TABLE = AtlasSampler::TILE_TABLE;
    static constexpr bool CYLINDER = true;
    static constexpr bool JOSEPH = false;
    static constexpr bool ROI = false;
    static constexpr bool DYRECT = false;
    static constexpr int MIN_BLOCKS = 0;  // 0: the shared forward kernel entry

    __device__ __forceinline__ void bind(float2 *table, int tid, int nthreads) { base.bind(table, tid, nthreads); }

    __device__ __forceinline__ float operator()(float qx, float qy, float qz, float &wsum) const
    {
        const float nphi = (float)C.n_phi;
        const float q2 = fmaf(qx, qx, qy * qy);
        const float r = q2 > 0.0f ? q2 * rsqrtf(q2) : 0.0f;
        float gp = fmaf(cyl_angle(qx, qy), C.inv_dphi, -0.5f);
        if (gp < 0.0f) gp += nphi;
        if (gp >= nphi) gp -= nphi;  // -tiny + N_phi rounded up to N_phi
        const float gr = fmaxf(fmaf(r, C.inv_dr, -0.5f), 0.0f);
        const float gz = fmaf(qz, C.inv_dz, C.zc);
        const float fr = floorf(gr), fp = floorf(gp), fz = floorf(gz);
        const int ir = (int)fr, ip = (int)fp, iz = (int)fz;
        const float ar = gr - fr, ap = gp - fp, az = gz - fz;
        const float wr0 = ir < C.n_r ? 1.0f - ar : 0.0f;
        const float wr1 = ir + 1 < C.n_r ? ar : 0.0f;
        const float wz0 = ((unsigned)iz < (unsigned)C.n_z) ? 1.0f - az : 0.0f;
        const float wz1 = ((unsigned)(iz + 1) < (unsigned)C.n_z) ? az : 0.0f;
        const int x0 = min(ir, C.n_r - 1);
        const int y0 = min(max(ip, 0), C.n_phi - 1);
        const Atlas &A = base.A;
        float a00, a10, a01, a11, b00, b10, b01, b11;
        const float2 o0 = base.origin(min(max(iz, 0), C.n_z - 1));
        const float2 o1 = base.origin(min(max(iz + 1, 0), C.n_z - 1));
        atlas_quad_at(A, o0.x + (float)x0, o0.y + (float)y0, a00, a10, a01, a11);
        atlas_quad_at(A, o1.x + (float)x0, o1.y + (float)y0, b00, b10, b01, b11);
        const float wp0 = 1.0f - ap, wp1 = ap;
        const float c0 = fmaf(wp0, fmaf(wr0, a00, wr1 * a10), wp1 * fmaf(wr0, a01, wr1 * a11));
        const float c1 = fmaf(wp0, fmaf(wr0, b00, wr1 * b10), wp1 * fmaf(wr0, b01, wr1 * b11));
        wsum = (wr0 + wr1) * (wz0 + wz1);
        return fmaf(wz0, c0, wz1 * c1);
    }
    // no interior short path: the mapping is not linear along the ray
    __device__ __forceinline__ float interior(float qx, float qy, float qz) const
    {
        float ws;
        return (*this)(qx, qy, qz, ws);
    }
};

// Frame position of the cylindrical voxel point at index coordinates
// (gr, gp, gz) (voxel centres at integers): r = (gr + 1/2) dr, phi = (gp +
// 1/2) dphi, z = (gz - zc) dz.
__device__ __forceinline__ void cyl_point(const CylGPU &C, float gr, float gp, float gz, float &x, float &y, float &z)
{
    const float r = (gr + 0.5f) * C.dr;
    float s, c;
    sincosf((gp + 0.5f) * C.dphi, &s, &c);
    x = r * c;
    y = r * s;
    z = (gz - C.zc) * C.dz;
}

}  // namespace ctrex

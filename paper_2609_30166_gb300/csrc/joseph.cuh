// joseph.cuh -- the classical Joseph projector (Sec. 4.1 cites Joseph's
// method; this is its slice-stepping form): a ray steps through the slices
// of its principal axis (the index coordinate that changes fastest along
// it), interpolates each slice bilinearly at the crossing (zero outside the
// grid), and weights every slice with the path length between neighbouring
// slice planes.
//
// Layout: one texture atlas holds the volume three times, as x-slices
// (tiles of ny x nz texels, (y, z)), y-slices ((x, z)) and z-slices ((x, y)),
// in tiles of W x H = max widths x max heights, so that every sample is one
// tex2Dgather of a 2x2 footprint whatever the ray's principal axis.  Tile t
// of stack m is t = tbase[m] + k.
#pragma once

#include "atlas.cuh"
#include "ray.cuh"

namespace ctrex {

struct JosephSampler {
    AtlasSampler base;  // the three-stack atlas and its per-CTA tile-origin table
    int n[3];           // nx, ny, nz
    int tbase[3];       // first tile of the x-, y- and z-slice stacks
    static constexpr int TILE_TABLE = AtlasSampler::TILE_TABLE;
    static constexpr bool CYLINDER = false;
    static constexpr bool JOSEPH = true;
    static constexpr bool ROI = false;
    static constexpr bool DYRECT = false;
    static constexpr int MIN_BLOCKS = 0;  // 0: the shared forward kernel entry

    __device__ __forceinline__ void bind(float2 *table, int tid, int nthreads) { base.bind(table, tid, nthreads); }
    // unused: the Joseph path never samples trilinearly
    __device__ __forceinline__ float operator()(float, float, float, float &ws) const
    {
        ws = 0.0f;
        return 0.0f;
    }
    __device__ __forceinline__ float interior(float, float, float) const { return 0.0f; }
};

// One ray in slice form: crossing of slice k at in-slice coordinates
// (p0 + k r1, q0 + k r2) of axes (a1, a2); slices [klo, khi] have a tap
// inside the grid; [kmin, kmax] are the slices of the grid in front of the
// source; dl = path length between neighbouring planes (mm).
struct JRay {
    float p0, q0, r1, r2, dl;
    int m, klo, khi, kmin, kmax;
};

// The two in-slice axes of principal axis m, in order.
__device__ __forceinline__ void joseph_axes(int m, int &a1, int &a2)
{
    a1 = m == 0 ? 1 : 0;
    a2 = m == 2 ? 1 : 2;
}

// Component i of a 3-vector by selects (no local-memory indexing).
__device__ __forceinline__ float jsel(const float v[3], int i) { return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]); }
__device__ __forceinline__ int jsel(int a, int b, int c, int i) { return i == 0 ? a : (i == 1 ? b : c); }

// Returns false if no slice crossing in front of the source has a tap
// inside the grid.
__device__ __forceinline__ bool joseph_setup(const Grid &G, const ViewGPU &V, float u, float v, JRay &J)
{
    float X[3], dg[3], len;
    ray_line(G, V, u, v, X, dg, len);
    int m = 0;
    if (fabsf(dg[1]) > fabsf(dg[m])) m = 1;
    if (fabsf(dg[2]) > fabsf(dg[m])) m = 2;
    int a1, a2;
    joseph_axes(m, a1, a2);
    const float dm = jsel(dg, m), Xm = jsel(X, m);
    const float inv = 1.0f / dm;  // mm per index unit along m (signed)
    J.m = m;
    J.dl = fabsf(inv);
    J.r1 = jsel(dg, a1) * inv;
    J.r2 = jsel(dg, a2) * inv;
    J.p0 = fmaf(-Xm, J.r1, jsel(X, a1));
    J.q0 = fmaf(-Xm, J.r2, jsel(X, a2));
    const int nm = jsel(G.nx, G.ny, G.nz, m), n1 = jsel(G.nx, G.ny, G.nz, a1), n2 = jsel(G.nx, G.ny, G.nz, a2);
    // closed bounds: the grid's slices, in front of the source (t >= -len)
    const float ksrc = fmaf(-len, dm, Xm);
    J.kmin = 0;
    J.kmax = nm - 1;
    if (inv > 0.0f)
        J.kmin = max(J.kmin, (int)ceilf(fmaxf(ksrc, -1.0f)));
    else
        J.kmax = min(J.kmax, (int)floorf(fminf(ksrc, (float)nm)));
    // open bounds: both in-slice coordinates in (-1, n_a)
    float lo = -INFINITY, hi = INFINITY;
    if (J.r1 != 0.0f) {
        const float ri = 1.0f / J.r1;
        const float ka = (-1.0f - J.p0) * ri, kb = ((float)n1 - J.p0) * ri;
        lo = fmaxf(lo, fminf(ka, kb));
        hi = fminf(hi, fmaxf(ka, kb));
    } else if (!(J.p0 > -1.0f && J.p0 < (float)n1)) {
        return false;
    }
    if (J.r2 != 0.0f) {
        const float ri = 1.0f / J.r2;
        const float ka = (-1.0f - J.q0) * ri, kb = ((float)n2 - J.q0) * ri;
        lo = fmaxf(lo, fminf(ka, kb));
        hi = fminf(hi, fmaxf(ka, kb));
    } else if (!(J.q0 > -1.0f && J.q0 < (float)n2)) {
        return false;
    }
    lo = fmaxf(lo, (float)J.kmin - 1.0f);  // keep the floats in int range
    hi = fminf(hi, (float)J.kmax + 1.0f);
    J.klo = max((int)floorf(lo) + 1, J.kmin);
    J.khi = min((int)ceilf(hi) - 1, J.kmax);
    return J.khi >= J.klo;
}

// Line integral and row sum of one ray.  The loop runs one slice past each
// end of the range (within the grid, in front of the source): the rounding
// of the range can move its ends by a slice, and a slice without taps inside
// the grid adds exactly zero.
__device__ __forceinline__ void joseph_integral(const Grid &G, const JosephSampler &smp, const ViewGPU &V, float u,
                                                float v, float &val, float &rs)
{
    val = 0.0f;
    rs = 0.0f;
    JRay J;
    if (!joseph_setup(G, V, u, v, J)) return;
    int a1, a2;
    joseph_axes(J.m, a1, a2);
    const int n1 = jsel(smp.n[0], smp.n[1], smp.n[2], a1), n2 = jsel(smp.n[0], smp.n[1], smp.n[2], a2);
    const int k0 = max(J.klo - 1, J.kmin), k1 = min(J.khi + 1, J.kmax);
    const int tb = jsel(smp.tbase[0], smp.tbase[1], smp.tbase[2], J.m);
    const Atlas &A = smp.base.A;
    float acc = 0.0f, wacc = 0.0f;
    // unrolled so that several independent gathers are in flight per thread
#pragma unroll 4
    for (int k = k0; k <= k1; ++k) {
        const float p = fmaf((float)k, J.r1, J.p0), q = fmaf((float)k, J.r2, J.q0);
        const float fp = floorf(p), fq = floorf(q);
        const int ip = (int)fp, iq = (int)fq;
        const float ap = p - fp, aq = q - fq;
        const float wp0 = ((unsigned)ip < (unsigned)n1) ? 1.0f - ap : 0.0f;
        const float wp1 = ((unsigned)(ip + 1) < (unsigned)n1) ? ap : 0.0f;
        const float wq0 = ((unsigned)iq < (unsigned)n2) ? 1.0f - aq : 0.0f;
        const float wq1 = ((unsigned)(iq + 1) < (unsigned)n2) ? aq : 0.0f;
        const float2 o = smp.base.origin(tb + k);
        const float x0 = fminf(fmaxf(fp, -1.0f), (float)(A.w - 1));
        const float y0 = fminf(fmaxf(fq, -1.0f), (float)(A.h - 1));
        float c00, c10, c01, c11;
        atlas_quad_at(A, o.x + x0, o.y + y0, c00, c10, c01, c11);
        acc += fmaf(wq0, fmaf(wp0, c00, wp1 * c10), wq1 * fmaf(wp0, c01, wp1 * c11));
        wacc += (wp0 + wp1) * (wq0 + wq1);
    }
    val = acc * J.dl;
    rs = wacc * J.dl;
}

}  // namespace ctrex

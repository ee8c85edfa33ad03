// backproject.cu -- voxel-driven backprojection with voxel weights, column-sum
// normalisation C and relaxation alpha (Sec. 4.1 "Backprojection operator",
// Sec. 4.3.2 weighted backprojection, Eq. (1) term 3).
//
// One thread per voxel, 32 x 4 x 2 voxels per CTA (x fastest, so a warp's
// voxels project onto neighbouring detector columns).  The per-view matrices
// are staged through shared memory in chunks; every thread walks the same
// view sequence, so the residual images are read view after view by all
// resident CTAs at once (one image band at a time sits in L2).  Grid order
// is x, y, then z: the CTAs resident together cover a z-slab of the volume,
// whose detector footprint over all views is a band of rows.
#include "atlas.cuh"
#include "ctrex_internal.cuh"
#include "cylinder.cuh"

namespace ctrex {

constexpr int BP_TX = 32, BP_TY = 4, BP_TZ = 2;
constexpr int BP_VZ = 2;  // voxels per thread along z (consecutive slices)
constexpr int BP_THREADS = BP_TX * BP_TY * BP_TZ;
constexpr int BP_CHUNK = 128;
#ifndef CTREX_BP_MIN_BLOCKS
#define CTREX_BP_MIN_BLOCKS 8  // CTAs per SM the register budget is sized for (full occupancy)
#endif
#ifndef CTREX_BP_UNROLL
#define CTREX_BP_UNROLL 2  // views per unrolled step of the view loop (2 measured fastest)
#endif
constexpr int BP_UNROLL = CTREX_BP_UNROLL;
#ifndef CTREX_BP_SUBV_MIN_BLOCKS
#define CTREX_BP_SUBV_MIN_BLOCKS 5  // the same for the sub-voxel variant (48 registers)
#endif
#ifndef CTREX_BP_DYR_MIN_BLOCKS
#define CTREX_BP_DYR_MIN_BLOCKS 5  // the event-model variant: eight accumulators (48 registers)
#endif

// Bilinear sample of one correction image at (u, v) = (iu + au, iv + av),
// zero outside the detector (taps outside get zero weight).  A Slot holds what
// a view's image needs (its base pointer or atlas tile origin); slots are
// computed once per view and staged in shared memory with the matrices.
template <typename TR>
struct LinearImages {
    const TR *r;
    int nu, nv;
    typedef const TR *Slot;
    __device__ __forceinline__ Slot slot(int k) const { return r + (size_t)k * nu * nv; }
    __device__ __forceinline__ float operator()(Slot img, int iu, int iv, float, float, float wu0, float wu1,
                                                float wv0, float wv1) const
    {
        const int u0 = max(iu, 0), u1 = min(iu + 1, nu - 1);
        const int v0 = max(iv, 0), v1 = min(iv + 1, nv - 1);
        const float r00 = Storage<TR>::load(img + v0 * nu + u0);
        const float r01 = Storage<TR>::load(img + v0 * nu + u1);
        const float r10 = Storage<TR>::load(img + v1 * nu + u0);
        const float r11 = Storage<TR>::load(img + v1 * nu + u1);
        return fmaf(wv0, fmaf(wu0, r00, wu1 * r01), wv1 * fmaf(wu0, r10, wu1 * r11));
    }
};

// The same sample from a texture atlas of the images: one gather, addressed
// at the footprint's shared corner (tile origin + floor(u) + 1, ...).
struct AtlasImages {
    Atlas A;
    typedef float2 Slot;
    __device__ __forceinline__ Slot slot(int k) const
    {
        k = min(max(k, 0), A.n - 1);
        return make_float2((float)((k & ((1 << A.tshift) - 1)) * A.w) + 1.0f, (float)((k >> A.tshift) * A.h) + 1.0f);
    }
    __device__ __forceinline__ float operator()(Slot o, int, int, float fu, float fv, float wu0, float wu1,
                                                float wv0, float wv1) const
    {
        float c00, c10, c01, c11;
        if (A.bf16) {
            const ushort4 q = tex2Dgather<ushort4>(A.tex, o.x + fu, o.y + fv, 0);
            c01 = __uint_as_float((unsigned)q.x << 16);
            c11 = __uint_as_float((unsigned)q.y << 16);
            c10 = __uint_as_float((unsigned)q.z << 16);
            c00 = __uint_as_float((unsigned)q.w << 16);
        } else {
            const float4 q = tex2Dgather<float4>(A.tex, o.x + fu, o.y + fv, 0);
            c01 = q.x;
            c11 = q.y;
            c10 = q.z;
            c00 = q.w;
        }
        return fmaf(wv0, fmaf(wu0, c00, wu1 * c10), wv1 * fmaf(wu0, c01, wu1 * c11));
    }
};

// 1/x: the hardware approximation refined by one Newton-Raphson step
// r1 = r0 (2 - x r0), which roughly doubles its correct bits.
__device__ __forceinline__ float recip(float x)
{
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(x));
    return r0 * fmaf(-x, r0, 2.0f);
}

// One voxel-view term: bilinear sample of the view's correction image at the
// projection (h1/h3, h2/h3) of the voxel centre, accumulated into b, and the
// in-range weight into c.  Taps outside the window [lo.x, hi.x] x [lo.y,
// hi.y] (the detector, or a per-view backprojection window) count as off the
// detector.  Projections whose four taps are all inside (the common case)
// take the short path: plain weights and c += 1.
template <typename Images>
__device__ __forceinline__ void bp_term(const Images &img, const typename Images::Slot &slot, float h1, float h2,
                                        float h3, float2 lo, float2 hi, float &b, float &c)
{
    if (!(h3 > 0.0f)) return;
    const float inv = recip(h3);
    const float u = h1 * inv, v = h2 * inv;
    const float fu = floorf(u), fv = floorf(v);
    const float au = u - fu, av = v - fv;
    if (u >= lo.x && u <= hi.x && v >= lo.y && v <= hi.y) {
        b += img(slot, (int)fu, (int)fv, fu, fv, 1.0f - au, au, 1.0f - av, av);
        c += 1.0f;
    } else if (u > lo.x - 1.0f && u < hi.x + 1.0f && v > lo.y - 1.0f && v < hi.y + 1.0f) {
        const float wu0 = fu >= lo.x ? 1.0f - au : 0.0f;
        const float wu1 = fu + 1.0f <= hi.x ? au : 0.0f;
        const float wv0 = fv >= lo.y ? 1.0f - av : 0.0f;
        const float wv1 = fv + 1.0f <= hi.y ? av : 0.0f;
        b += img(slot, (int)fu, (int)fv, fu, fv, wu0, wu1, wv0, wv1);
        c += (wu0 + wu1) * (wv0 + wv1);
    }
}

// SUBV: sub-voxel backprojection (Sec. 4.3.2, motion blur).  Each voxel's b
// and c are the means over sv^3 points at index offsets ((a + 1/2)/sv - 1/2)
// per axis; the points are visited inside the view loop, so the finer grid
// lives only in registers.  Its longer loop body gets a larger register
// budget (fewer resident CTAs per SM).
// CYL: the aligned cylindrical domain (Sec. 3.5): voxel (ix, iy, iz) is ring
// ix, sector iy, slice iz; its point is mapped to the cylinder frame (the
// frame the view matrices are expressed in) before projection, and the z
// neighbour lies dz further along the axis.
template <typename Images, typename TV, bool WINDOW, bool SUBV, bool CYL>
__global__ void __launch_bounds__(BP_THREADS, SUBV ? CTREX_BP_SUBV_MIN_BLOCKS : CTREX_BP_MIN_BLOCKS)
    bp_kernel(Grid G, const ViewGPU *__restrict__ views, const int *__restrict__ view_idx, int n_idx,
              const Images img, const int4 *__restrict__ window, TV *__restrict__ vol, const float *__restrict__ w,
              float alpha, int normalize, int accumulate, int sv, const CylGPU cyl)
{
    __shared__ float4 sP[BP_CHUNK][3];
    __shared__ typename Images::Slot sImg[BP_CHUNK];
    __shared__ float4 sWin[WINDOW ? BP_CHUNK : 1];  // per-view window (u_lo, u_hi, v_lo, v_hi)
    const int tid = (threadIdx.z * BP_TY + threadIdx.y) * BP_TX + threadIdx.x;
    const int ix = blockIdx.x * BP_TX + threadIdx.x;
    const int iy = blockIdx.y * BP_TY + threadIdx.y;
    const int iz = (blockIdx.z * BP_TZ + threadIdx.z) * BP_VZ;  // this thread: slices iz, iz + 1
    const bool inside = ix < G.nx && iy < G.ny && iz < G.nz;
    float fx = (float)ix, fy = (float)iy, fz = (float)iz;
    if (CYL && !SUBV) {
        float x, y, z;
        cyl_point(cyl, fx, fy, fz, x, y, z);
        fx = x;
        fy = y;
        fz = z;
    }
    float2 lo = make_float2(0.0f, 0.0f), hi = make_float2((float)(G.nu - 1), (float)(G.nv - 1));
    float b0 = 0.0f, c0 = 0.0f, b1 = 0.0f, c1 = 0.0f;
    const int total = n_idx * G.n_sub;
    for (int base = 0; base < total; base += BP_CHUNK) {
        const int cnt = min(BP_CHUNK, total - base);
        __syncthreads();
        for (int t = tid; t < cnt; t += BP_THREADS) {
            const int q = base + t;
            const int k = q / G.n_sub, s = q - k * G.n_sub;
            int view = view_idx ? view_idx[k] : k;
            const bool ok = view >= 0 && view < G.n_views;
            if (!ok) view = 0;
            const float *P = views[view * G.n_sub + s].P;
            sP[t][0] = make_float4(P[0], P[1], P[2], P[3]);
            sP[t][1] = make_float4(P[4], P[5], P[6], P[7]);
            // an invalid view index gets a zero depth row: it is skipped
            sP[t][2] = ok ? make_float4(P[8], P[9], P[10], P[11]) : make_float4(0.f, 0.f, 0.f, 0.f);
            sImg[t] = img.slot(k);
            if (WINDOW) {
                const int4 wd = window[view];
                sWin[t] = make_float4((float)wd.x, (float)wd.y, (float)wd.z, (float)wd.w);
            }
        }
        __syncthreads();
        if (!inside) continue;
#pragma unroll BP_UNROLL
        for (int m = 0; m < cnt; ++m) {
            const float4 p0 = sP[m][0], p1 = sP[m][1], p2 = sP[m][2];
            const typename Images::Slot slot = sImg[m];
            if (WINDOW) {
                const float4 wd = sWin[m];
                lo = make_float2(wd.x, wd.z);
                hi = make_float2(wd.y, wd.w);
            }
            if (SUBV) {
                const float d = 1.0f / (float)sv, o = 0.5f * d - 0.5f;
                for (int az = 0; az < sv; ++az) {
                    const float gz = fz + fmaf((float)az, d, o);
                    for (int ay = 0; ay < sv; ++ay) {
                        const float gy = fy + fmaf((float)ay, d, o);
                        float sn = 0.0f, cs = 0.0f;
                        if (CYL) sincosf((gy + 0.5f) * cyl.dphi, &sn, &cs);
                        for (int ax = 0; ax < sv; ++ax) {
                            const float gx = fx + fmaf((float)ax, d, o);
                            float X = gx, Y = gy, Z = gz;
                            if (CYL) {
                                const float r = (gx + 0.5f) * cyl.dr;
                                X = r * cs;
                                Y = r * sn;
                                Z = (gz - cyl.zc) * cyl.dz;
                            }
                            const float h3 = fmaf(p2.x, X, fmaf(p2.y, Y, fmaf(p2.z, Z, p2.w)));
                            const float h1 = fmaf(p0.x, X, fmaf(p0.y, Y, fmaf(p0.z, Z, p0.w)));
                            const float h2 = fmaf(p1.x, X, fmaf(p1.y, Y, fmaf(p1.z, Z, p1.w)));
                            bp_term(img, slot, h1, h2, h3, lo, hi, b0, c0);
                            if (CYL)
                                bp_term(img, slot, fmaf(p0.z, cyl.dz, h1), fmaf(p1.z, cyl.dz, h2),
                                        fmaf(p2.z, cyl.dz, h3), lo, hi, b1, c1);
                            else
                                bp_term(img, slot, h1 + p0.z, h2 + p1.z, h3 + p2.z, lo, hi, b1, c1);
                        }
                    }
                }
                continue;
            }
            // voxel (ix, iy, iz) and its z neighbour: h(z + 1) = h(z) + P[:, 2]
            // (+ dz P[:, 2] on the cylinder, whose matrices act on frame mm)
            const float h3 = fmaf(p2.x, fx, fmaf(p2.y, fy, fmaf(p2.z, fz, p2.w)));
            const float h1 = fmaf(p0.x, fx, fmaf(p0.y, fy, fmaf(p0.z, fz, p0.w)));
            const float h2 = fmaf(p1.x, fx, fmaf(p1.y, fy, fmaf(p1.z, fz, p1.w)));
            bp_term(img, slot, h1, h2, h3, lo, hi, b0, c0);
            if (CYL)
                bp_term(img, slot, fmaf(p0.z, cyl.dz, h1), fmaf(p1.z, cyl.dz, h2), fmaf(p2.z, cyl.dz, h3), lo, hi,
                        b1, c1);
            else
                bp_term(img, slot, h1 + p0.z, h2 + p1.z, h3 + p2.z, lo, hi, b1, c1);
        }
    }
    if (!inside) return;
    const float mean = SUBV ? G.inv_sub / (float)(sv * sv * sv) : G.inv_sub;
#pragma unroll
    for (int q = 0; q < BP_VZ; ++q) {
        if (iz + q >= G.nz) break;
        const float b = (q == 0 ? b0 : b1) * mean;
        const float c = (q == 0 ? c0 : c1) * mean;
        const size_t j = ((size_t)(iz + q) * G.ny + iy) * G.nx + ix;
        float scale = alpha;
        if (normalize) scale *= (c > 1e-6f ? 1.0f / c : 0.0f);
        if (w) scale *= __ldg(w + j);
        const float upd = scale * b;
        const float out = accumulate ? Storage<TV>::load(vol + j) + upd : upd;
        Storage<TV>::store(vol + j, out);
    }
}

// Event-based 4D model (Sec. 3.3): vol (and w) hold mu0 followed by mu1.
// Eq. (1) term 3 splits by the voxel's transition time tau_j: the views
// acquired before tau_j (t_v < tau_j) backproject into mu0_j and the others
// into mu1_j, each part normalised by its own column sum.  Cartesian grid,
// voxel centres, two z-neighbouring voxels per thread as in bp_kernel.
template <typename Images, typename TV, bool WINDOW>
__global__ void __launch_bounds__(BP_THREADS, CTREX_BP_DYR_MIN_BLOCKS)
    bp_dyrect_kernel(Grid G, const ViewGPU *__restrict__ views, const int *__restrict__ view_idx, int n_idx,
                     const Images img, const int4 *__restrict__ window, TV *__restrict__ vol,
                     const float *__restrict__ w, float alpha, int normalize, int accumulate,
                     const float *__restrict__ tau, const float *__restrict__ t_view)
{
    __shared__ float4 sP[BP_CHUNK][3];
    __shared__ typename Images::Slot sImg[BP_CHUNK];
    __shared__ float sT[BP_CHUNK];
    __shared__ float4 sWin[WINDOW ? BP_CHUNK : 1];
    const int tid = (threadIdx.z * BP_TY + threadIdx.y) * BP_TX + threadIdx.x;
    const int ix = blockIdx.x * BP_TX + threadIdx.x;
    const int iy = blockIdx.y * BP_TY + threadIdx.y;
    const int iz = (blockIdx.z * BP_TZ + threadIdx.z) * BP_VZ;
    const bool inside = ix < G.nx && iy < G.ny && iz < G.nz;
    const size_t nvox = (size_t)G.nx * G.ny * G.nz;
    const size_t j0 = ((size_t)iz * G.ny + iy) * G.nx + ix;
    const float tau0 = inside ? __ldg(tau + j0) : 0.0f;
    const float tau1 = inside && iz + 1 < G.nz ? __ldg(tau + j0 + (size_t)G.nx * G.ny) : 0.0f;
    const float fx = (float)ix, fy = (float)iy, fz = (float)iz;
    float2 lo = make_float2(0.0f, 0.0f), hi = make_float2((float)(G.nu - 1), (float)(G.nv - 1));
    // [voxel][part]: part 0 = views before the transition (mu0), 1 = after (mu1)
    float b00 = 0.f, c00 = 0.f, b01 = 0.f, c01 = 0.f, b10 = 0.f, c10 = 0.f, b11 = 0.f, c11 = 0.f;
    const int total = n_idx * G.n_sub;
    for (int base = 0; base < total; base += BP_CHUNK) {
        const int cnt = min(BP_CHUNK, total - base);
        __syncthreads();
        for (int t = tid; t < cnt; t += BP_THREADS) {
            const int q = base + t;
            const int k = q / G.n_sub, s = q - k * G.n_sub;
            int view = view_idx ? view_idx[k] : k;
            const bool ok = view >= 0 && view < G.n_views;
            if (!ok) view = 0;
            const float *P = views[view * G.n_sub + s].P;
            sP[t][0] = make_float4(P[0], P[1], P[2], P[3]);
            sP[t][1] = make_float4(P[4], P[5], P[6], P[7]);
            sP[t][2] = ok ? make_float4(P[8], P[9], P[10], P[11]) : make_float4(0.f, 0.f, 0.f, 0.f);
            sImg[t] = img.slot(k);
            sT[t] = __ldg(t_view + view);
            if (WINDOW) {
                const int4 wd = window[view];
                sWin[t] = make_float4((float)wd.x, (float)wd.y, (float)wd.z, (float)wd.w);
            }
        }
        __syncthreads();
        if (!inside) continue;
#pragma unroll BP_UNROLL
        for (int m = 0; m < cnt; ++m) {
            const float4 p0 = sP[m][0], p1 = sP[m][1], p2 = sP[m][2];
            const typename Images::Slot slot = sImg[m];
            const float tv = sT[m];
            if (WINDOW) {
                const float4 wd = sWin[m];
                lo = make_float2(wd.x, wd.z);
                hi = make_float2(wd.y, wd.w);
            }
            const float h3 = fmaf(p2.x, fx, fmaf(p2.y, fy, fmaf(p2.z, fz, p2.w)));
            const float h1 = fmaf(p0.x, fx, fmaf(p0.y, fy, fmaf(p0.z, fz, p0.w)));
            const float h2 = fmaf(p1.x, fx, fmaf(p1.y, fy, fmaf(p1.z, fz, p1.w)));
            float tb = 0.0f, tc = 0.0f;
            bp_term(img, slot, h1, h2, h3, lo, hi, tb, tc);
            const bool e0 = tv < tau0;
            b00 += e0 ? tb : 0.0f;
            c00 += e0 ? tc : 0.0f;
            b01 += e0 ? 0.0f : tb;
            c01 += e0 ? 0.0f : tc;
            tb = 0.0f;
            tc = 0.0f;
            bp_term(img, slot, h1 + p0.z, h2 + p1.z, h3 + p2.z, lo, hi, tb, tc);
            const bool e1 = tv < tau1;
            b10 += e1 ? tb : 0.0f;
            c10 += e1 ? tc : 0.0f;
            b11 += e1 ? 0.0f : tb;
            c11 += e1 ? 0.0f : tc;
        }
    }
    if (!inside) return;
    const float mean = G.inv_sub;
#pragma unroll
    for (int q = 0; q < BP_VZ; ++q) {
        if (iz + q >= G.nz) break;
        const size_t j = j0 + (size_t)q * G.nx * G.ny;
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            const float b = (q == 0 ? (part == 0 ? b00 : b01) : (part == 0 ? b10 : b11)) * mean;
            const float c = (q == 0 ? (part == 0 ? c00 : c01) : (part == 0 ? c10 : c11)) * mean;
            const size_t jo = j + (size_t)part * nvox;
            float scale = alpha;
            if (normalize) scale *= (c > 1e-6f ? 1.0f / c : 0.0f);
            if (w) scale *= __ldg(w + jo);
            const float upd = scale * b;
            const float out = accumulate ? Storage<TV>::load(vol + jo) + upd : upd;
            Storage<TV>::store(vol + jo, out);
        }
    }
}

template <typename Images, typename TV>
static cudaError_t bp_launch_dyrect(const BpArgs &a, const Images &img)
{
    const Grid &G = *a.grid;
    const dim3 block(BP_TX, BP_TY, BP_TZ);
    const dim3 grid((G.nx + BP_TX - 1) / BP_TX, (G.ny + BP_TY - 1) / BP_TY,
                    (G.nz + BP_TZ * BP_VZ - 1) / (BP_TZ * BP_VZ));
    if (a.cyl || a.subvox > 1) return cudaErrorInvalidValue;
    if (a.window)
        bp_dyrect_kernel<Images, TV, true><<<grid, block, 0, a.stream>>>(
            G, a.views, a.view_idx, a.n_idx, img, a.window, static_cast<TV *>(a.vol), a.w, a.alpha, a.normalize,
            a.accumulate, a.dyr->tau, a.dyr->t_view);
    else
        bp_dyrect_kernel<Images, TV, false><<<grid, block, 0, a.stream>>>(
            G, a.views, a.view_idx, a.n_idx, img, nullptr, static_cast<TV *>(a.vol), a.w, a.alpha, a.normalize,
            a.accumulate, a.dyr->tau, a.dyr->t_view);
    return cudaGetLastError();
}

template <typename Images, typename TV, bool SUBV, bool CYL>
static void bp_launch_window(const BpArgs &a, const Images &img, dim3 grid, dim3 block)
{
    const CylGPU cyl = a.cyl ? *a.cyl : CylGPU{};
    if (a.window)
        bp_kernel<Images, TV, true, SUBV, CYL><<<grid, block, 0, a.stream>>>(
            *a.grid, a.views, a.view_idx, a.n_idx, img, a.window, static_cast<TV *>(a.vol), a.w, a.alpha,
            a.normalize, a.accumulate, a.subvox, cyl);
    else
        bp_kernel<Images, TV, false, SUBV, CYL><<<grid, block, 0, a.stream>>>(
            *a.grid, a.views, a.view_idx, a.n_idx, img, nullptr, static_cast<TV *>(a.vol), a.w, a.alpha,
            a.normalize, a.accumulate, a.subvox, cyl);
}

template <typename Images, typename TV, bool CYL>
static void bp_launch_subv(const BpArgs &a, const Images &img, dim3 grid, dim3 block)
{
    if (a.subvox > 1)
        bp_launch_window<Images, TV, true, CYL>(a, img, grid, block);
    else
        bp_launch_window<Images, TV, false, CYL>(a, img, grid, block);
}

template <typename Images, typename TV>
static cudaError_t bp_launch(const BpArgs &a, const Images &img)
{
    const Grid &G = *a.grid;
    const dim3 block(BP_TX, BP_TY, BP_TZ);
    const dim3 grid((G.nx + BP_TX - 1) / BP_TX, (G.ny + BP_TY - 1) / BP_TY,
                    (G.nz + BP_TZ * BP_VZ - 1) / (BP_TZ * BP_VZ));
    if (a.cyl)
        bp_launch_subv<Images, TV, true>(a, img, grid, block);
    else
        bp_launch_subv<Images, TV, false>(a, img, grid, block);
    return cudaGetLastError();
}

template <typename Images>
static cudaError_t bp_dispatch_vol(const BpArgs &a, const Images &img)
{
    if (a.dyr) {
        if (a.vol_dtype == CTREX_F32) return bp_launch_dyrect<Images, float>(a, img);
        return bp_launch_dyrect<Images, __nv_bfloat16>(a, img);
    }
    if (a.vol_dtype == CTREX_F32) return bp_launch<Images, float>(a, img);
    return bp_launch<Images, __nv_bfloat16>(a, img);
}

cudaError_t launch_backproject(const BpArgs &a)
{
    const Grid &G = *a.grid;
    if (a.atlas) return bp_dispatch_vol(a, AtlasImages{*a.atlas});
    if (a.r_dtype == CTREX_F32)
        return bp_dispatch_vol(a, LinearImages<float>{static_cast<const float *>(a.r), G.nu, G.nv});
    return bp_dispatch_vol(a, LinearImages<__nv_bfloat16>{static_cast<const __nv_bfloat16 *>(a.r), G.nu, G.nv});
}

}  // namespace ctrex

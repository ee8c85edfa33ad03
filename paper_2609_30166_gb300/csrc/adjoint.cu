// adjoint.cu -- matched ray-driven adjoint A^T (exact transpose of the
// projector in project.cu, motion included) and the gradient of <g, A x> with
// respect to the motion parameters (chain rule through the pose and the
// B-spline warp; the deformation is recomputed per sample, never stored).
// The paper motivates geometry refinement and learned components (Sec. 5)
// but prints no such operator; both are the transpose / derivative of its
// Sec. 4.1 projector with the Sec. 2.2.2 / 3.1 warp.
#include "ray.cuh"

// Motion gradient CTA: CTREX_MGRAD_WARPS warps, each on an 8 x 4 pixel
// patch (the CTA covers 8 * warps detector columns x 4 rows), with
// CTREX_MGRAD_MIN_BLOCKS resident CTAs per SM (two warps and six CTAs cap
// the registers at 168; 5 or 4 CTAs with more registers, or 4-warp CTAs,
// were no faster).  The spline's y and z loops are unrolled
// (CTREX_MGRAD_UNROLL_Z): 616 -> 564 ms on the motion workload, with 4
// bytes of spills.  Few warps per CTA shorten the wait of warps with short
// rays for the CTA's final reduction.
#ifndef CTREX_MGRAD_WARPS
#define CTREX_MGRAD_WARPS 2
#endif
#ifndef CTREX_MGRAD_MIN_BLOCKS
#define CTREX_MGRAD_MIN_BLOCKS (12 / CTREX_MGRAD_WARPS)
#endif
#ifndef CTREX_MGRAD_UNROLL_Z
#define CTREX_MGRAD_UNROLL_Z 1
#endif

namespace ctrex {

constexpr int ADJ_TX = 32, ADJ_TY = 4;
constexpr int MG_WARPS = CTREX_MGRAD_WARPS, MG_THREADS = 32 * MG_WARPS;
constexpr int NCOEF = 8 * 8 * 8 * 3;

// ---------------------------------------------------------------------------
// Adjoint: scatter y_i * w_k * trilinear weight into the 8 taps (FP32 atomics)
// ---------------------------------------------------------------------------

// Trilinear scatter of val at the point with centred index coordinates gc
// (index coordinates minus the integer grid centre c: floor and fraction are
// exact in them).  Each (y, z) row of the 2 x 2 x 2 footprint adds w0, w1 to
// the neighbours x0, x0 + 1, consecutive floats.  When both lie in one
// 16-byte-aligned quad of the volume (x0 % 4 != 3 in element terms; 3 cases
// in 4), one vector reduction adds (.., w0, w1, ..) with zeros in the other
// two lanes, so a footprint issues about 5 reductions instead of 8 (the
// reductions' L1/TEX path bounds the kernel).  The zero lanes belong to
// neighbouring voxels (possibly of the adjacent row) inside the volume;
// adding +0 leaves them unchanged.  vec: the volume is 16-byte aligned;
// nvox: its element count.
// A footprint waiting to be scattered: the lower corner (ix, iy, iz) in
// voxel indices and the summed weight of each of its eight taps.  A ray's
// samples lie half a voxel apart, so consecutive ones often share the
// corner: their weights are added here and reduced into the volume once,
// when the corner moves or the ray ends.
struct Footprint {
    int ix = 0, iy = 0, iz = 0;
    bool live = false;
    float w[2][2][2] = {{{0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}}};
};

__device__ __forceinline__ void scatter_footprint(float *__restrict__ vol, int nx, int ny, int nz,
                                                  const Footprint &F, bool vec, long long nvox)
{
    const int ix = F.ix, iy = F.iy, iz = F.iz;
    const bool in0 = (unsigned)ix < (unsigned)nx, in1 = (unsigned)(ix + 1) < (unsigned)nx;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
        const int z = iz + dz;
        if ((unsigned)z >= (unsigned)nz) continue;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int y = iy + dy;
            if ((unsigned)y >= (unsigned)ny) continue;
            const long long e = ((long long)z * ny + y) * nx + ix;  // element of tap x0 (x0 may be -1)
            const float w0 = in0 ? F.w[dz][dy][0] : 0.0f, w1 = in1 ? F.w[dz][dy][1] : 0.0f;
            const int lane = (int)(e & 3);
            if (vec && lane != 3 && e >= 0 && (e | 3) < nvox) {
                float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (lane == 0) {
                    q.x = w0;
                    q.y = w1;
                } else if (lane == 1) {
                    q.y = w0;
                    q.z = w1;
                } else {
                    q.z = w0;
                    q.w = w1;
                }
                atomicAdd(reinterpret_cast<float4 *>(vol + (e - lane)), q);
            } else {
                if (in0) atomicAdd(vol + e, w0);
                if (in1) atomicAdd(vol + e + 1, w1);
            }
        }
    }
}

// Event-based 4D model (Sec. 3.3): the transpose sends each tap's share to
// mu0 (vol[j]) if the view's time t precedes the voxel's transition time
// tau_j, else to mu1 (vol[nvox + j]); scalar reductions.  The choice is the
// voxel's for the whole view, so merged weights route as their samples'.
__device__ __forceinline__ void scatter_footprint_dyrect(float *__restrict__ vol, int nx, int ny, int nz,
                                                         const Footprint &F, const float *__restrict__ tau, float t,
                                                         long long nvox)
{
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
        const int z = F.iz + dz;
        if ((unsigned)z >= (unsigned)nz) continue;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int y = F.iy + dy;
            if ((unsigned)y >= (unsigned)ny) continue;
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int x = F.ix + dx;
                if ((unsigned)x >= (unsigned)nx) continue;
                const long long j = ((long long)z * ny + y) * nx + x;
                atomicAdd(vol + (t < __ldg(tau + j) ? j : nvox + j), F.w[dz][dy][dx]);
            }
        }
    }
}

// Adds val at the point with centred index coordinates gc to the pending
// footprint F, first scattering F if the point's corner differs (DYR: into
// the event model's two fields, by tau and the view's time t).
template <bool DYR>
__device__ __forceinline__ void scatter_trilinear(float *__restrict__ vol, int nx, int ny, int nz, const float c[3],
                                                  const float gc[3], float val, bool vec, long long nvox,
                                                  Footprint &F, const float *__restrict__ tau, float t)
{
    const float fx = floorf(gc[0]), fy = floorf(gc[1]), fz = floorf(gc[2]);
    const int ix = (int)fx + (int)c[0], iy = (int)fy + (int)c[1], iz = (int)fz + (int)c[2];
    const float ax = gc[0] - fx, ay = gc[1] - fy, az = gc[2] - fz;
    const float wx[2] = {1.0f - ax, ax}, wy[2] = {1.0f - ay, ay}, wz[2] = {1.0f - az, az};
    if (F.live && (ix != F.ix || iy != F.iy || iz != F.iz)) {
        if (DYR)
            scatter_footprint_dyrect(vol, nx, ny, nz, F, tau, t, nvox);
        else
            scatter_footprint(vol, nx, ny, nz, F, vec, nvox);
        F.live = false;
    }
    if (!F.live) {
        F.ix = ix;
        F.iy = iy;
        F.iz = iz;
        F.live = true;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) F.w[dz][dy][dx] = 0.0f;
    }
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const float wzy = val * wz[dz] * wy[dy];
            F.w[dz][dy][0] = fmaf(wzy, wx[0], F.w[dz][dy][0]);
            F.w[dz][dy][1] = fmaf(wzy, wx[1], F.w[dz][dy][1]);
        }
}

template <bool MOTION, bool DYR>
__global__ void __launch_bounds__(ADJ_TX *ADJ_TY)
    adjoint_kernel(Grid G, const ViewGPU *__restrict__ views, const MotionGPU *__restrict__ motion,
                   const float *__restrict__ coef_g, const int *__restrict__ view_idx,
                   const float *__restrict__ proj, float *__restrict__ vol, unsigned *devcheck,
                   const float *__restrict__ tau, const float *__restrict__ t_view)
{
    __shared__ float4 s_coef[MOTION ? NCOEF_PAD : 1];  // zero-padded 9^3 float4 copy of the coefficients
    const int k = blockIdx.y;
    const int view = view_idx ? view_idx[k] : k;
    if (view < 0 || view >= G.n_views) {
        if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(devcheck, (unsigned)DEVCHECK_OOB);
        return;
    }
    MotionGPU mo;
    const float4 *coef = nullptr;
    if (MOTION) {
        mo = motion[view];
        if (coef_g) {
            load_coef_padded(s_coef, coef_g, threadIdx.y * ADJ_TX + threadIdx.x, ADJ_TX * ADJ_TY);
            coef = s_coef;
        }
        __syncthreads();
    }
    int iu, iv;
    tile_pixel<MOTION>(blockIdx.x * ADJ_TX, blockIdx.z * ADJ_TY, iu, iv);
    if (iu >= G.nu || iv >= G.nv) return;
    const float y = proj[((size_t)k * G.nv + iv) * G.nu + iu] * G.inv_sub;
    if (y == 0.0f) return;
    const bool vec = (reinterpret_cast<uintptr_t>(vol) & 15) == 0;
    const long long nvox = (long long)G.nx * G.ny * G.nz;
    const float t = DYR ? __ldg(t_view + view) : 0.0f;
    float cen[3];
    grid_centre(G, cen);
    Footprint F;  // the pending footprint of this thread's samples
    for (int s = 0; s < G.n_sub; ++s) {
        Ray R;  // sample positions relative to the grid centre
        if (!setup_ray(G, views[view * G.n_sub + s], (float)iu, (float)iv, R, cen)) continue;
        const float ys = y * G.step_mm;
        for (int kk = 0; kk < R.K; ++kk) {
            float g[3];
            float val = ys;
            if (kk < R.K - 1) {
                g[0] = fmaf((float)kk, R.sg[0], R.g0[0]);
                g[1] = fmaf((float)kk, R.sg[1], R.g0[1]);
                g[2] = fmaf((float)kk, R.sg[2], R.g0[2]);
            } else {
                if (!(R.w_last > 0.0f)) break;
                g[0] = R.g_last[0];
                g[1] = R.g_last[1];
                g[2] = R.g_last[2];
                val = y * R.w_last;
            }
            float gc[3];
            if (MOTION) {
                warp_sample_c(G, mo, coef, g, gc);
            } else {
                gc[0] = g[0];
                gc[1] = g[1];
                gc[2] = g[2];
            }
            if (!(gc[0] >= -1.0f - cen[0] && gc[0] < (float)G.nx - cen[0] && gc[1] >= -1.0f - cen[1] &&
                  gc[1] < (float)G.ny - cen[1] && gc[2] >= -1.0f - cen[2] && gc[2] < (float)G.nz - cen[2]))
                continue;
            scatter_trilinear<DYR>(vol, G.nx, G.ny, G.nz, cen, gc, val, vec, nvox, F, tau, t);
        }
    }
    if (F.live) {
        if (DYR)
            scatter_footprint_dyrect(vol, G.nx, G.ny, G.nz, F, tau, t, nvox);
        else
            scatter_footprint(vol, G.nx, G.ny, G.nz, F, vec, nvox);
    }
}

cudaError_t launch_adjoint(const FwdArgs &a, const float *proj, float *vol)
{
    if (a.n_idx == 0) return cudaSuccess;
    const Grid &G = *a.grid;
    const dim3 grid((G.nu + ADJ_TX - 1) / ADJ_TX, a.n_idx, (G.nv + ADJ_TY - 1) / ADJ_TY);
    const dim3 block(ADJ_TX, ADJ_TY);
    if (a.dyr && a.motion) return cudaErrorInvalidValue;  // the event model is defined without motion
    if (a.motion)
        adjoint_kernel<true, false><<<grid, block, 0, a.stream>>>(G, a.views, a.motion, a.coef_idx, a.view_idx,
                                                                 proj, vol, a.devcheck, nullptr, nullptr);
    else if (a.dyr)
        adjoint_kernel<false, true><<<grid, block, 0, a.stream>>>(G, a.views, nullptr, nullptr, a.view_idx, proj,
                                                                 vol, a.devcheck, a.dyr->tau, a.dyr->t_view);
    else
        adjoint_kernel<false, false><<<grid, block, 0, a.stream>>>(G, a.views, nullptr, nullptr, a.view_idx, proj,
                                                                  vol, a.devcheck, nullptr, nullptr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Motion gradient
// ---------------------------------------------------------------------------
//
// dL/dtheta and dL/dcoef of L = <g, A x> (chain rule of the Sec. 4.1
// projector through the Sec. 2.2.2 pose and the Sec. 3.1 warp).  Per sample
// k of ray i, with y = g' + s u(g'), g' = M g + b:
//   dL/dy  = g_i w_k grad mu(y)                 (trilinear gradient, index units)
//   dL/dg' = dL/dy (I + s du/dg')               -> dL/db += dL/dg', dL/dM += dL/dg' g^T
//   dL/dc_ijk[c] += s dL/dy[c] beta(xi - i) beta(eta - j) beta(zeta - k)
// Sample positions, the warp and the pose sums are formed relative to the
// integer grid centre c (as in the adjoint): dL/dM = sum dL/dg' (g - c)^T +
// (sum dL/dg') c^T, the last term added in FP64 by the finish kernel.

// Zero-padded trilinear interpolant's gradient (index units) inside the cell
// floor(y), at the point with centred index coordinates yc = y - c (floor and
// fraction exact in them).
template <typename TV>
__device__ __forceinline__ void trilinear_grad_c(const TV *__restrict__ vol, int nx, int ny, int nz, const float c[3],
                                                 const float yc[3], float grad[3])
{
    const float fx = floorf(yc[0]), fy = floorf(yc[1]), fz = floorf(yc[2]);
    const int ix = (int)fx + (int)c[0], iy = (int)fy + (int)c[1], iz = (int)fz + (int)c[2];
    const float ax = yc[0] - fx, ay = yc[1] - fy, az = yc[2] - fz;
    float v[2][2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int x = ix + dx, y = iy + dy, z = iz + dz;
                const bool in = (unsigned)x < (unsigned)nx && (unsigned)y < (unsigned)ny && (unsigned)z < (unsigned)nz;
                v[dz][dy][dx] = in ? Storage<TV>::load(vol + ((long long)z * ny + y) * nx + x) : 0.0f;
            }
    const float by0 = 1.0f - ay, bz0 = 1.0f - az, bx0 = 1.0f - ax;
    grad[0] = bz0 * (by0 * (v[0][0][1] - v[0][0][0]) + ay * (v[0][1][1] - v[0][1][0])) +
              az * (by0 * (v[1][0][1] - v[1][0][0]) + ay * (v[1][1][1] - v[1][1][0]));
    grad[1] = bz0 * (bx0 * (v[0][1][0] - v[0][0][0]) + ax * (v[0][1][1] - v[0][0][1])) +
              az * (bx0 * (v[1][1][0] - v[1][0][0]) + ax * (v[1][1][1] - v[1][0][1]));
    grad[2] = by0 * (bx0 * (v[1][0][0] - v[0][0][0]) + ax * (v[1][0][1] - v[0][0][1])) +
              ay * (bx0 * (v[1][1][0] - v[0][1][0]) + ax * (v[1][1][1] - v[0][1][1]));
}

// Displacement u and its derivatives with respect to the three spline
// coordinates, by sum factorisation over the separable 4 x 4 x 4 support:
// the x sums first (value and x-derivative weights), then y, then z --
// 576 FMAs instead of 64 taps x 12 accumulators with per-tap weight products.
__device__ __forceinline__ void spline_value_jacobian(const float4 *coef, const int i0[3], const float wx[4],
                                                      const float wy[4], const float wz[4], const float dx[4],
                                                      const float dy[4], const float dz[4], float u[3],
                                                      float Jx[3], float Jy[3], float Jz[3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = Jx[c] = Jy[c] = Jz[c] = 0.0f;
    const float4 *plane = coef_cell(coef, i0);
    // the z loop's two weights are picked by selects, which keeps the
    // arrays in registers when the loop stays rolled (CTREX_MGRAD_UNROLL_Z
    // 0); the y loop is unrolled: 16 independent float4 loads per plane.
#if CTREX_MGRAD_UNROLL_Z
#pragma unroll
#else
#pragma unroll 1
#endif
    for (int k = 0; k < 4; ++k, plane += CPAD * CPAD) {
        const float wzk = k == 0 ? wz[0] : (k == 1 ? wz[1] : (k == 2 ? wz[2] : wz[3]));
        const float dzk = k == 0 ? dz[0] : (k == 1 ? dz[1] : (k == 2 ? dz[2] : dz[3]));
        float a[3] = {0.f, 0.f, 0.f}, bx[3] = {0.f, 0.f, 0.f}, by[3] = {0.f, 0.f, 0.f};
        const float4 *row = plane;
#pragma unroll
        for (int j = 0; j < 4; ++j, row += CPAD) {
            const float wyj = wy[j], dyj = dy[j];
            float sx[3] = {0.f, 0.f, 0.f}, tx[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 cf = row[i];
                sx[0] = fmaf(wx[i], cf.x, sx[0]);
                sx[1] = fmaf(wx[i], cf.y, sx[1]);
                sx[2] = fmaf(wx[i], cf.z, sx[2]);
                tx[0] = fmaf(dx[i], cf.x, tx[0]);
                tx[1] = fmaf(dx[i], cf.y, tx[1]);
                tx[2] = fmaf(dx[i], cf.z, tx[2]);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a[c] = fmaf(wyj, sx[c], a[c]);
                bx[c] = fmaf(wyj, tx[c], bx[c]);
                by[c] = fmaf(dyj, sx[c], by[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            u[c] = fmaf(wzk, a[c], u[c]);
            Jx[c] = fmaf(wzk, bx[c], Jx[c]);
            Jy[c] = fmaf(wzk, by[c], Jy[c]);
            Jz[c] = fmaf(dzk, a[c], Jz[c]);
        }
    }
}

// --- coefficient gradient on the tensor cores --------------------------------
//
// Over the samples s of a warp that share one spline cell, the coefficient
// gradient of that cell is an outer-product sum
//   G[(c, kz)][(j, i)] = sum_s  (v_s[c] wz_s[kz]) (wy_s[j] wx_s[i]),
// v_s = s_view dL/dy_s: a 12 x 16 matrix = A (12 x samples) B (samples x 16),
// i.e. a GEMM with K = samples.  One warp step (32 samples) is 4 k-chunks of
// mma.m16n8k8 (TF32) per 8-column half of G, with rows 12..15 zero.  FP32
// accuracy comes from the 3-term split x = hi + lo (hi = tf32(x), lo =
// tf32(x - hi)): A B ~ Alo Bhi + Ahi Blo + Ahi Bhi, each product within about
// 3 * 2^-22 of the FP32 one.  A step's MMAs start from zero (a chain of 12
// k-steps), and its result is added to FP32 register sums of the warp's
// current cell; those go to the CTA's FP64 shared partials (atomics, once per
// change of cell) and, at the end, to FP64 global sums.
//
// Fragment layouts of mma.m16n8k8 .tf32 (g = lane / 4, t = lane % 4):
//   A (row-major 16 x 8): a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4)
//   B (col-major 8 x 8):  b0 (k = t, n = g), b1 (k = t + 4, n = g)
//   C/D (16 x 8):         d0 (g, 2t), d1 (g, 2t + 1), d2 (g + 8, 2t), d3 (g + 8, 2t + 1)
// With k = sample, lane (g, t) needs samples t and t + 4 of each chunk: it
// reads their spline fractions and v by shuffles and evaluates the B-spline
// basis functions its rows / columns need (kz = i = g % 4, j = g / 4 for the
// first half of G, 2 + g / 4 for the second) itself.

__device__ __forceinline__ unsigned tf32_bits(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x = hi + lo as two TF32 values.
__device__ __forceinline__ void tf32_split(float x, unsigned &hi, unsigned &lo)
{
    hi = tf32_bits(x);
    lo = tf32_bits(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32_16x8x8(float d[4], const unsigned a[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Power-basis coefficients (f^0 .. f^3) of the uniform cubic B-spline piece m
// (m = 0..3: weight of control point i0 - 1 + m at fraction f).
__device__ __forceinline__ float4 bspline_piece(int m)
{
    return m == 0 ? make_float4(1.0f / 6.0f, -0.5f, 0.5f, -1.0f / 6.0f)
                  : (m == 1 ? make_float4(2.0f / 3.0f, 0.0f, -1.0f, 0.5f)
                            : (m == 2 ? make_float4(1.0f / 6.0f, 0.5f, 0.5f, -0.5f)
                                      : make_float4(0.0f, 0.0f, 0.0f, 1.0f / 6.0f)));
}

__device__ __forceinline__ float horner(const float4 p, float f)
{
    return fmaf(fmaf(fmaf(p.w, f, p.z), f, p.y), f, p.x);
}

// The warp's coefficient-gradient state: FP32 sums of the current cell's
// 12 x 16 block in fragment layout (two 8-column halves).
struct CoefAcc {
    float acc[2][4];
    int cell;  // packed i0 of the current cell, -1 for none (warp-uniform)
};

// Adds the sums of acc's cell to the CTA's FP64 partials and clears them.
// Entries whose control point index passes 7 carry an exactly zero weight
// (cubic piece 3 at fraction 0) and are skipped.
__device__ __forceinline__ void coef_flush(CoefAcc &A, double *s_g64, int lane)
{
    if (A.cell >= 0) {
        const int i0x = A.cell & 7, i0y = (A.cell >> 3) & 7, i0z = A.cell >> 6;
        const int g = lane >> 2, t = lane & 3;
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = g + 8 * (q >> 1), col = 8 * h + 2 * t + (q & 1);
                const float v = A.acc[h][q];
                A.acc[h][q] = 0.0f;
                if (row >= 12 || v == 0.0f) continue;
                const int comp = row >> 2, kz = row & 3, j = col >> 2, i = col & 3;
                const int cx = i0x - 1 + i, cy = i0y - 1 + j, cz = i0z - 1 + kz;
                if (cx > 7 || cy > 7 || cz > 7) continue;
                atomicAdd(s_g64 + 3 * ((cz * 8 + cy) * 8 + cx) + comp, (double)v);
            }
    }
}

// One warp step of the coefficient gradient.  Per lane: cell = packed i0 of
// its sample, f = spline fractions, v = s_view dL/dy (zero when the lane has
// no contribution), live = whether it has one.  Warp-collective.
__device__ __forceinline__ void coef_step(CoefAcc &A, double *s_g64, int cell, const float f[3], const float v[3],
                                          bool live, const float4 *s_piece)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    // the B-spline pieces of this lane's rows and columns
    const float4 pz = s_piece[g & 3], px = pz, py0 = s_piece[g >> 2], py1 = s_piece[2 + (g >> 2)];
    unsigned pending = __ballot_sync(full, live);
    while (pending) {  // warp-uniform: one round per distinct cell of this step
        const int leader = __ffs(pending) - 1;
        const int lcell = __shfl_sync(full, cell, leader);
        const bool mine = ((pending >> lane) & 1u) && cell == lcell;
        if (lcell != A.cell) {
            coef_flush(A, s_g64, lane);
            A.cell = lcell;
        }
        const float pv0 = mine ? v[0] : 0.0f, pv1 = mine ? v[1] : 0.0f, pv2 = mine ? v[2] : 0.0f;
        const float pfx = mine ? f[0] : 0.0f, pfy = mine ? f[1] : 0.0f, pfz = mine ? f[2] : 0.0f;
        float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            float a[4], b[2][2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int src = 8 * q + t + 4 * h;
                const float fx = __shfl_sync(full, pfx, src), fy = __shfl_sync(full, pfy, src),
                            fz = __shfl_sync(full, pfz, src);
                const float x0 = __shfl_sync(full, pv0, src), x1 = __shfl_sync(full, pv1, src),
                            x2 = __shfl_sync(full, pv2, src);
                const float wz = horner(pz, fz), wx = horner(px, fx);
                a[2 * h] = (g < 4 ? x0 : x1) * wz;        // row g:     c = g / 4, kz = g % 4
                a[2 * h + 1] = g < 4 ? x2 * wz : 0.0f;    // row g + 8: c = 2 (rows 12..15 zero)
                b[0][h] = horner(py0, fy) * wx;           // column g of half 0: j = g / 4, i = g % 4
                b[1][h] = horner(py1, fy) * wx;           // column g of half 1: j = 2 + g / 4
            }
            unsigned ah[4], al[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) tf32_split(a[e], ah[e], al[e]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                unsigned bh0, bl0, bh1, bl1;
                tf32_split(b[h][0], bh0, bl0);
                tf32_split(b[h][1], bh1, bl1);
                mma_tf32_16x8x8(d[h], al, bh0, bh1);
                mma_tf32_16x8x8(d[h], ah, bl0, bl1);
                mma_tf32_16x8x8(d[h], ah, bh0, bh1);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 4; ++e) A.acc[h][e] += d[h][e];
        pending &= ~__ballot_sync(full, mine);
    }
}

template <typename TV>
__global__ void __launch_bounds__(MG_THREADS, CTREX_MGRAD_MIN_BLOCKS)
    motion_grad_kernel(Grid G, const ViewGPU *__restrict__ views, const MotionGPU *__restrict__ motion,
                       const float *__restrict__ coef_g, const int *__restrict__ view_idx,
                       const TV *__restrict__ vol, const float *__restrict__ gproj,
                       double *__restrict__ grad_M, double *__restrict__ grad_b,
                       double *__restrict__ grad_coef, unsigned *devcheck)
{
    __shared__ float4 s_coef[NCOEF_PAD];  // zero-padded 9^3 float4 copy of the coefficients
    __shared__ double s_g64[NCOEF];       // the CTA's coefficient-gradient partials
    __shared__ double s_red[12][MG_WARPS];
    __shared__ float4 s_piece[4];
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int lane = tid & 31;
    const int k = blockIdx.y;
    const int view = view_idx ? view_idx[k] : k;
    if (!(view >= 0 && view < G.n_views)) {
        if (tid == 0) atomicOr(devcheck, (unsigned)DEVCHECK_OOB);
        return;  // uniform over the CTA
    }
    const MotionGPU mo = motion[view];
    const bool spline = coef_g != nullptr && mo.s != 0.0f;
    const bool want_coef = spline && grad_coef != nullptr;
    if (spline) load_coef_padded(s_coef, coef_g, tid, MG_THREADS);
    if (want_coef)
        for (int i = tid; i < NCOEF; i += MG_THREADS) s_g64[i] = 0.0;
    if (tid < 4) s_piece[tid] = bspline_piece(tid);
    __syncthreads();
    float cen[3];
    grid_centre(G, cen);
    CoefAcc CA;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < 4; ++e) CA.acc[h][e] = 0.0f;
    CA.cell = -1;
    float G1[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
    int iu, iv;
    tile_pixel<true>(blockIdx.x * 8 * MG_WARPS, blockIdx.z * 4, iu, iv);
    const bool pix_ok = iu < G.nu && iv < G.nv;
    const float y = pix_ok ? gproj[((size_t)k * G.nv + iv) * G.nu + iu] * G.inv_sub : 0.0f;
    for (int s = 0; s < G.n_sub; ++s) {
        Ray R;  // sample positions relative to the grid centre
        const bool hit = pix_ok && setup_ray(G, views[view * G.n_sub + s], (float)(pix_ok ? iu : 0),
                                             (float)(pix_ok ? iv : 0), R, cen);
        // the warp-collective coefficient step needs every lane: lanes without
        // work run the loop with zero weight up to the warp's longest ray
        const int K = hit ? R.K : 0;
        int Kmax = K;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) Kmax = max(Kmax, __shfl_xor_sync(0xffffffffu, Kmax, off));
        for (int kk = 0; kk < Kmax; ++kk) {
            float gc[3] = {0.f, 0.f, 0.f};
            float sc = 0.0f;
            if (hit && kk < K - 1) {
                gc[0] = fmaf((float)kk, R.sg[0], R.g0[0]);
                gc[1] = fmaf((float)kk, R.sg[1], R.g0[1]);
                gc[2] = fmaf((float)kk, R.sg[2], R.g0[2]);
                sc = y * G.step_mm;
            } else if (hit && kk == K - 1) {
                gc[0] = R.g_last[0];
                gc[1] = R.g_last[1];
                gc[2] = R.g_last[2];
                sc = R.w_last > 0.0f ? y * R.w_last : 0.0f;
            }
            const bool act = hit && kk < K && sc != 0.0f;
            // warp: d = D gc + bc (+ s u), g' - c = gc + d
            float d[3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
                d[r] = fmaf(mo.D[3 * r], gc[0], fmaf(mo.D[3 * r + 1], gc[1], fmaf(mo.D[3 * r + 2], gc[2], mo.bc[r])));
            int i0[3] = {1, 1, 1};
            float f[3] = {0.f, 0.f, 0.f};
            float u[3] = {0.f, 0.f, 0.f}, Jx[3] = {0.f, 0.f, 0.f}, Jy[3] = {0.f, 0.f, 0.f},
                  Jz[3] = {0.f, 0.f, 0.f};
            if (spline) {
                bool on[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) spline_coord(gc[a] + d[a] + cen[a], G.spl_scale[a], i0[a], f[a], on[a]);
                float wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
                bspline_weights(f[0], wx);
                bspline_weights(f[1], wy);
                bspline_weights(f[2], wz);
                bspline_dweights(f[0], dx);
                bspline_dweights(f[1], dy);
                bspline_dweights(f[2], dz);
                spline_value_jacobian(s_coef, i0, wx, wy, wz, dx, dy, dz, u, Jx, Jy, Jz);
                const float sx = on[0] ? G.spl_scale[0] : 0.f, sy = on[1] ? G.spl_scale[1] : 0.f,
                            sz = on[2] ? G.spl_scale[2] : 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    Jx[c] *= sx;
                    Jy[c] *= sy;
                    Jz[c] *= sz;
                }
            }
            const float yc[3] = {gc[0] + fmaf(mo.s, u[0], d[0]), gc[1] + fmaf(mo.s, u[1], d[1]),
                                 gc[2] + fmaf(mo.s, u[2], d[2])};
            float gy[3] = {0.f, 0.f, 0.f};
            if (act && yc[0] >= -1.0f - cen[0] && yc[0] < (float)G.nx - cen[0] && yc[1] >= -1.0f - cen[1] &&
                yc[1] < (float)G.ny - cen[1] && yc[2] >= -1.0f - cen[2] && yc[2] < (float)G.nz - cen[2])
                trilinear_grad_c(vol, G.nx, G.ny, G.nz, cen, yc, gy);
#pragma unroll
            for (int c = 0; c < 3; ++c) gy[c] *= sc;  // dL/dy (index units)
            // dL/dg' = dL/dy (I + s J), J[c][a] = du_c / dg'_a
            const float gg[3] = {gy[0] + mo.s * (gy[0] * Jx[0] + gy[1] * Jx[1] + gy[2] * Jx[2]),
                                 gy[1] + mo.s * (gy[0] * Jy[0] + gy[1] * Jy[1] + gy[2] * Jy[2]),
                                 gy[2] + mo.s * (gy[0] * Jz[0] + gy[1] * Jz[1] + gy[2] * Jz[2])};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                gb[r] += gg[r];
                G1[3 * r + 0] = fmaf(gg[r], gc[0], G1[3 * r + 0]);
                G1[3 * r + 1] = fmaf(gg[r], gc[1], G1[3 * r + 1]);
                G1[3 * r + 2] = fmaf(gg[r], gc[2], G1[3 * r + 2]);
            }
            if (want_coef) {  // CTA-uniform
                const float v[3] = {mo.s * gy[0], mo.s * gy[1], mo.s * gy[2]};
                const bool live = act && (v[0] != 0.0f || v[1] != 0.0f || v[2] != 0.0f);
                const int cell = (i0[2] * 8 + i0[1]) * 8 + i0[0];
                coef_step(CA, s_g64, cell, f, v, live, s_piece);
            }
        }
    }
    if (want_coef) coef_flush(CA, s_g64, lane);
    // CTA reduction of the 12 pose-gradient entries: FP32 warp sums, FP64 over
    // the warps and across CTAs
    float vals[12];
#pragma unroll
    for (int q = 0; q < 9; ++q) vals[q] = G1[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) vals[9 + q] = gb[q];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        float v = vals[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) s_red[q][tid >> 5] = (double)v;
    }
    __syncthreads();
    if (tid < 12) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < MG_WARPS; ++w) v += s_red[tid][w];
        if (grad_M && tid < 9) atomicAdd(grad_M + 9 * view + tid, v);
        if (grad_b && tid >= 9) atomicAdd(grad_b + 3 * view + (tid - 9), v);
    }
    if (want_coef) {
        for (int i = tid; i < NCOEF; i += MG_THREADS) {
            const double v = s_g64[i];
            if (v != 0.0) atomicAdd(grad_coef + i, v);
        }
    }
}

cudaError_t launch_motion_grad(const FwdArgs &a, const float *gproj, double *grad_M, double *grad_b,
                               double *grad_coef_idx)
{
    if (a.n_idx == 0) return cudaSuccess;
    const Grid &G = *a.grid;
    const dim3 grid((G.nu + 8 * MG_WARPS - 1) / (8 * MG_WARPS), a.n_idx, (G.nv + 3) / 4);
    const dim3 block(32, MG_WARPS);
    if (a.vol_dtype == CTREX_F32)
        motion_grad_kernel<float><<<grid, block, 0, a.stream>>>(G, a.views, a.motion, a.coef_idx, a.view_idx,
                                                               (const float *)a.vol, gproj, grad_M, grad_b,
                                                               grad_coef_idx, a.devcheck);
    else
        motion_grad_kernel<__nv_bfloat16><<<grid, block, 0, a.stream>>>(
            G, a.views, a.motion, a.coef_idx, a.view_idx, (const __nv_bfloat16 *)a.vol, gproj, grad_M, grad_b,
            grad_coef_idx, a.devcheck);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-view motion set-up and the final chain rule to (omega, t, A, coef)
// ---------------------------------------------------------------------------

struct Frame {
    double vox[3];
    double origin[3];
    double cen[3];  // integer grid centre floor((n - 1) / 2) per axis (index coordinates)
};

// Rodrigues R = I + a K + b K^2 and dR/domega_i (FP64, one thread per view).
__device__ void rodrigues(const double w[3], double R[9], double dR[27])
{
    const double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double a, b, dat, dbt;
    if (th < 1e-4) {
        const double t2 = th * th;
        a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
        b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
        dat = -1.0 / 3.0 + t2 / 30.0;
        dbt = -1.0 / 12.0 + t2 / 180.0;
    } else {
        const double s = sin(th), c = cos(th);
        a = s / th;
        b = (1.0 - c) / (th * th);
        dat = (th * c - s) / (th * th * th);
        dbt = (th * s - 2.0 * (1.0 - c)) / (th * th * th * th);
    }
    const double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double K2[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) K2[3 * r + c] = K[3 * r] * K[c] + K[3 * r + 1] * K[3 + c] + K[3 * r + 2] * K[6 + c];
    for (int q = 0; q < 9; ++q) R[q] = (q % 4 == 0 ? 1.0 : 0.0) + a * K[q] + b * K2[q];
    for (int i = 0; i < 3; ++i) {
        double E[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (i == 0) { E[5] = -1; E[7] = 1; }
        if (i == 1) { E[2] = 1; E[6] = -1; }
        if (i == 2) { E[1] = -1; E[3] = 1; }
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double ek = 0.0, ke = 0.0;
                for (int q = 0; q < 3; ++q) {
                    ek += E[3 * r + q] * K[3 * q + c];
                    ke += K[3 * r + q] * E[3 * q + c];
                }
                dR[9 * i + 3 * r + c] = dat * w[i] * K[3 * r + c] + a * E[3 * r + c] +
                                        dbt * w[i] * K2[3 * r + c] + b * (ek + ke);
            }
    }
}

__global__ void motion_setup_kernel(const float *__restrict__ theta, const float *__restrict__ s_view,
                                    int n_views, Frame F, MotionGPU *__restrict__ motion,
                                    float *__restrict__ dRdw)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_views) return;
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, dR[27] = {0}, A[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    double t[3] = {0, 0, 0};
    if (theta) {
        const double w[3] = {theta[15 * v], theta[15 * v + 1], theta[15 * v + 2]};
        rodrigues(w, R, dR);
        for (int q = 0; q < 3; ++q) t[q] = theta[15 * v + 3 + q];
        for (int q = 0; q < 9; ++q) A[q] = theta[15 * v + 6 + q];
    }
    // world map x' = Mw x + bw with Mw = A R, bw = A t
    double Mw[9], bw[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) Mw[3 * r + c] = A[3 * r] * R[c] + A[3 * r + 1] * R[3 + c] + A[3 * r + 2] * R[6 + c];
        bw[r] = A[3 * r] * t[0] + A[3 * r + 1] * t[1] + A[3 * r + 2] * t[2];
    }
    // index map g' = M g + b: M = diag(1/vox) Mw diag(vox), b = (Mw o + bw - o) / vox
    MotionGPU m;
    for (int r = 0; r < 3; ++r) {
        double acc = bw[r] - F.origin[r];
        for (int c = 0; c < 3; ++c) {
            m.M[3 * r + c] = (float)(Mw[3 * r + c] * F.vox[c] / F.vox[r]);
            acc += Mw[3 * r + c] * F.origin[c];
        }
        const double b = acc / F.vox[r];
        m.b[r] = (float)b;
        double bc = b;
        for (int c = 0; c < 3; ++c) {
            const double Mrc = Mw[3 * r + c] * F.vox[c] / F.vox[r];
            const double Drc = Mrc - (r == c ? 1.0 : 0.0);
            m.D[3 * r + c] = (float)Drc;
            bc += Drc * F.cen[c];
        }
        m.bc[r] = (float)bc;
    }
    m.s = s_view ? s_view[v] : 0.0f;
    m.pad[0] = m.pad[1] = m.pad[2] = 0.0f;
    motion[v] = m;
    for (int q = 0; q < 27; ++q) dRdw[27 * v + q] = (float)dR[q];
}

__global__ void coef_to_index_kernel(const float *__restrict__ coef, Frame F, float *__restrict__ coef_idx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NCOEF) coef_idx[i] = (float)(coef[i] / F.vox[i % 3]);
}

cudaError_t launch_motion_setup(const float *theta, const float *coef, const float *s_view, int n_views,
                                const Grid &G, const double vox[3], const double origin[3], MotionGPU *motion,
                                float *coef_idx, float *dRdw, cudaStream_t stream)
{
    Frame F;
    const int n[3] = {G.nx, G.ny, G.nz};
    for (int a = 0; a < 3; ++a) {
        F.vox[a] = vox[a];
        F.origin[a] = origin[a];
        F.cen[a] = (double)((n[a] - 1) / 2);
    }
    motion_setup_kernel<<<(n_views + 127) / 128, 128, 0, stream>>>(theta, s_view, n_views, F, motion, dRdw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (coef) {
        coef_to_index_kernel<<<(NCOEF + 255) / 256, 256, 0, stream>>>(coef, F, coef_idx);
        e = cudaGetLastError();
    }
    return e;
}

// dL/d(omega, t, A) from dL/d(M, b) (index coordinates); one thread per view.
// gMc holds sum dL/dg' (g - c)^T, so dL/dM = gMc + gb c^T (c: integer grid
// centre).
__global__ void motion_finish_kernel(const float *__restrict__ theta, const float *__restrict__ dRdw,
                                     const double *__restrict__ gMc, const double *__restrict__ gb, int n_views,
                                     Frame F, float *__restrict__ grad_theta)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_views) return;
    double R[9], dR[27], A[9], t[3];
    const double w[3] = {theta[15 * v], theta[15 * v + 1], theta[15 * v + 2]};
    rodrigues(w, R, dR);
    for (int q = 0; q < 3; ++q) t[q] = theta[15 * v + 3 + q];
    for (int q = 0; q < 9; ++q) A[q] = theta[15 * v + 6 + q];
    // dL/dMw[r][c] = gM[r][c] vox[c]/vox[r] + gb[r] origin[c]/vox[r];  dL/dbw[r] = gb[r]/vox[r]
    double gMw[9], gbw[3];
    for (int r = 0; r < 3; ++r) {
        gbw[r] = gb[3 * v + r] / F.vox[r];
        for (int c = 0; c < 3; ++c) {
            const double gM = gMc[9 * v + 3 * r + c] + gb[3 * v + r] * F.cen[c];
            gMw[3 * r + c] = gM * F.vox[c] / F.vox[r] + gb[3 * v + r] * F.origin[c] / F.vox[r];
        }
    }
    // Mw = A R, bw = A t
    double gA[9], gR[9], gt[3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int q = 0; q < 3; ++q) s += gMw[3 * r + q] * R[3 * c + q];
            gA[3 * r + c] = s + gbw[r] * t[c];
            double s2 = 0.0;
            for (int q = 0; q < 3; ++q) s2 += A[3 * q + r] * gMw[3 * q + c];
            gR[3 * r + c] = s2;
        }
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int q = 0; q < 3; ++q) s += A[3 * q + c] * gbw[q];
        gt[c] = s;
    }
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int q = 0; q < 9; ++q) s += gR[q] * dR[9 * i + q];
        grad_theta[15 * v + i] += (float)s;
        grad_theta[15 * v + 3 + i] += (float)gt[i];
    }
    for (int q = 0; q < 9; ++q) grad_theta[15 * v + 6 + q] += (float)gA[q];
    (void)dRdw;
}

__global__ void coef_grad_finish_kernel(const double *__restrict__ g_idx, Frame F, float *__restrict__ grad_coef)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NCOEF) grad_coef[i] += (float)(g_idx[i] / F.vox[i % 3]);
}

cudaError_t launch_motion_grad_finish(const float *theta, const float *dRdw, const double *grad_M,
                                      const double *grad_b, const double *grad_coef_idx, int n_views,
                                      const Grid &G, const double vox[3], const double origin[3],
                                      float *grad_theta, float *grad_coef, cudaStream_t stream)
{
    Frame F;
    const int n[3] = {G.nx, G.ny, G.nz};
    for (int a = 0; a < 3; ++a) {
        F.vox[a] = vox[a];
        F.origin[a] = origin[a];
        F.cen[a] = (double)((n[a] - 1) / 2);
    }
    if (grad_theta && theta) {
        motion_finish_kernel<<<(n_views + 127) / 128, 128, 0, stream>>>(theta, dRdw, grad_M, grad_b, n_views, F,
                                                                        grad_theta);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (grad_coef && grad_coef_idx) {
        coef_grad_finish_kernel<<<(NCOEF + 255) / 256, 256, 0, stream>>>(grad_coef_idx, F, grad_coef);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace ctrex

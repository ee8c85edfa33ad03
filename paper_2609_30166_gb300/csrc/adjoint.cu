// adjoint.cu -- matched ray-driven adjoint A^T (exact transpose of the
// projector in project.cu, motion included) and the gradient of <g, A x> with
// respect to the motion parameters (chain rule through the pose and the
// B-spline warp; the deformation is recomputed per sample, never stored).
// The paper motivates geometry refinement and learned components (Sec. 5)
// but prints no such operator; both are the transpose / derivative of its
// Sec. 4.1 projector with the Sec. 2.2.2 / 3.1 warp.
#include "ray.cuh"

// 4 resident CTAs per SM for the motion gradient: registers capped at 128
// (a few bytes of spills), measured faster than 167 registers at 3 CTAs
#ifndef CTREX_MGRAD_MIN_BLOCKS
#define CTREX_MGRAD_MIN_BLOCKS 4
#endif

namespace ctrex {

constexpr int ADJ_TX = 32, ADJ_TY = 4;
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
// two lanes, so a sample issues about 5 reductions instead of 8 (the
// reductions' L1/TEX path bounds the kernel without motion; with motion the
// spline evaluation does).  The zero lanes belong to neighbouring voxels
// (possibly of the adjacent row) inside the volume; adding +0 leaves them
// unchanged.  vec: the volume is 16-byte aligned; nvox: its element count.
__device__ __forceinline__ void scatter_trilinear(float *__restrict__ vol, int nx, int ny, int nz, const float c[3],
                                                  const float gc[3], float val, bool vec, long long nvox)
{
    const float fx = floorf(gc[0]), fy = floorf(gc[1]), fz = floorf(gc[2]);
    const int ix = (int)fx + (int)c[0], iy = (int)fy + (int)c[1], iz = (int)fz + (int)c[2];
    const float ax = gc[0] - fx, ay = gc[1] - fy, az = gc[2] - fz;
    const float wx[2] = {1.0f - ax, ax}, wy[2] = {1.0f - ay, ay}, wz[2] = {1.0f - az, az};
    const bool in0 = (unsigned)ix < (unsigned)nx, in1 = (unsigned)(ix + 1) < (unsigned)nx;
#pragma unroll
    for (int dz = 0; dz < 2; ++dz) {
        const int z = iz + dz;
        if ((unsigned)z >= (unsigned)nz) continue;
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const int y = iy + dy;
            if ((unsigned)y >= (unsigned)ny) continue;
            const float wzy = val * wz[dz] * wy[dy];
            const long long e = ((long long)z * ny + y) * nx + ix;  // element of tap x0 (x0 may be -1)
            const int lane = (int)(e & 3);
            if (vec && lane != 3 && e >= 0 && (e | 3) < nvox) {
                float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                const float w0 = in0 ? wzy * wx[0] : 0.0f, w1 = in1 ? wzy * wx[1] : 0.0f;
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
                if (in0) atomicAdd(vol + e, wzy * wx[0]);
                if (in1) atomicAdd(vol + e + 1, wzy * wx[1]);
            }
        }
    }
}

template <bool MOTION>
__global__ void __launch_bounds__(ADJ_TX *ADJ_TY)
    adjoint_kernel(Grid G, const ViewGPU *__restrict__ views, const MotionGPU *__restrict__ motion,
                   const float *__restrict__ coef_g, const int *__restrict__ view_idx,
                   const float *__restrict__ proj, float *__restrict__ vol, unsigned *devcheck)
{
    __shared__ float4 s_coef[MOTION ? NCOEF / 3 : 1];  // padded: one vector load per coefficient
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
            for (int i = threadIdx.y * ADJ_TX + threadIdx.x; i < NCOEF / 3; i += ADJ_TX * ADJ_TY)
                s_coef[i] = make_float4(coef_g[3 * i], coef_g[3 * i + 1], coef_g[3 * i + 2], 0.0f);
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
    float cen[3];
    grid_centre(G, cen);
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
            scatter_trilinear(vol, G.nx, G.ny, G.nz, cen, gc, val, vec, nvox);
        }
    }
}

cudaError_t launch_adjoint(const FwdArgs &a, const float *proj, float *vol)
{
    if (a.n_idx == 0) return cudaSuccess;
    const Grid &G = *a.grid;
    const dim3 grid((G.nu + ADJ_TX - 1) / ADJ_TX, a.n_idx, (G.nv + ADJ_TY - 1) / ADJ_TY);
    const dim3 block(ADJ_TX, ADJ_TY);
    if (a.motion)
        adjoint_kernel<true><<<grid, block, 0, a.stream>>>(G, a.views, a.motion, a.coef_idx, a.view_idx,
                                                          proj, vol, a.devcheck);
    else
        adjoint_kernel<false><<<grid, block, 0, a.stream>>>(G, a.views, nullptr, nullptr, a.view_idx, proj,
                                                           vol, a.devcheck);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Motion gradient
// ---------------------------------------------------------------------------

// Zero-padded trilinear interpolant's gradient (index units) inside floor(g).
template <typename TV>
__device__ __forceinline__ void trilinear_grad(const TV *__restrict__ vol, int nx, int ny, int nz,
                                               const float g[3], float grad[3])
{
    const float fx = floorf(g[0]), fy = floorf(g[1]), fz = floorf(g[2]);
    const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
    const float ax = g[0] - fx, ay = g[1] - fy, az = g[2] - fz;
    float v[2][2][2];
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const int x = ix + dx, y = iy + dy, z = iz + dz;
                const bool in = (unsigned)x < (unsigned)nx && (unsigned)y < (unsigned)ny && (unsigned)z < (unsigned)nz;
                v[dz][dy][dx] = in ? Storage<TV>::load(vol + (z * ny + y) * nx + x) : 0.0f;
            }
    const float by0 = 1.0f - ay, bz0 = 1.0f - az, bx0 = 1.0f - ax;
    grad[0] = bz0 * (by0 * (v[0][0][1] - v[0][0][0]) + ay * (v[0][1][1] - v[0][1][0])) +
              az * (by0 * (v[1][0][1] - v[1][0][0]) + ay * (v[1][1][1] - v[1][1][0]));
    grad[1] = bz0 * (bx0 * (v[0][1][0] - v[0][0][0]) + ax * (v[0][1][1] - v[0][0][1])) +
              az * (bx0 * (v[1][1][0] - v[1][0][0]) + ax * (v[1][1][1] - v[1][0][1]));
    grad[2] = by0 * (bx0 * (v[1][0][0] - v[0][0][0]) + ax * (v[1][0][1] - v[0][0][1])) +
              ay * (bx0 * (v[1][1][0] - v[0][1][0]) + ax * (v[1][1][1] - v[0][1][1]));
}

// One sample of the motion gradient: accumulates dL/dM, dL/db (registers)
// and dL/dcoef (shared memory, warp-reduced when the warp shares one cell).
template <typename TV>
__device__ __forceinline__ void grad_sample(const Grid &G, const MotionGPU &m, const float *coef,
                                            const TV *__restrict__ vol, const float g[3], float scale,
                                            bool active, float gM[9], float gb[3], float *s_gcoef)
{
    float gp[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        gp[r] = fmaf(m.M[3 * r], g[0], fmaf(m.M[3 * r + 1], g[1], fmaf(m.M[3 * r + 2], g[2], m.b[r])));
    int i0[3] = {1, 1, 1};
    float f[3] = {0.f, 0.f, 0.f};
    bool act[3] = {false, false, false};
    float wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
    float u[3] = {0.f, 0.f, 0.f};
    float J[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // J[comp][axis]
    const bool spline = coef != nullptr && m.s != 0.0f;
    if (spline) {
#pragma unroll
        for (int a = 0; a < 3; ++a) spline_coord(gp[a], G.spl_scale[a], i0[a], f[a], act[a]);
        bspline_weights(f[0], wx);
        bspline_weights(f[1], wy);
        bspline_weights(f[2], wz);
        bspline_dweights(f[0], dx);
        bspline_dweights(f[1], dy);
        bspline_dweights(f[2], dz);
        const float sx = act[0] ? G.spl_scale[0] : 0.f, sy = act[1] ? G.spl_scale[1] : 0.f,
                    sz = act[2] ? G.spl_scale[2] : 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int cz = min(i0[2] - 1 + k, 7);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int cy = min(i0[1] - 1 + j, 7);
                const float *row = coef + 3 * ((cz * 8 + cy) * 8);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int cx = min(i0[0] - 1 + i, 7);
                    const float w0 = wx[i] * wy[j] * wz[k];
                    const float w1 = dx[i] * wy[j] * wz[k] * sx;
                    const float w2 = wx[i] * dy[j] * wz[k] * sy;
                    const float w3 = wx[i] * wy[j] * dz[k] * sz;
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float cv = row[3 * cx + c];
                        u[c] = fmaf(w0, cv, u[c]);
                        J[3 * c + 0] = fmaf(w1, cv, J[3 * c + 0]);
                        J[3 * c + 1] = fmaf(w2, cv, J[3 * c + 1]);
                        J[3 * c + 2] = fmaf(w3, cv, J[3 * c + 2]);
                    }
                }
            }
        }
    }
    const float yv[3] = {fmaf(m.s, u[0], gp[0]), fmaf(m.s, u[1], gp[1]), fmaf(m.s, u[2], gp[2])};
    float gy[3] = {0.f, 0.f, 0.f};
    if (active && yv[0] >= -1.0f && yv[0] < (float)G.nx && yv[1] >= -1.0f && yv[1] < (float)G.ny &&
        yv[2] >= -1.0f && yv[2] < (float)G.nz)
        trilinear_grad(vol, G.nx, G.ny, G.nz, yv, gy);
#pragma unroll
    for (int c = 0; c < 3; ++c) gy[c] *= scale;  // dL/dy (index units)
    // dL/dg' = dL/dy (I + s J)
    float ggp[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ggp[a] = gy[a] + m.s * (gy[0] * J[a] + gy[1] * J[3 + a] + gy[2] * J[6 + a]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        gb[r] += ggp[r];
        gM[3 * r + 0] = fmaf(ggp[r], g[0], gM[3 * r + 0]);
        gM[3 * r + 1] = fmaf(ggp[r], g[1], gM[3 * r + 1]);
        gM[3 * r + 2] = fmaf(ggp[r], g[2], gM[3 * r + 2]);
    }
    if (s_gcoef == nullptr || m.s == 0.0f) return;
    // dL/dcoef[cell + (i, j, k)][c] += s * dL/dy[c] * wx[i] wy[j] wz[k] for the
    // 4 x 4 x 4 support of each lane's spline cell.  Lanes are served one cell
    // at a time (a warp's rays usually share one cell, rarely two); for the
    // lanes of that cell the 192 contributions are summed across the warp by
    // a reduce-scatter in six passes of 32 entries (31 shuffles each), after
    // which lane l owns entry 32 p + l and adds it to shared memory: no two
    // lanes of a warp touch the same address.
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int cell = (i0[2] * 8 + i0[1]) * 8 + i0[0];
    unsigned pending = __ballot_sync(full, active && scale != 0.0f);
    const float vs[3] = {m.s * gy[0], m.s * gy[1], m.s * gy[2]};
    while (pending) {  // warp-uniform
        const int leader = __ffs(pending) - 1;
        const int lcell = __shfl_sync(full, cell, leader);
        const bool mine = ((pending >> lane) & 1u) && cell == lcell;
        const float on = mine ? 1.0f : 0.0f;
        const int li0[3] = {__shfl_sync(full, i0[0], leader), __shfl_sync(full, i0[1], leader),
                            __shfl_sync(full, i0[2], leader)};
        // entry e = c * 64 + (k * 16 + j * 4 + i): pass p (32 entries) holds one
        // component c = p / 2 and the two z planes k = 2 (p % 2) + {0, 1}
#pragma unroll 1
        for (int pass = 0; pass < 6; ++pass) {
            const float vc = on * (pass < 2 ? vs[0] : (pass < 4 ? vs[1] : vs[2]));
            const float wz0 = (pass & 1) ? wz[2] : wz[0], wz1 = (pass & 1) ? wz[3] : wz[1];
            float v[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = vc * (q < 16 ? wz0 : wz1) * wy[(q >> 2) & 3] * wx[q & 3];
            // recursive halving: after the offset-o stage a lane keeps the half
            // of its entries whose bit matches its own lane bit o
#pragma unroll
            for (int o = 16, half = 16; o > 0; o >>= 1, half >>= 1) {
                const bool upper = (lane & o) != 0;
#pragma unroll
                for (int q = 0; q < half; ++q) {
                    const float send = upper ? v[q] : v[q + half];
                    const float keep = upper ? v[q + half] : v[q];
                    v[q] = keep + __shfl_xor_sync(full, send, o);
                }
            }
            // lane owns entry 32 pass + lane: c = pass / 2, (i, j, k) from the lane
            const int c = pass >> 1;
            const int cx = min(li0[0] - 1 + (lane & 3), 7), cy = min(li0[1] - 1 + ((lane >> 2) & 3), 7),
                      cz = min(li0[2] - 1 + 2 * (pass & 1) + (lane >> 4), 7);
            if (v[0] != 0.0f) atomicAdd(s_gcoef + 3 * ((cz * 8 + cy) * 8 + cx) + c, v[0]);
        }
        pending &= ~__ballot_sync(full, mine);
    }
}

template <typename TV>
__global__ void __launch_bounds__(ADJ_TX *ADJ_TY, CTREX_MGRAD_MIN_BLOCKS)
    motion_grad_kernel(Grid G, const ViewGPU *__restrict__ views, const MotionGPU *__restrict__ motion,
                       const float *__restrict__ coef_g, const int *__restrict__ view_idx,
                       const TV *__restrict__ vol, const float *__restrict__ gproj,
                       float *__restrict__ grad_M, float *__restrict__ grad_b,
                       float *__restrict__ grad_coef, unsigned *devcheck)
{
    __shared__ float s_coef[NCOEF];
    __shared__ float s_gcoef[NCOEF];
    __shared__ float s_red[12][ADJ_TX * ADJ_TY / 32];
    const int tid = threadIdx.y * ADJ_TX + threadIdx.x;
    const int k = blockIdx.y;
    int view = view_idx ? view_idx[k] : k;
    const bool view_ok = view >= 0 && view < G.n_views;
    if (!view_ok) {
        if (tid == 0) atomicOr(devcheck, (unsigned)DEVCHECK_OOB);
        return;  // uniform over the CTA
    }
    const MotionGPU mo = motion[view];
    const float *coef = nullptr;
    if (coef_g) {
        for (int i = tid; i < NCOEF; i += ADJ_TX * ADJ_TY) {
            s_coef[i] = coef_g[i];
            s_gcoef[i] = 0.0f;
        }
        coef = s_coef;
    }
    __syncthreads();
    float gM[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, gb[3] = {0.f, 0.f, 0.f};
    int iu, iv;
    tile_pixel<true>(blockIdx.x * ADJ_TX, blockIdx.z * ADJ_TY, iu, iv);
    const bool pix_ok = iu < G.nu && iv < G.nv;
    const float y = pix_ok ? gproj[((size_t)k * G.nv + iv) * G.nu + iu] * G.inv_sub : 0.0f;
    float *gco = (coef_g && grad_coef) ? s_gcoef : nullptr;
    for (int s = 0; s < G.n_sub; ++s) {
        Ray R;
        bool hit = pix_ok && setup_ray(G, views[view * G.n_sub + s], (float)(pix_ok ? iu : 0),
                                       (float)(pix_ok ? iv : 0), R);
        // the warp-collective shared-memory reduction needs every lane: lanes
        // without work run the loop with zero weight up to the warp's longest ray
        int K = hit ? R.K : 0;
        int Kmax = K;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) Kmax = max(Kmax, __shfl_xor_sync(0xffffffffu, Kmax, off));
        for (int kk = 0; kk < Kmax; ++kk) {
            float g[3] = {0.f, 0.f, 0.f};
            float sc = 0.0f;
            const bool act = hit && kk < K && y != 0.0f;
            if (hit && kk < K - 1) {
                g[0] = fmaf((float)kk, R.sg[0], R.g0[0]);
                g[1] = fmaf((float)kk, R.sg[1], R.g0[1]);
                g[2] = fmaf((float)kk, R.sg[2], R.g0[2]);
                sc = y * G.step_mm;
            } else if (hit && kk == K - 1) {
                g[0] = R.g_last[0];
                g[1] = R.g_last[1];
                g[2] = R.g_last[2];
                sc = R.w_last > 0.0f ? y * R.w_last : 0.0f;
            }
            grad_sample(G, mo, coef, vol, g, act ? sc : 0.0f, act, gM, gb, gco);
        }
    }
    // CTA reduction of the 12 pose-gradient entries, one atomic each
    float vals[12];
#pragma unroll
    for (int q = 0; q < 9; ++q) vals[q] = gM[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) vals[9 + q] = gb[q];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        float v = vals[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if ((tid & 31) == 0) s_red[q][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < 12) {
        float v = 0.0f;
#pragma unroll
        for (int w = 0; w < ADJ_TX * ADJ_TY / 32; ++w) v += s_red[tid][w];
        if (grad_M && tid < 9) atomicAdd(grad_M + 9 * view + tid, v);
        if (grad_b && tid >= 9) atomicAdd(grad_b + 3 * view + (tid - 9), v);
    }
    if (gco) {
        for (int i = tid; i < NCOEF; i += ADJ_TX * ADJ_TY) {
            const float v = s_gcoef[i];
            if (v != 0.0f) atomicAdd(grad_coef + i, v);
        }
    }
}

cudaError_t launch_motion_grad(const FwdArgs &a, const float *gproj, float *grad_M, float *grad_b,
                               float *grad_coef_idx)
{
    if (a.n_idx == 0) return cudaSuccess;
    const Grid &G = *a.grid;
    const dim3 grid((G.nu + ADJ_TX - 1) / ADJ_TX, a.n_idx, (G.nv + ADJ_TY - 1) / ADJ_TY);
    const dim3 block(ADJ_TX, ADJ_TY);
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
__global__ void motion_finish_kernel(const float *__restrict__ theta, const float *__restrict__ dRdw,
                                     const float *__restrict__ gM, const float *__restrict__ gb, int n_views,
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
        for (int c = 0; c < 3; ++c)
            gMw[3 * r + c] = gM[9 * v + 3 * r + c] * F.vox[c] / F.vox[r] + gb[3 * v + r] * F.origin[c] / F.vox[r];
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

__global__ void coef_grad_finish_kernel(const float *__restrict__ g_idx, Frame F, float *__restrict__ grad_coef)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NCOEF) grad_coef[i] += (float)(g_idx[i] / F.vox[i % 3]);
}

cudaError_t launch_motion_grad_finish(const float *theta, const float *dRdw, const float *grad_M,
                                      const float *grad_b, const float *grad_coef_idx, int n_views,
                                      const double vox[3], const double origin[3], float *grad_theta,
                                      float *grad_coef, cudaStream_t stream)
{
    Frame F;
    for (int a = 0; a < 3; ++a) {
        F.vox[a] = vox[a];
        F.origin[a] = origin[a];
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

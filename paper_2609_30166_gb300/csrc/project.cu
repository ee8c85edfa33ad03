// project.cu -- ray-driven cone-beam forward projector A (Sec. 4.1
// "Projection operator"), its angular sub-sample loop (Sec. 3.4, Sec. 4.2.2),
// the per-sample motion warp (Sec. 3.1.1, Sec. 4.2.1) and the fused
// detector-space correction R (p - A x) with residual norms (Sec. 4.1
// "Correction kernel", Eq. (1) terms 1-2).
//
// Launch shape: one thread per detector pixel, 32 x 4 pixels per CTA so that
// a warp covers 32 neighbouring pixels of one detector row (neighbouring rays
// sample neighbouring voxels at every step).  Grid = (u tiles, views, v
// tiles): the CTAs resident at one time cover a band of detector rows across
// many views, whose rays all cross the same z-slab of the volume, so that
// slab stays in L2 while it is being sampled.
#include "atlas.cuh"
#include "cylinder.cuh"
#include "dyrect.cuh"
#include "fwd_common.cuh"
#include "joseph.cuh"
#include "ray.cuh"
#include "roi.cuh"

namespace ctrex {


template <typename TV>
__device__ __forceinline__ float LinearSampler<TV>::operator()(float gx, float gy, float gz, float &wsum) const
{
    return trilinear(vol, nx, ny, nz, gx, gy, gz, wsum);
}

template <typename TV>
__device__ __forceinline__ float LinearSampler<TV>::interior(float gx, float gy, float gz) const
{
    float ws;
    return trilinear(vol, nx, ny, nz, gx, gy, gz, ws);
}

// Integral of one pixel (mean over its sub-angle rays): value and row sum.
// On the cylindrical domain the ray is clipped to the bounding cylinder and
// every sample is mapped to (r, phi, z) by the sampler; the rest is shared.
template <typename Sampler, bool MOTION>
__device__ __forceinline__ void pixel_integral(const Grid &G, const ViewGPU *__restrict__ views,
                                               const MotionGPU &mo, const float4 *coef,
                                               const Sampler &vol, int view, float u,
                                               float v, float &val, float &rs)
{
    float acc = 0.0f, acc_rs = 0.0f;
    for (int s = 0; s < G.n_sub; ++s) {
        const ViewGPU V = views[view * G.n_sub + s];
        if constexpr (Sampler::ROI) {
            float a, ars;
            roi_integral<false>(G, vol, V, u, v, a, ars);
            acc += a;
            acc_rs += ars;
            continue;
        }
        if constexpr (Sampler::JOSEPH) {
            float a, ars;
            joseph_integral(G, vol, V, u, v, a, ars);
            acc += a;
            acc_rs += ars;
            continue;
        }
        Ray R;
        if constexpr (Sampler::CYLINDER) {
            if (!setup_ray_cyl(G, vol.C, V, u, v, R)) continue;
        } else {
            if (!setup_ray(G, V, u, v, R)) continue;
        }
        float a = 0.0f, ars = 0.0f;
        const int Km1 = R.K - 1;
        int ka = Km1, kb = Km1;
        if (!MOTION && !Sampler::CYLINDER) interior_range(G, R, ka, kb);
        auto general = [&](int k) {
            float g[3];
            g[0] = fmaf((float)k, R.sg[0], R.g0[0]);
            g[1] = fmaf((float)k, R.sg[1], R.g0[1]);
            g[2] = fmaf((float)k, R.sg[2], R.g0[2]);
            if (MOTION) {
                float y[3];
                warp_sample(G, mo, coef, g, y);
                g[0] = y[0];
                g[1] = y[1];
                g[2] = y[2];
            }
            float ws;
            a += vol(g[0], g[1], g[2], ws);
            ars += ws;
        };
        const int kstop = MOTION ? Km1 : ka;
        for (int k = 0; k < kstop; ++k) general(k);
        if (!MOTION) {
            for (int k = ka; k < kb; ++k)
                a += vol.interior(fmaf((float)k, R.sg[0], R.g0[0]), fmaf((float)k, R.sg[1], R.g0[1]),
                                  fmaf((float)k, R.sg[2], R.g0[2]));
            ars += (float)(kb - ka);
            for (int k = kb; k < Km1; ++k) general(k);
        }
        a *= G.step_mm;
        ars *= G.step_mm;
        if (R.w_last > 0.0f) {
            float g[3] = {R.g_last[0], R.g_last[1], R.g_last[2]};
            if (MOTION) {
                float y[3];
                warp_sample(G, mo, coef, g, y);
                g[0] = y[0];
                g[1] = y[1];
                g[2] = y[2];
            }
            float ws;
            a = fmaf(R.w_last, vol(g[0], g[1], g[2], ws), a);
            ars = fmaf(R.w_last, ws, ars);
        }
        acc += a;
        acc_rs += ars;
    }
    val = acc * G.inv_sub;
    rs = acc_rs * G.inv_sub;
}

template <typename Sampler, typename TP, int MODE, bool MOTION>
__device__ __forceinline__ void fwd_body(Grid G, const ViewGPU *__restrict__ views,
                                         const MotionGPU *__restrict__ motion, const float *__restrict__ coef_g,
                                         const Sampler &vol_in, const int *__restrict__ view_idx,
                                         TP *__restrict__ out, float *__restrict__ rowsum_out,
                                         const TP *__restrict__ p, float *__restrict__ partials, unsigned *devcheck,
                                         int p_by_view)
{
    __shared__ float4 s_coef[MOTION ? NCOEF_PAD : 1];  // zero-padded 9^3 float4 copy of the coefficients
    __shared__ float s_red[2][FWD_TX * FWD_TY / 32];
    __shared__ float2 s_tile[Sampler::TILE_TABLE];
    Sampler vol = vol_in;
    vol.bind(s_tile, threadIdx.y * FWD_TX + threadIdx.x, FWD_TX * FWD_TY);
    const int k = blockIdx.y;
    int view = view_idx ? view_idx[k] : k;
    bool ok = true;
    if (view < 0 || view >= G.n_views) {
        if (threadIdx.x == 0 && threadIdx.y == 0) atomicOr(devcheck, (unsigned)DEVCHECK_OOB);
        ok = false;
        view = 0;
    }
    if constexpr (Sampler::DYRECT) vol.set_view(view);  // the view's acquisition time
    MotionGPU mo;
    const float4 *coef = nullptr;
    if (MOTION) {
        mo = motion[view];
        if (coef_g != nullptr) {
            load_coef_padded(s_coef, coef_g, threadIdx.y * FWD_TX + threadIdx.x, FWD_TX * FWD_TY);
            coef = s_coef;
        }
        __syncthreads();
    }
    int iu, iv;
    tile_pixel<MOTION>(blockIdx.x * FWD_TX, blockIdx.z * FWD_TY, iu, iv);
    const bool in_pix = iu < G.nu && iv < G.nv;
    const bool inside = ok && in_pix;
    float val = 0.0f, rs = 0.0f;
    if (inside) pixel_integral<Sampler, MOTION>(G, views, mo, coef, vol, view, (float)iu, (float)iv, val, rs);
    fwd_epilogue<TP, MODE>(G, k, view, ok, in_pix, iu, iv, val, rs, out, rowsum_out, p, partials, p_by_view,
                           s_red);
}

template <typename Sampler, typename TP, int MODE, bool MOTION>
__global__ void __launch_bounds__(FWD_TX *FWD_TY)
    fwd_kernel(Grid G, const ViewGPU *__restrict__ views, const MotionGPU *__restrict__ motion,
               const float *__restrict__ coef_g, const Sampler vol_in, const int *__restrict__ view_idx,
               TP *__restrict__ out, float *__restrict__ rowsum_out, const TP *__restrict__ p,
               float *__restrict__ partials, unsigned *devcheck, int p_by_view)
{
    fwd_body<Sampler, TP, MODE, MOTION>(G, views, motion, coef_g, vol_in, view_idx, out, rowsum_out, p, partials,
                                        devcheck, p_by_view);
}

// Projectors whose sampler declares MIN_BLOCKS > 0 (the event model and
// the multi-resolution ROI) run through this entry, compiled for that many
// resident CTAs per SM; the others keep fwd_kernel's bounds.  Event model:
// 72 registers and 7 CTAs gave 1128 ms on the 512^3 event workload, 56
// registers and 9 CTAs 1058 ms.
template <typename Sampler, typename TP, int MODE>
__global__ void __launch_bounds__(FWD_TX *FWD_TY, Sampler::MIN_BLOCKS > 0 ? Sampler::MIN_BLOCKS : 1)
    fwd_kernel_mb(Grid G, const ViewGPU *__restrict__ views, const Sampler vol_in, const int *__restrict__ view_idx,
                  TP *__restrict__ out, float *__restrict__ rowsum_out, const TP *__restrict__ p,
                  float *__restrict__ partials, unsigned *devcheck, int p_by_view)
{
    fwd_body<Sampler, TP, MODE, false>(G, views, nullptr, nullptr, vol_in, view_idx, out, rowsum_out, p, partials,
                                       devcheck, p_by_view);
}

// Second pass of the residual reduction: one CTA, fixed order, FP64.
__global__ void __launch_bounds__(1024) finish_sums_kernel(const float *__restrict__ partials, size_t n,
                                                           double *__restrict__ sums)
{
    __shared__ double s[2][1024];
    double a = 0.0, b = 0.0;
    for (size_t i = threadIdx.x; i < n; i += blockDim.x) {
        a += (double)partials[2 * i];
        b += (double)partials[2 * i + 1];
    }
    s[0][threadIdx.x] = a;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            s[0][threadIdx.x] += s[0][threadIdx.x + off];
            s[1][threadIdx.x] += s[1][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        sums[0] = s[0][0];
        sums[1] = s[1][0];
    }
}

// Exact sample count (same set-up arithmetic as the projector): ray
// segments, or for the Joseph projector slice crossings with a tap inside.
enum CountKind { COUNT_BOX = 0, COUNT_CYL = 1, COUNT_JOSEPH = 2, COUNT_ROI = 3 };
template <int KIND>
__global__ void __launch_bounds__(FWD_TX *FWD_TY)
    count_kernel(Grid G, CylGPU C, RoiGPU Q, const ViewGPU *__restrict__ views, const int *__restrict__ view_idx,
                 unsigned long long *out)
{
    const int k = blockIdx.y;
    const int view = view_idx ? view_idx[k] : k;
    if (view < 0 || view >= G.n_views) return;
    const int iu = blockIdx.x * FWD_TX + threadIdx.x;
    const int iv = blockIdx.z * FWD_TY + threadIdx.y;
    unsigned long long n = 0;
    if (iu < G.nu && iv < G.nv) {
        for (int s = 0; s < G.n_sub; ++s) {
            Ray R;
            const ViewGPU &V = views[view * G.n_sub + s];
            if (KIND == COUNT_ROI) {
                RoiSampler rs{};
                rs.R = Q;
                float a, b;
                n += (unsigned long long)roi_integral<true>(G, rs, V, (float)iu, (float)iv, a, b);
                continue;
            }
            if (KIND == COUNT_JOSEPH) {
                JRay J;
                if (joseph_setup(G, V, (float)iu, (float)iv, J)) n += (unsigned long long)(J.khi - J.klo + 1);
                continue;
            }
            const bool hit = KIND == COUNT_CYL ? setup_ray_cyl(G, C, V, (float)iu, (float)iv, R)
                                               : setup_ray(G, V, (float)iu, (float)iv, R);
            if (hit) n += (unsigned long long)R.K;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) n += __shfl_xor_sync(0xffffffffu, n, off);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(out, n);
}

static dim3 fwd_grid(const Grid &G, int n_idx)
{
    return dim3((G.nu + FWD_TX - 1) / FWD_TX, n_idx, (G.nv + FWD_TY - 1) / FWD_TY);
}

int forward_partials_needed(const Grid &G, int n_idx)
{
    const dim3 g = fwd_grid(G, n_idx);
    return (int)(g.x * g.y * g.z);
}

template <typename Sampler, typename TP, int MODE>
static cudaError_t fwd_launch(const FwdArgs &a, const Sampler &smp, TP *out, float *rowsum, const TP *p,
                              float *partials)
{
    const Grid &G = *a.grid;
    const dim3 grid = fwd_grid(G, a.n_idx), block(FWD_TX, FWD_TY);
    if constexpr (!Sampler::CYLINDER && !Sampler::JOSEPH && !Sampler::ROI && !Sampler::DYRECT) {
        if (a.motion) {
            fwd_kernel<Sampler, TP, MODE, true><<<grid, block, 0, a.stream>>>(
                G, a.views, a.motion, a.coef_idx, smp, a.view_idx, out, rowsum, p, partials, a.devcheck,
                a.p_by_view);
            return cudaGetLastError();
        }
    } else if (a.motion) {
        return cudaErrorNotSupported;  // the motion warp is defined for the trilinear Cartesian projector only
    }
    if constexpr (Sampler::MIN_BLOCKS > 0)
        fwd_kernel_mb<Sampler, TP, MODE><<<grid, block, 0, a.stream>>>(G, a.views, smp, a.view_idx, out, rowsum, p,
                                                                      partials, a.devcheck, a.p_by_view);
    else
        fwd_kernel<Sampler, TP, MODE, false><<<grid, block, 0, a.stream>>>(
            G, a.views, nullptr, nullptr, smp, a.view_idx, out, rowsum, p, partials, a.devcheck, a.p_by_view);
    return cudaGetLastError();
}

// Texture-atlas sampling when the context has uploaded the volume into one;
// row-major loads otherwise (volumes beyond the 2D texture limits).
template <typename TP, int MODE>
static cudaError_t fwd_dispatch_sampler(const FwdArgs &a, TP *out, float *rowsum, const TP *p, float *partials)
{
    if (a.roi) {  // context and ROI grids, each from its own atlas
        if (!a.atlas || !a.roi_atlas || a.cyl || a.joseph) return cudaErrorInvalidValue;
        RoiSampler rs{RoiAtlasSampler{*a.atlas}, RoiAtlasSampler{*a.roi_atlas}, *a.roi};
        return fwd_launch<RoiSampler, TP, MODE>(a, rs, out, rowsum, p, partials);
    }
    if (a.dyr) {  // mu0 from the volume atlas, mu1 and tau from their own
        if (!a.atlas || !a.dyr->mu1 || !a.dyr->tau_atlas || a.cyl || a.joseph) return cudaErrorInvalidValue;
        DyrectSampler ds{*a.atlas, *a.dyr->mu1, *a.dyr->tau_atlas, a.dyr->t_view, a.dyr->tau_brick, a.dyr->bnx,
                         a.dyr->bny};
        return fwd_launch<DyrectSampler, TP, MODE>(a, ds, out, rowsum, p, partials);
    }
    if (a.joseph) {  // the Joseph projector reads its three-stack atlas only
        if (!a.atlas || a.cyl) return cudaErrorInvalidValue;
        const Grid &G = *a.grid;
        JosephSampler js{AtlasSampler{*a.atlas}, {G.nx, G.ny, G.nz}, {0, G.nx, G.nx + G.ny}};
        return fwd_launch<JosephSampler, TP, MODE>(a, js, out, rowsum, p, partials);
    }
    if (a.cyl) {  // the cylindrical domain is sampled from its atlas only
        if (!a.atlas) return cudaErrorInvalidValue;
        return fwd_launch<CylSampler, TP, MODE>(a, CylSampler{AtlasSampler{*a.atlas}, *a.cyl}, out, rowsum, p,
                                               partials);
    }
    if (a.atlas) return fwd_launch<AtlasSampler, TP, MODE>(a, AtlasSampler{*a.atlas}, out, rowsum, p, partials);
    const Grid &G = *a.grid;
    if (a.vol_dtype == CTREX_F32)
        return fwd_launch<LinearSampler<float>, TP, MODE>(
            a, LinearSampler<float>{static_cast<const float *>(a.vol), G.nx, G.ny, G.nz}, out, rowsum, p, partials);
    return fwd_launch<LinearSampler<__nv_bfloat16>, TP, MODE>(
        a, LinearSampler<__nv_bfloat16>{static_cast<const __nv_bfloat16 *>(a.vol), G.nx, G.ny, G.nz}, out, rowsum,
        p, partials);
}

template <int MODE>
static cudaError_t fwd_dispatch(const FwdArgs &a, int pdt, void *out, float *rowsum, const void *p,
                                float *partials)
{
    if (pdt == CTREX_F32)
        return fwd_dispatch_sampler<float, MODE>(a, (float *)out, rowsum, (const float *)p, partials);
    return fwd_dispatch_sampler<__nv_bfloat16, MODE>(a, (__nv_bfloat16 *)out, rowsum, (const __nv_bfloat16 *)p,
                                                     partials);
}

cudaError_t launch_forward(const FwdArgs &a, void *proj, int proj_dtype, float *rowsum)
{
    if (a.n_idx == 0) return cudaSuccess;
    return fwd_dispatch<MODE_PROJECT>(a, proj_dtype, proj, rowsum, nullptr, nullptr);
}

cudaError_t launch_forward_correct(const FwdArgs &a, const void *p, int p_dtype, void *r, int r_dtype,
                                   float *partials, int n_partials_cap, double *sums)
{
    if (p_dtype != r_dtype) return cudaErrorInvalidValue;
    if (a.n_idx == 0) {
        if (sums) return cudaMemsetAsync(sums, 0, 2 * sizeof(double), a.stream);
        return cudaSuccess;
    }
    const int n = forward_partials_needed(*a.grid, a.n_idx);
    if (n > n_partials_cap) return cudaErrorInvalidValue;
    cudaError_t e = fwd_dispatch<MODE_CORRECT>(a, p_dtype, r, nullptr, p, partials);
    if (e != cudaSuccess || sums == nullptr) return e;
    finish_sums_kernel<<<1, 1024, 0, a.stream>>>(partials, (size_t)n, sums);
    return cudaGetLastError();
}

cudaError_t launch_count_samples(const FwdArgs &a, unsigned long long *out)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), a.stream);
    if (e != cudaSuccess || a.n_idx == 0) return e;
    const dim3 grid = fwd_grid(*a.grid, a.n_idx), block(FWD_TX, FWD_TY);
    if (a.cyl)
        count_kernel<COUNT_CYL><<<grid, block, 0, a.stream>>>(*a.grid, *a.cyl, RoiGPU{}, a.views, a.view_idx, out);
    else if (a.joseph)
        count_kernel<COUNT_JOSEPH><<<grid, block, 0, a.stream>>>(*a.grid, CylGPU{}, RoiGPU{}, a.views, a.view_idx,
                                                                 out);
    else if (a.roi)
        count_kernel<COUNT_ROI><<<grid, block, 0, a.stream>>>(*a.grid, CylGPU{}, *a.roi, a.views, a.view_idx, out);
    else
        count_kernel<COUNT_BOX><<<grid, block, 0, a.stream>>>(*a.grid, CylGPU{}, RoiGPU{}, a.views, a.view_idx,
                                                              out);
    return cudaGetLastError();
}

// (min, max) of tau over each 8^3 brick and the voxel past each of its
// upper faces: one thread per brick (run once, by ctrex_set_dyrect).
__global__ void tau_brick_kernel(const float *__restrict__ tau, int nx, int ny, int nz, int bnx, int bny, int bnz,
                                 float2 *__restrict__ out)
{
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= (long long)bnx * bny * bnz) return;
    const int bx = (int)(b % bnx), by = (int)((b / bnx) % bny), bz = (int)(b / ((long long)bnx * bny));
    const int x1 = min(8 * bx + 8, nx - 1), y1 = min(8 * by + 8, ny - 1), z1 = min(8 * bz + 8, nz - 1);
    float lo = INFINITY, hi = -INFINITY;
    bool nan = false;
    for (int z = 8 * bz; z <= z1; ++z)
        for (int y = 8 * by; y <= y1; ++y) {
            const float *row = tau + ((size_t)z * ny + y) * nx;
            for (int x = 8 * bx; x <= x1; ++x) {
                const float v = __ldg(row + x);
                nan |= v != v;
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
            }
        }
    // a NaN transition time sends its tap to mu1 (t < NaN is false): such a
    // brick never takes the mu0 shortcut, and the mu1 one only for t = +inf
    out[b] = nan ? make_float2(-INFINITY, INFINITY) : make_float2(lo, hi);
}

cudaError_t launch_tau_bricks(const float *tau, int nx, int ny, int nz, float2 *out, cudaStream_t stream)
{
    const int bnx = (nx + 7) / 8, bny = (ny + 7) / 8, bnz = (nz + 7) / 8;
    const long long n = (long long)bnx * bny * bnz;
    tau_brick_kernel<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(tau, nx, ny, nz, bnx, bny, bnz, out);
    return cudaGetLastError();
}

}  // namespace ctrex

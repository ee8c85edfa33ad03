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
#include "ctrex_internal.cuh"

namespace ctrex {

constexpr int BP_TX = 32, BP_TY = 4, BP_TZ = 2;
constexpr int BP_THREADS = BP_TX * BP_TY * BP_TZ;
constexpr int BP_CHUNK = 128;

template <typename TR, typename TV>
__global__ void __launch_bounds__(BP_THREADS)
    bp_kernel(Grid G, const ViewGPU *__restrict__ views, const int *__restrict__ view_idx, int n_idx,
              const TR *__restrict__ r, TV *__restrict__ vol, const float *__restrict__ w, float alpha,
              int normalize, int accumulate)
{
    __shared__ float4 sP[BP_CHUNK][3];
    __shared__ int sImg[BP_CHUNK];
    const int tid = (threadIdx.z * BP_TY + threadIdx.y) * BP_TX + threadIdx.x;
    const int ix = blockIdx.x * BP_TX + threadIdx.x;
    const int iy = blockIdx.y * BP_TY + threadIdx.y;
    const int iz = blockIdx.z * BP_TZ + threadIdx.z;
    const bool inside = ix < G.nx && iy < G.ny && iz < G.nz;
    const float fx = (float)ix, fy = (float)iy, fz = (float)iz;
    const int nu = G.nu, nv = G.nv;
    const size_t npix = (size_t)nu * nv;
    float b = 0.0f, c = 0.0f;
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
            sImg[t] = k;
        }
        __syncthreads();
        if (!inside) continue;
        for (int m = 0; m < cnt; ++m) {
            const float4 p2 = sP[m][2];
            const float h3 = fmaf(p2.x, fx, fmaf(p2.y, fy, fmaf(p2.z, fz, p2.w)));
            if (!(h3 > 0.0f)) continue;
            const float4 p0 = sP[m][0], p1 = sP[m][1];
            const float h1 = fmaf(p0.x, fx, fmaf(p0.y, fy, fmaf(p0.z, fz, p0.w)));
            const float h2 = fmaf(p1.x, fx, fmaf(p1.y, fy, fmaf(p1.z, fz, p1.w)));
            const float inv = __frcp_rn(h3);
            const float u = h1 * inv, v = h2 * inv;
            if (!(u > -1.0f && u < (float)nu && v > -1.0f && v < (float)nv)) continue;
            const float fu = floorf(u), fv = floorf(v);
            const int iu = (int)fu, iv = (int)fv;
            const float au = u - fu, av = v - fv;
            const float wu0 = iu >= 0 ? 1.0f - au : 0.0f;
            const float wu1 = iu + 1 < nu ? au : 0.0f;
            const float wv0 = iv >= 0 ? 1.0f - av : 0.0f;
            const float wv1 = iv + 1 < nv ? av : 0.0f;
            const int u0 = max(iu, 0), u1 = min(iu + 1, nu - 1);
            const int v0 = max(iv, 0), v1 = min(iv + 1, nv - 1);
            const TR *img = r + (size_t)sImg[m] * npix;
            const float r00 = Storage<TR>::load(img + v0 * nu + u0);
            const float r01 = Storage<TR>::load(img + v0 * nu + u1);
            const float r10 = Storage<TR>::load(img + v1 * nu + u0);
            const float r11 = Storage<TR>::load(img + v1 * nu + u1);
            b += fmaf(wv0, fmaf(wu0, r00, wu1 * r01), wv1 * fmaf(wu0, r10, wu1 * r11));
            c += (wu0 + wu1) * (wv0 + wv1);
        }
    }
    if (!inside) return;
    b *= G.inv_sub;
    c *= G.inv_sub;
    const size_t j = ((size_t)iz * G.ny + iy) * G.nx + ix;
    float scale = alpha;
    if (normalize) scale *= (c > 1e-6f ? 1.0f / c : 0.0f);
    if (w) scale *= __ldg(w + j);
    const float upd = scale * b;
    const float out = accumulate ? Storage<TV>::load(vol + j) + upd : upd;
    Storage<TV>::store(vol + j, out);
}

template <typename TR, typename TV>
static cudaError_t bp_launch(const BpArgs &a)
{
    const Grid &G = *a.grid;
    const dim3 block(BP_TX, BP_TY, BP_TZ);
    const dim3 grid((G.nx + BP_TX - 1) / BP_TX, (G.ny + BP_TY - 1) / BP_TY, (G.nz + BP_TZ - 1) / BP_TZ);
    bp_kernel<TR, TV><<<grid, block, 0, a.stream>>>(G, a.views, a.view_idx, a.n_idx,
                                                   static_cast<const TR *>(a.r), static_cast<TV *>(a.vol),
                                                   a.w, a.alpha, a.normalize, a.accumulate);
    return cudaGetLastError();
}

cudaError_t launch_backproject(const BpArgs &a)
{
    if (a.r_dtype == CTREX_F32) {
        if (a.vol_dtype == CTREX_F32) return bp_launch<float, float>(a);
        return bp_launch<float, __nv_bfloat16>(a);
    }
    if (a.vol_dtype == CTREX_F32) return bp_launch<__nv_bfloat16, float>(a);
    return bp_launch<__nv_bfloat16, __nv_bfloat16>(a);
}

}  // namespace ctrex

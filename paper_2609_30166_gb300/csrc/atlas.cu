// atlas.cu -- allocation, texture/surface objects and upload of slice atlases.
#include "atlas.cuh"

namespace ctrex {

// Zero every texel of a new array (its content is undefined): taps outside a
// slice read neighbouring tiles, unused tiles or padding with weight zero,
// and zero times a stale NaN would not be zero.
__global__ void __launch_bounds__(256) clear_kernel(cudaSurfaceObject_t surf, int W, int H, int bytes)
{
    const int x = blockIdx.x * 64 + (threadIdx.x & 63);
    const int y = blockIdx.y * 4 + (threadIdx.x >> 6);
    if (x >= W || y >= H) return;
    if (bytes == 4)
        surf2Dwrite(0u, surf, x * 4, y);
    else
        surf2Dwrite((unsigned short)0, surf, x * 2, y);
}

cudaError_t atlas_clear(cudaSurfaceObject_t surf, int W, int H, int bytes)
{
    const dim3 grid((W + 63) / 64, (H + 3) / 4);
    clear_kernel<<<grid, 256>>>(surf, W, H, bytes);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

void atlas_release(AtlasStore &s)
{
    if (s.tex) cudaDestroyTextureObject(s.tex);
    if (s.surf) cudaDestroySurfaceObject(s.surf);
    if (s.array) cudaFreeArray(s.array);
    s = AtlasStore();
}

cudaError_t atlas_ensure(AtlasStore &s, int w, int h, int n, bool bf16, int device, bool packed, bool wrap)
{
    packed = packed && bf16;
    if (wrap) h += 1;
    if (s.array && s.w == w && s.h == h && s.n == n && s.bf16 == (bf16 ? 1 : 0) && s.packed == (packed ? 1 : 0) &&
        s.wrap == (wrap ? 1 : 0))
        return cudaSuccess;
    atlas_release(s);
    int maxw = 0, maxh = 0;
    cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxSurface2DWidth, device);
    cudaDeviceGetAttribute(&maxh, cudaDevAttrMaxSurface2DHeight, device);
    int tw = 0, th = 0;
    cudaDeviceGetAttribute(&tw, cudaDevAttrMaxTexture2DWidth, device);
    cudaDeviceGetAttribute(&th, cudaDevAttrMaxTexture2DHeight, device);
    maxw = min(maxw, tw);
    maxh = min(maxh, th);
    // tiles per row: a power of two giving a roughly square atlas
    int tshift = 0;
    while ((1LL << tshift) * (long long)w * (1LL << tshift) * (long long)w < (long long)n * w * h) ++tshift;
    long long W = (1LL << tshift) * (long long)w;
    long long rows = (n + (1 << tshift) - 1) >> tshift;
    while (W > maxw && tshift > 0) {
        --tshift;
        W = (1LL << tshift) * (long long)w;
        rows = (n + (1 << tshift) - 1) >> tshift;
    }
    const long long H = rows * h;
    if (W > maxw || H > maxh || W < 1 || H < 1) return cudaErrorInvalidValue;
    cudaChannelFormatDesc desc = packed ? cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindUnsigned)
                                 : bf16 ? cudaCreateChannelDesc(16, 0, 0, 0, cudaChannelFormatKindUnsigned)
                                        : cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindFloat);
    cudaError_t e = cudaMallocArray(&s.array, &desc, (size_t)W, (size_t)H, cudaArraySurfaceLoadStore);
    if (e != cudaSuccess) {
        s.array = nullptr;
        return e;
    }
    cudaResourceDesc rd = {};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = s.array;
    cudaTextureDesc td = {};
    td.addressMode[0] = cudaAddressModeBorder;
    td.addressMode[1] = cudaAddressModeBorder;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    e = cudaCreateTextureObject(&s.tex, &rd, &td, nullptr);
    if (e == cudaSuccess) e = cudaCreateSurfaceObject(&s.surf, &rd);
    if (e == cudaSuccess) e = atlas_clear(s.surf, (int)W, (int)H, packed || !bf16 ? 4 : 2);
    if (e != cudaSuccess) {
        atlas_release(s);
        return e;
    }
    s.w = w;
    s.h = h;
    s.n = n;
    s.tshift = tshift;
    s.bf16 = bf16 ? 1 : 0;
    s.packed = packed ? 1 : 0;
    s.wrap = wrap ? 1 : 0;
    return cudaSuccess;
}

Atlas atlas_view(const AtlasStore &s)
{
    Atlas a;
    a.tex = s.tex;
    a.w = s.w;
    a.h = s.h;
    a.n = s.n;
    a.tshift = s.tshift;
    a.bf16 = s.bf16;
    a.packed = s.packed;
    return a;
}

// Tile rows y < hd come from source row y; a wrap row (y == hd) repeats row 0.
template <typename T>
__global__ void __launch_bounds__(256) upload_kernel(const T *__restrict__ src, cudaSurfaceObject_t surf, int w,
                                                     int h, int n, int tshift, int hd)
{
    const int x = blockIdx.x * 64 + (threadIdx.x & 63);
    const int y = blockIdx.y * 4 + (threadIdx.x >> 6);
    const int z = blockIdx.z;
    if (x >= w || y >= h || z >= n) return;
    const T v = src[((size_t)z * hd + (y < hd ? y : 0)) * w + x];
    const int X = (z & ((1 << tshift) - 1)) * w + x;
    const int Y = (z >> tshift) * h + y;
    surf2Dwrite(v, surf, X * (int)sizeof(T), Y);
}

// Packed BF16 slice pairs: texel (x, y) of slice z = (v[z] | v[z + 1] << 16).
__global__ void __launch_bounds__(256) upload_packed_kernel(const unsigned short *__restrict__ src,
                                                            cudaSurfaceObject_t surf, int w, int h, int n, int tshift)
{
    const int x = blockIdx.x * 64 + (threadIdx.x & 63);
    const int y = blockIdx.y * 4 + (threadIdx.x >> 6);
    const int z = blockIdx.z;
    if (x >= w || y >= h || z >= n) return;
    const size_t o = ((size_t)z * h + y) * w + x;
    const unsigned lo = src[o];
    const unsigned hi = z + 1 < n ? src[o + (size_t)w * h] : 0u;
    const int X = (z & ((1 << tshift) - 1)) * w + x;
    const int Y = (z >> tshift) * h + y;
    surf2Dwrite(lo | (hi << 16), surf, X * 4, Y);
}

cudaError_t atlas_upload(const AtlasStore &s, const void *src, cudaStream_t stream)
{
    const dim3 grid((s.w + 63) / 64, (s.h + 3) / 4, s.n);
    if (s.packed) {
        upload_packed_kernel<<<grid, 256, 0, stream>>>(static_cast<const unsigned short *>(src), s.surf, s.w, s.h,
                                                       s.n, s.tshift);
        return cudaGetLastError();
    }
    const int hd = s.h - s.wrap;  // rows of source data per slice
    if (s.bf16)
        upload_kernel<unsigned short><<<grid, 256, 0, stream>>>(static_cast<const unsigned short *>(src), s.surf, s.w,
                                                                s.h, s.n, s.tshift, hd);
    else
        upload_kernel<float><<<grid, 256, 0, stream>>>(static_cast<const float *>(src), s.surf, s.w, s.h, s.n,
                                                       s.tshift, hd);
    return cudaGetLastError();
}

// Three-stack atlas of the Joseph projector: tile t at ((t & mask) W, (t >>
// tshift) H).  x-slice k is tile k with texel (y, z); y-slice k is tile nx + k
// with texel (x, z); z-slice k is tile nx + ny + k with texel (x, y).
template <typename T>
__device__ __forceinline__ void jos_write(cudaSurfaceObject_t surf, int W, int H, int tshift, int t, int u, int v,
                                          T val)
{
    const int X = (t & ((1 << tshift) - 1)) * W + u;
    const int Y = (t >> tshift) * H + v;
    surf2Dwrite(val, surf, X * (int)sizeof(T), Y);
}

// y- and z-slice stacks: reads and writes both run along x.
template <typename T>
__global__ void __launch_bounds__(256) jos_upload_yz(const T *__restrict__ src, cudaSurfaceObject_t surf, int nx,
                                                     int ny, int nz, int W, int H, int tshift)
{
    const int x = blockIdx.x * 64 + (threadIdx.x & 63);
    const int y = blockIdx.y * 4 + (threadIdx.x >> 6);
    const int z = blockIdx.z;
    if (x >= nx || y >= ny || z >= nz) return;
    const T v = src[((size_t)z * ny + y) * nx + x];
    jos_write(surf, W, H, tshift, nx + ny + z, x, y, v);
    jos_write(surf, W, H, tshift, nx + y, x, z, v);
}

// x-slice stack: a 32 x 32 (x, y) block of one z-slice is transposed in
// shared memory, so the writes run along y.
template <typename T>
__global__ void __launch_bounds__(256) jos_upload_x(const T *__restrict__ src, cudaSurfaceObject_t surf, int nx,
                                                    int ny, int nz, int W, int H, int tshift)
{
    __shared__ T tile[32][33];
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32, z = blockIdx.z;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int y = y0 + ty + 8 * r, x = x0 + tx;
        if (x < nx && y < ny) tile[ty + 8 * r][tx] = src[((size_t)z * ny + y) * nx + x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int x = x0 + ty + 8 * r, y = y0 + tx;
        if (x < nx && y < ny) jos_write(surf, W, H, tshift, x, y, z, tile[tx][ty + 8 * r]);
    }
}

cudaError_t atlas_upload_joseph(const AtlasStore &s, const void *src, int nx, int ny, int nz, cudaStream_t stream)
{
    if (s.n != nx + ny + nz || s.w < max(nx, ny) || s.h < max(ny, nz) || s.packed) return cudaErrorInvalidValue;
    const dim3 g1((nx + 63) / 64, (ny + 3) / 4, nz), g2((nx + 31) / 32, (ny + 31) / 32, nz);
    if (s.bf16) {
        const unsigned short *p = static_cast<const unsigned short *>(src);
        jos_upload_yz<unsigned short><<<g1, 256, 0, stream>>>(p, s.surf, nx, ny, nz, s.w, s.h, s.tshift);
        jos_upload_x<unsigned short><<<g2, 256, 0, stream>>>(p, s.surf, nx, ny, nz, s.w, s.h, s.tshift);
    } else {
        const float *p = static_cast<const float *>(src);
        jos_upload_yz<float><<<g1, 256, 0, stream>>>(p, s.surf, nx, ny, nz, s.w, s.h, s.tshift);
        jos_upload_x<float><<<g2, 256, 0, stream>>>(p, s.surf, nx, ny, nz, s.w, s.h, s.tshift);
    }
    return cudaGetLastError();
}

}  // namespace ctrex

// atlas.cu -- allocation, texture/surface objects and upload of slice atlases.
#include "atlas.cuh"

namespace ctrex {

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

}  // namespace ctrex

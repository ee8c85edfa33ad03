// atlas.cuh -- a stack of 2D slices (volume z-slices, or detector images)
// laid out as tiles of one 2D cudaArray, read through the texture path.
//
// The array is block-linear: a 2x2 neighbourhood of one slice sits in one or
// two cache lines whatever the direction a warp's rays travel in, which a
// row-major volume cannot offer.  One tex2Dgather returns the four texels of
// a bilinear footprint in a single instruction; the interpolation weights are
// computed in FP32 registers by the caller (the texture unit's own filtering
// uses low-precision fixed-point weights and is not used).  The footprint is
// addressed at the exact corner shared by its four texels, an integer
// coordinate, so the texture unit's coordinate rounding cannot move it.
#pragma once

#include "ctrex_internal.cuh"

namespace ctrex {

struct Atlas {
    cudaTextureObject_t tex = 0;  // point sampling, border = 0, unnormalised coordinates
    int w = 0, h = 0;             // slice width and height (texels)
    int n = 0;                    // number of slices
    int tshift = 0;               // tiles per atlas row = 1 << tshift
    int bf16 = 0;                 // texels are raw BF16 bit patterns (16-bit unsigned)
    int packed = 0;               // 32-bit texels: BF16 of slice s (low half) and s + 1 (high half)
};

// Four texels of one footprint addressed by their shared corner (X, Y) in
// atlas coordinates (tile origin + (x0, y0) + 1); see atlas_quad.
__device__ __forceinline__ void atlas_quad_at(const Atlas &A, float X, float Y, float &c00, float &c10, float &c01,
                                              float &c11)
{
    if (A.bf16) {
        const ushort4 q = tex2Dgather<ushort4>(A.tex, X, Y, 0);
        c01 = __uint_as_float((unsigned)q.x << 16);
        c11 = __uint_as_float((unsigned)q.y << 16);
        c10 = __uint_as_float((unsigned)q.z << 16);
        c00 = __uint_as_float((unsigned)q.w << 16);
    } else {
        const float4 q = tex2Dgather<float4>(A.tex, X, Y, 0);
        c01 = q.x;
        c11 = q.y;
        c10 = q.z;
        c00 = q.w;
    }
}

// Four texels (x0,y0) (x0+1,y0) (x0,y0+1) (x0+1,y0+1) of slice s (clamped to a
// valid slice; out-of-slice texels are the neighbouring tile's, so callers
// give them zero weight).
__device__ __forceinline__ void atlas_quad(const Atlas &A, int s, int x0, int y0, float &c00, float &c10,
                                           float &c01, float &c11)
{
    s = min(max(s, 0), A.n - 1);
    const float X = (float)(((s & ((1 << A.tshift) - 1)) * A.w) + x0) + 1.0f;
    const float Y = (float)(((s >> A.tshift) * A.h) + y0) + 1.0f;
    atlas_quad_at(A, X, Y, c00, c10, c01, c11);
}

// Zero-padded trilinear interpolation of a volume atlas at index coordinate
// (gx, gy, gz); same weights as the row-major sampler, two gathers.
// TT: slices whose tile origins the shared-memory table holds (origins of
// later slices are computed on the fly).
template <int TT>
struct AtlasSamplerT {
    Atlas A;
    const float2 *tile = nullptr;  // shared-memory table: slice -> (atlas x, y of its tile) + 1

    static constexpr int TILE_TABLE = TT;
    static constexpr bool CYLINDER = false;
    static constexpr bool JOSEPH = false;
    static constexpr bool ROI = false;
    static constexpr bool DYRECT = false;
    static constexpr int MIN_BLOCKS = 0;  // 0: the shared forward kernel entry
    // Fills the per-CTA tile-origin table (all threads call; barrier inside).
    __device__ __forceinline__ void bind(float2 *table, int tid, int nthreads)
    {
        const int n = min(A.n, TILE_TABLE);
        for (int s = tid; s < n; s += nthreads)
            table[s] = make_float2((float)((s & ((1 << A.tshift) - 1)) * A.w) + 1.0f,
                                   (float)((s >> A.tshift) * A.h) + 1.0f);
        __syncthreads();
        tile = table;
    }
    __device__ __forceinline__ float2 origin(int s) const
    {
        if (s < TILE_TABLE) return tile[s];
        return make_float2((float)((s & ((1 << A.tshift) - 1)) * A.w) + 1.0f, (float)((s >> A.tshift) * A.h) + 1.0f);
    }

    // Interior sample: all eight taps inside the grid (0 <= g < n - 1 on each
    // axis), so no zero-padding weights; the row-sum weight is 1.
    __device__ __forceinline__ float interior(float gx, float gy, float gz) const
    {
        const float fx = floorf(gx), fy = floorf(gy), fz = floorf(gz);
        const int iz = (int)fz;
        const float ax = gx - fx, ay = gy - fy, az = gz - fz;
        const float2 o0 = origin(iz);
        float a00, a10, a01, a11, b00, b10, b01, b11;
        if (A.packed) {
            const uint4 q = tex2Dgather<uint4>(A.tex, o0.x + fx, o0.y + fy, 0);
            a01 = __uint_as_float(q.x << 16);
            a11 = __uint_as_float(q.y << 16);
            a10 = __uint_as_float(q.z << 16);
            a00 = __uint_as_float(q.w << 16);
            b01 = __uint_as_float(q.x & 0xFFFF0000u);
            b11 = __uint_as_float(q.y & 0xFFFF0000u);
            b10 = __uint_as_float(q.z & 0xFFFF0000u);
            b00 = __uint_as_float(q.w & 0xFFFF0000u);
        } else {
            const float2 o1 = origin(iz + 1);
            if (A.bf16) {
                const ushort4 q = tex2Dgather<ushort4>(A.tex, o0.x + fx, o0.y + fy, 0);
                const ushort4 r = tex2Dgather<ushort4>(A.tex, o1.x + fx, o1.y + fy, 0);
                a01 = __uint_as_float((unsigned)q.x << 16);
                a11 = __uint_as_float((unsigned)q.y << 16);
                a10 = __uint_as_float((unsigned)q.z << 16);
                a00 = __uint_as_float((unsigned)q.w << 16);
                b01 = __uint_as_float((unsigned)r.x << 16);
                b11 = __uint_as_float((unsigned)r.y << 16);
                b10 = __uint_as_float((unsigned)r.z << 16);
                b00 = __uint_as_float((unsigned)r.w << 16);
            } else {
                const float4 q = tex2Dgather<float4>(A.tex, o0.x + fx, o0.y + fy, 0);
                const float4 r = tex2Dgather<float4>(A.tex, o1.x + fx, o1.y + fy, 0);
                a01 = q.x;
                a11 = q.y;
                a10 = q.z;
                a00 = q.w;
                b01 = r.x;
                b11 = r.y;
                b10 = r.z;
                b00 = r.w;
            }
        }
        const float c0 = fmaf(ay, fmaf(ax, a11 - a01, a01) - fmaf(ax, a10 - a00, a00), fmaf(ax, a10 - a00, a00));
        const float c1 = fmaf(ay, fmaf(ax, b11 - b01, b01) - fmaf(ax, b10 - b00, b00), fmaf(ax, b10 - b00, b00));
        return fmaf(az, c1 - c0, c0);
    }

    __device__ __forceinline__ float operator()(float gx, float gy, float gz, float &wsum) const
    {
        const float fx = floorf(gx), fy = floorf(gy), fz = floorf(gz);
        const int ix = (int)fx, iy = (int)fy, iz = (int)fz;
        const float ax = gx - fx, ay = gy - fy, az = gz - fz;
        const float wx0 = ((unsigned)ix < (unsigned)A.w) ? 1.0f - ax : 0.0f;
        const float wx1 = ((unsigned)(ix + 1) < (unsigned)A.w) ? ax : 0.0f;
        const float wy0 = ((unsigned)iy < (unsigned)A.h) ? 1.0f - ay : 0.0f;
        const float wy1 = ((unsigned)(iy + 1) < (unsigned)A.h) ? ay : 0.0f;
        const float wz0 = ((unsigned)iz < (unsigned)A.n) ? 1.0f - az : 0.0f;
        const float wz1 = ((unsigned)(iz + 1) < (unsigned)A.n) ? az : 0.0f;
        // keep the gathered footprint inside the tile's neighbourhood
        const int x0 = min(max(ix, -1), A.w - 1), y0 = min(max(iy, -1), A.h - 1);
        float a00, a10, a01, a11, b00, b10, b01, b11;
        if (A.packed) {
            // one gather: low halves = slice iz, high halves = slice iz + 1.  Below
            // the first slice, slice 0 (low halves) plays the role of iz + 1.
            const int s = min(max(iz, 0), A.n - 1);
            const float X = (float)(((s & ((1 << A.tshift) - 1)) * A.w) + x0) + 1.0f;
            const float Y = (float)(((s >> A.tshift) * A.h) + y0) + 1.0f;
            const uint4 q = tex2Dgather<uint4>(A.tex, X, Y, 0);
            a01 = __uint_as_float(q.x << 16);
            a11 = __uint_as_float(q.y << 16);
            a10 = __uint_as_float(q.z << 16);
            a00 = __uint_as_float(q.w << 16);
            if (iz >= 0) {
                b01 = __uint_as_float(q.x & 0xFFFF0000u);
                b11 = __uint_as_float(q.y & 0xFFFF0000u);
                b10 = __uint_as_float(q.z & 0xFFFF0000u);
                b00 = __uint_as_float(q.w & 0xFFFF0000u);
            } else {
                b00 = a00;
                b10 = a10;
                b01 = a01;
                b11 = a11;
            }
        } else {
            atlas_quad(A, iz, x0, y0, a00, a10, a01, a11);
            atlas_quad(A, iz + 1, x0, y0, b00, b10, b01, b11);
        }
        const float c0 = fmaf(wy0, fmaf(wx0, a00, wx1 * a10), wy1 * fmaf(wx0, a01, wx1 * a11));
        const float c1 = fmaf(wy0, fmaf(wx0, b00, wx1 * b10), wy1 * fmaf(wx0, b01, wx1 * b11));
        wsum = (wx0 + wx1) * (wy0 + wy1) * (wz0 + wz1);
        return fmaf(wz0, c0, wz1 * c1);
    }
};

using AtlasSampler = AtlasSamplerT<2048>;

// Row-major (linear memory) sampler with the same semantics.
template <typename TV>
struct LinearSampler {
    const TV *vol;
    int nx, ny, nz;
    static constexpr int TILE_TABLE = 1;
    static constexpr bool CYLINDER = false;
    static constexpr bool JOSEPH = false;
    static constexpr bool ROI = false;
    static constexpr bool DYRECT = false;
    static constexpr int MIN_BLOCKS = 0;  // 0: the shared forward kernel entry
    __device__ __forceinline__ void bind(float2 *, int, int) {}
    __device__ __forceinline__ float interior(float gx, float gy, float gz) const;
    __device__ __forceinline__ float operator()(float gx, float gy, float gz, float &wsum) const;
};

// Host side (atlas.cu).
struct AtlasStore {
    cudaArray_t array = nullptr;
    cudaTextureObject_t tex = 0;
    cudaSurfaceObject_t surf = 0;
    int w = 0, h = 0, n = 0, tshift = 0, bf16 = -1, packed = 0;
    int wrap = 0;  // tiles carry one extra row repeating row 0 (periodic axis); h counts it
};
// Creates (or keeps, if the shape matches) an atlas for n slices of w x h;
// packed: 32-bit texels holding BF16 slice pairs (s, s + 1); wrap: every
// tile gets an extra row h that repeats row 0 (the atlas's h is then h + 1).
// Returns cudaErrorInvalidValue if it cannot fit the device's 2D texture limits.
cudaError_t atlas_ensure(AtlasStore &s, int w, int h, int n, bool bf16, int device, bool packed = false,
                         bool wrap = false);
void atlas_release(AtlasStore &s);
Atlas atlas_view(const AtlasStore &s);
// Copies a [nz][ny][nx] volume into a three-stack atlas of nx + ny + nz tiles
// of at least max(nx, ny) x max(ny, nz) texels (x-, y- then z-slices).
cudaError_t atlas_upload_joseph(const AtlasStore &s, const void *src, int nx, int ny, int nz, cudaStream_t stream);
// Zeroes a W x H array of 2- or 4-byte texels (called on every new atlas).
cudaError_t atlas_clear(cudaSurfaceObject_t surf, int W, int H, int bytes);
// Copies slices [n][h][w] (row-major, FP32 or BF16 as the atlas) into the
// atlas; for a packed atlas, texel s holds slices s and s + 1 (zero past n).
cudaError_t atlas_upload(const AtlasStore &s, const void *src, cudaStream_t stream);

}  // namespace ctrex

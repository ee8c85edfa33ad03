// probe.cu -- measured ceilings the projectors are rated against: the texture
// unit's gather throughput on an L1-resident texture (the projectors are
// bound by the texture return path, not by HBM), and the L2 read bandwidth
// (the graded gather roofline: algorithmic gather bytes over what L2 can
// deliver when L1 does not hold the footprint).
#include "atlas.cuh"

namespace {

constexpr int PROBE_W = 128;  // 128 x 128 FP32 texels = 64 KiB, L1 resident

__global__ void __launch_bounds__(128) gather_probe_kernel(cudaTextureObject_t tex, int iters, float *sink)
{
    float acc = 0.0f;
    unsigned x = (blockIdx.x * 37u + threadIdx.x) & (PROBE_W - 1);
    unsigned y = (blockIdx.x * 11u + threadIdx.x * 3u) & (PROBE_W - 1);
    for (int i = 0; i < iters; ++i) {
        const float4 q = tex2Dgather<float4>(tex, (float)x + 1.0f, (float)y + 1.0f, 0);
        acc += q.x + q.y + q.z + q.w;
        x = (x + 5u) & (PROBE_W - 1);
        y = (y + 3u) & (PROBE_W - 1);
    }
    if (acc == 123456.0f) sink[0] = acc;  // keeps the loop alive
}

// L2 read probe: every thread streams 16-byte vectors through the L2-only
// load path (ld.global.cg: no L1 allocation, so every load is an L2 access),
// grid-striding over a buffer that fits in L2; the sum goes to a sink so the
// loads stay live.
__global__ void __launch_bounds__(256) l2_read_probe_kernel(const float4 *__restrict__ buf, long long n_vec,
                                                            int passes, float *sink)
{
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_vec; i += 4 * stride) {
            float4 a = __ldcg(buf + i);
            float4 b = i + stride < n_vec ? __ldcg(buf + i + stride) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 c = i + 2 * stride < n_vec ? __ldcg(buf + i + 2 * stride) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 d = i + 3 * stride < n_vec ? __ldcg(buf + i + 3 * stride) : make_float4(0.f, 0.f, 0.f, 0.f);
            acc += (a.x + b.y) + (c.z + d.w);
        }
    }
    if (acc == 123456.0f) sink[0] = acc;  // keeps the loads alive
}

}  // namespace

extern "C" int ctrex_probe_l2_read_bandwidth(void *cuda_stream, double *gb_per_s)
{
    if (!gb_per_s) return CTREX_E_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0) {
        cudaGetLastError();
        return CTREX_E_CUDA;
    }
    // half of L2, a whole number of 16-byte vectors
    const long long bytes = ((long long)l2 / 2) & ~15LL;
    const long long n_vec = bytes / 16;
    float4 *buf = nullptr;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CTREX_E_CUDA;
    if (cudaMalloc((void **)&buf, bytes) == cudaSuccess && cudaMalloc((void **)&sink, 4) == cudaSuccess &&
        cudaMemsetAsync(buf, 0, bytes, stream) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess) {
        const int blocks = sms * 8, passes = 512;  // about 33 GB read: > 1 ms
        l2_read_probe_kernel<<<blocks, 256, 0, stream>>>(buf, n_vec, 4, sink);  // brings the buffer into L2
        cudaEventRecord(e0, stream);
        l2_read_probe_kernel<<<blocks, 256, 0, stream>>>(buf, n_vec, passes, sink);
        cudaEventRecord(e1, stream);
        float ms = 0.0f;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms > 0.0f) {
            *gb_per_s = (double)bytes * passes / (ms * 1e-3) / 1e9;
            rc = CTREX_OK;
        }
    }
    cudaGetLastError();
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

extern "C" int ctrex_probe_gather_rate(void *cuda_stream, double *gathers_per_s)
{
    if (!gathers_per_s) return CTREX_E_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return CTREX_E_CUDA;
    }
    cudaChannelFormatDesc desc = cudaCreateChannelDesc(32, 0, 0, 0, cudaChannelFormatKindFloat);
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CTREX_E_CUDA;
    if (cudaMallocArray(&arr, &desc, PROBE_W, PROBE_W) == cudaSuccess && cudaMalloc((void **)&sink, 4) == cudaSuccess &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = td.addressMode[1] = cudaAddressModeBorder;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        if (cudaCreateTextureObject(&tex, &rd, &td, nullptr) == cudaSuccess) {
            const int blocks = sms * 16, iters = 2048;
            gather_probe_kernel<<<blocks, 128, 0, stream>>>(tex, 64, sink);  // warm-up
            cudaEventRecord(e0, stream);
            gather_probe_kernel<<<blocks, 128, 0, stream>>>(tex, iters, sink);
            cudaEventRecord(e1, stream);
            float ms = 0.0f;
            if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                ms > 0.0f) {
                *gathers_per_s = (double)blocks * 128.0 * iters / (ms * 1e-3);
                rc = CTREX_OK;
            }
        }
    }
    cudaGetLastError();
    if (tex) cudaDestroyTextureObject(tex);
    if (arr) cudaFreeArray(arr);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

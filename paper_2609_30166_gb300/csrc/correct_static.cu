// correct_static.cu -- the detector-space correction r = R (p - q) with the
// residual norms, as a stand-alone launch that allocates no memory.
//
// Why it exists: the context-based entry points grow their scratch buffers
// with cudaMalloc on demand.  Some callers cannot allow that: a host whose
// own caching allocator has already reserved the device memory, an
// acquisition loop that must not stall in the driver's allocator (cudaMalloc
// may synchronise the device and take unbounded time), or a plugin host that
// forbids allocation inside its processing callback.  This entry point needs
// no context and no allocation: the caller passes inputs and outputs, and the
// only scratch (the per-CTA partial sums of the two-pass, fixed-order
// reduction) lives in the file-scope device array below.
//
// The array is 1 MiB and every GPU that loads the library keeps it until the
// process exits.  All calls share it: two calls whose kernels overlap on the
// GPU (different streams, or different host threads) race on it and must be
// serialised by the caller.  Pass one writes every partial that pass two
// reads, so nothing needs clearing between calls.
#include <mutex>

#include "ctrex_internal.cuh"

namespace {

constexpr int CS_THREADS = 256;
constexpr long long CS_PER_BLOCK = 8192;  // elements per CTA in pass one
constexpr int CS_MAX_BLOCKS = 65536;      // partial pairs the scratch holds
constexpr long long CS_MAX_N = CS_PER_BLOCK * CS_MAX_BLOCKS;  // 2^29 elements
constexpr int CS_MAX_DEVICES = 64;

// (sum (p-q)^2, sum p^2) per CTA of pass one.
static __device__ __align__(256) double g_cs_partials[2 * CS_MAX_BLOCKS];

// Host code must not take the address of g_cs_partials directly (in host
// code the name is a host-side stand-in): the device address is looked up
// once per device with cudaGetSymbolAddress and cached here.  With lazy
// module loading that first lookup loads the module (array and kernels),
// so callers make one call per device before any allocation-free region.
// The cache belongs to the device's primary context and is not refreshed
// after a cudaDeviceReset.
std::mutex g_cs_mutex;
double *g_cs_ptr[CS_MAX_DEVICES] = {};

int scratch_for_current_device(double **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CTREX_E_CUDA;
    }
    if (dev < 0 || dev >= CS_MAX_DEVICES) return CTREX_E_CUDA;
    std::lock_guard<std::mutex> lock(g_cs_mutex);
    if (g_cs_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_cs_partials) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return CTREX_E_CUDA;
        }
        g_cs_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_cs_ptr[dev];
    return CTREX_OK;
}

template <typename T>
__global__ void __launch_bounds__(CS_THREADS)
    correct_partials_kernel(const T *__restrict__ p, const T *__restrict__ q, const float *__restrict__ rowsum,
                            T *__restrict__ r, long long n, float eps_R, double *__restrict__ partials)
{
    __shared__ double s_red[2][CS_THREADS / 32];
    const long long begin = (long long)blockIdx.x * CS_PER_BLOCK;
    const long long end = begin + CS_PER_BLOCK < n ? begin + CS_PER_BLOCK : n;
    float e2 = 0.0f, p2 = 0.0f;
    for (long long i = begin + threadIdx.x; i < end; i += CS_THREADS) {
        const float pm = ctrex::Storage<T>::load(p + i);
        const float e = pm - ctrex::Storage<T>::load(q + i);
        const float rs = __ldg(rowsum + i);
        const float Rw = rs > eps_R ? 1.0f / rs : 0.0f;
        ctrex::Storage<T>::store(r + i, Rw * e);
        e2 = fmaf(e, e, e2);
        p2 = fmaf(pm, pm, p2);
    }
    double a = e2, b = p2;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    if ((threadIdx.x & 31) == 0) {
        s_red[0][threadIdx.x >> 5] = a;
        s_red[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
#pragma unroll
        for (int w = 0; w < CS_THREADS / 32; ++w) {
            sa += s_red[0][w];
            sb += s_red[1][w];
        }
        partials[2 * blockIdx.x] = sa;
        partials[2 * blockIdx.x + 1] = sb;
    }
}

__global__ void __launch_bounds__(1024) correct_finish_kernel(const double *__restrict__ partials, int nblocks,
                                                              double *__restrict__ sums)
{
    __shared__ double s[2][1024];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        a += partials[2 * i];
        b += partials[2 * i + 1];
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

template <typename T>
cudaError_t launch(const void *p, const void *q, const float *rowsum, void *r, long long n, float eps_R,
                   double *sums, double *scratch, cudaStream_t stream)
{
    const int nblocks = (int)((n + CS_PER_BLOCK - 1) / CS_PER_BLOCK);
    correct_partials_kernel<T><<<nblocks, CS_THREADS, 0, stream>>>(
        static_cast<const T *>(p), static_cast<const T *>(q), rowsum, static_cast<T *>(r), n, eps_R, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || sums == nullptr) return e;
    correct_finish_kernel<<<1, 1024, 0, stream>>>(scratch, nblocks, sums);
    return cudaGetLastError();
}

}  // namespace

namespace ctrex {

long long correct_scratch_pairs(long long n) { return (n + CS_PER_BLOCK - 1) / CS_PER_BLOCK; }

cudaError_t launch_correct(const void *p, const void *q, const float *rowsum, void *r, int dtype, long long n,
                           float eps_R, double *sums, double *scratch, cudaStream_t stream)
{
    if (n <= 0) return cudaSuccess;
    return dtype == CTREX_F32 ? launch<float>(p, q, rowsum, r, n, eps_R, sums, scratch, stream)
                              : launch<__nv_bfloat16>(p, q, rowsum, r, n, eps_R, sums, scratch, stream);
}

}  // namespace ctrex

extern "C" int ctrex_correct_static(const void *p, const void *q, const float *rowsum, void *r, int dtype,
                                    long long n, float eps_R, double *sums, void *cuda_stream)
{
    if (n < 0 || n > CS_MAX_N) return CTREX_E_SHAPE;
    if (dtype != CTREX_F32 && dtype != CTREX_BF16) return CTREX_E_DTYPE;
    if (!(eps_R >= 0.0f)) return CTREX_E_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    if (n == 0) {
        if (sums && cudaMemsetAsync(sums, 0, 2 * sizeof(double), stream) != cudaSuccess) {
            cudaGetLastError();
            return CTREX_E_CUDA;
        }
        return CTREX_OK;
    }
    if (!p || !q || !rowsum || !r) return CTREX_E_ARG;
    double *scratch = nullptr;
    const int e = scratch_for_current_device(&scratch);
    if (e != CTREX_OK) return e;
    const cudaError_t ce = dtype == CTREX_F32
                               ? launch<float>(p, q, rowsum, r, n, eps_R, sums, scratch, stream)
                               : launch<__nv_bfloat16>(p, q, rowsum, r, n, eps_R, sums, scratch, stream);
    return ce == cudaSuccess ? CTREX_OK : CTREX_E_CUDA;
}

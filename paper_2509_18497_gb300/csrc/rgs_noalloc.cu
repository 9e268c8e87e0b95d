// rgs_residual_norm_noalloc: the FP64 residual norm ||x - y||_2 of two float arrays,
// computed without allocating any device memory.
//
// Some callers cannot allocate: a host application that reserves its whole device-memory
// budget up front and hands the library only the buffers it owns (a renderer or a serving
// process with a fixed pool), or a latency-critical loop where a cudaMalloc would
// synchronise the device and stall other streams.  For them this entry point keeps its
// scratch -- one FP64 partial sum per block -- in a file-scope __device__ array that is
// part of the library image: every GPU that loads librgs.so holds these
// RGS_NOALLOC_MAX_BLOCKS * 8 bytes (64 KiB) until the process exits.
//
// Host code must not pass the array's name to a kernel: on the host it names a stand-in,
// not a device address.  The device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached for the life of the process;
// a device reset (cudaDeviceReset) unloads the module and leaves that cached address stale,
// so this entry point must not be used after one.
#include <mutex>

#include "rgs_internal.cuh"

#define RGS_NOALLOC_THREADS 256
#define RGS_NOALLOC_ITEMS 32
#define RGS_NOALLOC_CHUNK (RGS_NOALLOC_THREADS * RGS_NOALLOC_ITEMS) // elements per block
#define RGS_NOALLOC_MAX_BLOCKS 8192                                   // scratch: 8192 doubles
#define RGS_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_partials[RGS_NOALLOC_MAX_BLOCKS];

namespace {

std::mutex g_noalloc_mu;
double *g_noalloc_ptr[RGS_NOALLOC_MAX_DEVICES] = {};

// each block writes the FP64 sum of (x - y)^2 over its chunk to partials[blockIdx.x]
__global__ void __launch_bounds__(RGS_NOALLOC_THREADS) k_norm_partials(const float *__restrict__ x,
                                                                     const float *__restrict__ y, long long n,
                                                                     double *partials) {
    const long long base = (long long)blockIdx.x * RGS_NOALLOC_CHUNK;
    double s = 0.0;
    for (int q = 0; q < RGS_NOALLOC_ITEMS; ++q) {
        const long long i = base + (long long)q * RGS_NOALLOC_THREADS + threadIdx.x;
        if (i < n) {
            const double d = (double)x[i] - (double)y[i];
            s += d * d;
        }
    }
    __shared__ double red[RGS_NOALLOC_THREADS / 32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RGS_NOALLOC_THREADS / 32; ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// one block: sums the first `blocks` partials and writes the square root
__global__ void __launch_bounds__(RGS_NOALLOC_THREADS) k_norm_final(const double *partials, int blocks,
                                                                  double *out) {
    double s = 0.0;
    for (int b = threadIdx.x; b < blocks; b += RGS_NOALLOC_THREADS) s += partials[b];
    __shared__ double red[RGS_NOALLOC_THREADS / 32];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < RGS_NOALLOC_THREADS / 32; ++w) t += red[w];
        *out = sqrt(t);
    }
}

// device address of the scratch array for the current device (looked up once per device)
rgs_status noalloc_scratch(double **ptr) {
    int dev = 0;
    RGS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= RGS_NOALLOC_MAX_DEVICES) {
        rgs_set_error("rgs_residual_norm_noalloc: device %d beyond the %d supported", dev, RGS_NOALLOC_MAX_DEVICES);
        return RGS_ERR_ARG;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        RGS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partials));
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *ptr = g_noalloc_ptr[dev];
    return RGS_OK;
}

} // namespace

extern "C" rgs_status rgs_residual_norm_noalloc(const float *x, const float *y, int64_t n, double *norm_out,
                                                void *stream) {
    if (!x || !y || !norm_out) {
        rgs_set_error("rgs_residual_norm_noalloc: NULL argument");
        return RGS_ERR_ARG;
    }
    if (n < 0 || n > (int64_t)RGS_NOALLOC_MAX_BLOCKS * RGS_NOALLOC_CHUNK) {
        rgs_set_error("rgs_residual_norm_noalloc: n = %lld outside [0, %lld] (the fixed scratch holds %d block "
                      "partials of %d elements each)",
                      (long long)n, (long long)RGS_NOALLOC_MAX_BLOCKS * RGS_NOALLOC_CHUNK, RGS_NOALLOC_MAX_BLOCKS,
                      RGS_NOALLOC_CHUNK);
        return RGS_ERR_ARG;
    }
    double *partials = nullptr;
    rgs_status r = noalloc_scratch(&partials);
    if (r != RGS_OK) return r;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int blocks = (int)((n + RGS_NOALLOC_CHUNK - 1) / RGS_NOALLOC_CHUNK);
    // an error left pending by earlier, unrelated work is not this call's: clear it first,
    // then check each launch on its own
    (void)cudaGetLastError();
    if (blocks > 0) {
        {
            ProfScope ps_("k_norm_partials", st);
            k_norm_partials<<<blocks, RGS_NOALLOC_THREADS, 0, st>>>(x, y, (long long)n, partials);
        }
        RGS_LAUNCH("residual_norm_noalloc: k_norm_partials");
    }
    {
        ProfScope ps_("k_norm_final", st);
        k_norm_final<<<1, RGS_NOALLOC_THREADS, 0, st>>>(partials, blocks, norm_out);
    }
    RGS_LAUNCH("residual_norm_noalloc: k_norm_final");
    return RGS_OK;
}

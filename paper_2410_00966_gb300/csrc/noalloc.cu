// Coupling sum X = V_c sum_i Ms_i m_i . B_rms,i on caller-provided device
// arrays, with no device allocation anywhere on the call path.
//
// The paper has no counterpart: this exists for callers that cannot call
// cudaMalloc -- code living inside a host framework whose own pool owns the
// device memory and forbids allocations behind its back, or a latency-critical
// loop where cudaMalloc's implicit device-wide synchronisation is not
// acceptable.  Instead of allocating, the kernel's scratch (one FP64 partial
// per chunk of cells, plus the finishing counter and the result) lives in a
// file-scope static __device__ array of fixed size, which every GPU that loads
// the library holds until the process exits.
#include <cuda_runtime.h>

#include "mmcq.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_CHUNK = 4096;           // cells reduced by one block
constexpr int NA_MAX_CHUNKS = 4096;            // -> at most 16,777,216 cells
constexpr int NA_COUNTER = NA_MAX_CHUNKS;      // slot holding the block counter
constexpr int NA_RESULT = NA_MAX_CHUNKS + 1;   // slot holding the result
constexpr int NA_MAX_DEVICES = 64;

// The whole scratch of the entry point: partials, counter, result (32.8 KB).
static __device__ __align__(256) double na_scratch[NA_MAX_CHUNKS + 32];

// Device address of na_scratch on each device, filled by the first call made
// with that device current.  In host code the name na_scratch is only a
// host-side stand-in, so kernels must be given this address instead.
static double* na_addr[NA_MAX_DEVICES];

__device__ double na_block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;  // valid in thread 0
}

// One block per chunk of NA_CHUNK cells; the last block to finish adds the
// chunk partials in chunk order (deterministic) and stores V_c * sum.
__global__ void __launch_bounds__(NA_THREADS) k_coupling_noalloc(const float* __restrict__ m,
                                                                 const float* __restrict__ ms,
                                                                 const float* __restrict__ brms, long long n,
                                                                 double vc, int nchunks, double* scratch) {
    __shared__ double red[NA_THREADS / 32];
    __shared__ int last;
    const long long c0 = (long long)blockIdx.x * NA_CHUNK;
    const long long c1 = c0 + NA_CHUNK < n ? c0 + NA_CHUNK : n;
    double acc = 0.0;
    for (long long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
        double dot = (double)m[3 * i] * brms[3 * i] + (double)m[3 * i + 1] * brms[3 * i + 1] +
                     (double)m[3 * i + 2] * brms[3 * i + 2];
        acc += (double)ms[i] * dot;
    }
    acc = na_block_sum(acc, red);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = acc;
        __threadfence();
        unsigned prev = atomicAdd(reinterpret_cast<unsigned*>(scratch + NA_COUNTER), 1u);
        last = prev == (unsigned)(nchunks - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) s += __ldcg(scratch + c);
    s = na_block_sum(s, red);
    if (threadIdx.x == 0) {
        scratch[NA_RESULT] = s * vc;
        *reinterpret_cast<unsigned*>(scratch + NA_COUNTER) = 0u;
    }
}

}  // namespace

extern "C" int mmcq_coupling_sum_noalloc(const float* m, const float* ms, const float* brms, int64_t n, double vc,
                                         double* out, void* stream) {
    if (!m || !ms || !brms || !out || n < 1 || !(vc > 0)) return MMCQ_ERR_ARG;
    if (n > (int64_t)NA_CHUNK * NA_MAX_CHUNKS) return MMCQ_ERR_UNSUPPORTED;  // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MMCQ_ERR_CUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return MMCQ_ERR_UNSUPPORTED;
    if (!na_addr[dev]) {
        // set-up, once per device, with that device current
        double* p = nullptr;
        if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), na_scratch) != cudaSuccess || !p) return MMCQ_ERR_CUDA;
        na_addr[dev] = p;
    }
    double* scratch = na_addr[dev];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nchunks = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
    // the counter must start at zero; the array keeps whatever the last call left
    if (cudaMemsetAsync(scratch + NA_COUNTER, 0, sizeof(double), s) != cudaSuccess) return MMCQ_ERR_CUDA;
    k_coupling_noalloc<<<nchunks, NA_THREADS, 0, s>>>(m, ms, brms, (long long)n, vc, nchunks, scratch);
    if (cudaGetLastError() != cudaSuccess) return MMCQ_ERR_CUDA;
    if (cudaMemcpyAsync(out, scratch + NA_RESULT, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MMCQ_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MMCQ_ERR_CUDA;
    return MMCQ_OK;
}

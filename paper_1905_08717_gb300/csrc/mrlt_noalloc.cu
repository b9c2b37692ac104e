// mrlt_noalloc.cu -- leaf-mass reduction that allocates no device memory.
//
// Some callers cannot call cudaMalloc: for example a process whose device
// memory is entirely reserved up front by another allocator (a caching
// allocator or a fixed serving budget), or a latency-critical loop that must
// not pay for an allocation and its implicit device synchronisation.  For them
// mr_leaf_mass_noalloc computes the same per-variable total
// sum_leaves q_v |cell| that MR_READ_STATS reports, from leaf keys and values
// that the caller already holds in its own device buffers.  Its only scratch
// is the file-scope array below, a fixed 10 KiB (256 x 5 doubles) held by every
// GPU that loads the library until the process exits.
#include "mrlt.h"

#include <cuda_runtime.h>

#include <atomic>
#include <climits>
#include <cstdio>
#include <cstring>

namespace {

constexpr int kBlocks = 256;   // partial sums per call (fixed reduction shape)
constexpr int kThreads = 256;
constexpr int kMaxVars = 5;    // largest number of variables (3D Euler)
constexpr int kMaxDevices = 64;

// per-block partial sums of the last call; every call overwrites the slots it
// reads, so nothing needs clearing, but concurrent calls share this array
static __device__ __align__(256) double g_noalloc_partial[kBlocks * kMaxVars];

// device address of g_noalloc_partial per device, looked up on the first call
// on that device; atomic, so that host threads making their first calls at
// the same time never race on the cache (they store the same value)
std::atomic<double*> g_partial_addr[kMaxDevices] = {};

void put_msg(char* msg, size_t cap, const char* text)
{
    if (msg && cap) {
        strncpy(msg, text, cap - 1);
        msg[cap - 1] = '\0';
    }
}

__global__ void k_mass_partial(const int* keys, const double* vals, long long n, int m, double vol0,
                               int dim, double* partial)
{
    __shared__ double sh[kThreads];
    for (int v = 0; v < m; ++v) {
        double acc = 0.0;
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
             t += (long long)gridDim.x * blockDim.x) {
            const int l = keys[4 * t];
            // |cell| of level l = vol0 / 2^{dim l}
            acc += vals[t * m + v] * ldexp(vol0, -dim * l);
        }
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int o = kThreads / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[blockIdx.x * kMaxVars + v] = sh[0];
        __syncthreads();
    }
}

__global__ void k_mass_final(const double* partial, int m, double* out)
{
    const int v = threadIdx.x;
    if (v >= m) return;
    double s = 0.0;
    for (int b = 0; b < kBlocks; ++b) s += partial[b * kMaxVars + v];
    out[v] = s;
}

} // namespace

extern "C" mr_status mr_leaf_mass_noalloc(int dim, const double* lo, const double* hi, const int* keys_dev,
                                          const double* values_dev, long long n_leaves, int m,
                                          double* mass_dev, void* cuda_stream, char* msg, size_t msg_cap)
{
    char buf[160];
    if (dim < 1 || dim > 3 || !lo || !hi || !mass_dev || n_leaves < 0 ||
        (n_leaves > 0 && (!keys_dev || !values_dev))) {
        put_msg(msg, msg_cap, "mr_leaf_mass_noalloc: invalid argument (dim 1..3, box, buffers)");
        return MR_E_INVALID;
    }
    if (m < 1 || m > kMaxVars) {
        snprintf(buf, sizeof buf, "mr_leaf_mass_noalloc: m = %d variables, the fixed scratch holds at most %d",
                 m, kMaxVars);
        put_msg(msg, msg_cap, buf);
        return MR_E_INVALID;
    }
    if (n_leaves > (long long)INT_MAX) {
        snprintf(buf, sizeof buf, "mr_leaf_mass_noalloc: %lld leaves exceeds the maximum %d", n_leaves, INT_MAX);
        put_msg(msg, msg_cap, buf);
        return MR_E_INVALID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        put_msg(msg, msg_cap, "mr_leaf_mass_noalloc: no usable current CUDA device");
        return MR_E_CUDA;
    }
    // once per device, with that device current: device address of the scratch
    double* partial = g_partial_addr[dev].load(std::memory_order_acquire);
    if (!partial) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess || !p) {
            snprintf(buf, sizeof buf, "mr_leaf_mass_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            put_msg(msg, msg_cap, buf);
            return MR_E_CUDA;
        }
        partial = (double*)p;
        g_partial_addr[dev].store(partial, std::memory_order_release);
    }
    double vol0 = 1.0;
    for (int k = 0; k < dim; ++k) vol0 *= hi[k] - lo[k];
    cudaStream_t st = (cudaStream_t)cuda_stream;
    k_mass_partial<<<kBlocks, kThreads, 0, st>>>(keys_dev, values_dev, n_leaves, m, vol0, dim, partial);
    k_mass_final<<<1, 32, 0, st>>>(partial, m, mass_dev);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(buf, sizeof buf, "mr_leaf_mass_noalloc: launch failed: %s", cudaGetErrorString(e));
        put_msg(msg, msg_cap, buf);
        return MR_E_CUDA;
    }
    put_msg(msg, msg_cap, "");
    return MR_OK;
}

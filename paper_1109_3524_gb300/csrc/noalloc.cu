// Residual norms of the pinned Poisson system without any device allocation.
//
// Callers that cannot allocate device memory at the point of the call - a
// process that runs under a fixed device-memory plan (a serving process whose
// allocator is frozen after start-up), code running from a host callback where
// cudaMalloc would synchronise the device, or a host program that has no
// framework allocator to borrow a workspace from - can still check a solution
// of Eq. 9b with this entry point: its residual vector and its reduction
// scratch live in one file-scope device array that is part of the loaded
// library.  The paper has no counterpart; this is a service of the library.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/ibm.h"
#include "device.cuh"
#include "kernels.h"

namespace ibm {
int internal_poisson_residual(ibm_ctx* c, const double* x, const double* b, double* r, long long* n,
                              cudaStream_t* st);
int internal_fail(ibm_ctx* c, int code, const std::string& m);
void internal_count_launch(ibm_ctx* c);
int internal_device(const ibm_ctx* c);
}  // namespace ibm

namespace {

constexpr long long kStaticMaxN = 1LL << 21;   // residual entries (n_lambda) the array holds
constexpr int kStaticBlocks = 1024;            // reduction blocks (partial-sum slots)
constexpr int kNormThreads = 256;
// [0, kStaticMaxN): residual; then 2 * kStaticBlocks partial sums; then the two
// results; then the block counter.  16.8 MB, held by every device that loads
// the library until the process exits.
constexpr long long kScratchDoubles = kStaticMaxN + 2LL * kStaticBlocks + 4;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_addr[256] = {};   // device address of g_noalloc_scratch per device ordinal

// [b.b, r.r] with per-block partials in the static scratch; the last block to
// finish (atomic ticket) sums them in a fixed order.  The counter is cleared
// by the host before every launch (the only reset); neither that nor anything
// else protects calls that overlap on the GPU, which share the counter.
__global__ void __launch_bounds__(kNormThreads) k_norms_static(long long n, const double* __restrict__ b,
                                                               const double* __restrict__ r, double* partials,
                                                               unsigned int* counter, double* result) {
    __shared__ double sh[2][kNormThreads / 32];
    __shared__ bool last;
    double s0 = 0.0, s1 = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        s0 += b[k] * b[k];
        s1 += r[k] * r[k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        sh[0][wid] = s0;
        sh[1][wid] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < nw; ++w) {
            a += sh[0][w];
            c += sh[1][w];
        }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = c;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double a = 0.0, c = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) {
        a += __ldcg(&partials[2 * k]);
        c += __ldcg(&partials[2 * k + 1]);
    }
    result[0] = a;
    result[1] = c;
}

// Device address of the static scratch on the current device, looked up once
// per device (with that device current) and cached.  The cache assumes the
// device's primary context is never reset while the library is loaded.
int scratch_address(double** out, std::string* err) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return IBM_ERR_CUDA;
    }
    if (dev < 0 || dev >= 256) {
        *err = "device ordinal out of range";
        return IBM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return IBM_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return IBM_OK;
}

}  // namespace

extern "C" int ibm_poisson_residual_norms_noalloc(ibm_ctx* ctx, const double* d_lambda, const double* d_rhs,
                                                  double* norms_out) {
    if (!ctx || !d_lambda || !d_rhs || !norms_out) return IBM_ERR_ARG;
    int64_t nl = 0;
    int rc = ibm_sizes(ctx, nullptr, &nl, nullptr);
    if (rc) return rc;
    if (nl > kStaticMaxN)
        return ibm::internal_fail(ctx, IBM_ERR_ARG,
                                  "n_lambda = " + std::to_string(nl) + " exceeds the static scratch maximum of " +
                                      std::to_string(kStaticMaxN) + " entries (use ibm_apply_poisson)");
    // the context's stream belongs to the device bound at ibm_bind_workspace;
    // the scratch address must be that device's
    const int bound_dev = ibm::internal_device(ctx);
    int cur_dev = -1;
    if (cudaGetDevice(&cur_dev) != cudaSuccess || cur_dev != bound_dev)
        return ibm::internal_fail(ctx, IBM_ERR_STATE,
                                  "current device " + std::to_string(cur_dev) + " is not the context's device " +
                                      std::to_string(bound_dev));
    double* base = nullptr;
    std::string err;
    if ((rc = scratch_address(&base, &err))) return ibm::internal_fail(ctx, rc, err);
    double* r = base;
    double* partials = base + kStaticMaxN;
    double* result = partials + 2LL * kStaticBlocks;
    unsigned int* counter = reinterpret_cast<unsigned int*>(result + 2);
    long long n = 0;
    cudaStream_t st = nullptr;
    // the call copies to host memory and synchronises: never during a capture
    if ((rc = ibm::internal_poisson_residual(ctx, nullptr, nullptr, nullptr, &n, &st))) return rc;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return ibm::internal_fail(ctx, IBM_ERR_STATE, "the context's stream is capturing a graph");
    if ((rc = ibm::internal_poisson_residual(ctx, d_lambda, d_rhs, r, &n, &st))) return rc;
    // the counter must start at zero for the last-block detection
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        long long blocks = (n + kNormThreads - 1) / kNormThreads;
        if (blocks < 1) blocks = 1;
        if (blocks > kStaticBlocks) blocks = kStaticBlocks;
        k_norms_static<<<int(blocks), kNormThreads, 0, st>>>(n, d_rhs, r, partials, counter, result);
        ibm::internal_count_launch(ctx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(norms_out, result, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ibm::internal_fail(ctx, IBM_ERR_CUDA, std::string("noalloc residual: ") + cudaGetErrorString(e));
    return IBM_OK;
}

// Device-side views, reductions and kernel launchers of the GB300 library.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace ibm {

constexpr int kThreads = 256;             // threads per block of the streaming kernels
constexpr int kMaxPartialBlocks = 4096;   // partial-sum slots per reduction value

// Scalars of one CG solve, resident on the device.  Finalising blocks write
// them; the host reads them only between chunks of iterations.
struct CgScalars {
    double bb;          // ||b||^2
    double rr;          // ||r||^2 (current)
    double rr0;         // ||r0||^2
    double rz;          // r.z of the current preconditioned residual
    double rz_old;
    double pq;          // p.Ap
    double pq_old;
    double zq;          // z.q_prev (flexible CG)
    double alpha, beta;
    double tol2;        // tol^2
    int32_t iter, max_iter;
    int32_t done, status;
    int32_t flexible;   // 1: Notay FCG(1) beta, 0: Fletcher-Reeves
    int32_t restart;    // 1: next preconditioned residual starts a new direction
    int32_t guard;      // loop-body executions of the device-side iteration loop
    int32_t pad;
    unsigned int counter[4];
};

// Velocity / pressure 5-point operator on nblk stacked nx*ny arrays:
// y = diag x - cE x_E - cE_W x_W - cN x_N - cN_S x_S  (couplings inside a block).
template <typename T>
struct Stencil {
    int nx, ny, nblk;
    long long nc;                 // nx*ny
    const T* cE;
    const T* cN;
    const T* diag;
    const T* idiag;
};

// Extra rows/columns of the pinned Q^T B^1 Q coming from the bodies:
// touched cells gain sum_k C_ck f_k; force rows are sparse rows over lambda.
template <typename T>
struct Coupling {
    int ntc;                      // touched cells
    const long long* tcell;       // their cell index
    const long long* tc_ptr;      // CSR over touched cells
    const int* tc_col;            // lambda column (forces)
    const T* tc_val;
    int nf;                       // force rows (2 n_b)
    long long f0;                 // lambda index of the first force row (nx*ny)
    const long long* f_ptr;
    const int* f_col;
    const T* f_val;
    const T* f_idiag;             // 1/diag of force rows
};

template <typename T>
struct CsrView {
    long long n;
    const long long* ptr;
    const int* col;
    const T* val;
    long long nnz;    // entries (host-side launch shaping)
};

// FP32 pressure block of the pinned Q^T B^1 Q (Eq. 9b) from the 1D metrics:
// the east link of cell (i,j) is ax[i] ay[j], the north link bx[i] by[j]
// (ax[nx-1] = by[ny-1] = 0); the diagonal is the sum of the cell's four links
// before pinning, and the links touching the pinned cell are removed.
struct Sep32 {
    int nx, ny;
    long long pin;
    const float* ax;      // nx: 1/dxf[i+1]
    const float* ay;      // ny: dt dy[j]
    const float* bx;      // nx: dt dx[i]
    const float* by;      // ny: 1/dyf[j+1]
};

// Sliced ELLPACK, 32-row slices: entry k of row 32 s + t at off[s] + 32 k + t
// (padding: value 0, valid column).  A warp owns a slice, a lane a row, so
// every value and column load of a warp is one contiguous 128-byte line.
template <typename T>
struct SellView {
    long long n;          // rows
    long long nslices;    // ceil(n / 32)
    const long long* off; // nslices + 1
    const int* col;
    const T* val;
    long long entries;    // stored entries, padding included
};

// One lane's row of a sliced-ELLPACK slice: sum over k < w of
// val[p0 + 32 k] * g(col[p0 + 32 k]), summed in k order.  The column and
// value loads of the first 16 entries are all issued before the gathers, so a
// row costs about two memory round trips instead of one per batch.
template <typename T, class G>
__device__ __forceinline__ T sell_row(const int* col, const T* val, long long p0, int w, G&& g) {
    constexpr int K = 16;
    int c[K];
    T v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        c[k] = k < w ? col[p0 + 32 * k] : 0;
        v[k] = k < w ? val[p0 + 32 * k] : T(0);
    }
    T acc = T(0);
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (k < w) acc += v[k] * g(c[k]);
    for (int k = K; k < w; ++k) acc += val[p0 + 32 * k] * g(col[p0 + 32 * k]);
    return acc;
}

// The first K entries of one lane's row of a sliced-ELLPACK slice, loaded
// ahead of their use.  A matrix never depends on the preceding kernel, so a
// kernel launched with programmatic dependent launch issues these loads
// before griddepcontrol.wait and keeps only the gathers of the vector behind
// it.  apply() sums in the same order as sell_row.
template <typename T, int K = 16>
struct SellPre {
    long long p0;
    int w;
    int c[K];
    T v[K];
    __device__ __forceinline__ void fetch(const long long* off, const int* col, const T* val, long long s, int lane) {
        const long long o0 = off[s];
        w = int((off[s + 1] - o0) >> 5);
        p0 = o0 + lane;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            c[k] = k < w ? col[p0 + 32 * k] : 0;
            v[k] = k < w ? val[p0 + 32 * k] : T(0);
        }
    }
    template <class G>
    __device__ __forceinline__ T apply(const int* col, const T* val, G&& g) const {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (k < w) acc += v[k] * g(c[k]);
        for (int k = K; k < w; ++k) acc += val[p0 + 32 * k] * g(col[p0 + 32 * k]);
        return acc;
    }
};

struct GridView {
    int nx, ny;
    long long nc;
    const double* dx;
    const double* dy;
    const double* idx;
    const double* idy;
    const double* dxf;
    const double* dyf;
    const double* idxf;
    const double* idyf;
};

struct BoundaryView {
    const double* u_left;     // ny
    const double* u_right;    // ny   (time n)
    const double* u_right1;   // ny   (time n+1)
    const double* v_bottom;   // nx
    const double* v_top;      // nx
    const double* u_bottom;   // nx+1
    const double* u_top;      // nx+1
    const double* v_left;     // ny+1
    const double* v_right;    // ny+1 (time n)
    const double* v_right1;   // ny+1 (time n+1)
};

// Programmatic dependent launch (kernels of the solver path are launched with
// it): wait until the preceding kernel of the stream has completed and its
// writes are visible, then allow the next kernel's blocks to be scheduled, so
// the next launch overlaps this one instead of following its drain.  Both are
// no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- block reduction ------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void warp_sum(double (&v)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// Sums v over the block into partials[k*kMaxPartialBlocks + slot].  Returns
// true in every thread of the block that arrives last among `expected`
// participating blocks; that block then holds in v the totals over all
// slots 0..expected-1, summed in a fixed order (deterministic).
template <int NV>
__device__ bool block_reduce_last(double (&v)[NV], double* partials, int slot, int expected,
                                  unsigned int* counter) {
    __shared__ double sh[NV][kThreads / 32];
    __shared__ bool last;
    warp_sum<NV>(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][wid] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[k][w];
            partials[k * kMaxPartialBlocks + slot] = s;
        }
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == unsigned(expected - 1));
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < expected; b += blockDim.x)
            s += __ldcg(&partials[k * kMaxPartialBlocks + b]);
        v[k] = s;
    }
    warp_sum<NV>(v);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][wid] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += sh[k][w];
        v[k] = s;
    }
    if (threadIdx.x == 0) *counter = 0u;
    return true;
}

inline int grid_for(long long n, int threads = kThreads, int cap = kMaxPartialBlocks) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return int(b);
}

}  // namespace ibm

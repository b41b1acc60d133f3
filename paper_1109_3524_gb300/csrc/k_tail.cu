// The coarse end of the smoothed-aggregation V-cycle (section 3: the
// preconditioner of the Poisson solve of Eq. 9b) in one kernel.
//
// Below a few ten thousand rows a level's sweep moves well under a megabyte,
// so a separate kernel per sweep is bound by launch latency, not by memory.
// Here one thread-block cluster runs the whole sub-cycle: damped-Jacobi
// pre-sweeps, residual, restriction, the dense coarsest solve, prolongation
// and post-sweeps of every level from `lev[0]` down, with a hardware cluster
// barrier between dependent phases.  The cluster is co-scheduled by
// construction, so no software spin-wait is involved.  Vectors written in one
// phase and read by other blocks in the next are loaded through L2 (ld.cg),
// after the barrier's release/acquire ordering.
#include <cooperative_groups.h>

#include "kernels.h"

namespace cg = cooperative_groups;

namespace ibm {
namespace {

template <typename T>
__device__ __forceinline__ T ldv(const T* p) { return __ldcg(p); }

// One damped-Jacobi-family pass over a level in sliced ELLPACK (one warp per
// 32-row slice): MODE_JAC0 y = w D^-1 b, MODE_JAC y = x + w D^-1 (b - A x),
// MODE_RESID y = b - A x.
template <typename T>
__device__ void pass(int mode, const SellView<T>& A, const T* idiag, const T* x, const T* b, T* y, T omega,
                     long long warp, long long nwarps, int lane) {
    for (long long s = warp; s < A.nslices; s += nwarps) {
        const long long i = s * 32 + lane;
        if (mode == MODE_JAC0) {
            if (i < A.n) y[i] = omega * idiag[i] * ldv(b + i);
            continue;
        }
        const long long o0 = A.off[s], o1 = A.off[s + 1];
        T acc = T(0);
        if (mode == MODE_JAC2) {
            // neighbours after the first sweep from zero: w D^-1 b
#pragma unroll 8
            for (long long p = o0 + lane; p < o1; p += 32) {
                const int c = A.col[p];
                acc += A.val[p] * (omega * idiag[c] * ldv(b + c));
            }
        } else {
#pragma unroll 8
            for (long long p = o0 + lane; p < o1; p += 32) acc += A.val[p] * ldv(x + A.col[p]);
        }
        if (i < A.n) {
            const T bi = ldv(b + i);
            if (mode == MODE_RESID) y[i] = bi - acc;
            else if (mode == MODE_JAC2) y[i] = omega * idiag[i] * bi + omega * idiag[i] * (bi - acc);
            else y[i] = ldv(x + i) + omega * idiag[i] * (bi - acc);
        }
    }
}

// y (+)= M x for a prolongator or restriction in sliced ELLPACK
template <typename T>
__device__ void mv(const SellView<T>& M, const T* x, T* y, bool acc_into, long long warp, long long nwarps,
                   int lane) {
    for (long long s = warp; s < M.nslices; s += nwarps) {
        const long long i = s * 32 + lane;
        const long long o0 = M.off[s], o1 = M.off[s + 1];
        T acc = T(0);
#pragma unroll 8
        for (long long p = o0 + lane; p < o1; p += 32) acc += M.val[p] * ldv(x + M.col[p]);
        if (i < M.n) y[i] = acc_into ? ldv(y + i) + acc : acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_tail(TailArgs<T> a) {
    if (a.sc && *((volatile const int*)&a.sc->done)) return;   // uniform: no kernel writes it meanwhile
    cg::cluster_group cl = cg::this_cluster();
    const int lane = threadIdx.x & 31;
    const long long warp = (long long)(cl.block_rank() * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = (long long)(cl.num_blocks() * blockDim.x) >> 5;
    T* cur[kMaxTailLevels];
    T* oth[kMaxTailLevels];
    // restriction down to the coarsest level
    for (int l = 0; l + 1 < a.nlev; ++l) {
        const TailLevel<T>& L = a.lev[l];
        T* x = L.x;
        T* x2 = L.x2;
        pass(a.pre >= 2 ? MODE_JAC2 : MODE_JAC0, L.A, L.idiag, x, L.b, x, L.omega, warp, nwarps, lane);
        cl.sync();
        for (int s = a.pre >= 2 ? 2 : 1; s < a.pre; ++s) {
            pass(MODE_JAC, L.A, L.idiag, x, L.b, x2, L.omega, warp, nwarps, lane);
            T* t = x;
            x = x2;
            x2 = t;
            cl.sync();
        }
        pass(MODE_RESID, L.A, L.idiag, x, L.b, L.r, L.omega, warp, nwarps, lane);
        cl.sync();
        mv(L.R, L.r, a.lev[l + 1].b, false, warp, nwarps, lane);
        cl.sync();
        cur[l] = x;
        oth[l] = x2;
    }
    // dense coarsest solve x = Ainv b (warp per row)
    {
        const TailLevel<T>& C = a.lev[a.nlev - 1];
        const int n = a.nc;
        for (long long i = warp; i < n; i += nwarps) {
            T acc = T(0);
            for (int j = lane; j < n; j += 32) acc += a.cinv[i * (long long)n + j] * ldv(C.b + j);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) C.x[i] = acc;
        }
        cl.sync();
    }
    // prolongation and post-smoothing back up
    for (int l = a.nlev - 2; l >= 0; --l) {
        const TailLevel<T>& L = a.lev[l];
        const T* xc = (l + 2 == a.nlev) ? a.lev[l + 1].x : cur[l + 1];
        T* x = cur[l];
        T* x2 = oth[l];
        mv(L.P, xc, x, true, warp, nwarps, lane);
        cl.sync();
        for (int s = 0; s < a.post; ++s) {
            pass(MODE_JAC, L.A, L.idiag, x, L.b, x2, L.omega, warp, nwarps, lane);
            T* t = x;
            x = x2;
            x2 = t;
            cl.sync();
        }
        cur[l] = x;
    }
}

}  // namespace

template <typename T>
int tail_cluster_size(int device) {
    (void)device;
    static int cached = -1;   // per process: every device of one build has the same limits
    if (cached >= 0) return cached;
    int cs = 0;
    if (cudaFuncSetAttribute(k_tail<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        for (int want : {16, 8}) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(want);
            cfg.blockDim = dim3(kTailThreads);
            cudaLaunchAttribute at;
            at.id = cudaLaunchAttributeClusterDimension;
            at.val.clusterDim.x = want;
            at.val.clusterDim.y = 1;
            at.val.clusterDim.z = 1;
            cfg.attrs = &at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            if (cudaOccupancyMaxActiveClusters(&nclusters, k_tail<T>, &cfg) == cudaSuccess && nclusters > 0) {
                cs = want;
                break;
            }
        }
    }
    cudaGetLastError();   // clear a refused attribute or query
    cached = cs;
    return cs;
}

template <typename T>
cudaError_t launch_tail(const TailArgs<T>& a, int cluster, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(kTailThreads);
    cfg.stream = st;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeClusterDimension;
    at.val.clusterDim.x = cluster;
    at.val.clusterDim.y = 1;
    at.val.clusterDim.z = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tail<T>, a);
}

template int tail_cluster_size<float>(int);
template int tail_cluster_size<double>(int);
template cudaError_t launch_tail<float>(const TailArgs<float>&, int, cudaStream_t);
template cudaError_t launch_tail<double>(const TailArgs<double>&, int, cudaStream_t);

}  // namespace ibm

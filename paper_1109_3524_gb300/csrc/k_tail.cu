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

#include <algorithm>
#include <vector>

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
        const long long o0 = A.off[s];
        const int w = int((A.off[s + 1] - o0) >> 5);
        T acc;
        if (mode == MODE_JAC2)   // neighbours after the first sweep from zero: w D^-1 b
            acc = sell_row(A.col, A.val, o0 + lane, w, [&](int c) { return omega * idiag[c] * ldv(b + c); });
        else
            acc = sell_row(A.col, A.val, o0 + lane, w, [&](int c) { return ldv(x + c); });
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
        const long long o0 = M.off[s];
        const T acc = sell_row(M.col, M.val, o0 + lane, int((M.off[s + 1] - o0) >> 5), [&](int c) { return ldv(x + c); });
        if (i < M.n) y[i] = acc_into ? ldv(y + i) + acc : acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_tail(TailArgs<T> a) {
    pdl_entry();
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
    // dense coarsest solve x = Ainv b in FP64 (warp per row)
    {
        const TailLevel<T>& C = a.lev[a.nlev - 1];
        const int n = a.nc;
        for (long long i = warp; i < n; i += nwarps) {
            double acc = 0.0;
            for (int j = lane; j < n; j += 32) acc += __ldg(a.cinv + i * (long long)n + j) * double(ldv(C.b + j));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) C.x[i] = T(acc);
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

// ---- staged variant: every block keeps the slices it owns in shared memory ----------
//
// The blocks of the cluster split each operator's slices (and the rows of the
// dense coarsest inverse) into contiguous ranges.  Each block copies its
// operator ranges into shared memory once per launch, so the sweeps read
// matrix entries from shared memory and only the vectors through L2.  The
// FP64 coarsest inverse stays in global memory (L2-resident after the first
// V-cycle); each block reads its rows once per launch.
template <typename T>
struct StagedOp {
    long long s0, s1;      // owned slices
    long long n;           // rows of the operator
    const int* off;        // s1 - s0 + 1 entry offsets relative to the first owned entry
    const int* col;
    const T* val;
};

__device__ __forceinline__ char* carve16(char*& p, long long bytes) {
    p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    char* r = p;
    p += bytes;
    return r;
}

// Block-wide copy of n elements of type V, eight loads in flight per thread.
template <typename V>
__device__ __forceinline__ void copy_block(V* d, const V* s, long long n) {
    constexpr int B = 8;
    const long long step = (long long)blockDim.x * B;
    for (long long k0 = threadIdx.x; k0 < n; k0 += step) {
        V v[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const long long k = k0 + (long long)u * blockDim.x;
            if (k < n) v[u] = __ldg(s + k);
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const long long k = k0 + (long long)u * blockDim.x;
            if (k < n) d[k] = v[u];
        }
    }
}

// bytes: a multiple of 16; both pointers 16-byte aligned
__device__ __forceinline__ void copy16(void* dst, const void* src, long long bytes) {
    copy_block(static_cast<int4*>(dst), static_cast<const int4*>(src), bytes / 16);
}

template <typename T>
__device__ StagedOp<T> stage(const SellView<T>& M, int rank, int cs, char*& sm) {
    StagedOp<T> o;
    o.s0 = M.nslices * rank / cs;
    o.s1 = M.nslices * (rank + 1) / cs;
    o.n = M.n;
    const long long e0 = M.off[o.s0], ne = M.off[o.s1] - e0;   // multiples of 32 entries
    int* off = reinterpret_cast<int*>(carve16(sm, (o.s1 - o.s0 + 1) * 4));
    int* col = reinterpret_cast<int*>(carve16(sm, ne * 4));
    T* val = reinterpret_cast<T*>(carve16(sm, ne * (long long)sizeof(T)));
    for (long long k = threadIdx.x; k <= o.s1 - o.s0; k += blockDim.x) off[k] = int(M.off[o.s0 + k] - e0);
    copy16(col, M.col + e0, ne * 4);
    copy16(val, M.val + e0, ne * (long long)sizeof(T));
    o.off = off;
    o.col = col;
    o.val = val;
    return o;
}

template <typename T>
__device__ void pass_st(int mode, const StagedOp<T>& A, const T* idiag, const T* x, const T* b, T* y, T omega,
                        int wb, int nwb, int lane) {
    for (long long s = A.s0 + wb; s < A.s1; s += nwb) {
        const long long i = s * 32 + lane;
        if (mode == MODE_JAC0) {
            if (i < A.n) y[i] = omega * idiag[i] * ldv(b + i);
            continue;
        }
        const int o0 = A.off[s - A.s0];
        const int w = (A.off[s - A.s0 + 1] - o0) >> 5;
        T acc;
        if (mode == MODE_JAC2)
            acc = sell_row(A.col, A.val, o0 + lane, w, [&](int c) { return omega * idiag[c] * ldv(b + c); });
        else
            acc = sell_row(A.col, A.val, o0 + lane, w, [&](int c) { return ldv(x + c); });
        if (i < A.n) {
            const T bi = ldv(b + i);
            if (mode == MODE_RESID) y[i] = bi - acc;
            else if (mode == MODE_JAC2) y[i] = omega * idiag[i] * bi + omega * idiag[i] * (bi - acc);
            else y[i] = ldv(x + i) + omega * idiag[i] * (bi - acc);
        }
    }
}

template <typename T>
__device__ void mv_st(const StagedOp<T>& M, const T* x, T* y, bool acc_into, int wb, int nwb, int lane) {
    for (long long s = M.s0 + wb; s < M.s1; s += nwb) {
        const long long i = s * 32 + lane;
        const int o0 = M.off[s - M.s0];
        const T acc = sell_row(M.col, M.val, o0 + lane, (M.off[s - M.s0 + 1] - o0) >> 5, [&](int c) { return ldv(x + c); });
        if (i < M.n) y[i] = acc_into ? ldv(y + i) + acc : acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(kTailThreads) k_tail_staged(TailArgs<T> a) {
    pdl_entry();
    if (a.sc && *((volatile const int*)&a.sc->done)) return;   // uniform: no kernel writes it meanwhile
    extern __shared__ __align__(16) char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = int(cl.block_rank()), cs = int(cl.num_blocks());
    const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    char* sm = smem;
    StagedOp<T> A[kMaxTailLevels], Rs[kMaxTailLevels], Ps[kMaxTailLevels];
    for (int l = 0; l + 1 < a.nlev; ++l) {
        A[l] = stage(a.lev[l].A, rank, cs, sm);
        Rs[l] = stage(a.lev[l].R, rank, cs, sm);
        Ps[l] = stage(a.lev[l].P, rank, cs, sm);
    }
    const int n = a.nc;
    const int r0 = n * rank / cs, r1 = n * (rank + 1) / cs;
    double* bsh = reinterpret_cast<double*>(carve16(sm, (long long)n * (long long)sizeof(double)));
    __syncthreads();
    T* cur[kMaxTailLevels];
    T* oth[kMaxTailLevels];
    for (int l = 0; l + 1 < a.nlev; ++l) {
        const TailLevel<T>& L = a.lev[l];
        T* x = L.x;
        T* x2 = L.x2;
        pass_st(a.pre >= 2 ? MODE_JAC2 : MODE_JAC0, A[l], L.idiag, x, L.b, x, L.omega, wb, nwb, lane);
        cl.sync();
        for (int s = a.pre >= 2 ? 2 : 1; s < a.pre; ++s) {
            pass_st(MODE_JAC, A[l], L.idiag, x, L.b, x2, L.omega, wb, nwb, lane);
            T* t = x;
            x = x2;
            x2 = t;
            cl.sync();
        }
        pass_st(MODE_RESID, A[l], L.idiag, x, L.b, L.r, L.omega, wb, nwb, lane);
        cl.sync();
        mv_st(Rs[l], L.r, a.lev[l + 1].b, false, wb, nwb, lane);
        cl.sync();
        cur[l] = x;
        oth[l] = x2;
    }
    {   // dense coarsest solve in FP64: b widened into shared memory, x narrowed
        const TailLevel<T>& C = a.lev[a.nlev - 1];
        for (int k = threadIdx.x; k < n; k += blockDim.x) bsh[k] = double(ldv(C.b + k));
        __syncthreads();
        for (int i = r0 + wb; i < r1; i += nwb) {
            const double* row = a.cinv + (long long)i * n;
            double acc = 0.0;
#pragma unroll 4
            for (int j = lane; j < n; j += 32) acc += __ldg(row + j) * bsh[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) C.x[i] = T(acc);
        }
        cl.sync();
    }
    for (int l = a.nlev - 2; l >= 0; --l) {
        const TailLevel<T>& L = a.lev[l];
        const T* xc = (l + 2 == a.nlev) ? a.lev[l + 1].x : cur[l + 1];
        T* x = cur[l];
        T* x2 = oth[l];
        mv_st(Ps[l], xc, x, true, wb, nwb, lane);
        cl.sync();
        for (int s = 0; s < a.post; ++s) {
            pass_st(MODE_JAC, A[l], L.idiag, x, L.b, x2, L.omega, wb, nwb, lane);
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

// Shared-memory bytes one block of the staged kernel needs (the same carving
// as the kernel), from the host copies of the slice offsets.
long long tail_staged_bytes(const std::vector<const std::vector<long long>*>& offs, int coarse_n, int cs,
                            size_t ts) {
    long long worst = 0;
    auto a16 = [](long long b) { return (b + 15) & ~15LL; };
    for (int rank = 0; rank < cs; ++rank) {
        long long b = 0;
        for (const auto* off : offs) {
            const long long ns = (long long)off->size() - 1;
            const long long s0 = ns * rank / cs, s1 = ns * (rank + 1) / cs;
            const long long ne = (*off)[s1] - (*off)[s0];
            b = a16(b) + (s1 - s0 + 1) * 4;
            b = a16(b) + ne * 4;
            b = a16(b) + ne * (long long)ts;
        }
        b = a16(b) + (long long)coarse_n * (long long)sizeof(double);   // widened coarsest right-hand side
        worst = std::max(worst, b + 16);
    }
    return worst;
}

template <typename T>
bool tail_staged_ready(int cluster, long long smem) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        smem > optin) {
        cudaGetLastError();
        return false;
    }
    bool ok = cudaFuncSetAttribute(k_tail_staged<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess &&
              cudaFuncSetAttribute(k_tail_staged<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) == cudaSuccess;
    if (ok) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cluster);
        cfg.blockDim = dim3(kTailThreads);
        cfg.dynamicSmemBytes = size_t(smem);
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = cluster;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        cfg.attrs = &at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        ok = cudaOccupancyMaxActiveClusters(&nclusters, k_tail_staged<T>, &cfg) == cudaSuccess && nclusters > 0;
    }
    cudaGetLastError();
    return ok;
}

template <typename T>
cudaError_t launch_tail(const TailArgs<T>& a, int cluster, long long staged_smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(kTailThreads);
    cfg.stream = st;
    cfg.dynamicSmemBytes = staged_smem > 0 ? size_t(staged_smem) : 0;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 2 : 1;
    if (staged_smem > 0) return cudaLaunchKernelEx(&cfg, k_tail_staged<T>, a);
    return cudaLaunchKernelEx(&cfg, k_tail<T>, a);
}

template int tail_cluster_size<float>(int);
template int tail_cluster_size<double>(int);
template cudaError_t launch_tail<float>(const TailArgs<float>&, int, long long, cudaStream_t);
template cudaError_t launch_tail<double>(const TailArgs<double>&, int, long long, cudaStream_t);
template bool tail_staged_ready<float>(int, long long);
template bool tail_staged_ready<double>(int, long long);

}  // namespace ibm

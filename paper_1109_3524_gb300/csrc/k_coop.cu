// The coarse levels of the smoothed-aggregation V-cycle (section 3: the
// preconditioner of the Poisson solve of Eq. 9b) as one cooperative kernel
// over the whole GPU.
//
// Below the finest level every phase of the V-cycle - a damped-Jacobi sweep,
// a residual, a restriction, a prolongation - touches at most a few megabytes
// that sit in L2, so a launch per phase is bound by launch and ramp latency,
// not by memory.  Here all blocks of one cooperative launch (co-resident by
// construction) run the phases in order: the restriction from the parent
// level, pre-sweeps, residual and restriction of every level, the dense FP64
// coarsest solve, prolongation and post-sweeps back up, and the prolongation
// into the parent level, with a grid barrier between dependent phases.  Each
// wait of the barrier is bounded: after kSpinLimit polls the block records an
// error (and, when the solve's scalars are given, ends the solve with status
// 6) and every block leaves at its next barrier.  Vectors written in one phase
// and read by other blocks in the next are read through L2 (ld.cg) after the
// barrier's release / acquire ordering.
#include <algorithm>

#include "kernels.h"

namespace ibm {
namespace {

constexpr int kCoopThreads = 512;
constexpr long long kSpinLimit = 1LL << 22;   // polls of one barrier wait (about 0.3 s with the back-off)

template <typename T>
__device__ __forceinline__ T ldv(const T* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_i(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Sense-free generation barrier over all blocks of the grid.  Returns false in
// every thread of every block once any block has given up waiting.
__device__ __noinline__ bool grid_sync(GridBarrier* gb, unsigned& gen, CgScalars* sc) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = gen + 1;
        __threadfence();   // this block's writes before its arrival
        const unsigned arrived = atomicAdd(&gb->count, 1u) + 1u;
        int good = 1;
        if (arrived == gridDim.x) {
            atomicExch(&gb->count, 0u);
            __threadfence();
            atomicExch(&gb->gen, target);   // release every waiting block
        } else {
            long long spins = 0;
            while (ld_acquire(&gb->gen) != target) {
                if (ld_relaxed_i(&gb->err)) {
                    good = 0;
                    break;
                }
                if (++spins > kSpinLimit) {
                    atomicExch(&gb->err, 1);
                    if (sc) {
                        sc->status = 6;
                        sc->done = 1;
                    }
                    good = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        gen = target;
        ok = good && ld_relaxed_i(&gb->err) == 0;
    }
    __syncthreads();
    return ok != 0;
}

// One damped-Jacobi-family pass over a level in sliced ELLPACK (one warp per
// 32-row slice, warps of the whole grid): MODE_JAC0 y = w D^-1 b, MODE_JAC
// y = x + w D^-1 (b - A x), MODE_JAC2 two sweeps from zero, MODE_RESID
// y = b - A x.
template <typename T>
__device__ void pass(int mode, const SellView<T>& A, const T* idiag, const T* x, const T* b, T* y, T omega,
                     long long warp, long long nwarps, int lane) {
    for (long long s = warp; s < A.nslices; s += nwarps) {
        const long long i = s * 32 + lane;
        if (mode == MODE_JAC0) {
            if (i < A.n) y[i] = omega * __ldg(idiag + i) * ldv(b + i);
            continue;
        }
        const long long o0 = __ldg(A.off + s);
        const int w = int((__ldg(A.off + s + 1) - o0) >> 5);
        T acc;
        if (mode == MODE_JAC2)
            acc = sell_row(A.col, A.val, o0 + lane, w, [&](int c) { return omega * __ldg(idiag + c) * ldv(b + c); });
        else
            acc = sell_row(A.col, A.val, o0 + lane, w, [&](int c) { return ldv(x + c); });
        if (i < A.n) {
            const T bi = ldv(b + i), id = __ldg(idiag + i);
            if (mode == MODE_RESID) y[i] = bi - acc;
            else if (mode == MODE_JAC2) y[i] = omega * id * bi + omega * id * (bi - acc);
            else y[i] = ldv(x + i) + omega * id * (bi - acc);
        }
    }
}

// y (+)= M x for a prolongator or restriction in sliced ELLPACK
template <typename T>
__device__ void mv(const SellView<T>& M, const T* x, T* y, bool acc_into, long long warp, long long nwarps,
                   int lane) {
    for (long long s = warp; s < M.nslices; s += nwarps) {
        const long long i = s * 32 + lane;
        const long long o0 = __ldg(M.off + s);
        const T acc = sell_row(M.col, M.val, o0 + lane, int((__ldg(M.off + s + 1) - o0) >> 5),
                               [&](int c) { return ldv(x + c); });
        if (i < M.n) y[i] = acc_into ? ldv(y + i) + acc : acc;
    }
}

template <typename T>
__global__ void __launch_bounds__(kCoopThreads) k_coarse_coop(CoopArgs<T> a) {
    if (a.sc && *((volatile const int*)&a.sc->done)) return;   // uniform: nothing writes it meanwhile
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = ld_acquire(&a.bar->gen);
    CgScalars* sc = a.sc;
    if (a.has_parent) {   // b of the first level = R_parent r_parent
        mv(a.Rp, a.rp, a.lev[0].b, false, warp, nwarps, lane);
        if (!grid_sync(a.bar, gen, sc)) return;
    }
    T* cur[kMaxCoopLevels];
    T* oth[kMaxCoopLevels];
    for (int l = 0; l + 1 < a.nlev; ++l) {
        const CoopLevel<T>& L = a.lev[l];
        T* x = L.x;
        T* x2 = L.x2;
        pass(a.pre >= 2 ? MODE_JAC2 : MODE_JAC0, L.A, L.idiag, x, L.b, x, L.omega, warp, nwarps, lane);
        if (!grid_sync(a.bar, gen, sc)) return;
        for (int s = a.pre >= 2 ? 2 : 1; s < a.pre; ++s) {
            pass(MODE_JAC, L.A, L.idiag, x, L.b, x2, L.omega, warp, nwarps, lane);
            T* t = x;
            x = x2;
            x2 = t;
            if (!grid_sync(a.bar, gen, sc)) return;
        }
        pass(MODE_RESID, L.A, L.idiag, x, L.b, L.r, L.omega, warp, nwarps, lane);
        if (!grid_sync(a.bar, gen, sc)) return;
        mv(L.R, L.r, a.lev[l + 1].b, false, warp, nwarps, lane);
        if (!grid_sync(a.bar, gen, sc)) return;
        cur[l] = x;
        oth[l] = x2;
    }
    {   // dense coarsest solve in FP64 (warp per row): b widened, x narrowed
        const CoopLevel<T>& C = a.lev[a.nlev - 1];
        const int n = a.nc;
        for (long long i = warp; i < n; i += nwarps) {
            const double* row = a.cinv + i * (long long)n;
            double acc = 0.0;
#pragma unroll 4
            for (int j = lane; j < n; j += 32) acc += __ldg(row + j) * double(ldv(C.b + j));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) C.x[i] = T(acc);
        }
        if (!grid_sync(a.bar, gen, sc)) return;
    }
    for (int l = a.nlev - 2; l >= 0; --l) {
        const CoopLevel<T>& L = a.lev[l];
        const T* xc = (l + 2 == a.nlev) ? a.lev[l + 1].x : cur[l + 1];
        T* x = cur[l];
        T* x2 = oth[l];
        mv(L.P, xc, x, true, warp, nwarps, lane);
        if (!grid_sync(a.bar, gen, sc)) return;
        for (int s = 0; s < a.post; ++s) {
            pass(MODE_JAC, L.A, L.idiag, x, L.b, x2, L.omega, warp, nwarps, lane);
            T* t = x;
            x = x2;
            x2 = t;
            if (!grid_sync(a.bar, gen, sc)) return;
        }
        cur[l] = x;
    }
    if (a.has_parent)   // x_parent += P_parent x of the first level
        mv(a.Pp, a.nlev > 1 ? cur[0] : a.lev[0].x, a.xp, true, warp, nwarps, lane);
}

}  // namespace

template <typename T>
int coop_grid(int device) {
    static int cached = -1;   // per process: every device of one build has the same limits
    if (cached >= 0) return cached;
    int per_sm = 0, sms = 0, coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_coop<T>, kCoopThreads, 0) != cudaSuccess) {
        cudaGetLastError();
        cached = 0;
        return 0;
    }
    cached = sms * std::min(per_sm, 2);
    return cached;
}

template <typename T>
cudaError_t launch_coop(const CoopArgs<T>& a, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kCoopThreads);
    cfg.stream = st;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeCooperative;
    at.val.cooperative = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_coarse_coop<T>, a);
}

template int coop_grid<float>(int);
template int coop_grid<double>(int);
template cudaError_t launch_coop<float>(const CoopArgs<float>&, int, cudaStream_t);
template cudaError_t launch_coop<double>(const CoopArgs<double>&, int, cudaStream_t);

}  // namespace ibm

// The coarse levels of the smoothed-aggregation V-cycle (section 3: the
// preconditioner of the Poisson solve of Eq. 9b) as one cooperative kernel
// over the whole GPU.
//
// Below the finest level every phase of the V-cycle - a damped-Jacobi sweep,
// a residual, a restriction, a prolongation - touches at most a few megabytes
// that sit in L2, so a launch per phase is bound by launch and memory latency,
// not by bandwidth.  Here all blocks of one cooperative launch (co-resident by
// construction) run the phases in order: the restriction from the parent
// level, pre-sweeps, residual and restriction of every level, the dense FP64
// coarsest solve, prolongation and post-sweeps back up, and the prolongation
// into the parent level, with a grid barrier between dependent phases.
//
// Latency, not bandwidth, sets the time of a phase: a sliced-ELLPACK row costs
// a chain of dependent loads (slice offset, then column / value, then the
// gathered vector entry).  So each block copies its share of the small
// operators (the coarse levels' A, R and P, chosen by the host to fit) into
// shared memory once per launch, which leaves one L2 round trip (the gather)
// per row of those phases; the operators read from global memory (the larger
// levels and the transfers to the parent) keep several slices' loads in
// flight per warp.
//
// Each wait of the grid barrier is bounded: after kSpinLimit polls the block
// records an error (and, when the solve's scalars are given, ends the solve
// with status 6) and every block leaves at its next barrier.  Vectors written
// in one phase and read by other blocks in the next are read through L2
// (ld.cg) after the barrier's release / acquire ordering.
#include <algorithm>
#include <vector>

#include "kernels.h"

namespace ibm {
namespace {

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

// Generation barrier over all blocks of the grid.  Returns false in every
// thread of every block once any block has given up waiting.
__device__ __forceinline__ bool grid_sync(GridBarrier* gb, unsigned& gen, CgScalars* sc) {
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
                __nanosleep(32);
            }
        }
        __threadfence();
        gen = target;
        ok = good && ld_relaxed_i(&gb->err) == 0;
    }
    __syncthreads();
    return ok != 0;
}

// ---- operators: staged (this block's slices in shared memory) or global -----------
// Staged operator of this block: slices [s0, s1) with entry offsets relative
// to the first owned entry, its columns and values at byte offsets of the
// block's dynamic shared memory.
struct StagedDesc {
    int s0, s1;
    unsigned off_o, col_o, val_o;
    int staged;
};

template <typename T>
struct Op {
    SellView<T> g;          // the operator in global memory
    bool staged;
    int s0, s1;
    const int* off;
    const int* col;
    const T* val;
};

__device__ __forceinline__ char* carve16(char*& p, long long bytes) {
    p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    char* r = p;
    p += bytes;
    return r;
}

// Block-wide copy of n 16-byte words, eight loads in flight per thread.
__device__ __forceinline__ void copy16(void* dst, const void* src, long long bytes) {
    int4* d = static_cast<int4*>(dst);
    const int4* s = static_cast<const int4*>(src);
    const long long n = bytes / 16;
    constexpr int B = 8;
    const long long step = (long long)blockDim.x * B;
    for (long long k0 = threadIdx.x; k0 < n; k0 += step) {
        int4 v[B];
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

// Copies this block's slices of M into shared memory (all threads; thread 0
// records the descriptor).
template <typename T>
__device__ void stage(const SellView<T>& M, bool staged, char* base, char*& sm, StagedDesc* desc) {
    if (!staged) {
        if (threadIdx.x == 0) desc->staged = 0;
        return;
    }
    const int s0 = int(M.nslices * blockIdx.x / gridDim.x);
    const int s1 = int(M.nslices * (blockIdx.x + 1) / gridDim.x);
    const long long e0 = M.off[s0], ne = M.off[s1] - e0;   // multiples of 32 entries
    int* off = reinterpret_cast<int*>(carve16(sm, (long long)(s1 - s0 + 1) * 4));
    int* col = reinterpret_cast<int*>(carve16(sm, ne * 4));
    T* val = reinterpret_cast<T*>(carve16(sm, ne * (long long)sizeof(T)));
    for (int k = threadIdx.x; k <= s1 - s0; k += blockDim.x) off[k] = int(M.off[s0 + k] - e0);
    copy16(col, M.col + e0, ne * 4);
    copy16(val, M.val + e0, ne * (long long)sizeof(T));
    if (threadIdx.x == 0) {
        desc->staged = 1;
        desc->s0 = s0;
        desc->s1 = s1;
        desc->off_o = unsigned(reinterpret_cast<char*>(off) - base);
        desc->col_o = unsigned(reinterpret_cast<char*>(col) - base);
        desc->val_o = unsigned(reinterpret_cast<char*>(val) - base);
    }
}

template <typename T>
__device__ __forceinline__ Op<T> get_op(const SellView<T>& M, const StagedDesc& d, const char* base) {
    Op<T> o;
    o.g = M;
    o.staged = d.staged != 0;
    o.s0 = d.s0;
    o.s1 = d.s1;
    o.off = reinterpret_cast<const int*>(base + d.off_o);
    o.col = reinterpret_cast<const int*>(base + d.col_o);
    o.val = reinterpret_cast<const T*>(base + d.val_o);
    return o;
}

// row value of one lane: sum_k val[p0 + 32k] * g(col[p0 + 32k]) over the slice width
template <typename T, int K, class G>
__device__ __forceinline__ T row_dot(const int* col, const T* val, long long p0, int w, G&& g) {
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

// The value of row i = 32 s + lane of a sweep, residual or product for slice s
// of the operator (staged: local slice index ls).
template <typename T, class G>
__device__ __forceinline__ T op_row(const Op<T>& o, long long s, int lane, G&& g) {
    if (o.staged) {
        const int ls = int(s - o.s0);
        const int e0 = o.off[ls];
        return row_dot<T, 8>(o.col, o.val, e0 + lane, (o.off[ls + 1] - e0) >> 5, g);
    }
    const long long e0 = __ldg(o.g.off + s);
    return row_dot<T, 8>(o.g.col, o.g.val, e0 + lane, int((__ldg(o.g.off + s + 1) - e0) >> 5), g);
}

// Slice loop of a phase: the block's own slices when staged (warps of the
// block), else a grid-stride loop over all warps.
template <typename T, class F>
__device__ __forceinline__ void for_slices(const Op<T>& o, long long warp, long long nwarps, F&& f) {
    if (o.staged) {
        const int wb = threadIdx.x >> 5, nwb = blockDim.x >> 5;
        for (long long s = o.s0 + wb; s < o.s1; s += nwb) f(s);
    } else {
        for (long long s = warp; s < o.g.nslices; s += nwarps) f(s);
    }
}

// MODE_JAC0 y = w D^-1 b, MODE_JAC y = x + w D^-1 (b - A x), MODE_JAC2 two
// sweeps from zero, MODE_RESID y = b - A x
template <typename T>
__device__ void pass(int mode, const Op<T>& A, const T* idiag, const T* x, const T* b, T* y, T omega, long long warp,
                     long long nwarps, int lane) {
    const long long n = A.g.n;
    for_slices(A, warp, nwarps, [&](long long s) {
        const long long i = s * 32 + lane;
        if (mode == MODE_JAC0) {
            if (i < n) y[i] = omega * __ldg(idiag + i) * ldv(b + i);
            return;
        }
        T acc;
        if (mode == MODE_JAC2)
            acc = op_row(A, s, lane, [&](int c) { return omega * __ldg(idiag + c) * ldv(b + c); });
        else
            acc = op_row(A, s, lane, [&](int c) { return ldv(x + c); });
        if (i < n) {
            const T bi = ldv(b + i), id = __ldg(idiag + i);
            if (mode == MODE_RESID) y[i] = bi - acc;
            else if (mode == MODE_JAC2) y[i] = omega * id * bi + omega * id * (bi - acc);
            else y[i] = ldv(x + i) + omega * id * (bi - acc);
        }
    });
}

// y (+)= M x for a prolongator or restriction
template <typename T>
__device__ void mv(const Op<T>& M, const T* x, T* y, bool acc_into, long long warp, long long nwarps, int lane) {
    const long long n = M.g.n;
    for_slices(M, warp, nwarps, [&](long long s) {
        const long long i = s * 32 + lane;
        const T acc = op_row(M, s, lane, [&](int c) { return ldv(x + c); });
        if (i < n) y[i] = acc_into ? ldv(y + i) + acc : acc;
    });
}

// y (+)= M x for a large operator in global memory with narrow rows (the
// transfers to and from the parent level): U slices per warp iteration, every
// load of the U slices issued before the gathers
template <typename T, int U, int K>
__device__ void mv_wide(const SellView<T>& M, const T* x, T* y, bool acc_into, long long warp, long long nwarps,
                        int lane) {
    for (long long s0 = warp; s0 < M.nslices; s0 += nwarps * U) {
        long long e[U];
        int w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long s = s0 + u * nwarps;
            const bool in = s < M.nslices;
            e[u] = in ? __ldg(M.off + s) : 0;
            w[u] = in ? int((__ldg(M.off + s + 1) - e[u]) >> 5) : 0;
        }
        int c[U][K];
        T v[U][K];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < K; ++k) {
                c[u][k] = k < w[u] ? __ldg(M.col + e[u] + lane + 32 * k) : 0;
                v[u][k] = k < w[u] ? __ldg(M.val + e[u] + lane + 32 * k) : T(0);
            }
        T acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            acc[u] = T(0);
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (k < w[u]) acc[u] += v[u][k] * ldv(x + c[u][k]);
            for (int k = K; k < w[u]; ++k)
                acc[u] += __ldg(M.val + e[u] + lane + 32 * k) * ldv(x + __ldg(M.col + e[u] + lane + 32 * k));
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long i = (s0 + u * nwarps) * 32 + lane;
            if (i < M.n) y[i] = acc_into ? ldv(y + i) + acc[u] : acc[u];
        }
    }
}

// Dense coarsest solve x = Ainv b in FP64 (b widened, x narrowed): the rows
// are split over the blocks, each row over all warps of its block, partial
// sums combined in shared memory.
template <typename T>
__device__ void coarse_solve(const double* cinv, int n, const T* b, T* x, double* red) {
    const int r0 = int((long long)n * blockIdx.x / gridDim.x), r1 = int((long long)n * (blockIdx.x + 1) / gridDim.x);
    const int wb = threadIdx.x >> 5, lane = threadIdx.x & 31, nwb = blockDim.x >> 5;
    for (int i = r0; i < r1; ++i) {
        const double* row = cinv + (long long)i * n;
        double acc = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) acc += __ldg(row + j) * double(ldv(b + j));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) red[wb] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < nwb; ++w) s += red[w];
            x[i] = T(s);
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kCoopThreads, 1) k_coarse_coop(CoopArgs<T> a) {
    if (a.sc && *((volatile const int*)&a.sc->done)) return;   // uniform: nothing writes it meanwhile
    extern __shared__ __align__(16) char coop_smem[];
    __shared__ double red[kCoopThreads / 32];
    __shared__ StagedDesc desc[3 * kMaxCoopLevels];
    const CoopTable<T>* __restrict__ tab = a.tab;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = ld_acquire(&a.bar->gen);
    CgScalars* sc = a.sc;
    // this block's slices of the staged operators
    {
        char* sm = coop_smem;
        for (int l = 0; l + 1 < a.nlev; ++l) {
            stage(tab->lev[l].A, (a.staged >> (3 * l)) & 1u, coop_smem, sm, &desc[3 * l]);
            stage(tab->lev[l].R, (a.staged >> (3 * l + 1)) & 1u, coop_smem, sm, &desc[3 * l + 1]);
            stage(tab->lev[l].P, (a.staged >> (3 * l + 2)) & 1u, coop_smem, sm, &desc[3 * l + 2]);
        }
    }
    __syncthreads();
    if (a.has_parent) {   // b of the first level = R_parent r_parent
        mv_wide<T, 2, 4>(tab->Rp, a.rp, tab->lev[0].b, false, warp, nwarps, lane);
        if (!grid_sync(a.bar, gen, sc)) return;
    }
    // per-level result and spare buffers of the down leg (shared: every thread
    // takes the same path; the barriers order the write before the reads)
    __shared__ T* cur[kMaxCoopLevels];
    __shared__ T* oth[kMaxCoopLevels];
    for (int l = 0; l + 1 < a.nlev; ++l) {
        const CoopLevel<T>& L = tab->lev[l];
        const Op<T> A = get_op(L.A, desc[3 * l], coop_smem);
        const T omega = L.omega;
        const T* idiag = L.idiag;
        const T* b = L.b;
        T* x = L.x;
        T* x2 = L.x2;
        pass(a.pre >= 2 ? MODE_JAC2 : MODE_JAC0, A, idiag, x, b, x, omega, warp, nwarps, lane);
        if (!grid_sync(a.bar, gen, sc)) return;
        for (int s = a.pre >= 2 ? 2 : 1; s < a.pre; ++s) {
            pass(MODE_JAC, A, idiag, x, b, x2, omega, warp, nwarps, lane);
            T* t = x;
            x = x2;
            x2 = t;
            if (!grid_sync(a.bar, gen, sc)) return;
        }
        pass(MODE_RESID, A, idiag, x, b, L.r, omega, warp, nwarps, lane);
        if (!grid_sync(a.bar, gen, sc)) return;
        mv(get_op(L.R, desc[3 * l + 1], coop_smem), L.r, tab->lev[l + 1].b, false, warp, nwarps, lane);
        if (threadIdx.x == 0) {
            cur[l] = x;
            oth[l] = x2;
        }
        if (!grid_sync(a.bar, gen, sc)) return;
    }
    {
        const CoopLevel<T>& C = tab->lev[a.nlev - 1];
        coarse_solve<T>(a.cinv, a.nc, C.b, C.x, red);
        if (!grid_sync(a.bar, gen, sc)) return;
    }
    for (int l = a.nlev - 2; l >= 0; --l) {
        const CoopLevel<T>& L = tab->lev[l];
        const T* xc = (l + 2 == a.nlev) ? tab->lev[l + 1].x : cur[l + 1];
        T* x = cur[l];
        T* x2 = oth[l];
        mv(get_op(L.P, desc[3 * l + 2], coop_smem), xc, x, true, warp, nwarps, lane);
        if (!grid_sync(a.bar, gen, sc)) return;
        const Op<T> A = get_op(L.A, desc[3 * l], coop_smem);
        for (int s = 0; s < a.post; ++s) {
            pass(MODE_JAC, A, L.idiag, x, L.b, x2, L.omega, warp, nwarps, lane);
            T* t = x;
            x = x2;
            x2 = t;
            if (!grid_sync(a.bar, gen, sc)) return;
        }
        if (threadIdx.x == 0) cur[l] = x;
        __syncthreads();
    }
    if (a.has_parent)   // x_parent += P_parent x of the first level
        mv_wide<T, 4, 4>(tab->Pp, a.nlev > 1 ? cur[0] : tab->lev[0].x, a.xp, true, warp, nwarps, lane);
}

}  // namespace

// The kernel's dynamic shared-memory attribute is process-wide: it only
// grows (to the largest size any context asked for), so a launch of one
// context never exceeds what another context set later.
template <typename T>
int coop_blocks_per_sm(int device, long long smem) {
    static long long reserved = 0;
    int per_sm = 0, coop = 0, optin = 0;
    const long long want = std::max(reserved, smem);
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) != cudaSuccess || !coop ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        want > optin ||
        cudaFuncSetAttribute(k_coarse_coop<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(want)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_coop<T>, kCoopThreads, size_t(want)) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    reserved = want;
    return per_sm;
}

// Shared-memory bytes per block of the staged operators (the same carving as
// the kernel) for a grid of `grid` blocks, from the host copies of the slice
// offsets in kernel order (A, R, P of each level; null entries unstaged).
long long coop_staged_bytes(const std::vector<const std::vector<long long>*>& offs, const std::vector<size_t>& tsz,
                            int grid) {
    long long worst = 0;
    auto a16 = [](long long b) { return (b + 15) & ~15LL; };
    for (int rank = 0; rank < grid; ++rank) {
        long long b = 0;
        for (size_t m = 0; m < offs.size(); ++m) {
            const std::vector<long long>* off = offs[m];
            if (!off) continue;
            const long long ns = (long long)off->size() - 1;
            const long long s0 = ns * rank / grid, s1 = ns * (rank + 1) / grid;
            const long long ne = (*off)[s1] - (*off)[s0];
            b = a16(b) + (s1 - s0 + 1) * 4;
            b = a16(b) + ne * 4;
            b = a16(b) + ne * (long long)tsz[m];
        }
        worst = std::max(worst, b + 16);
    }
    return worst;
}

template <typename T>
cudaError_t launch_coop(const CoopArgs<T>& a, int grid, long long smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kCoopThreads);
    cfg.dynamicSmemBytes = size_t(smem);
    cfg.stream = st;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeCooperative;
    at.val.cooperative = 1;
    cfg.attrs = &at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_coarse_coop<T>, a);
}

template int coop_blocks_per_sm<float>(int, long long);
template int coop_blocks_per_sm<double>(int, long long);
template cudaError_t launch_coop<float>(const CoopArgs<float>&, int, long long, cudaStream_t);
template cudaError_t launch_coop<double>(const CoopArgs<double>&, int, long long, cudaStream_t);

}  // namespace ibm

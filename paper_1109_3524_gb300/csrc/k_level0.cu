// Finest level of the FP32 pressure-block V-cycle (the smoothed-aggregation
// preconditioner of the Poisson solve, Eq. 9b, section 3) with temporal
// blocking: the pre-smoothing sweeps and the residual run in one kernel, and
// the post-smoothing sweeps (after the prolongation) in another.
//
// A block owns a box of 64 columns by TY + 2 S rows in shared memory: a tile
// of (64 - 2 S) x TY cells and a halo of S cells (S = number of sweeps).  After
// sweep p the iterate is exact on the tile grown by S - p cells, so after S
// sweeps it is exact on the tile itself and one pass over the inputs serves
// all S sweeps.  Halo cells are recomputed by every block that needs them.
// A thread owns two columns (tx and tx + 32) and every eighth row of the box
// and issues all its global loads before using any.  The block keeps the 1D
// link factors of its columns and rows (east link of cell (i, j) = ax_i ay_j,
// north link = bx_i by_j) and each cell's diagonal and w / diagonal in shared
// memory, formed once per launch, and checks grid edges and the pinned cell
// only in the blocks whose box reaches them.  The arithmetic of a sweep is the
// same sequence of FP32 operations as in the one-kernel-per-sweep path.
#include <algorithm>

#include "device.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace ibm {
namespace {

constexpr int kL0Threads = 256;   // 32 columns x 8 rows of threads
constexpr int kBoxW = 64;         // box width (two columns per thread)
constexpr int kTY = 32;           // tile rows

template <int S>
struct Box {
    static constexpr int W = kBoxW, H = kTY + 2 * S, TX = kBoxW - 2 * S, U = (H + 7) / 8;
};

__device__ __forceinline__ float fac(const float* a, int i, int n) { return (i >= 0 && i < n) ? __ldg(a + i) : 0.f; }

// Shared memory of a block: the box's right-hand side, two iterates, w / the
// unpinned diagonal of every cell, and the 1D factors of the
// box's columns and rows (for smem column c, global i = i0 + c:
// ax(i - 1) = ax[c], ax(i) = ax[c + 1]; for row r, global j = j0 + r:
// by(j - 1) = by[r], by(j) = by[r + 1]; zero outside the grid).
template <int S>
struct Smem {
    static constexpr int N = Box<S>::H * Box<S>::W;
    float sb[N], xa[N], xb[N], swd[N];
    float ax[Box<S>::W + 1], bx[Box<S>::W], ay[Box<S>::H], by[Box<S>::H + 1];
};

// Per-thread geometry: which of its cells lie in the grid, and the
// block-uniform flags of the slow paths.
template <int S>
struct Cells {
    int i0, j0, tx, ty;
    unsigned in_mask;   // bit 2u + h: cell (u, h) lies in the box and in the grid
    bool edge;          // the box reaches beyond the grid
    bool pin_near;      // the pinned cell or a neighbour of it lies in the box
    float axl[2], axr[2], bxc[2];   // factors of the thread's two columns: ax(i - 1), ax(i), bx(i)

    __device__ __forceinline__ void init(const Sep32& s, Smem<S>& m, float omega, int bx, int by) {
        using B = Box<S>;
        tx = threadIdx.x & 31;
        ty = threadIdx.x >> 5;
        i0 = bx * B::TX - S;
        j0 = by * kTY - S;
        for (int t = threadIdx.x; t < B::W + 1; t += blockDim.x) m.ax[t] = fac(s.ax, i0 + t - 1, s.nx);
        for (int t = threadIdx.x; t < B::W; t += blockDim.x) m.bx[t] = fac(s.bx, i0 + t, s.nx);
        for (int t = threadIdx.x; t < B::H; t += blockDim.x) m.ay[t] = fac(s.ay, j0 + t, s.ny);
        for (int t = threadIdx.x; t < B::H + 1; t += blockDim.x) m.by[t] = fac(s.by, j0 + t - 1, s.ny);
        in_mask = 0u;
#pragma unroll
        for (int u = 0; u < B::U; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = ty + 8 * u, i = i0 + tx + 32 * h, j = j0 + r;
                if (r < B::H && i >= 0 && i < s.nx && j >= 0 && j < s.ny) in_mask |= 1u << (2 * u + h);
            }
        edge = i0 < 0 || j0 < 0 || i0 + B::W > s.nx || j0 + B::H > s.ny;
        const int pi = int(s.pin % s.nx), pj = int(s.pin / s.nx);
        pin_near = pi >= i0 - 1 && pi <= i0 + B::W && pj >= j0 - 1 && pj <= j0 + B::H;
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            axl[h] = m.ax[tx + 32 * h];
            axr[h] = m.ax[tx + 32 * h + 1];
            bxc[h] = m.bx[tx + 32 * h];
        }
        // w / diagonal table (the diagonal itself is formed again from the links)
#pragma unroll
        for (int u = 0; u < B::U; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = ty + 8 * u, c = tx + 32 * h;
                if (r >= B::H) continue;
                const int idx = r * B::W + c;
                const float dg = inside(u, h) ? diag(h, m.ay[r], m.by[r], m.by[r + 1]) : 1.f;
                m.swd[idx] = omega * __frcp_rn(dg);
            }
    }
    // unpinned diagonal of a cell in column h of a row with factors ay, by(j - 1), by(j)
    __device__ __forceinline__ float diag(int h, float ayj, float bys, float byn) const {
        return (axr[h] + axl[h]) * ayj + bxc[h] * (byn + bys);
    }
    __device__ __forceinline__ bool inside(int u, int h) const { return (in_mask >> (2 * u + h)) & 1u; }
};

// y = x + w D^-1 (b - A x) (JAC) or b - A x (RESID) at box cell (u, h) from
// the shared box; links touching the pinned cell removed when pin_near.
// Row factors ayj = ay(j), bys = by(j - 1), byn = by(j) come from the caller
// (one load per row for the thread's two columns).
template <int S, bool RESID>
__device__ __forceinline__ float update(const Sep32& s, const Cells<S>& g, const Smem<S>& m, int u, int h,
                                        const float* x, float ayj, float bys, float byn) {
    constexpr int W = Box<S>::W;
    const int r = g.ty + 8 * u, c = g.tx + 32 * h, idx = r * W + c;
    const float dg = g.diag(h, ayj, bys, byn);
    float e = g.axr[h] * ayj, w = g.axl[h] * ayj, n = g.bxc[h] * byn, so = g.bxc[h] * bys;
    if (g.pin_near) {
        const long long k = (long long)(g.j0 + r) * s.nx + (g.i0 + c);
        if (k == s.pin) e = w = n = so = 0.f;
        if (k + 1 == s.pin) e = 0.f;
        if (k - 1 == s.pin) w = 0.f;
        if (k + s.nx == s.pin) n = 0.f;
        if (k - s.nx == s.pin) so = 0.f;
    }
    const float xc = x[idx];
    const float ax = dg * xc - e * x[idx + 1] - w * x[idx - 1] - n * x[idx + W] - so * x[idx - W];
    if (RESID) return m.sb[idx] - ax;
    return xc + m.swd[idx] * (m.sb[idx] - ax);
}

// Sweeps at margins M .. S-1 of the box, ping-ponging x and y; returns the
// buffer holding the last iterate.
template <int S, int M>
__device__ __forceinline__ float* sweeps(const Sep32& s, const Cells<S>& g, const Smem<S>& m, float* x, float* y) {
    using B = Box<S>;
    if constexpr (M >= S) {
        return x;
    } else {
#pragma unroll
        for (int u = 0; u < B::U; ++u) {
            const int r = g.ty + 8 * u;
            if (r < M || r >= B::H - M) continue;
            const float ayj = m.ay[r], bys = m.by[r], byn = m.by[r + 1];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = g.tx + 32 * h;
                if (c < M || c >= B::W - M) continue;
                const int idx = r * B::W + c;
                if (g.edge && !g.inside(u, h)) {
                    y[idx] = 0.f;
                    continue;
                }
                y[idx] = update<S, false>(s, g, m, u, h, x, ayj, bys, byn);
            }
        }
        __syncthreads();
        return sweeps<S, M + 1>(s, g, m, y, x);
    }
}

// Pre-smoothing of the finest level fused with its residual: S damped-Jacobi
// sweeps from x = 0 on b (FP64 in, read once), then r = b - A x_S.  Writes
// b32 = float(b) (the right-hand side of the post-smoother), x = x_S and r.
template <int S>
__global__ void __launch_bounds__(kL0Threads, 4) k_l0_pre(Sep32 s, const double* __restrict__ b,
                                                          float* __restrict__ b32, float* __restrict__ xo,
                                                          float* __restrict__ ro, float omega, DotArgs d,
                                                          int ntx, int ntiles) {
    pdl_entry();
    if (skip(d)) return;
    using B = Box<S>;
    extern __shared__ __align__(16) unsigned char l0_smem[];
    Smem<S>& m = *reinterpret_cast<Smem<S>*>(l0_smem);
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tbx = t % ntx, tby = t / ntx;
        Cells<S> g;
        // all loads of b first (they overlap the set-up), then x1 = w b / d
        double bv[B::U][2];
        {
            const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
            const int i0 = tbx * B::TX - S, j0 = tby * kTY - S;
#pragma unroll
            for (int u = 0; u < B::U; ++u)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = ty + 8 * u, i = i0 + tx + 32 * h, j = j0 + r;
                    bv[u][h] = (r < B::H && i >= 0 && i < s.nx && j >= 0 && j < s.ny)
                                   ? __ldg(b + (long long)j * s.nx + i) : 0.0;
                }
        }
        g.init(s, m, omega, tbx, tby);
#pragma unroll
        for (int u = 0; u < B::U; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g.ty + 8 * u;
                if (r >= B::H) continue;
                const int idx = r * B::W + g.tx + 32 * h;
                const float bf = float(bv[u][h]);
                m.sb[idx] = bf;
                m.xa[idx] = g.inside(u, h) ? m.swd[idx] * bf : 0.f;
            }
        __syncthreads();
        const float* x = sweeps<S, 1>(s, g, m, m.xa, m.xb);
        // residual on the tile; outputs
#pragma unroll
        for (int u = 0; u < B::U; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g.ty + 8 * u, c = g.tx + 32 * h;
                if (r < S || r >= B::H - S || c < S || c >= B::W - S || !g.inside(u, h)) continue;
                const long long k = (long long)(g.j0 + r) * s.nx + (g.i0 + c);
                const int idx = r * B::W + c;
                const float res = update<S, true>(s, g, m, u, h, x, m.ay[r], m.by[r], m.by[r + 1]);
                b32[k] = m.sb[idx];
                xo[k] = x[idx];
                ro[k] = res;
            }
        __syncthreads();   // the next tile overwrites the shared box
    }
}

// Post-smoothing of the finest level: S damped-Jacobi sweeps on b32 from x
// (the pre-smoothed iterate plus the prolongated correction), the last one
// written to out (TYo) - with DK_ZR the dots z.r and z.q of z = out (or
// z = base - out) into the reduction described by d.
template <typename TYo, int S, int DK>
__global__ void __launch_bounds__(kL0Threads, 4) k_l0_post(Sep32 s, const float* __restrict__ xin,
                                                           const float* __restrict__ b32, TYo* __restrict__ out,
                                                           float omega, DotArgs d, int ntx, int ntiles) {
    pdl_entry();
    if (skip(d)) return;
    using B = Box<S>;
    extern __shared__ __align__(16) unsigned char l0_smem[];
    Smem<S>& m = *reinterpret_cast<Smem<S>*>(l0_smem);
    double acc[2] = {0.0, 0.0};
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tbx = t % ntx, tby = t / ntx;
        Cells<S> g;
        float xv[B::U][2], bf[B::U][2];
        {
            const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
            const int i0 = tbx * B::TX - S, j0 = tby * kTY - S;
#pragma unroll
            for (int u = 0; u < B::U; ++u)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int r = ty + 8 * u, i = i0 + tx + 32 * h, j = j0 + r;
                    const bool in = r < B::H && i >= 0 && i < s.nx && j >= 0 && j < s.ny;
                    const long long k = (long long)j * s.nx + i;
                    xv[u][h] = in ? __ldg(xin + k) : 0.f;
                    bf[u][h] = in ? __ldg(b32 + k) : 0.f;
                }
        }
        g.init(s, m, omega, tbx, tby);
#pragma unroll
        for (int u = 0; u < B::U; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g.ty + 8 * u;
                if (r >= B::H) continue;
                const int idx = r * B::W + g.tx + 32 * h;
                m.sb[idx] = bf[u][h];
                m.xa[idx] = xv[u][h];
            }
        __syncthreads();
        const float* x = sweeps<S, 1>(s, g, m, m.xa, m.xb);
        // last sweep on the tile, then the FP64 dots of its output (loads of r, q
        // and base issued for a whole row group at a time)
#pragma unroll
        for (int u = 0; u < B::U; ++u) {
            float o[2];
            long long k[2];
            bool on[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = g.ty + 8 * u, c = g.tx + 32 * h;
                on[h] = r >= S && r < B::H - S && c >= S && c < B::W - S && g.inside(u, h);
                k[h] = (long long)(g.j0 + r) * s.nx + (g.i0 + c);
                o[h] = on[h] ? update<S, false>(s, g, m, u, h, x, m.ay[r], m.by[r], m.by[r + 1]) : 0.f;
            }
            if (DK == DK_ZR) {
                double rr[2], qq[2];
                float bs[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    rr[h] = on[h] ? __ldg(d.r + k[h]) : 0.0;
                    qq[h] = on[h] ? __ldg(d.q + k[h]) : 0.0;
                    bs[h] = (on[h] && d.base) ? __ldg(static_cast<const float*>(d.base) + k[h]) : 0.f;
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!on[h]) continue;
                    const double z = d.base ? double(bs[h]) - double(o[h]) : double(TYo(o[h]));
                    out[k[h]] = TYo(z);
                    acc[0] += z * rr[h];
                    acc[1] += z * qq[h];
                }
            } else {
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    if (on[h]) out[k[h]] = TYo(o[h]);
            }
        }
        __syncthreads();   // the next tile overwrites the shared box
    }
    if (DK == DK_ZR) reduce_and_finalize<2>(acc, d, d.slot0 + blockIdx.x);
}

// Tiles of a grid (x tiles, all tiles); a launch has min(tiles, kL0MaxBlocks)
// blocks, each looping over tiles, so that the reduction of the post-sweep
// kernel fits its partial-sum slots on any grid.
template <int S>
int2 tiles_s(int nx, int ny) {
    const int ntx = (nx + Box<S>::TX - 1) / Box<S>::TX;
    return make_int2(ntx, ntx * ((ny + kTY - 1) / kTY));
}
template <int S>
dim3 grid_s(int nx, int ny) {
    return dim3(unsigned(std::min(tiles_s<S>(nx, ny).y, kL0MaxBlocks)));
}

}  // namespace

dim3 l0_grid(int sweeps, int nx, int ny) {
    switch (sweeps) {
        case 1: return grid_s<1>(nx, ny);
        case 2: return grid_s<2>(nx, ny);
        case 3: return grid_s<3>(nx, ny);
        case 4: return grid_s<4>(nx, ny);
        case 5: return grid_s<5>(nx, ny);
        case 6: return grid_s<6>(nx, ny);
        default: return dim3(0, 0, 0);
    }
}

bool l0_fused_ok(int sweeps) { return sweeps >= 1 && sweeps <= kL0MaxSweeps; }

// Dynamic shared memory of a fused kernel (above the 48 KB default from
// S = 3 on): the attribute is set once per kernel instantiation.
template <int S>
void pre_s(const Sep32& s, const double* b, float* b32, float* x, float* r, float omega, const DotArgs& d,
           cudaStream_t st) {
    static const bool attr =
        cudaFuncSetAttribute(k_l0_pre<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sizeof(Smem<S>))) ==
        cudaSuccess;
    (void)attr;
    const int2 t = tiles_s<S>(s.nx, s.ny);
    launch_k(k_l0_pre<S>, grid_s<S>(s.nx, s.ny), kL0Threads, sizeof(Smem<S>), st, s, b, b32, x, r, omega, d, t.x,
             t.y);
}

template <typename TYo, int S, int DK>
void post_s(const Sep32& s, const float* xin, const float* b32, TYo* out, float omega, const DotArgs& d,
            cudaStream_t st) {
    static const bool attr = cudaFuncSetAttribute(k_l0_post<TYo, S, DK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  int(sizeof(Smem<S>))) == cudaSuccess;
    (void)attr;
    const int2 t = tiles_s<S>(s.nx, s.ny);
    launch_k(k_l0_post<TYo, S, DK>, grid_s<S>(s.nx, s.ny), kL0Threads, sizeof(Smem<S>), st, s, xin, b32, out, omega,
             d, t.x, t.y);
}

void launch_l0_pre(int sweeps, const Sep32& s, const double* b, float* b32, float* x, float* r, float omega,
                   const DotArgs& d, cudaStream_t st) {
    switch (sweeps) {
        case 1: pre_s<1>(s, b, b32, x, r, omega, d, st); break;
        case 2: pre_s<2>(s, b, b32, x, r, omega, d, st); break;
        case 3: pre_s<3>(s, b, b32, x, r, omega, d, st); break;
        case 4: pre_s<4>(s, b, b32, x, r, omega, d, st); break;
        case 5: pre_s<5>(s, b, b32, x, r, omega, d, st); break;
        case 6: pre_s<6>(s, b, b32, x, r, omega, d, st); break;
        default: break;
    }
}

template <typename TYo>
void launch_l0_post(int sweeps, int dk, const Sep32& s, const float* xin, const float* b32, TYo* out, float omega,
                    const DotArgs& d, cudaStream_t st) {
#define IBM_L0P(S)                                                 \
    do {                                                           \
        if (dk == DK_ZR) post_s<TYo, S, DK_ZR>(s, xin, b32, out, omega, d, st); \
        else post_s<TYo, S, DK_NONE>(s, xin, b32, out, omega, d, st);           \
    } while (0)
    switch (sweeps) {
        case 1: IBM_L0P(1); break;
        case 2: IBM_L0P(2); break;
        case 3: IBM_L0P(3); break;
        case 4: IBM_L0P(4); break;
        case 5: IBM_L0P(5); break;
        case 6: IBM_L0P(6); break;
        default: break;
    }
#undef IBM_L0P
}
template void launch_l0_post<float>(int, int, const Sep32&, const float*, const float*, float*, float,
                                    const DotArgs&, cudaStream_t);
template void launch_l0_post<double>(int, int, const Sep32&, const float*, const float*, double*, float,
                                     const DotArgs&, cudaStream_t);

}  // namespace ibm

// Solver kernels: matrix-free 5-point operators with the sparse body rows of
// Q^T B^1 Q (Eq. 9b), CG / flexible-CG vector updates with fused dot products
// (Eq. 9a, 9b), and the smoothed-aggregation V-cycle (section 3): damped
// Jacobi smoothing, residual, restriction, prolongation, coarsest solve.
#include "device.cuh"
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "kernels.h"
#include "reduce.cuh"

namespace ibm {

bool pdl_enabled() {
    static const bool on = std::getenv("IBM_NO_PDL") == nullptr;
    return on;
}

// ---------------------------------------------------------------------------
// 5-point operator (stencil part).  MODE: APPLY y = A x, RESID y = b - A x,
// JAC y = x + w D^-1 (b - A x), JAC0 y = w D^-1 b.  DK selects fused dots.
// ---------------------------------------------------------------------------
template <typename T, typename TB, typename TY, int MODE, int DK>
__global__ void __launch_bounds__(kThreads) k_stencil(Stencil<T> s, const T* __restrict__ x,
                                                      const TB* __restrict__ b, TY* __restrict__ y,
                                                      T omega, DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    // rows of nblk stacked nx*ny arrays: blockIdx.y strides over rows, threads over x
    const int nx = s.nx, ny = s.ny, nrows = ny * s.nblk;
    double acc[2] = {0.0, 0.0};
    for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
        const int j = row % ny;
        const int base = row * nx;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
            const int k = base + i;
            T out;
            if (MODE == MODE_JAC0) {
                out = omega * ld(s.idiag, k) * T(ld(b, k));
            } else {
                const T xc = ld(x, k);
                T ax = ld(s.diag, k) * xc;
                if (i + 1 < nx) ax -= ld(s.cE, k) * ld(x, k + 1);
                if (i > 0) ax -= ld(s.cE, k - 1) * ld(x, k - 1);
                if (j + 1 < ny) ax -= ld(s.cN, k) * ld(x, k + nx);
                if (j > 0) ax -= ld(s.cN, k - nx) * ld(x, k - nx);
                if (MODE == MODE_APPLY) out = ax;
                else if (MODE == MODE_RESID) out = T(ld(b, k)) - ax;
                else out = xc + omega * ld(s.idiag, k) * (T(ld(b, k)) - ax);
                if (DK == DK_XY) acc[0] += double(xc) * double(out);
            }
            if (DK == DK_ZR && d.base) {   // z = base - x (second V-cycle of the Schur preconditioner)
                const double z = double(static_cast<const T*>(d.base)[k]) - double(out);
                y[k] = TY(z);
                acc[0] += z * d.r[k];
                acc[1] += z * d.q[k];
                continue;
            }
            y[k] = TY(out);
            if (DK == DK_RESID) {
                const double bv = double(ld(b, k));
                acc[0] += bv * bv;
                acc[1] += double(out) * double(out);
            } else if (DK == DK_ZR) {
                const double z = double(TY(out));
                acc[0] += z * d.r[k];
                acc[1] += z * d.q[k];
            }
        }
    }
    if (DK != DK_NONE) reduce_and_finalize<2>(acc, d, d.slot0 + blockIdx.y * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------------------
// Finest pressure level of the FP32 V-cycle with couplings from 1D arrays:
// 12-16 bytes per cell and sweep instead of 32 with stored coefficients.
// A thread updates a strip of kV0Rows rows of one column, so the loads of
// the strip (centre column with a halo row each side, east and west
// neighbours, b) are all in flight together.
// ---------------------------------------------------------------------------
constexpr int kV0Rows = 4;

__device__ __forceinline__ float sep_ax(const Sep32& s, int i) { return (i >= 0 && i < s.nx) ? __ldg(s.ax + i) : 0.f; }
__device__ __forceinline__ float sep_by(const Sep32& s, int j) { return (j >= 0 && j < s.ny) ? __ldg(s.by + j) : 0.f; }

// unpinned diagonal of cell (i, j): the sum of its four links
__device__ __forceinline__ float sep_diag(const Sep32& s, int i, int j) {
    return (sep_ax(s, i) + sep_ax(s, i - 1)) * __ldg(s.ay + j) + __ldg(s.bx + i) * (sep_by(s, j) + sep_by(s, j - 1));
}

// V0_JAC / V0_RESID sweeps on b32 (DK_ZR: with the dots of the last sweep)
template <typename TY, int MODE, int DK>
__global__ void __launch_bounds__(kThreads) k_vc0(Sep32 s, const float* __restrict__ x, const double* __restrict__ b,
                                                  float* __restrict__ b32, TY* __restrict__ y, float omega,
                                                  DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    constexpr int R = kV0Rows;
    const int nx = s.nx, ny = s.ny;
    const int pin = int(s.pin);
    double acc[2] = {0.0, 0.0};
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (int j0 = blockIdx.y * R; j0 < ny && i < nx; j0 += gridDim.y * R) {
        const float axi = sep_ax(s, i), axw = sep_ax(s, i - 1), bxi = __ldg(s.bx + i);
        // centre column v[0..R+1] = rows j0-1 .. j0+R; east/west for the strip rows
        float vc[R + 2], ve[R], vw[R], bk[R];
#pragma unroll
        for (int r = 0; r < R + 2; ++r) {
            const int j = j0 - 1 + r;
            vc[r] = (j >= 0 && j < ny) ? x[j * nx + i] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = j0 + r;
            const int k = j * nx + i;
            const bool in = j < ny;
            ve[r] = (in && i + 1 < nx) ? x[k + 1] : 0.f;
            vw[r] = (in && i > 0) ? x[k - 1] : 0.f;
            bk[r] = in ? b32[k] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int j = j0 + r;
            if (j >= ny) break;
            const int k = j * nx + i;
            const float ayj = __ldg(s.ay + j), byn = sep_by(s, j), bys = sep_by(s, j - 1);
            float wE = axi * ayj, wW = axw * ayj, wN = bxi * byn, wS = bxi * bys;
            const float dg = (axi + axw) * ayj + bxi * (byn + bys);   // as sep_diag
            if (k == pin) wE = wW = wN = wS = 0.f;
            if (k + 1 == pin) wE = 0.f;
            if (k - 1 == pin) wW = 0.f;
            if (k + nx == pin) wN = 0.f;
            if (k - nx == pin) wS = 0.f;
            const float id = __frcp_rn(dg);
            const float xc = vc[r + 1];
            const float ax = dg * xc - wE * ve[r] - wW * vw[r] - wN * vc[r + 2] - wS * vc[r];
            const float out = MODE == V0_RESID ? bk[r] - ax : xc + omega * id * (bk[r] - ax);
            if (DK == DK_ZR) {
                const double z = d.base ? double(static_cast<const float*>(d.base)[k]) - double(out)
                                        : double(TY(out));
                y[k] = TY(z);
                acc[0] += z * d.r[k];
                acc[1] += z * d.q[k];
            } else {
                y[k] = TY(out);
            }
        }
    }
    if (DK == DK_ZR) reduce_and_finalize<2>(acc, d, d.slot0 + blockIdx.y * gridDim.x + blockIdx.x);
}

// First sweeps from x = 0 (V0_PRE2 / V0_PRE1): every cell's first iterate
// x1 = w b / d is formed once, into a shared tile of the block's columns (one
// halo column each side) and the strip rows (one halo row each side), so b is
// read and converted from FP64 once per cell.
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_vc0_pre(Sep32 s, const double* __restrict__ b,
                                                      float* __restrict__ b32, float* __restrict__ y, float omega,
                                                      DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    constexpr int R = kV0Rows;
    __shared__ float t[R + 2][kThreads + 2];
    const int nx = s.nx, ny = s.ny;
    const int pin = int(s.pin);
    const int i0 = blockIdx.x * blockDim.x;
    const int i = i0 + threadIdx.x;
    const bool col_in = i < nx;
    for (int j0 = blockIdx.y * R; j0 < ny; j0 += gridDim.y * R) {
        float bk[R];
#pragma unroll
        for (int r = 0; r < R + 2; ++r) {
            const int j = j0 - 1 + r;
            float v = 0.f;
            if (col_in && j >= 0 && j < ny) {
                const float bv = float(b[j * nx + i]);
                v = omega * bv * __frcp_rn(sep_diag(s, i, j));
                if (r >= 1 && r <= R) bk[r - 1] = bv;
            }
            t[r][threadIdx.x + 1] = v;
        }
        if (MODE == V0_PRE2 && (threadIdx.x == 0 || threadIdx.x == blockDim.x - 1)) {
            const int ih = threadIdx.x == 0 ? i0 - 1 : i0 + int(blockDim.x);
            const int th = threadIdx.x == 0 ? 0 : int(blockDim.x) + 1;
#pragma unroll
            for (int r = 1; r <= R; ++r) {
                const int j = j0 - 1 + r;
                t[r][th] = (ih >= 0 && ih < nx && j < ny) ? omega * float(b[j * nx + ih]) * __frcp_rn(sep_diag(s, ih, j))
                                                          : 0.f;
            }
        }
        __syncthreads();
        if (col_in) {
            const float axi = sep_ax(s, i), axw = sep_ax(s, i - 1), bxi = __ldg(s.bx + i);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j = j0 + r;
                if (j >= ny) break;
                const int k = j * nx + i;
                const float xc = t[r + 1][threadIdx.x + 1];
                float out = xc;
                if (MODE == V0_PRE2) {
                    const float ayj = __ldg(s.ay + j), byn = sep_by(s, j), bys = sep_by(s, j - 1);
                    float wE = axi * ayj, wW = axw * ayj, wN = bxi * byn, wS = bxi * bys;
                    const float dg = (axi + axw) * ayj + bxi * (byn + bys);   // as sep_diag
                    if (k == pin) wE = wW = wN = wS = 0.f;
                    if (k + 1 == pin) wE = 0.f;
                    if (k - 1 == pin) wW = 0.f;
                    if (k + nx == pin) wN = 0.f;
                    if (k - nx == pin) wS = 0.f;
                    const float ax = dg * xc - wE * t[r + 1][threadIdx.x + 2] - wW * t[r + 1][threadIdx.x] -
                                     wN * t[r + 2][threadIdx.x + 1] - wS * t[r][threadIdx.x + 1];
                    out = xc + omega * __frcp_rn(dg) * (bk[r] - ax);
                }
                b32[k] = bk[r];
                y[k] = out;
            }
        }
        __syncthreads();
    }
}

template <typename TY>
void launch_vc0(int mode, int dk, const Sep32& s, const float* x, const double* b, float* b32, TY* y, float omega,
                const DotArgs& d, dim3 grid, cudaStream_t st) {
#define IBM_V0(M, K) launch_k(k_vc0<TY, M, K>, grid, kThreads, 0, st, s, x, b, b32, y, omega, d)
    if (dk == DK_ZR) {
        if (mode == V0_JAC) IBM_V0(V0_JAC, DK_ZR);
        return;
    }
    if constexpr (std::is_same<TY, float>::value) {
        if (mode == V0_PRE2) {
            launch_k(k_vc0_pre<V0_PRE2>, grid, kThreads, 0, st, s, b, b32, y, omega, d);
            return;
        }
        if (mode == V0_PRE1) {
            launch_k(k_vc0_pre<V0_PRE1>, grid, kThreads, 0, st, s, b, b32, y, omega, d);
            return;
        }
    }
    switch (mode) {
        case V0_JAC: IBM_V0(V0_JAC, DK_NONE); break;
        case V0_RESID: IBM_V0(V0_RESID, DK_NONE); break;
        default: break;
    }
#undef IBM_V0
}
template void launch_vc0<float>(int, int, const Sep32&, const float*, const double*, float*, float*, float,
                                const DotArgs&, dim3, cudaStream_t);
template void launch_vc0<double>(int, int, const Sep32&, const float*, const double*, float*, double*, float,
                                 const DotArgs&, dim3, cudaStream_t);

// ---------------------------------------------------------------------------
// Body rows: touched cells and force rows (same MODE semantics; y of the
// touched cells already holds the stencil part).
// ---------------------------------------------------------------------------
template <typename T, typename TB, typename TY, int MODE, int DK>
__global__ void __launch_bounds__(kThreads) k_coupling(Coupling<T> c, const T* __restrict__ x,
                                                       const TB* __restrict__ b, TY* __restrict__ y,
                                                       const T* __restrict__ idiag, T omega, DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    double acc[2] = {0.0, 0.0};
    // items: the touched cells (padded to whole warps), then one warp per force row
    const long long ntc_pad = ((long long)c.ntc + 31) / 32 * 32;
    const long long total = ntc_pad + 32LL * c.nf;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        if (t < ntc_pad) {
            if (t >= c.ntc) continue;
            if (MODE == MODE_JAC0) continue;   // x = 0: no coupling term
            const long long cell = c.tcell[t];
            T e = T(0);
            for (long long p = c.tc_ptr[t]; p < c.tc_ptr[t + 1]; ++p) e += c.tc_val[p] * x[c.tc_col[p]];
            T cur = T(y[cell]);
            T out;
            if (MODE == MODE_APPLY) out = cur + e;
            else if (MODE == MODE_RESID) out = cur - e;
            else out = cur - omega * idiag[cell] * e;
            y[cell] = TY(out);
            if (DK == DK_XY) acc[0] += double(x[cell]) * double(e);
            if (DK == DK_ZR) {
                const double z = double(TY(out)) - double(TY(cur));
                acc[0] += z * d.r[cell];
                acc[1] += z * d.q[cell];
            }
            if (DK == DK_RESID) acc[1] += double(out) * double(out) - double(cur) * double(cur);
        } else {
            // a whole warp per force row: the row's entries over the lanes
            const long long u = t - ntc_pad;
            const long long r = u >> 5;
            const int lane = int(u & 31);
            const long long row = c.f0 + r;
            T out;
            if (MODE == MODE_JAC0) {
                out = omega * c.f_idiag[r] * T(b[row]);
            } else {
                T ax = T(0);
                for (long long p = c.f_ptr[r] + lane; p < c.f_ptr[r + 1]; p += 32) ax += c.f_val[p] * x[c.f_col[p]];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ax += __shfl_xor_sync(0xffffffffu, ax, o);
                if (MODE == MODE_APPLY) out = ax;
                else if (MODE == MODE_RESID) out = T(b[row]) - ax;
                else out = x[row] + omega * c.f_idiag[r] * (T(b[row]) - ax);
                if (DK == DK_XY && lane == 0) acc[0] += double(x[row]) * double(out);
            }
            if (lane != 0) continue;
            y[row] = TY(out);
            if (DK == DK_RESID) {
                const double bv = double(b[row]);
                acc[0] += bv * bv;
                acc[1] += double(out) * double(out);
            } else if (DK == DK_ZR) {
                const double z = double(TY(out));
                acc[0] += z * d.r[row];
                acc[1] += z * d.q[row];
            }
        }
    }
    if (DK != DK_NONE) reduce_and_finalize<2>(acc, d, d.slot0 + blockIdx.x);
}

// ---------------------------------------------------------------------------
// End of a loop body of the device-side iteration loop (conditional while
// node of a CUDA graph): continue while not done.  The guard bounds the
// number of bodies independently of the solver's own iteration count, so the
// loop ends even if a reduction never reported completion (status 2).
// ---------------------------------------------------------------------------
__global__ void k_loop_cond(cudaGraphConditionalHandle h, CgScalars* sc) {
    pdl_entry();
    if (threadIdx.x == 0) {
        const int g = ++sc->guard;
        if (!sc->done && g > sc->max_iter + 8) {
            sc->done = 1;
            sc->status = 2;
        }
        cudaGraphSetConditional(h, sc->done ? 0u : 1u);
    }
}
void launch_loop_cond(cudaGraphConditionalHandle h, CgScalars* sc, cudaStream_t st) {
    launch_k(k_loop_cond, 1, 32, 0, st, h, sc);
}

// ---------------------------------------------------------------------------
// CG vector kernels (FP64)
// ---------------------------------------------------------------------------
// p = z + beta p
__global__ void __launch_bounds__(kThreads) k_pupdate(long long n, const double* __restrict__ z,
                                                      double* __restrict__ p, DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    const double beta = d.sc->beta;
    if (beta == 0.0) {   // first direction: p = z (p may hold stale values)
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
             k += (long long)gridDim.x * blockDim.x)
            p[k] = z[k];
        return;
    }
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        p[k] = z[k] + beta * p[k];
}

// x += alpha p, r -= alpha q, rr; PW: z = idiag r (or z = r when idiag null), rz
template <int PW>
__global__ void __launch_bounds__(kThreads) k_cg_update(long long n, double* __restrict__ x,
                                                        double* __restrict__ r, const double* __restrict__ p,
                                                        const double* __restrict__ q, double* __restrict__ z,
                                                        const double* __restrict__ idiag, DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    const double alpha = d.sc->alpha;
    double acc[2] = {0.0, 0.0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        x[k] += alpha * p[k];
        const double rn = r[k] - alpha * q[k];
        r[k] = rn;
        acc[0] += rn * rn;
        if (PW) {
            const double zn = idiag ? idiag[k] * rn : rn;
            z[k] = zn;
            acc[1] += rn * zn;
        }
    }
    reduce_and_finalize<2>(acc, d, blockIdx.x);
}

// [a.a, b.b] (residual norms of the coupled system, formed after both the
// stencil and body-row kernels have written r)
__global__ void __launch_bounds__(kThreads) k_dot2(long long n, const double* __restrict__ a,
                                                   const double* __restrict__ b, DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    double acc[2] = {0.0, 0.0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const double av = a[k], bv = b[k];
        acc[0] += av * av;
        acc[1] += bv * bv;
    }
    reduce_and_finalize<2>(acc, d, blockIdx.x);
}

// z = idiag r (or r), rz: first pointwise-preconditioned residual
__global__ void __launch_bounds__(kThreads) k_pw_precond(long long n, const double* __restrict__ r,
                                                         double* __restrict__ z, const double* __restrict__ idiag,
                                                         DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    double acc[1] = {0.0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const double zn = idiag ? idiag[k] * r[k] : r[k];
        z[k] = zn;
        acc[0] += r[k] * zn;
    }
    reduce_and_finalize<1>(acc, d, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Schur-complement block preconditioner of [Lp C; C^T F]:
//   y1 = V r_p,  z_f = S^-1 (r_f - C^T y1),  z_p = y1 - V (C z_f),
// S = F - C^T V C (dense, 2 n_b square), V the pressure-block V-cycle.
// ---------------------------------------------------------------------------
// v[c] = C[c, row] for the cells of force row `row` (or 0 when clear)
__global__ void k_col_scatter(CsrView<double> Cf, long long f0, int row, double* __restrict__ v, int clear) {
    pdl_entry();
    for (long long p = Cf.ptr[row] + threadIdx.x; p < Cf.ptr[row + 1]; p += blockDim.x) {
        const int col = Cf.col[p];
        if (col < f0) v[col] = clear ? 0.0 : Cf.val[p];
    }
}

// S[k, col] = F[k, col] - (C^T w)_k for all force rows k
template <typename T>
__global__ void k_schur_col(CsrView<double> Cf, long long f0, int col, const T* __restrict__ w,
                            double* __restrict__ S) {
    pdl_entry();
    const int nf = int(Cf.n);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) {
        double ctw = 0.0, f = 0.0;
        for (long long p = Cf.ptr[k]; p < Cf.ptr[k + 1]; ++p) {
            const int cc = Cf.col[p];
            if (cc < f0) ctw += Cf.val[p] * double(w[cc]);
            else if (cc - f0 == col) f = Cf.val[p];
        }
        S[(long long)k * nf + col] = f - ctw;
    }
}

// ---- dense SPD inverse of the Schur complement on the device (Gauss-Jordan) ----
// S <- (S + S^T) / 2: the V-cycle-built complement is symmetric up to rounding
__global__ void k_symmetrize(int n, double* S) {
    pdl_entry();
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = int(t / n), j = int(t % n);
        if (j <= i) continue;
        const double a = 0.5 * (S[(long long)i * n + j] + S[(long long)j * n + i]);
        S[(long long)i * n + j] = a;
        S[(long long)j * n + i] = a;
    }
}

// Blocked in-place Gauss-Jordan inversion (no pivoting: S is SPD, so every
// pivot block is SPD; a non-positive scalar pivot inside a block sets *flag).
// Step k over the rows/columns [k, k+b) of the pivot block P:
//   P <- P^-1;  row panel (columns outside the block) <- P^-1 * row panel;
//   other rows: M_ij -= M_iK(old) * rowpanel_Kj,  M_iK <- -M_iK(old) * P^-1.
constexpr int kGJ = 32;

// (1) P^-1 of the b x b pivot block into pinv, and the old column panel of
// every row into cpan (n x b)
template <typename T>
__global__ void __launch_bounds__(1024) k_gj_block(int n, const T* M, int k, int b, T* pinv, T* cpan, int* flag) {
    pdl_entry();
    __shared__ T P[kGJ][kGJ + 1];
    const int tx = threadIdx.x % kGJ, ty = threadIdx.x / kGJ;
    if (blockIdx.x == 0) {
        P[ty][tx] = (ty < b && tx < b) ? M[(long long)(k + ty) * n + k + tx] : T(ty == tx ? 1 : 0);
        __syncthreads();
        for (int t = 0; t < b; ++t) {
            const T p = P[t][t];
            __syncthreads();
            if (ty == 0 && tx == 0 && !(p > T(0))) *flag = 1;
            const T pp = p > T(0) ? p : T(1);
            const T cit = P[ty][t];   // old column t
            __syncthreads();
            if (ty == t) P[t][tx] = (tx == t ? T(1) : P[t][tx]) / pp;
            __syncthreads();
            if (ty != t) P[ty][tx] = (tx == t ? T(0) : P[ty][tx]) - cit * P[t][tx];
            __syncthreads();
        }
        pinv[ty * kGJ + tx] = P[ty][tx];   // the padding stays identity / zero
    }
    // old column panel, all rows (the pivot rows included, unused)
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * b;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = t / b;
        const int c = int(t % b);
        cpan[i * kGJ + c] = M[i * n + k + c];
    }
}

// (2) row panel <- P^-1 * row panel (columns outside the block), pivot block <- P^-1
template <typename T>
__global__ void k_gj_rows(int n, T* M, int k, int b, const T* pinv) {
    pdl_entry();
    __shared__ T Pi[kGJ][kGJ];
    for (int t = threadIdx.x; t < kGJ * kGJ; t += blockDim.x) Pi[t / kGJ][t % kGJ] = pinv[t];
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    T col[kGJ];
    const bool inblk = j >= k && j < k + b;
#pragma unroll
    for (int r = 0; r < kGJ; ++r) col[r] = r < b ? M[(long long)(k + r) * n + j] : T(0);
#pragma unroll 4
    for (int r = 0; r < b; ++r) {
        T acc = T(0);
        if (inblk) {
            acc = Pi[r][j - k];
        } else {
#pragma unroll
            for (int q = 0; q < kGJ; ++q) acc += Pi[r][q] * col[q];
        }
        M[(long long)(k + r) * n + j] = acc;
    }
}

// (3) every other row: M_ij -= cpan_i . rowpanel_j (j outside the block),
// M_iK <- -cpan_i * P^-1 (j inside the block, where the row panel holds P^-1)
template <typename T>
__global__ void k_gj_update(int n, T* M, int k, int b, const T* cpan) {
    pdl_entry();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const bool inblk = j >= k && j < k + b;
    T rp[kGJ];
#pragma unroll
    for (int r = 0; r < kGJ; ++r) rp[r] = r < b ? M[(long long)(k + r) * n + j] : T(0);
    for (int i = blockIdx.y * 8; i < n && i < blockIdx.y * 8 + 8; ++i) {
        if (i >= k && i < k + b) continue;
        const T* ci = cpan + (long long)i * kGJ;
        T acc = T(0);
#pragma unroll
        for (int r = 0; r < kGJ; ++r)
            if (r < b) acc += ci[r] * rp[r];   // entries past b of the panel are not written
        const long long q = (long long)i * n + j;
        M[q] = (inblk ? T(0) : M[q]) - acc;
    }
}

__global__ void k_to_f32(long long n, const double* a, float* b) {
    pdl_entry();
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        b[t] = float(a[t]);
}

// ---- cache of V-cycle responses for moving bodies ----------------------------------
// v[cell] = val
__global__ void k_set_entry(double* v, long long cell, double val) {
    pdl_entry();
    if (threadIdx.x == 0) v[cell] = val;
}
// slot[cell] = s for the staged (cell, s) pairs; cell_of[s] = cell
__global__ void k_cache_map(int n, const long long* pairs, int* slot, long long* cell_of) {
    pdl_entry();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const long long c = pairs[2 * k], s = pairs[2 * k + 1];
        slot[c] = int(s);
        cell_of[s] = c;
    }
}
// forget the cached cells: slot[cell_of[s]] = -1
__global__ void k_cache_clear(int n, int* slot, const long long* cell_of) {
    pdl_entry();
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) slot[cell_of[s]] = -1;
}
// row and column sv of G from the response w = V e_v (V is symmetric)
template <typename T>
__global__ void k_cache_store(int nu, const long long* cell_of, const T* w, int sv, T* G, long long ld) {
    pdl_entry();
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += gridDim.x * blockDim.x) {
        const T val = w[cell_of[u]];
        G[(long long)sv * ld + u] = val;
        G[(long long)u * ld + sv] = val;
    }
}
// S = F - C^T G C from the force rows [C^T | F] (cells < f0, forces >= f0)
template <typename T>
__global__ void k_schur_cached(CsrView<double> Cf, long long f0, const int* slot, const T* G, long long ld,
                               double* S) {
    pdl_entry();
    const int nf = int(Cf.n);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= nf || i >= nf) return;
    double acc = 0.0, f = 0.0;
    for (long long p = Cf.ptr[i]; p < Cf.ptr[i + 1]; ++p) {
        const long long a = Cf.col[p];
        if (a >= f0) {
            if (a - f0 == j) f = Cf.val[p];
            continue;
        }
        const T* Ga = G + (long long)slot[a] * ld;
        double t = 0.0;
        for (long long q = Cf.ptr[j]; q < Cf.ptr[j + 1]; ++q) {
            const long long b = Cf.col[q];
            if (b < f0) t += Cf.val[q] * double(Ga[slot[b]]);
        }
        acc += Cf.val[p] * t;
    }
    S[(long long)i * nf + j] = f - acc;
}

void launch_set_entry(double* v, long long cell, double val, cudaStream_t st) {
    launch_k(k_set_entry, 1, 32, 0, st, v, cell, val);
}
void launch_cache_map(int n, const long long* pairs, int* slot, long long* cell_of, cudaStream_t st) {
    if (n > 0) launch_k(k_cache_map, (n + kThreads - 1) / kThreads, kThreads, 0, st, n, pairs, slot, cell_of);
}
void launch_cache_clear(int n, int* slot, const long long* cell_of, cudaStream_t st) {
    if (n > 0) launch_k(k_cache_clear, (n + kThreads - 1) / kThreads, kThreads, 0, st, n, slot, cell_of);
}
template <typename T>
void launch_cache_store(int nu, const long long* cell_of, const T* w, int sv, T* G, long long ld, cudaStream_t st) {
    launch_k(k_cache_store<T>, (nu + kThreads - 1) / kThreads, kThreads, 0, st, nu, cell_of, w, sv, G, ld);
}
template <typename T>
void launch_schur_cached(const CsrView<double>& Cf, long long f0, const int* slot, const T* G, long long ld, double* S,
                         cudaStream_t st) {
    const int nf = int(Cf.n);
    launch_k(k_schur_cached<T>, dim3((nf + 127) / 128, nf), 128, 0, st, Cf, f0, slot, G, ld, S);
}
template void launch_cache_store<float>(int, const long long*, const float*, int, float*, long long, cudaStream_t);
template void launch_cache_store<double>(int, const long long*, const double*, int, double*, long long, cudaStream_t);
template void launch_schur_cached<float>(const CsrView<double>&, long long, const int*, const float*, long long,
                                         double*, cudaStream_t);
template void launch_schur_cached<double>(const CsrView<double>&, long long, const int*, const double*, long long,
                                          double*, cudaStream_t);

template <typename T>
void gj_invert(int n, T* M, T* scratch, int* flag, cudaStream_t st) {
    T* pinv = scratch;                 // kGJ x kGJ
    T* cpan = scratch + kGJ * kGJ;     // n x kGJ
    const int gr = (n + kThreads - 1) / kThreads;
    const dim3 gu(gr, (n + 7) / 8);
    const int gb = int(std::min<long long>(((long long)n * kGJ + 1023) / 1024, 1024));
    for (int k = 0; k < n; k += kGJ) {
        const int b = std::min(kGJ, n - k);
        launch_k(k_gj_block<T>, gb, 1024, 0, st, n, (const T*)M, k, b, pinv, cpan, flag);
        launch_k(k_gj_rows<T>, gr, kThreads, 0, st, n, M, k, b, (const T*)pinv);
        launch_k(k_gj_update<T>, gu, kThreads, 0, st, n, M, k, b, (const T*)cpan);
    }
}

void launch_spd_inverse(int n, double* M, double* scratch, int* flag, float* M32, cudaStream_t st) {
    const long long nn = (long long)n * n;
    const int g1 = int(std::min<long long>((nn + kThreads - 1) / kThreads, 4096));
    launch_k(k_symmetrize, g1, kThreads, 0, st, n, M);
    if (M32) {   // S narrowed to FP32 and inverted there; M keeps S
        launch_k(k_to_f32, g1, kThreads, 0, st, nn, (const double*)M, M32);
        gj_invert<float>(n, M32, reinterpret_cast<float*>(scratch), flag, st);
    } else {
        gj_invert<double>(n, M, scratch, flag, st);
    }
}

// tf = r_f - C^T y1
template <typename T>
__global__ void k_schur_tf(CsrView<double> Cf, long long f0, const double* __restrict__ r, const T* __restrict__ y1,
                           double* __restrict__ tf, const CgScalars* sc) {
    pdl_entry();
    if (sc && *((volatile const int*)&sc->done)) return;
    const int nf = int(Cf.n);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) {
        double s = r[f0 + k];
        for (long long p = Cf.ptr[k]; p < Cf.ptr[k + 1]; ++p) {
            const int cc = Cf.col[p];
            if (cc < f0) s -= Cf.val[p] * double(y1[cc]);
        }
        tf[k] = s;
    }
}

// out = add + sign M v (one warp per row of the dense nf x nf M; add
// nullable); DOTS: with the force part of z.r, z.q of z = out into d
template <typename T, bool DOTS>
__device__ __forceinline__ void k_dense_mv_body(int nf, const T* __restrict__ Sinv, const double* __restrict__ tf,
                                                const double* __restrict__ add, double sign, double* __restrict__ zf,
                                                const DotArgs& d) {
    pdl_entry();
    if (skip(d)) return;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    double acc[2] = {0.0, 0.0};
    // FP64 products and sums (an FP32 accumulation of S^-1 t measurably raised
    // the iteration count), four independent partial sums per lane
    for (int k = warp; k < nf; k += nwarps) {
        const T* row = Sinv + (long long)k * nf;
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        int j = lane;
        for (; j + 96 < nf; j += 128) {
            a[0] += double(row[j]) * tf[j];
            a[1] += double(row[j + 32]) * tf[j + 32];
            a[2] += double(row[j + 64]) * tf[j + 64];
            a[3] += double(row[j + 96]) * tf[j + 96];
        }
        for (; j < nf; j += 32) a[0] += double(row[j]) * tf[j];
        double s = (a[0] + a[1]) + (a[2] + a[3]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            const double z = add ? add[k] + sign * s : s;
            zf[k] = z;
            if (DOTS) {
                acc[0] += z * d.r[k];
                acc[1] += z * d.q[k];
            }
        }
    }
    if (DOTS) reduce_and_finalize<2>(acc, d, d.slot0 + blockIdx.x);
}

// z_f = S^-1 tf (one warp per row, dense) with the force part of z.r, z.q
template <typename T>
__global__ void __launch_bounds__(kThreads) k_schur_zf(int nf, const T* __restrict__ Sinv, const double* __restrict__ tf,
                                                       double* __restrict__ zf, DotArgs d) {
    k_dense_mv_body<T, true>(nf, Sinv, tf, nullptr, 1.0, zf, d);
}

// out = add + sign M v for a dense nf x nf M (add nullable), no dots
template <typename T>
__global__ void __launch_bounds__(kThreads) k_dense_mv(int nf, const T* __restrict__ M, const double* __restrict__ v,
                                                       const double* __restrict__ add, double sign,
                                                       double* __restrict__ out, DotArgs d) {
    k_dense_mv_body<T, false>(nf, M, v, add, sign, out, d);
}

// s[tcell] = (C z_f)[tcell]  (other entries of s stay zero)
__global__ void k_schur_sp(int ntc, const long long* __restrict__ tcell, CsrView<double> Cc, long long f0,
                           const double* __restrict__ z, double* __restrict__ s, const CgScalars* sc) {
    pdl_entry();
    if (sc && *((volatile const int*)&sc->done)) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntc; t += gridDim.x * blockDim.x) {
        double a = 0.0;
        for (long long p = Cc.ptr[t]; p < Cc.ptr[t + 1]; ++p) a += Cc.val[p] * z[Cc.col[p]];
        s[tcell[t]] = a;
    }
}

// ---------------------------------------------------------------------------
// AMG levels of the V-cycle (sliced ELLPACK)
// ---------------------------------------------------------------------------
// One warp per 32-row slice, one lane per row: y = A x, b - A x,
// x + w D^-1 (b - A x) or w D^-1 b (MODE as for the stencil).
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_sell(SellView<T> A, const T* __restrict__ idiag,
                                                   const T* __restrict__ x, const T* __restrict__ b,
                                                   T* __restrict__ y, T omega, const CgScalars* sc) {
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    // the warp's first slice of A is loaded before the wait on the preceding kernel
    SellPre<T> pa;
    if (MODE != MODE_JAC0 && s < A.nslices) pa.fetch(A.off, A.col, A.val, s, lane);
    pdl_entry();
    if (sc && *((volatile const int*)&sc->done)) return;
    for (bool first = true; s < A.nslices; s += nwarps, first = false) {
        const long long i = s * 32 + lane;
        if (MODE == MODE_JAC0) {
            if (i < A.n) y[i] = omega * idiag[i] * b[i];
            continue;
        }
        if (!first) pa.fetch(A.off, A.col, A.val, s, lane);
        T acc;
        if (MODE == MODE_JAC2)   // neighbours after the first sweep from zero: w D^-1 b
            acc = pa.apply(A.col, A.val, [&](int c) { return omega * idiag[c] * b[c]; });
        else
            acc = pa.apply(A.col, A.val, [&](int c) { return x[c]; });
        if (i < A.n) {
            if (MODE == MODE_APPLY) y[i] = acc;
            else if (MODE == MODE_RESID) y[i] = b[i] - acc;
            else if (MODE == MODE_JAC2) {
                const T x1 = omega * idiag[i] * b[i];
                y[i] = x1 + omega * idiag[i] * (b[i] - acc);
            } else y[i] = x[i] + omega * idiag[i] * (b[i] - acc);
        }
    }
}

// y (+)= A x  (restriction: y = R r; prolongation: y += P xc)
template <typename T, int ACC>
__global__ void __launch_bounds__(kThreads) k_sell_mv(SellView<T> A, const T* __restrict__ x,
                                                      T* __restrict__ y, const CgScalars* sc) {
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    SellPre<T> pa;   // first slice loaded before the wait on the preceding kernel
    if (s < A.nslices) pa.fetch(A.off, A.col, A.val, s, lane);
    pdl_entry();
    if (sc && *((volatile const int*)&sc->done)) return;
    for (bool first = true; s < A.nslices; s += nwarps, first = false) {
        const long long i = s * 32 + lane;
        if (!first) pa.fetch(A.off, A.col, A.val, s, lane);
        const T acc = pa.apply(A.col, A.val, [&](int c) { return x[c]; });
        if (i < A.n) {
            if (ACC) y[i] += acc;
            else y[i] = acc;
        }
    }
}

// Pre-smoothing and restriction of a level in one launch.  Blocks [0, nbA)
// form x = PRE damped-Jacobi sweeps from x = 0 (PRE 1: w D^-1 b; PRE 2: the
// second sweep with the neighbours' first sweep formed on the fly), blocks
// [nbA, ..) the coarse right-hand side b_c = Rt b with Rt = R (I - A w D^-1)^PRE:
// the residual left by those sweeps is (I - A w D^-1)^PRE b, so both halves
// need only b.  Rt rows are wide (tens of entries): LPR lanes per row.
template <typename T, int PRE, int LPR>
__global__ void __launch_bounds__(kThreads) k_sell_down(SellView<T> A, const T* __restrict__ idiag,
                                                        const T* __restrict__ b, T* __restrict__ x, T omega,
                                                        CsrView<T> Rt, T* __restrict__ bc, int nbA,
                                                        const CgScalars* sc) {
    const int lane = threadIdx.x & 31;
    if (int(blockIdx.x) < nbA) {
        const long long nwarps = ((long long)nbA * blockDim.x) >> 5;
        long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
        SellPre<T> pa;   // first slice loaded before the wait on the preceding kernel
        if (PRE == 2 && s < A.nslices) pa.fetch(A.off, A.col, A.val, s, lane);
        pdl_entry();
        if (sc && *((volatile const int*)&sc->done)) return;
        for (bool first = true; s < A.nslices; s += nwarps, first = false) {
            const long long i = s * 32 + lane;
            if (PRE == 1) {
                if (i < A.n) x[i] = omega * idiag[i] * b[i];
                continue;
            }
            if (!first) pa.fetch(A.off, A.col, A.val, s, lane);
            const T acc = pa.apply(A.col, A.val, [&](int c) { return omega * idiag[c] * b[c]; });
            if (i < A.n) {
                const T x1 = omega * idiag[i] * b[i];
                x[i] = x1 + omega * idiag[i] * (b[i] - acc);
            }
        }
        return;
    }
    constexpr int RPW = 32 / LPR;   // rows per warp
    const long long gw = ((long long)(blockIdx.x - nbA) * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)(gridDim.x - nbA) * blockDim.x) >> 5;
    const int g = lane / LPR, sub = lane % LPR;
    // the first chunk of the warp's first rows is loaded before the wait on
    // the preceding kernel
    long long r0 = gw * RPW;
    long long pb = 0, pe = 0;
    int c0[4];
    T v0[4];
    if (r0 + g < Rt.n) {
        pb = Rt.ptr[r0 + g] + sub;
        pe = Rt.ptr[r0 + g + 1];
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long q = pb + k * LPR;
        c0[k] = q < pe ? Rt.col[q] : 0;
        v0[k] = q < pe ? Rt.val[q] : T(0);
    }
    pdl_entry();
    if (sc && *((volatile const int*)&sc->done)) return;
    // the loop bound is the same for every lane of the warp (the shuffles below
    // need the whole warp)
    for (bool first = true; r0 < Rt.n; r0 += nw * RPW, first = false) {
        const long long r = r0 + g;
        T acc = T(0);
        if (r < Rt.n) {
            long long p, p1;
            if (first) {
#pragma unroll
                for (int k = 0; k < 4; ++k) acc += v0[k] * b[c0[k]];
                p = pb + 4 * LPR;
                p1 = pe;
            } else {
                p = Rt.ptr[r] + sub;
                p1 = Rt.ptr[r + 1];
            }
            for (; p < p1; p += 4 * LPR) {
                int c[4];
                T v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const long long q = p + k * LPR;
                    c[k] = q < p1 ? Rt.col[q] : 0;
                    v[k] = q < p1 ? Rt.val[q] : T(0);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) acc += v[k] * b[c[k]];
            }
        }
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (r < Rt.n && sub == 0) bc[r] = acc;
    }
}

// The coarse correction and the first post-sweep in one launch:
// y = x + w D^-1 (b - A x) + Q x_c with Q = (I - w D^-1 A) P, which is the
// sweep applied to x + P x_c.  Q has the level's rows, so its slices line up
// with A's.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_sell_up(SellView<T> A, const T* __restrict__ idiag,
                                                      const T* __restrict__ x, const T* __restrict__ b,
                                                      T* __restrict__ y, T omega, SellView<T> Q,
                                                      const T* __restrict__ xc, const CgScalars* sc) {
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    SellPre<T> pa, pq;   // first slice of A and Q loaded before the wait on the preceding kernel
    if (s < A.nslices) {
        pa.fetch(A.off, A.col, A.val, s, lane);
        pq.fetch(Q.off, Q.col, Q.val, s, lane);
    }
    pdl_entry();
    if (sc && *((volatile const int*)&sc->done)) return;
    for (bool first = true; s < A.nslices; s += nwarps, first = false) {
        const long long i = s * 32 + lane;
        if (!first) {
            pa.fetch(A.off, A.col, A.val, s, lane);
            pq.fetch(Q.off, Q.col, Q.val, s, lane);
        }
        const T acc = pa.apply(A.col, A.val, [&](int c) { return x[c]; });
        const T cor = pq.apply(Q.col, Q.val, [&](int c) { return xc[c]; });
        if (i < A.n) y[i] = x[i] + omega * idiag[i] * (b[i] - acc) + cor;
    }
}

// Poisson operator Q^T B^N Q (N > 1) held as an FP64 sliced-ELLPACK matrix:
// y = A x (MODE_APPLY) or b - A x (MODE_RESID) with the fused reductions of
// the 5-point path: DK_XY [x.y], DK_RESID [b.b, y.y].
template <int MODE, int DK>
__global__ void __launch_bounds__(kThreads) k_sell_op(SellView<double> A, const double* __restrict__ x,
                                                      const double* __restrict__ b, double* __restrict__ y,
                                                      DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    double acc[2] = {0.0, 0.0};
    for (long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; s < A.nslices; s += nwarps) {
        const long long i = s * 32 + lane;
        const long long o0 = A.off[s];
        const double ax = sell_row(A.col, A.val, o0 + lane, int((A.off[s + 1] - o0) >> 5), [&](int c) { return x[c]; });
        if (i < A.n) {
            const double out = MODE == MODE_RESID ? b[i] - ax : ax;
            y[i] = out;
            if (DK == DK_XY) {
                acc[0] += x[i] * out;
            } else if (DK == DK_RESID) {
                acc[0] += b[i] * b[i];
                acc[1] += out * out;
            }
        }
    }
    if (DK != DK_NONE) reduce_and_finalize<2>(acc, d, d.slot0 + blockIdx.x);
}

// level-0 right-hand side of a V-cycle in the level's type
template <typename T>
__global__ void __launch_bounds__(kThreads) k_narrow(long long n, const double* __restrict__ a, T* __restrict__ b,
                                                     const CgScalars* sc) {
    pdl_entry();
    if (sc && *((volatile const int*)&sc->done)) return;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        b[k] = T(a[k]);
}

// z = x widened to FP64; DK_ZR: [z.r, z.q] into the reduction d
template <typename T, int DK>
__global__ void __launch_bounds__(kThreads) k_widen(long long n, const T* __restrict__ x, double* __restrict__ z,
                                                    DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    double acc[2] = {0.0, 0.0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double v = double(x[k]);
        z[k] = v;
        if (DK == DK_ZR) {
            acc[0] += v * d.r[k];
            acc[1] += v * d.q[k];
        }
    }
    if (DK == DK_ZR) reduce_and_finalize<2>(acc, d, d.slot0 + blockIdx.x);
}

// x = Ainv b, dense FP64 inverse of the coarsest operator
template <typename T>
__global__ void __launch_bounds__(kThreads) k_coarse(int n, const double* __restrict__ Ainv,
                                                     const T* __restrict__ b, T* __restrict__ x,
                                                     const CgScalars* sc) {
    __shared__ double bs[2048];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    // the first KC entries per lane of the warp's first row of the inverse are
    // loaded before the wait on the preceding kernel
    constexpr int KC = 24;
    double a0[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) {
        const int j = lane + 32 * k;
        a0[k] = (warp < n && j < n) ? Ainv[(long long)warp * n + j] : 0.0;
    }
    pdl_entry();
    if (sc && *((volatile const int*)&sc->done)) return;
    for (int i = threadIdx.x; i < n; i += blockDim.x) bs[i] = double(b[i]);
    __syncthreads();
    for (int i = warp; i < n; i += nwarps) {
        double s = 0.0;
        int j = lane;
        if (i == warp) {
#pragma unroll
            for (int k = 0; k < KC; ++k, j += 32)
                if (j < n) s += a0[k] * bs[j];
        }
        for (; j < n; j += 32) s += Ainv[(long long)i * n + j] * bs[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) x[i] = T(s);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T, typename TB, typename TY>
void launch_stencil(int mode, int dk, const Stencil<T>& s, const T* x, const TB* b, TY* y, T omega,
                    const DotArgs& d, dim3 grid, cudaStream_t st) {
#define IBM_ST(M, K) launch_k(k_stencil<T, TB, TY, M, K>, grid, kThreads, 0, st, s, x, b, y, omega, d)
    switch (mode * 4 + dk) {
        case MODE_APPLY * 4 + DK_NONE: IBM_ST(MODE_APPLY, DK_NONE); break;
        case MODE_APPLY * 4 + DK_XY: IBM_ST(MODE_APPLY, DK_XY); break;
        case MODE_RESID * 4 + DK_NONE: IBM_ST(MODE_RESID, DK_NONE); break;
        case MODE_RESID * 4 + DK_RESID: IBM_ST(MODE_RESID, DK_RESID); break;
        case MODE_JAC * 4 + DK_NONE: IBM_ST(MODE_JAC, DK_NONE); break;
        case MODE_JAC * 4 + DK_ZR: IBM_ST(MODE_JAC, DK_ZR); break;
        case MODE_JAC0 * 4 + DK_NONE: IBM_ST(MODE_JAC0, DK_NONE); break;
        case MODE_JAC0 * 4 + DK_ZR: IBM_ST(MODE_JAC0, DK_ZR); break;
        default: break;
    }
#undef IBM_ST
}

template <typename T, typename TB, typename TY>
void launch_coupling(int mode, int dk, const Coupling<T>& c, const T* x, const TB* b, TY* y,
                     const T* idiag, T omega, const DotArgs& d, int grid, cudaStream_t st) {
#define IBM_CP(M, K) launch_k(k_coupling<T, TB, TY, M, K>, grid, kThreads, 0, st, c, x, b, y, idiag, omega, d)
    switch (mode * 4 + dk) {
        case MODE_APPLY * 4 + DK_NONE: IBM_CP(MODE_APPLY, DK_NONE); break;
        case MODE_APPLY * 4 + DK_XY: IBM_CP(MODE_APPLY, DK_XY); break;
        case MODE_RESID * 4 + DK_NONE: IBM_CP(MODE_RESID, DK_NONE); break;
        case MODE_RESID * 4 + DK_RESID: IBM_CP(MODE_RESID, DK_RESID); break;
        case MODE_JAC * 4 + DK_NONE: IBM_CP(MODE_JAC, DK_NONE); break;
        case MODE_JAC * 4 + DK_ZR: IBM_CP(MODE_JAC, DK_ZR); break;
        case MODE_JAC0 * 4 + DK_NONE: IBM_CP(MODE_JAC0, DK_NONE); break;
        case MODE_JAC0 * 4 + DK_ZR: IBM_CP(MODE_JAC0, DK_ZR); break;
        default: break;
    }
#undef IBM_CP
}

template void launch_stencil<double, double, double>(int, int, const Stencil<double>&, const double*,
                                                     const double*, double*, double, const DotArgs&, dim3,
                                                     cudaStream_t);
template void launch_stencil<float, double, float>(int, int, const Stencil<float>&, const float*,
                                                   const double*, float*, float, const DotArgs&, dim3,
                                                   cudaStream_t);
template void launch_stencil<float, double, double>(int, int, const Stencil<float>&, const float*,
                                                    const double*, double*, float, const DotArgs&, dim3,
                                                    cudaStream_t);
template void launch_coupling<double, double, double>(int, int, const Coupling<double>&, const double*,
                                                      const double*, double*, const double*, double,
                                                      const DotArgs&, int, cudaStream_t);
template void launch_coupling<float, double, float>(int, int, const Coupling<float>&, const float*,
                                                    const double*, float*, const float*, float,
                                                    const DotArgs&, int, cudaStream_t);
template void launch_coupling<float, double, double>(int, int, const Coupling<float>&, const float*,
                                                     const double*, double*, const float*, float,
                                                     const DotArgs&, int, cudaStream_t);

void launch_pupdate(long long n, const double* z, double* p, const DotArgs& d, int grid, cudaStream_t st) {
    launch_k(k_pupdate, grid, kThreads, 0, st, n, z, p, d);
}
void launch_cg_update(int pw, long long n, double* x, double* r, const double* p, const double* q, double* z,
                      const double* idiag, const DotArgs& d, int grid, cudaStream_t st) {
    if (pw) launch_k(k_cg_update<1>, grid, kThreads, 0, st, n, x, r, p, q, z, idiag, d);
    else launch_k(k_cg_update<0>, grid, kThreads, 0, st, n, x, r, p, q, z, idiag, d);
}
void launch_col_scatter(const CsrView<double>& Cf, long long f0, int row, double* v, int clear, cudaStream_t st) {
    launch_k(k_col_scatter, 1, 64, 0, st, Cf, f0, row, v, clear);
}
template <typename T>
void launch_schur_col(const CsrView<double>& Cf, long long f0, int col, const T* w, double* S, cudaStream_t st) {
    launch_k(k_schur_col<T>, int((Cf.n + 127) / 128), 128, 0, st, Cf, f0, col, w, S);
}
template <typename T>
void launch_schur_tf(const CsrView<double>& Cf, long long f0, const double* r, const T* y1, double* tf,
                     const CgScalars* sc, cudaStream_t st) {
    launch_k(k_schur_tf<T>, int((Cf.n + 127) / 128), 128, 0, st, Cf, f0, r, y1, tf, sc);
}
template <typename T>
void launch_schur_zf(int nf, const T* Sinv, const double* tf, double* zf, const DotArgs& d, int grid,
                     cudaStream_t st) {
    launch_k(k_schur_zf<T>, grid, kThreads, 0, st, nf, Sinv, tf, zf, d);
}
template <typename T>
void launch_dense_mv(int nf, const T* M, const double* v, const double* add, double sign, double* out,
                     const CgScalars* sc, int grid, cudaStream_t st) {
    DotArgs d;
    d.sc = const_cast<CgScalars*>(sc);
    launch_k(k_dense_mv<T>, grid, kThreads, 0, st, nf, M, v, add, sign, out, d);
}
// v[k] in [-0.5, 0.5) from a multiplicative hash of k (a fixed probe vector)
__global__ void k_probe_fill(int n, double* __restrict__ v) {
    pdl_entry();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        v[k] = double((unsigned(k) + 1u) * 2654435761u) * (1.0 / 4294967296.0) - 0.5;
}
void launch_probe_fill(int n, double* v, cudaStream_t st) {
    launch_k(k_probe_fill, std::max(1, std::min((n + kThreads - 1) / kThreads, 1024)), kThreads, 0, st, n, v);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_dense_mv_dots(int nf, const T* __restrict__ M, const double* __restrict__ v,
                                                            const double* __restrict__ add, double* __restrict__ out,
                                                            DotArgs d) {
    k_dense_mv_body<T, true>(nf, M, v, add, 1.0, out, d);
}
template <typename T>
void launch_dense_mv_dots(int nf, const T* M, const double* v, const double* add, double* out, const DotArgs& d,
                          int grid, cudaStream_t st) {
    launch_k(k_dense_mv_dots<T>, grid, kThreads, 0, st, nf, M, v, add, out, d);
}
template void launch_dense_mv_dots<float>(int, const float*, const double*, const double*, double*, const DotArgs&, int,
                                          cudaStream_t);
template void launch_dense_mv<double>(int, const double*, const double*, const double*, double, double*,
                                      const CgScalars*, int, cudaStream_t);
template void launch_dense_mv<float>(int, const float*, const double*, const double*, double, double*,
                                     const CgScalars*, int, cudaStream_t);
void launch_schur_sp(int ntc, const long long* tcell, const CsrView<double>& Cc, long long f0, const double* z,
                     double* s, const CgScalars* sc, cudaStream_t st) {
    if (ntc <= 0) return;
    launch_k(k_schur_sp, (ntc + 127) / 128, 128, 0, st, ntc, tcell, Cc, f0, z, s, sc);
}
template void launch_schur_col<double>(const CsrView<double>&, long long, int, const double*, double*, cudaStream_t);
template void launch_schur_col<float>(const CsrView<double>&, long long, int, const float*, double*, cudaStream_t);
template void launch_schur_tf<double>(const CsrView<double>&, long long, const double*, const double*, double*,
                                      const CgScalars*, cudaStream_t);
template void launch_schur_tf<float>(const CsrView<double>&, long long, const double*, const float*, double*,
                                     const CgScalars*, cudaStream_t);
template void launch_schur_zf<double>(int, const double*, const double*, double*, const DotArgs&, int, cudaStream_t);
template void launch_schur_zf<float>(int, const float*, const double*, double*, const DotArgs&, int, cudaStream_t);

void launch_dot2(long long n, const double* a, const double* b, const DotArgs& d, int grid, cudaStream_t st) {
    launch_k(k_dot2, grid, kThreads, 0, st, n, a, b, d);
}
void launch_pw_precond(long long n, const double* r, double* z, const double* idiag, const DotArgs& d, int grid,
                       cudaStream_t st) {
    launch_k(k_pw_precond, grid, kThreads, 0, st, n, r, z, idiag, d);
}

// one warp per slice; grid-stride beyond 65535 blocks
inline int grid_slices(long long nslices) {
    long long b = (nslices * 32 + kThreads - 1) / kThreads;
    return int(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

template <typename T>
void launch_sell(int mode, const SellView<T>& A, const T* idiag, const T* x, const T* b, T* y, T omega,
                 const CgScalars* sc, cudaStream_t st) {
    const int g = grid_slices(A.nslices);
    switch (mode) {
        case MODE_APPLY: launch_k(k_sell<T, MODE_APPLY>, g, kThreads, 0, st, A, idiag, x, b, y, omega, sc); break;
        case MODE_RESID: launch_k(k_sell<T, MODE_RESID>, g, kThreads, 0, st, A, idiag, x, b, y, omega, sc); break;
        case MODE_JAC: launch_k(k_sell<T, MODE_JAC>, g, kThreads, 0, st, A, idiag, x, b, y, omega, sc); break;
        case MODE_JAC0: launch_k(k_sell<T, MODE_JAC0>, g, kThreads, 0, st, A, idiag, x, b, y, omega, sc); break;
        case MODE_JAC2: launch_k(k_sell<T, MODE_JAC2>, g, kThreads, 0, st, A, idiag, x, b, y, omega, sc); break;
        default: break;
    }
}
template <typename T>
void launch_sell_mv(int acc, const SellView<T>& A, const T* x, T* y, const CgScalars* sc, cudaStream_t st) {
    const int g = grid_slices(A.nslices);
    if (acc) launch_k(k_sell_mv<T, 1>, g, kThreads, 0, st, A, x, y, sc);
    else launch_k(k_sell_mv<T, 0>, g, kThreads, 0, st, A, x, y, sc);
}
template <typename T, int PRE, int LPR>
void down_lpr(const SellView<T>& A, const T* idiag, const T* b, T* x, T omega, const CsrView<T>& Rt, T* bc,
              const CgScalars* sc, cudaStream_t st) {
    const int nbA = grid_slices(A.nslices);
    long long nbR = (Rt.n * LPR + kThreads - 1) / kThreads;
    nbR = nbR < 1 ? 1 : (nbR > 32768 ? 32768 : nbR);
    launch_k(k_sell_down<T, PRE, LPR>, nbA + int(nbR), kThreads, 0, st, A, idiag, b, x, omega, Rt, bc, nbA, sc);
}
template <typename T, int PRE>
void down_pre(const SellView<T>& A, const T* idiag, const T* b, T* x, T omega, const CsrView<T>& Rt, T* bc,
              const CgScalars* sc, cudaStream_t st) {
    const double avg = Rt.n > 0 ? double(Rt.nnz) / double(Rt.n) : 0.0;
    if (avg <= 24.0) down_lpr<T, PRE, 4>(A, idiag, b, x, omega, Rt, bc, sc, st);
    else if (avg <= 64.0) down_lpr<T, PRE, 8>(A, idiag, b, x, omega, Rt, bc, sc, st);
    else down_lpr<T, PRE, 16>(A, idiag, b, x, omega, Rt, bc, sc, st);
}
template <typename T>
void launch_sell_down(int pre, const SellView<T>& A, const T* idiag, const T* b, T* x, T omega,
                      const CsrView<T>& Rt, T* bc, const CgScalars* sc, cudaStream_t st) {
    if (pre == 1) down_pre<T, 1>(A, idiag, b, x, omega, Rt, bc, sc, st);
    else down_pre<T, 2>(A, idiag, b, x, omega, Rt, bc, sc, st);
}
template <typename T>
void launch_sell_up(const SellView<T>& A, const T* idiag, const T* x, const T* b, T* y, T omega,
                    const SellView<T>& Q, const T* xc, const CgScalars* sc, cudaStream_t st) {
    launch_k(k_sell_up<T>, grid_slices(A.nslices), kThreads, 0, st, A, idiag, x, b, y, omega, Q, xc, sc);
}
template <typename T>
void launch_coarse(int n, const double* Ainv, const T* b, T* x, const CgScalars* sc, cudaStream_t st) {
    const int grid = (n * 32 + kThreads - 1) / kThreads;
    launch_k(k_coarse<T>, grid < 1 ? 1 : grid, kThreads, 0, st, n, Ainv, b, x, sc);
}
void launch_sell_op(int mode, int dk, const SellView<double>& A, const double* x, const double* b, double* y,
                    const DotArgs& d, int grid, cudaStream_t st) {
    if (mode == MODE_RESID) {
        if (dk == DK_RESID) launch_k(k_sell_op<MODE_RESID, DK_RESID>, grid, kThreads, 0, st, A, x, b, y, d);
        else launch_k(k_sell_op<MODE_RESID, DK_NONE>, grid, kThreads, 0, st, A, x, b, y, d);
    } else {
        if (dk == DK_XY) launch_k(k_sell_op<MODE_APPLY, DK_XY>, grid, kThreads, 0, st, A, x, b, y, d);
        else launch_k(k_sell_op<MODE_APPLY, DK_NONE>, grid, kThreads, 0, st, A, x, b, y, d);
    }
}
template <typename T>
void launch_narrow(long long n, const double* a, T* b, const CgScalars* sc, int grid, cudaStream_t st) {
    launch_k(k_narrow<T>, grid, kThreads, 0, st, n, a, b, sc);
}
template <typename T>
void launch_widen(int dk, long long n, const T* x, double* z, const DotArgs& d, int grid, cudaStream_t st) {
    if (dk == DK_ZR) launch_k(k_widen<T, DK_ZR>, grid, kThreads, 0, st, n, x, z, d);
    else launch_k(k_widen<T, DK_NONE>, grid, kThreads, 0, st, n, x, z, d);
}
template void launch_narrow<double>(long long, const double*, double*, const CgScalars*, int, cudaStream_t);
template void launch_narrow<float>(long long, const double*, float*, const CgScalars*, int, cudaStream_t);
template void launch_widen<double>(int, long long, const double*, double*, const DotArgs&, int, cudaStream_t);
template void launch_widen<float>(int, long long, const float*, double*, const DotArgs&, int, cudaStream_t);
template void launch_sell<double>(int, const SellView<double>&, const double*, const double*, const double*,
                                  double*, double, const CgScalars*, cudaStream_t);
template void launch_sell<float>(int, const SellView<float>&, const float*, const float*, const float*, float*,
                                 float, const CgScalars*, cudaStream_t);
template void launch_sell_down<double>(int, const SellView<double>&, const double*, const double*, double*, double,
                                       const CsrView<double>&, double*, const CgScalars*, cudaStream_t);
template void launch_sell_down<float>(int, const SellView<float>&, const float*, const float*, float*, float,
                                      const CsrView<float>&, float*, const CgScalars*, cudaStream_t);
template void launch_sell_up<double>(const SellView<double>&, const double*, const double*, const double*, double*,
                                     double, const SellView<double>&, const double*, const CgScalars*, cudaStream_t);
template void launch_sell_up<float>(const SellView<float>&, const float*, const float*, const float*, float*, float,
                                    const SellView<float>&, const float*, const CgScalars*, cudaStream_t);
template void launch_sell_mv<double>(int, const SellView<double>&, const double*, double*, const CgScalars*,
                                     cudaStream_t);
template void launch_sell_mv<float>(int, const SellView<float>&, const float*, float*, const CgScalars*,
                                    cudaStream_t);
template void launch_coarse<double>(int, const double*, const double*, double*, const CgScalars*, cudaStream_t);
template void launch_coarse<float>(int, const double*, const float*, float*, const CgScalars*, cudaStream_t);

}  // namespace ibm

// Time-step kernels of the projection method: convective outflow, the
// explicit right-hand side r1 (AB2 convection + CN diffusion, Eq. 7), the
// right-hand side of Eq. 9b, the projection Eq. 9c and the force sums.
#include "device.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace ibm {

// u velocity at x-face i (0..nx), row j; boundary columns from b (time n)
__device__ __forceinline__ double Uval(const GridView& g, const double* q, const BoundaryView& b, int i, int j) {
    if (i == 0) return b.u_left[j];
    if (i == g.nx) return b.u_right[j];
    return q[(long long)j * g.nx + i] * g.idy[j];
}
// v velocity at column i, y-face j (0..ny)
__device__ __forceinline__ double Vval(const GridView& g, const double* q, const BoundaryView& b, int i, int j) {
    if (j == 0) return b.v_bottom[i];
    if (j == g.ny) return b.v_top[i];
    return q[g.nc + (long long)j * g.nx + i] * g.idx[i];
}

// Convective outflow on the right edge (section 5.2): explicit upwind update
// of the normal u and tangential v with speed uinf, then a uniform shift of
// u on the edge so that the net boundary flux vanishes.  One block.
__global__ void __launch_bounds__(1024) k_outflow(GridView g, StepParams p, const double* __restrict__ q,
                                                   BoundaryView b, double* __restrict__ ur1,
                                                   double* __restrict__ vr1) {
    pdl_entry();
    __shared__ double sh[32];
    const int nx = g.nx, ny = g.ny;
    if (p.bc != 0) {
        for (int j = threadIdx.x; j < ny; j += blockDim.x) ur1[j] = b.u_right[j];
        for (int j = threadIdx.x; j <= ny; j += blockDim.x) vr1[j] = b.v_right[j];
        return;
    }
    const double cu = p.uinf * p.dt / g.dx[nx - 1];
    const double cv = p.uinf * p.dt / (0.5 * g.dx[nx - 1]);
    double s = 0.0;
    for (int j = threadIdx.x; j < ny; j += blockDim.x) {
        const double ub = b.u_right[j];
        const double ui = q[(long long)j * nx + nx - 1] * g.idy[j];
        const double un = ub - cu * (ub - ui);
        ur1[j] = un;
        s += un * g.dy[j];
    }
    for (int j = threadIdx.x; j <= ny; j += blockDim.x) {
        if (j == 0 || j == ny) {
            vr1[j] = b.v_right[j];
        } else {
            const double vb = b.v_right[j];
            const double vi = q[g.nc + (long long)j * nx + nx - 1] * g.idx[nx - 1];
            vr1[j] = vb - cv * (vb - vi);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    double out = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) out += sh[w];
    const double shift = (p.inflow - out) / p.ly;
    for (int j = threadIdx.x; j < ny; j += blockDim.x) ur1[j] += shift;
}

// Explicit right-hand side of Eq. 9a on the padded velocity array:
// r1 = (M/dt) q + L q / 2 + (bc^n + bc^{n+1}) / 2 - (3/2 N^n - 1/2 N^{n-1}),
// with L q / 2 = (M/dt) q - A q.  Also writes N^n.
__global__ void __launch_bounds__(kThreads) k_rhs(GridView g, StepParams p, Stencil<double> A,
                                                  const double* __restrict__ mdt, const double* __restrict__ q,
                                                  BoundaryView b, const double* __restrict__ nprev,
                                                  double* __restrict__ ncur, double* __restrict__ r1) {
    pdl_entry();
    const int nx = g.nx, ny = g.ny;
    const double nu = p.nu;
    for (int row = blockIdx.y; row < 2 * ny; row += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
        const int blk = row >= ny ? 1 : 0;
        const int j = row - blk * ny;
        const long long k = (long long)row * nx + i;
        if ((blk == 0 && i == 0) || (blk == 1 && j == 0)) {
            r1[k] = 0.0;
            ncur[k] = 0.0;
            continue;
        }
        double N, bc;
        if (blk == 0) {
            const double uc = Uval(g, q, b, i, j);
            const double ue = Uval(g, q, b, i + 1, j), uw = Uval(g, q, b, i - 1, j);
            const double uE = 0.5 * (uc + ue), uW = 0.5 * (uw + uc);
            const double uN = (j < ny - 1) ? uc + (Uval(g, q, b, i, j + 1) - uc) * (0.5 * g.dy[j] * g.idyf[j + 1])
                                           : b.u_top[i];
            double uS;
            if (j > 0) {
                const double us = Uval(g, q, b, i, j - 1);
                uS = us + (uc - us) * (0.5 * g.dy[j - 1] * g.idyf[j]);
            } else {
                uS = b.u_bottom[i];
            }
            const double wx = 0.5 * g.dx[i - 1] * g.idxf[i];
            const double vnw = Vval(g, q, b, i - 1, j + 1), vne = Vval(g, q, b, i, j + 1);
            const double vsw = Vval(g, q, b, i - 1, j), vse = Vval(g, q, b, i, j);
            const double vN = vnw + (vne - vnw) * wx, vS = vsw + (vse - vsw) * wx;
            N = (uE * uE - uW * uW) + (uN * vN - uS * vS) * (g.dxf[i] * g.idy[j]);
            // boundary part of the viscous term, averaged over t^n and t^{n+1}
            bc = 0.0;
            if (i + 1 == nx) bc += nu * 0.5 * (b.u_right[j] + b.u_right1[j]) * g.idx[i];
            if (i - 1 == 0) bc += nu * b.u_left[j] * g.idx[0];
            if (j == ny - 1) bc += 2.0 * nu * g.dxf[i] * b.u_top[i] * g.idy[j] * g.idy[j];
            if (j == 0) bc += 2.0 * nu * g.dxf[i] * b.u_bottom[i] * g.idy[j] * g.idy[j];
        } else {
            const double vc = Vval(g, q, b, i, j);
            const double vN = 0.5 * (vc + Vval(g, q, b, i, j + 1)), vS = 0.5 * (Vval(g, q, b, i, j - 1) + vc);
            const double wy = 0.5 * g.dy[j - 1] * g.idyf[j];
            const double ues = Uval(g, q, b, i + 1, j - 1), uen = Uval(g, q, b, i + 1, j);
            const double uws = Uval(g, q, b, i, j - 1), uwn = Uval(g, q, b, i, j);
            const double uE = ues + (uen - ues) * wy, uW = uws + (uwn - uws) * wy;
            double vE, vW;
            if (i < nx - 1) vE = vc + (Vval(g, q, b, i + 1, j) - vc) * (0.5 * g.dx[i] * g.idxf[i + 1]);
            else vE = b.v_right[j];
            if (i > 0) {
                const double vw = Vval(g, q, b, i - 1, j);
                vW = vw + (vc - vw) * (0.5 * g.dx[i - 1] * g.idxf[i]);
            } else {
                vW = b.v_left[j];
            }
            N = (uE * vE - uW * vW) * (g.dyf[j] * g.idx[i]) + (vN * vN - vS * vS);
            bc = 0.0;
            if (j + 1 == ny) bc += nu * b.v_top[i] * g.idy[j];
            if (j - 1 == 0) bc += nu * b.v_bottom[i] * g.idy[0];
            if (i == nx - 1) bc += 2.0 * nu * g.dyf[j] * 0.5 * (b.v_right[j] + b.v_right1[j]) * g.idx[i] * g.idx[i];
            if (i == 0) bc += 2.0 * nu * g.dyf[j] * b.v_left[j] * g.idx[i] * g.idx[i];
        }
        // A q (homogeneous 5-point part)
        const double qc = q[k];
        double aq = A.diag[k] * qc;
        if (i + 1 < nx) aq -= A.cE[k] * q[k + 1];
        if (i > 0) aq -= A.cE[k - 1] * q[k - 1];
        if (j + 1 < ny) aq -= A.cN[k] * q[k + nx];
        if (j > 0) aq -= A.cN[k - nx] * q[k - nx];
        const double np = p.first ? N : nprev[k];
        r1[k] = 2.0 * mdt[k] * qc - aq + bc - (1.5 * N - 0.5 * np);
        ncur[k] = N;
    }
}

// b2 = [-(net outflow of q* per cell, boundary faces at t^{n+1}) ; E q* - u_B],
// b2[pin] = 0  (Eq. 9b with G^T = -divergence).
__global__ void __launch_bounds__(kThreads) k_poisson_rhs(GridView g, StepParams p, const double* __restrict__ qs,
                                                          BoundaryView b, CsrView<double> E,
                                                          const double* __restrict__ ub, double* __restrict__ b2) {
    pdl_entry();
    const int nx = g.nx, ny = g.ny;
    const long long nc = g.nc, n = nc + E.n;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        if (k < nc) {
            const int i = int(k % nx), j = int(k / nx);
            const double qw = (i == 0) ? b.u_left[j] * g.dy[j] : qs[k];
            const double qe = (i == nx - 1) ? b.u_right1[j] * g.dy[j] : qs[k + 1];
            const double qsouth = (j == 0) ? b.v_bottom[i] * g.dx[i] : qs[nc + k];
            const double qn = (j == ny - 1) ? b.v_top[i] * g.dx[i] : qs[nc + k + nx];
            b2[k] = (k == p.pin) ? 0.0 : -((qe - qw) + (qn - qsouth));
        } else {
            const long long r = k - nc;
            double s = 0.0;
            for (long long t = E.ptr[r]; t < E.ptr[r + 1]; ++t) s += E.val[t] * qs[E.col[t]];
            b2[k] = s - ub[r];
        }
    }
}

// q = q* - B^1 G phi on all interior faces (Eq. 9c, pressure part); B^1 = dt M^-1.
// qs null: q* = 0.  pin >= 0: phi[pin] is taken as 0 (the pinned column of
// Q^T B Q keeps only its diagonal).
__global__ void __launch_bounds__(kThreads) k_project(GridView g, double dt, const double* __restrict__ qs,
                                                      const double* __restrict__ lam, double* __restrict__ q,
                                                      long long pin) {
    pdl_entry();
    const int nx = g.nx, ny = g.ny;
    const long long nc = g.nc;
    auto phi = [&](long long k) { return k == pin ? 0.0 : lam[k]; };
    for (int row = blockIdx.y; row < 2 * ny; row += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
        const int blk = row >= ny ? 1 : 0;
        const int j = row - blk * ny;
        const long long k = (long long)row * nx + i;
        const long long kk = k - blk * nc;
        const double s = qs ? qs[k] : 0.0;
        double out = 0.0;
        if (blk == 0 && i > 0) out = s - dt * g.dy[j] * g.idxf[i] * (phi(kk) - phi(kk - 1));
        else if (blk == 1 && j > 0) out = s - dt * g.dx[i] * g.idyf[j] * (phi(kk) - phi(kk - nx));
        q[k] = out;
    }
}

// The Poisson operator Q^T B^N Q of Eq. 9b applied without assembling it,
// last stage: q = -B^N Q x (the projection of x with q* = 0, its N - 1
// further terms included) gives Q^T B^N Q x = -Q^T q = [div q; -E q]
// (G^T = -div, homogeneous boundary faces); the pinned row keeps its
// diagonal: y[pin] = dpin x[pin].  MODE_RESID: y = b - (Q^T B^N Q) x.  Dots as
// in the assembled operator: DK_XY x.y, DK_RESID [b.b, y.y].
template <int MODE, int DK>
__global__ void __launch_bounds__(kThreads) k_qt_apply(GridView g, long long pin, double dpin,
                                                       const double* __restrict__ q, CsrView<double> E,
                                                       const double* __restrict__ x, const double* __restrict__ b,
                                                       double* __restrict__ y, DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    const int nx = g.nx, ny = g.ny;
    const long long nc = g.nc, n = nc + E.n;
    double acc[2] = {0.0, 0.0};
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        double a;
        if (k == pin) {
            a = dpin * x[k];
        } else if (k < nc) {
            const int i = int(k % nx), j = int(k / nx);
            const double qw = i == 0 ? 0.0 : q[k];
            const double qe = i == nx - 1 ? 0.0 : q[k + 1];
            const double qsouth = j == 0 ? 0.0 : q[nc + k];
            const double qn = j == ny - 1 ? 0.0 : q[nc + k + nx];
            a = (qe - qw) + (qn - qsouth);
        } else {
            const long long r = k - nc;
            double s = 0.0;
            for (long long t = E.ptr[r]; t < E.ptr[r + 1]; ++t) s += E.val[t] * q[E.col[t]];
            a = -s;
        }
        const double out = MODE == MODE_RESID ? b[k] - a : a;
        y[k] = out;
        if (DK == DK_XY) {
            acc[0] += x[k] * out;
        } else if (DK == DK_RESID) {
            acc[0] += b[k] * b[k];
            acc[1] += out * out;
        }
    }
    if (DK != DK_NONE) reduce_and_finalize<2>(acc, d, d.slot0 + blockIdx.x);
}

// q -= B^1 E^T f~ on the faces touched by the bodies (face-major E^T, no atomics).
__global__ void __launch_bounds__(kThreads) k_project_body(GridView g, double dt, int nfaces,
                                                           const int* __restrict__ faces, CsrView<double> ET,
                                                           const double* __restrict__ f, double* __restrict__ q) {
    pdl_entry();
    const int nx = g.nx;
    const long long nc = g.nc;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nfaces; t += gridDim.x * blockDim.x) {
        const long long fidx = faces[t];
        double s = 0.0;
        for (long long p = ET.ptr[t]; p < ET.ptr[t + 1]; ++p) s += ET.val[p] * f[ET.col[p]];
        double B;
        if (fidx < nc) {
            const int i = int(fidx % nx), j = int(fidx / nx);
            B = dt * g.dy[j] * g.idxf[i];
        } else {
            const long long kk = fidx - nc;
            const int i = int(kk % nx), j = int(kk / nx);
            B = dt * g.dx[i] * g.idyf[j];
        }
        q[fidx] -= B * s;
    }
}

// out[0] = sum f~x, out[1] = sum f~y (one block, fixed summation order)
__global__ void __launch_bounds__(1024) k_forces(int n_b, const double* __restrict__ f, double* __restrict__ out) {
    pdl_entry();
    __shared__ double sh[2][32];
    double sx = 0.0, sy = 0.0;
    for (int k = threadIdx.x; k < n_b; k += blockDim.x) {
        sx += f[k];
        sy += f[n_b + k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = sx; sh[1][threadIdx.x >> 5] = sy; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) { a += sh[0][w]; c += sh[1][w]; }
        out[0] = a;
        out[1] = c;
        out[2] = 0.0;   // maxima of k_constraints, which runs next
        out[3] = 0.0;
    }
}

// FP64 check of the constraints of Eq. 8 on q^{n+1} after the projection:
// out[2] = max |G^T q + bc2| over the cells other than the pinned one (boundary
// fluxes at t^{n+1}), out[3] = max |E q - u_B| over the body rows.  The maxima
// of non-negative doubles are combined as their bit patterns (integer order
// equals value order; a NaN compares above every number and is kept).
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(addr), static_cast<unsigned long long>(__double_as_longlong(v)));
}
// max that keeps a NaN (fmax would drop it)
__device__ __forceinline__ double nan_max(double a, double b) { return a != a ? a : (b != b ? b : fmax(a, b)); }

__global__ void __launch_bounds__(kThreads) k_constraints(GridView g, StepParams p, const double* __restrict__ q,
                                                          BoundaryView b, CsrView<double> E,
                                                          const double* __restrict__ ub, double* __restrict__ out) {
    pdl_entry();
    __shared__ double sh[2][kThreads / 32];
    const int nx = g.nx, ny = g.ny;
    const long long nc = g.nc;
    double mdiv = 0.0, mslip = 0.0;
    // cells: blockIdx.y strides over rows, threads over the row (2D launch shape)
    for (int j = blockIdx.y; j < ny; j += gridDim.y) {
        const long long row = (long long)j * nx;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
            const long long k = row + i;
            if (k == p.pin) continue;
            const double qw = (i == 0) ? b.u_left[j] * g.dy[j] : q[k];
            const double qe = (i == nx - 1) ? b.u_right1[j] * g.dy[j] : q[k + 1];
            const double qsouth = (j == 0) ? b.v_bottom[i] * g.dx[i] : q[nc + k];
            const double qn = (j == ny - 1) ? b.v_top[i] * g.dx[i] : q[nc + k + nx];
            mdiv = nan_max(mdiv, fabs((qe - qw) + (qn - qsouth)));
        }
    }
    // body rows: one thread each, over the whole grid
    const long long tid = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * gridDim.y * blockDim.x;
    for (long long r = tid; r < E.n; r += nthr) {
        double s = -ub[r];
        for (long long t = E.ptr[r]; t < E.ptr[r + 1]; ++t) s += E.val[t] * q[E.col[t]];
        mslip = nan_max(mslip, fabs(s));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mdiv = nan_max(mdiv, __shfl_xor_sync(0xffffffffu, mdiv, o));
        mslip = nan_max(mslip, __shfl_xor_sync(0xffffffffu, mslip, o));
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = mdiv;
        sh[1][threadIdx.x >> 5] = mslip;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) {
            a = nan_max(a, sh[0][w]);
            c = nan_max(c, sh[1][w]);
        }
        atomic_max_nonneg(out + 2, fabs(a));
        atomic_max_nonneg(out + 3, fabs(c));
    }
}

// lambda0 = 2 lambda^n - lambda^{n-1}; lambda^{n-1} <- lambda^n (one pass)
__global__ void __launch_bounds__(kThreads) k_extrapolate(long long n, double* __restrict__ lam,
                                                          double* __restrict__ prev, int first) {
    pdl_entry();
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const double t = lam[k];
        if (!first) lam[k] = 2.0 * t - prev[k];
        prev[k] = t;
    }
}
void launch_extrapolate(long long n, double* lam, double* prev, int first, int grid, cudaStream_t st) {
    launch_k(k_extrapolate, grid, kThreads, 0, st, n, lam, prev, first);
}

// ---- warm start by projection onto the previous solutions -----------------------
// The basis X_0 .. X_{m-1} (columns of stride ld) is K-orthonormal for the
// Poisson operator K; KX holds K X_i.  Dot products are summed per block, then
// in one block in a fixed order (deterministic).

// part[i * gridDim.x + block] = X_i . (a - b) over the block's entries (b nullable)
__global__ void __launch_bounds__(kThreads) k_proj_dots(long long n, int m, const double* __restrict__ X, long long ld,
                                                        const double* __restrict__ a, const double* __restrict__ b,
                                                        double* __restrict__ part) {
    pdl_entry();
    __shared__ double sh[kProjMax][kThreads / 32];
    double acc[kProjMax];
#pragma unroll
    for (int i = 0; i < kProjMax; ++i) acc[i] = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double v = b ? a[k] - b[k] : a[k];
#pragma unroll
        for (int i = 0; i < kProjMax; ++i)
            if (i < m) acc[i] += X[i * ld + k] * v;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < kProjMax; ++i) {
        if (i >= m) break;
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[i][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double t = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
        part[threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// coef[i] = sum of the nb partials of dot i in a fixed order; one warp per
// coefficient (block of 32 m threads)
__global__ void k_proj_sum(int m, int nb, const double* __restrict__ part, double* __restrict__ coef) {
    pdl_entry();
    const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (i >= m) return;
    double t = 0.0;
    for (int b = lane; b < nb; b += 32) t += part[i * nb + b];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) coef[i] = t;
}

// v = base - sign sum_i coef_i X_i (base null: 0); with w non-null also
// w = (y - r) - sign sum_i coef_i KX_i (r nullable); in place allowed
__global__ void __launch_bounds__(kThreads) k_proj_combine(long long n, int m, const double* __restrict__ X,
                                                           const double* __restrict__ KX, long long ld,
                                                           const double* __restrict__ coef,
                                                           const double* __restrict__ base, double* __restrict__ v,
                                                           const double* __restrict__ y, const double* __restrict__ r,
                                                           double* __restrict__ w, double sign) {
    pdl_entry();
    double c[kProjMax];
#pragma unroll
    for (int i = 0; i < kProjMax; ++i) c[i] = i < m ? sign * coef[i] : 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        double a = base ? base[k] : 0.0;
#pragma unroll
        for (int i = 0; i < kProjMax; ++i)
            if (i < m) a -= c[i] * X[i * ld + k];
        v[k] = a;
        if (w) {
            double b = r ? y[k] - r[k] : y[k];
#pragma unroll
            for (int i = 0; i < kProjMax; ++i)
                if (i < m) b -= c[i] * KX[i * ld + k];
            w[k] = b;
        }
    }
}

// X_new = v / sqrt(g), KX_new = w / sqrt(g) with g = coef[0] = v.w; a vector
// that adds nothing (g <= tiny * ref, ref = coef[1]) is stored as zero
__global__ void __launch_bounds__(kThreads) k_proj_store(long long n, const double* __restrict__ v,
                                                         const double* __restrict__ w, const double* __restrict__ coef,
                                                         double* __restrict__ X, double* __restrict__ KX) {
    pdl_entry();
    const double g = coef[0], ref = coef[1];
    const double s = (g > 1e-24 * fabs(ref) && g > 0.0) ? 1.0 / sqrt(g) : 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        X[k] = s * v[k];
        KX[k] = s * w[k];
    }
}

void launch_proj_dots(long long n, int m, const double* X, long long ld, const double* a, const double* b,
                      double* part, double* coef, cudaStream_t st) {
    launch_k(k_proj_dots, kProjBlocks, kThreads, 0, st, n, m, X, ld, a, b, part);
    launch_k(k_proj_sum, 1, 32 * m, 0, st, m, kProjBlocks, (const double*)part, coef);
}
void launch_proj_combine(long long n, int m, const double* X, const double* KX, long long ld, const double* coef,
                         const double* base, double* v, const double* y, const double* r, double* w, double sign,
                         int grid, cudaStream_t st) {
    launch_k(k_proj_combine, grid, kThreads, 0, st, n, m, X, KX, ld, coef, base, v, y, r, w, sign);
}
void launch_proj_store(long long n, const double* v, const double* w, const double* coef, double* X, double* KX,
                       int grid, cudaStream_t st) {
    launch_k(k_proj_store, grid, kThreads, 0, st, n, v, w, coef, X, KX);
}

// Further terms of B^N Q lam (N > 1) in the projection, t_k = (dt/2) M^-1 L t_{k-1}
// written as t_{k-1} - (A t_{k-1}) / (M/dt) with A = M/dt - L/2 (Eq. 9c).
__global__ void __launch_bounds__(kThreads) k_bn_start(long long n, const double* __restrict__ mdt,
                                                       const double* __restrict__ q, const double* __restrict__ qs,
                                                       double* __restrict__ t) {
    pdl_entry();
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        t[k] = mdt[k] > 0.0 ? q[k] - (qs ? qs[k] : 0.0) : 0.0;
}
__global__ void __launch_bounds__(kThreads) k_bn_term(long long n, const double* __restrict__ mdt,
                                                      const double* __restrict__ At, double* __restrict__ t,
                                                      double* __restrict__ q) {
    pdl_entry();
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double m = mdt[k];
        const double v = m > 0.0 ? t[k] - At[k] / m : 0.0;
        t[k] = v;
        q[k] += v;
    }
}
void launch_bn_start(long long n, const double* mdt, const double* q, const double* qs, double* t, int grid,
                     cudaStream_t st) {
    launch_k(k_bn_start, grid, kThreads, 0, st, n, mdt, q, qs, t);
}
void launch_bn_term(long long n, const double* mdt, const double* At, double* t, double* q, int grid,
                    cudaStream_t st) {
    launch_k(k_bn_term, grid, kThreads, 0, st, n, mdt, At, t, q);
}

void launch_outflow(const GridView& g, const StepParams& p, const double* q, BoundaryView b, double* ur1,
                    double* vr1, cudaStream_t st) {
    launch_k(k_outflow, 1, 1024, 0, st, g, p, q, b, ur1, vr1);
}
void launch_rhs(const GridView& g, const StepParams& p, const Stencil<double>& A, const double* mdt,
                const double* q, BoundaryView b, const double* nprev, double* ncur, double* r1, dim3 grid,
                cudaStream_t st) {
    launch_k(k_rhs, grid, kThreads, 0, st, g, p, A, mdt, q, b, nprev, ncur, r1);
}
void launch_poisson_rhs(const GridView& g, const StepParams& p, const double* qs, BoundaryView b,
                        const CsrView<double>& E, const double* ub, double* b2, int grid, cudaStream_t st) {
    launch_k(k_poisson_rhs, grid, kThreads, 0, st, g, p, qs, b, E, ub, b2);
}
void launch_project(const GridView& g, double dt, const double* qs, const double* lam, double* q, dim3 grid,
                    cudaStream_t st, long long pin) {
    launch_k(k_project, grid, kThreads, 0, st, g, dt, qs, lam, q, pin);
}
void launch_qt_apply(int mode, int dk, const GridView& g, long long pin, double dpin, const double* q,
                     const CsrView<double>& E, const double* x, const double* b, double* y, const DotArgs& d, int grid,
                     cudaStream_t st) {
#define IBM_QT(M, K) launch_k(k_qt_apply<M, K>, grid, kThreads, 0, st, g, pin, dpin, q, E, x, b, y, d)
    if (mode == MODE_RESID) {
        if (dk == DK_RESID) IBM_QT(MODE_RESID, DK_RESID);
        else IBM_QT(MODE_RESID, DK_NONE);
    } else {
        if (dk == DK_XY) IBM_QT(MODE_APPLY, DK_XY);
        else IBM_QT(MODE_APPLY, DK_NONE);
    }
#undef IBM_QT
}
void launch_project_body(const GridView& g, double dt, int nfaces, const int* faces, const CsrView<double>& ET,
                         const double* f, double* q, cudaStream_t st) {
    if (nfaces <= 0) return;
    launch_k(k_project_body, (nfaces + kThreads - 1) / kThreads, kThreads, 0, st, g, dt, nfaces, faces, ET, f, q);
}
void launch_forces(int n_b, const double* f, double* out, cudaStream_t st) {
    launch_k(k_forces, 1, 1024, 0, st, n_b, f, out);
}
void launch_constraints(const GridView& g, const StepParams& p, const double* q, BoundaryView b,
                        const CsrView<double>& E, const double* ub, double* out, dim3 grid, cudaStream_t st) {
    launch_k(k_constraints, grid, kThreads, 0, st, g, p, q, b, E, ub, out);
}

}  // namespace ibm

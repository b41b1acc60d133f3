// Inner FP32 solve of the mixed-precision velocity solve (Eq. 9a, A q* = r1).
//
// The outer loop (api.cu) forms the residual r = r1 - A q in FP64, solves
// A e = r approximately with the Jacobi-preconditioned CG below in FP32, adds
// e to q in FP64 and forms the FP64 residual again, until that residual meets
// the solve's tolerance.  The inner solve stores its vectors and the
// operator's coefficients in FP32 and forms products and per-thread partial
// sums in FP32; the block and grid sums of its dot products and its step
// lengths stay in FP64 (the reductions of the FP64 loops).  On GB300 an FP64
// operation per unknown costs about as much as moving 16 bytes per unknown,
// so the FP64 CG loop is bound by its arithmetic; the inner loop is bound by
// memory and launch latency instead.
#include "device.cuh"
#include "kernels.h"
#include "reduce.cuh"

namespace ibm {
namespace {

// r = float(r64), e = 0, z = D^-1 r; [r.r, r.z] start the inner solve's
// scalars over (FIN_INIT_PW) with tolerance tol2_in and max_iter iterations
__global__ void __launch_bounds__(kThreads) k_v32_init(long long n, const double* __restrict__ r64,
                                                       float* __restrict__ r, float* __restrict__ e,
                                                       float* __restrict__ z, const float* __restrict__ idiag,
                                                       double tol2_in, int max_iter, DotArgs d) {
    pdl_entry();
    float a0 = 0.f, a1 = 0.f;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const float rv = float(r64[k]);
        const float zv = idiag[k] * rv;
        r[k] = rv;
        e[k] = 0.f;
        z[k] = zv;
        a0 += rv * rv;
        a1 += rv * zv;
    }
    double acc[2] = {double(a0), double(a1)};
    if (block_reduce_last<2>(acc, d.partials, blockIdx.x, d.expected, &d.sc->counter[d.counter_id]) &&
        threadIdx.x == 0) {
        d.sc->tol2 = tol2_in;
        d.sc->max_iter = max_iter;
        d.sc->guard = 0;
        finalize(FIN_INIT_PW, acc, d.sc);
    }
}

// p = z + beta p (p = z for the first direction)
__global__ void __launch_bounds__(kThreads) k_v32_pupdate(long long n, const float* __restrict__ z,
                                                          float* __restrict__ p, DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    const double beta = d.sc->beta;
    const float bf = float(beta);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        p[k] = beta == 0.0 ? z[k] : z[k] + bf * p[k];
}

// q = A p on nblk stacked nx x ny blocks (5-point couplings inside a block)
// with [p.q] (FIN_ALPHA)
__global__ void __launch_bounds__(kThreads) k_v32_apply(Stencil<float> s, const float* __restrict__ p,
                                                        float* __restrict__ q, DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    const int nx = s.nx, ny = s.ny, nrows = ny * s.nblk;
    float a = 0.f;
    for (int row = blockIdx.y; row < nrows; row += gridDim.y) {
        const int j = row % ny;
        const int base = row * nx;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += gridDim.x * blockDim.x) {
            const int k = base + i;
            const float pc = __ldg(p + k);
            float ax = __ldg(s.diag + k) * pc;
            if (i + 1 < nx) ax -= __ldg(s.cE + k) * __ldg(p + k + 1);
            if (i > 0) ax -= __ldg(s.cE + k - 1) * __ldg(p + k - 1);
            if (j + 1 < ny) ax -= __ldg(s.cN + k) * __ldg(p + k + nx);
            if (j > 0) ax -= __ldg(s.cN + k - nx) * __ldg(p + k - nx);
            q[k] = ax;
            a += pc * ax;
        }
    }
    double acc[2] = {double(a), 0.0};
    reduce_and_finalize<2>(acc, d, d.slot0 + blockIdx.y * gridDim.x + blockIdx.x);
}

// e += alpha p, r -= alpha q, z = D^-1 r; [r.r, r.z] (FIN_UPDATE_PW)
__global__ void __launch_bounds__(kThreads) k_v32_update(long long n, float* __restrict__ e, float* __restrict__ r,
                                                         const float* __restrict__ p, const float* __restrict__ q,
                                                         float* __restrict__ z, const float* __restrict__ idiag,
                                                         DotArgs d) {
    pdl_entry();
    if (skip(d)) return;
    const float alpha = float(d.sc->alpha);
    float a0 = 0.f, a1 = 0.f;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        e[k] += alpha * p[k];
        const float rn = r[k] - alpha * q[k];
        const float zn = idiag[k] * rn;
        r[k] = rn;
        z[k] = zn;
        a0 += rn * rn;
        a1 += rn * zn;
    }
    double acc[2] = {double(a0), double(a1)};
    reduce_and_finalize<2>(acc, d, blockIdx.x);
}

// x += double(e)
__global__ void __launch_bounds__(kThreads) k_v32_correct(long long n, double* __restrict__ x,
                                                          const float* __restrict__ e) {
    pdl_entry();
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        x[k] += double(e[k]);
}

}  // namespace

void launch_v32_init(long long n, const double* r64, float* r, float* e, float* z, const float* idiag, double tol2_in,
                     int max_iter, const DotArgs& d, int grid, cudaStream_t st) {
    launch_k(k_v32_init, grid, kThreads, 0, st, n, r64, r, e, z, idiag, tol2_in, max_iter, d);
}
void launch_v32_pupdate(long long n, const float* z, float* p, const DotArgs& d, int grid, cudaStream_t st) {
    launch_k(k_v32_pupdate, grid, kThreads, 0, st, n, z, p, d);
}
void launch_v32_apply(const Stencil<float>& s, const float* p, float* q, const DotArgs& d, dim3 grid, cudaStream_t st) {
    launch_k(k_v32_apply, grid, kThreads, 0, st, s, p, q, d);
}
void launch_v32_update(long long n, float* e, float* r, const float* p, const float* q, float* z, const float* idiag,
                       const DotArgs& d, int grid, cudaStream_t st) {
    launch_k(k_v32_update, grid, kThreads, 0, st, n, e, r, p, q, z, idiag, d);
}
void launch_v32_correct(long long n, double* x, const float* e, int grid, cudaStream_t st) {
    launch_k(k_v32_correct, grid, kThreads, 0, st, n, x, e);
}

}  // namespace ibm

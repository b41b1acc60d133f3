// Body rows of a moving body on the device (Eq. 5, Eq. 6, and the coupling
// blocks of the pinned Q^T B^1 Q of Eq. 9b): given the sparsity pattern the
// host derived from the point positions (integer work only) and the index
// maps that say which entries of E build each coupling entry, every weight
// and coupling value is formed here in FP64:
//   E          u row of point k at face (i, j): dxf_i d(xf_i - xi_k) d(yc_j - eta_k),
//              v row: dyf_j d(xc_i - xi_k) d(yf_j - eta_k)   (Eq. 6 on fluxes),
//   E^T        the same values, face-major,
//   C^T part   of a force row: +/- B_f E_(r,f) for the one or two faces of row r
//              beside the cell (B = dt M^-1 of the face),
//   F part     F_(r,r') = sum over the faces both rows touch of E_(r,f) B_f E_(r',f),
//   diagonal   of every force row (and its inverse), FP32 copies for the
//              mixed-precision V-cycle path.
// d is the three-point discrete delta of Roma, Peskin & Berger (Eq. 5).
#include <algorithm>

#include "kernels.h"

namespace ibm {
namespace {

__device__ __forceinline__ double roma(double r, double h) {
    const double a = fabs(r) / h;
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / (3.0 * h);
    if (a <= 1.5) {
        const double s = 1.0 - 3.0 * (1.0 - a) * (1.0 - a);
        return (5.0 - 3.0 * a - sqrt(s > 0.0 ? s : 0.0)) / (6.0 * h);
    }
    return 0.0;
}

// B = dt M^-1 of face f of the padded velocity layout
__device__ __forceinline__ double face_B(const BodyGeo& g, long long f) {
    if (f < g.nc) {
        const int i = int(f % g.nx), j = int(f / g.nx);
        return g.dt * g.dy[j] * g.idxf[i];
    }
    const long long s = f - g.nc;
    const int i = int(s % g.nx), j = int(s / g.nx);
    return g.dt * g.dx[i] * g.idyf[j];
}

// E values, one thread per row
__global__ void __launch_bounds__(256) k_body_E(BodyGeo g, CsrView<double> E, double* __restrict__ val,
                                               const int* __restrict__ point, const double* __restrict__ xb,
                                               const double* __restrict__ yb) {
    pdl_entry();
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < E.n; r += (long long)gridDim.x * blockDim.x) {
        const int k = point[r];
        const double xi = xb[k], eta = yb[k];
        for (long long e = E.ptr[r]; e < E.ptr[r + 1]; ++e) {
            const long long f = E.col[e];
            double v;
            if (f < g.nc) {
                const int i = int(f % g.nx), j = int(f / g.nx);
                v = g.dxf[i] * roma(g.xf[i] - xi, g.h) * roma(g.yc[j] - eta, g.h);
            } else {
                const long long s = f - g.nc;
                const int i = int(s % g.nx), j = int(s / g.nx);
                v = g.dyf[j] * roma(g.xc[i] - xi, g.h) * roma(g.yf[j] - eta, g.h);
            }
            val[e] = v;
        }
    }
}

// E^T values, the force rows [C^T | F] (a warp per row) and the force-row
// diagonal (and its inverse) of the Poisson operator
__global__ void __launch_bounds__(256) k_body_rows(BodyGeo g, CsrView<double> E, CsrView<double> ET, double* __restrict__ etv,
                                                  CsrView<double> Cf, double* __restrict__ cfv,
                                                  const int* __restrict__ et_src, const int* __restrict__ cf_a,
                                                  const int* __restrict__ cf_b, const int* __restrict__ diag_idx,
                                                  double* __restrict__ pdiag, double* __restrict__ pidiag,
                                                  float* __restrict__ pdiag32, float* __restrict__ pidiag32) {
    pdl_entry();
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    for (long long p = tid; p < ET.nnz; p += nthr) etv[p] = E.val[et_src[p]];
    const int lane = threadIdx.x & 31;
    for (long long r = tid >> 5; r < Cf.n; r += nthr >> 5) {
        for (long long p = Cf.ptr[r] + lane; p < Cf.ptr[r + 1]; p += 32) {
            double v = 0.0;
            if (cf_a[p] >= 0) {   // C^T: the row's faces beside this cell
                for (int s = 0; s < 2; ++s) {
                    const int code = s == 0 ? cf_a[p] : cf_b[p];
                    if (code < 0) continue;
                    const long long e = code >> 1;
                    const double t = face_B(g, E.col[e]) * E.val[e];
                    v += (code & 1) ? -t : t;
                }
            } else {              // F: faces shared with row r2
                const long long r2 = Cf.col[p] - g.nc;
                for (long long e = E.ptr[r]; e < E.ptr[r + 1]; ++e) {
                    const long long f = E.col[e];
                    for (long long e2 = E.ptr[r2]; e2 < E.ptr[r2 + 1]; ++e2)
                        if (E.col[e2] == f) {
                            v += E.val[e] * face_B(g, f) * E.val[e2];
                            break;
                        }
                }
            }
            cfv[p] = v;
            if (p == diag_idx[r]) {
                pdiag[g.nc + r] = v;
                pidiag[g.nc + r] = 1.0 / v;
                if (pdiag32) {
                    pdiag32[g.nc + r] = float(v);
                    pidiag32[g.nc + r] = float(1.0 / v);
                }
            }
        }
    }
}

// touched-cell rows C from the force rows; FP32 copies of both (mixed path)
__global__ void __launch_bounds__(256) k_body_cc(CsrView<double> Cc, double* __restrict__ ccv, const int* __restrict__ cc_src,
                                                const double* __restrict__ cfv, long long cf_nnz, float* __restrict__ cc32,
                                                float* __restrict__ cf32) {
    pdl_entry();
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nthr = (long long)gridDim.x * blockDim.x;
    for (long long q = tid; q < Cc.nnz; q += nthr) {
        const double v = cfv[cc_src[q]];
        ccv[q] = v;
        if (cc32) cc32[q] = float(v);
    }
    if (cf32)
        for (long long p = tid; p < cf_nnz; p += nthr) cf32[p] = float(cfv[p]);
}

inline int grid_n(long long n) { return int(std::max<long long>(1, std::min<long long>((n + 255) / 256, 1024))); }

}  // namespace

void launch_body_values(const BodyGeo& g, const BodyDev& b, cudaStream_t st) {
    launch_k(k_body_E, grid_n(b.E.n), 256, 0, st, g, b.E, b.Ev, b.point, b.xb, b.yb);
    CsrView<double> E = b.E;
    E.val = b.Ev;
    launch_k(k_body_rows, grid_n(std::max<long long>(b.ET.nnz, 32LL * b.Cf.n)), 256, 0, st, g, E, b.ET, b.ETv, b.Cf,
             b.Cfv, b.et_src, b.cf_a, b.cf_b, b.diag, b.pdiag, b.pidiag, b.pdiag32, b.pidiag32);
    launch_k(k_body_cc, grid_n(std::max(b.Cc.nnz, b.Cf.nnz)), 256, 0, st, b.Cc, b.Ccv, b.cc_src,
             (const double*)b.Cfv, b.Cf.nnz, b.Cc32, b.Cf32);
}

}  // namespace ibm

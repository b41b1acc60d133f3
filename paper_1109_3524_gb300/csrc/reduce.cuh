// Fused reductions of the CG / flexible-CG drivers: the finalising block of a
// reduction updates the solve's scalars (alpha, beta, convergence) on the
// device.  Shared by the kernel files that take part in a reduction.
#pragma once
#include "device.cuh"
#include "kernels.h"

namespace ibm {

// ---------------------------------------------------------------------------
// Scalar finalisation (runs in the last block of a reduction)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize(int fin, const double* v, CgScalars* sc) {
    switch (fin) {
        case FIN_INIT: {            // v = [b.b, r.r]
            sc->bb = v[0];
            sc->rr = v[1];
            sc->rr0 = v[1];
            sc->iter = 0;
            sc->status = 0;
            sc->beta = 0.0;
            sc->rz = 0.0;
            sc->done = (v[0] == 0.0) || (v[1] <= sc->tol2 * v[0]) || (sc->max_iter <= 0);
            if (!isfinite(v[0]) || !isfinite(v[1])) { sc->done = 1; sc->status = 5; }
            break;
        }
        case FIN_PRECOND: {         // v = [r.z, z.q_prev]
            if (sc->iter == 0 || sc->restart) sc->beta = 0.0;
            else if (sc->flexible) sc->beta = -v[1] / sc->pq_old;
            else sc->beta = v[0] / sc->rz;
            sc->rz_old = sc->rz;
            sc->rz = v[0];
            sc->zq = v[1];
            sc->restart = 0;
            if (!isfinite(v[0])) { sc->done = 1; sc->status = 5; }
            break;
        }
        case FIN_ALPHA: {           // v = [p.q]
            sc->pq = v[0];
            if (!(v[0] > 0.0) || !isfinite(v[0])) { sc->done = 1; sc->status = 5; break; }
            sc->alpha = sc->rz / v[0];
            sc->pq_old = v[0];
            break;
        }
        case FIN_UPDATE: {          // v = [r.r, r.z]  (r.z used with pointwise preconditioners)
            sc->iter += 1;
            sc->rr = v[0];
            if (!isfinite(v[0])) { sc->done = 1; sc->status = 5; break; }
            if (v[0] <= sc->tol2 * sc->bb) { sc->done = 1; sc->status = 0; }
            else if (sc->iter >= sc->max_iter) { sc->done = 1; sc->status = 4; }
            break;
        }
        case FIN_UPDATE_PW: {       // pointwise preconditioner: also beta (Fletcher-Reeves)
            sc->iter += 1;
            sc->rr = v[0];
            if (!isfinite(v[0]) || !isfinite(v[1])) { sc->done = 1; sc->status = 5; break; }
            sc->beta = v[1] / sc->rz;
            sc->rz_old = sc->rz;
            sc->rz = v[1];
            if (v[0] <= sc->tol2 * sc->bb) { sc->done = 1; sc->status = 0; }
            else if (sc->iter >= sc->max_iter) { sc->done = 1; sc->status = 4; }
            break;
        }
        case FIN_PW_INIT: {         // first pointwise-preconditioned residual: v = [r.z]
            sc->rz = v[0];
            sc->beta = 0.0;
            break;
        }
        case FIN_STORE_RR: {        // true residual at exit: v = [b.b, r.r]
            sc->rr = v[1];
            break;
        }
        case FIN_INIT_PW: {         // start of a pointwise-preconditioned solve from x = 0: v = [r.r, r.z]
            sc->bb = v[0];
            sc->rr = v[0];
            sc->rr0 = v[0];
            sc->rz = v[1];
            sc->iter = 0;
            sc->status = 0;
            sc->beta = 0.0;
            sc->restart = 0;
            sc->done = (v[0] == 0.0) || (sc->max_iter <= 0);
            if (!isfinite(v[0]) || !isfinite(v[1])) { sc->done = 1; sc->status = 5; }
            break;
        }
        default: break;
    }
}

template <int NV>
__device__ __forceinline__ void reduce_and_finalize(double (&v)[NV], const DotArgs& d, int slot) {
    double w[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) w[k] = v[k];
    if (block_reduce_last<NV>(w, d.partials, slot, d.expected, &d.sc->counter[d.counter_id])) {
        if (threadIdx.x == 0) {
            double t[2] = {w[0], NV > 1 ? w[NV > 1 ? 1 : 0] : 0.0};
            finalize(d.fin, t, d.sc);
        }
    }
}

__device__ __forceinline__ bool skip(const DotArgs& d) {
    return d.sc != nullptr && !d.ignore_done && *((volatile const int*)&d.sc->done);
}

template <typename TI> __device__ __forceinline__ TI ld(const TI* p, long long i) { return __ldg(p + i); }

}  // namespace ibm

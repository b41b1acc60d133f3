// Kernel launchers shared between the kernel files and the C ABI.
#pragma once
#include <vector>

#include "device.cuh"

namespace ibm {

// Solver kernels are launched with programmatic stream serialisation (every
// such kernel starts with pdl_entry()); IBM_NO_PDL=1 in the environment turns
// it off.
bool pdl_enabled();
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at;
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// MODE_JAC2 (sliced-ELLPACK levels): two damped-Jacobi sweeps from x = 0 in one pass
enum { MODE_APPLY = 0, MODE_RESID = 1, MODE_JAC = 2, MODE_JAC0 = 3, MODE_JAC2 = 4 };
enum { DK_NONE = 0, DK_XY = 1, DK_RESID = 2, DK_ZR = 3 };
enum { FIN_NONE = 0, FIN_INIT, FIN_PRECOND, FIN_ALPHA, FIN_UPDATE, FIN_UPDATE_PW, FIN_PW_INIT, FIN_STORE_RR,
       FIN_INIT_PW };

// Arguments of a fused reduction: partial sums per block, the number of
// participating blocks (over one or two kernels) and what the last block does.
struct DotArgs {
    CgScalars* sc = nullptr;
    double* partials = nullptr;
    int expected = 0;        // blocks contributing (all kernels of the reduction)
    int slot0 = 0;           // first partial slot of this kernel
    int counter_id = 0;
    int fin = FIN_NONE;
    int ignore_done = 0;     // run even after convergence (true-residual check)
    const double* r = nullptr;   // DK_ZR: z.r
    const double* q = nullptr;   // DK_ZR: z.q_prev
    const void* base = nullptr;  // DK_ZR: output z = base - x (level type), stencil-only V-cycles
};

template <typename T, typename TB, typename TY>
void launch_stencil(int mode, int dk, const Stencil<T>& s, const T* x, const TB* b, TY* y, T omega,
                    const DotArgs& d, dim3 grid, cudaStream_t st);
// 2D launch shape of the 5-point kernels: x-blocks over a row, y-blocks over
// rows (strided); at most `target` blocks in total
inline dim3 stencil_grid(int nx, int nrows, int target) {
    int gx = (nx + kThreads - 1) / kThreads;
    int gy = target / gx;
    if (gy < 1) gy = 1;
    if (gy > nrows) gy = nrows;
    return dim3(gx, gy, 1);
}
template <typename T, typename TB, typename TY>
void launch_coupling(int mode, int dk, const Coupling<T>& c, const T* x, const TB* b, TY* y, const T* idiag,
                     T omega, const DotArgs& d, int grid, cudaStream_t st);
void launch_loop_cond(cudaGraphConditionalHandle h, CgScalars* sc, cudaStream_t st);
void launch_pupdate(long long n, const double* z, double* p, const DotArgs& d, int grid, cudaStream_t st);
void launch_cg_update(int pw, long long n, double* x, double* r, const double* p, const double* q, double* z,
                      const double* idiag, const DotArgs& d, int grid, cudaStream_t st);
void launch_dot2(long long n, const double* a, const double* b, const DotArgs& d, int grid, cudaStream_t st);
void launch_pw_precond(long long n, const double* r, double* z, const double* idiag, const DotArgs& d, int grid,
                       cudaStream_t st);
// Finest level of the pressure-block V-cycle in FP32 from the 1D metrics.
// V0_PRE2: y = two damped-Jacobi sweeps from x = 0 (b read once, FP64) and
// b32 = float(b); V0_PRE1: y = one sweep, b32 = float(b); V0_JAC: y = x +
// w D^-1 (b32 - A x); V0_RESID: y = b32 - A x.  DK_ZR (V0_JAC only) forms
// z.r and z.q of z = y (or z = base - y) into the reduction described by d.
enum { V0_PRE2 = 0, V0_PRE1 = 1, V0_JAC = 2, V0_RESID = 3 };
template <typename TY>
void launch_vc0(int mode, int dk, const Sep32& s, const float* x, const double* b, float* b32, TY* y, float omega,
                const DotArgs& d, dim3 grid, cudaStream_t st);

// Finest level of the FP32 pressure-block V-cycle with temporal blocking
// (k_level0.cu): launch_l0_pre runs `sweeps` damped-Jacobi sweeps from x = 0
// and the residual in one pass (writes b32 = float(b), x and r);
// launch_l0_post runs `sweeps` sweeps from xin (after the prolongation), the
// last one into out (DK_ZR: with z.r, z.q into d).  Both launch on
// l0_grid(sweeps, nx, ny) blocks (the reduction's block count), at most
// kL0MaxBlocks, each block looping over 58 x 32-cell tiles (S = 3).
constexpr int kL0MaxSweeps = 6;
constexpr int kL0MaxBlocks = 2048;   // blocks of a fused launch (each loops over tiles)
bool l0_fused_ok(int sweeps);
dim3 l0_grid(int sweeps, int nx, int ny);
void launch_l0_pre(int sweeps, const Sep32& s, const double* b, float* b32, float* x, float* r, float omega,
                   const DotArgs& d, cudaStream_t st);
template <typename TYo>
void launch_l0_post(int sweeps, int dk, const Sep32& s, const float* xin, const float* b32, TYo* out, float omega,
                    const DotArgs& d, cudaStream_t st);

// AMG level operators, prolongators and restrictions (sliced ELLPACK)
template <typename T>
void launch_sell(int mode, const SellView<T>& A, const T* idiag, const T* x, const T* b, T* y, T omega,
                 const CgScalars* sc, cudaStream_t st);
template <typename T>
void launch_sell_mv(int acc, const SellView<T>& A, const T* x, T* y, const CgScalars* sc, cudaStream_t st);
// pre-sweeps from zero and the restriction of their residual (Rt = R (I - A w D^-1)^pre, pre 1 or 2)
template <typename T>
void launch_sell_down(int pre, const SellView<T>& A, const T* idiag, const T* b, T* x, T omega,
                      const CsrView<T>& Rt, T* bc, const CgScalars* sc, cudaStream_t st);
// the coarse correction and the first post-sweep (Q = (I - w D^-1 A) P)
template <typename T>
void launch_sell_up(const SellView<T>& A, const T* idiag, const T* x, const T* b, T* y, T omega,
                    const SellView<T>& Q, const T* xc, const CgScalars* sc, cudaStream_t st);
template <typename T>
void launch_coarse(int n, const double* Ainv, const T* b, T* x, const CgScalars* sc, cudaStream_t st);
// Q^T B^N Q (N > 1) as an FP64 sliced-ELLPACK matrix: MODE_APPLY / MODE_RESID
// with the reductions DK_NONE, DK_XY (APPLY) or DK_RESID (RESID)
void launch_sell_op(int mode, int dk, const SellView<double>& A, const double* x, const double* b, double* y,
                    const DotArgs& d, int grid, cudaStream_t st);
// b = T(a); z = double(x) with [z.r, z.q] when dk == DK_ZR
template <typename T>
void launch_narrow(long long n, const double* a, T* b, const CgScalars* sc, int grid, cudaStream_t st);
template <typename T>
void launch_widen(int dk, long long n, const T* x, double* z, const DotArgs& d, int grid, cudaStream_t st);

// ---- coarse end of the V-cycle on one thread-block cluster (k_tail.cu) ----------
constexpr int kTailThreads = 1024;
constexpr int kMaxTailLevels = 8;
template <typename T>
struct TailLevel {
    SellView<T> A, P, R;       // P, R: to and from the next level (unused on the coarsest)
    const T* idiag;
    T* b;
    T* x;
    T* x2;
    T* r;
    T omega;
};
template <typename T>
struct TailArgs {
    TailLevel<T> lev[kMaxTailLevels];
    const double* cinv;        // dense FP64 inverse of the coarsest operator, row-major nc x nc
                               // (the coarsest solve is FP64 in both precisions: b widened,
                               // FP64 products and sums, x narrowed to T)
    const CgScalars* sc;       // nullable; the kernel returns at once when sc->done is set
    int nlev, pre, post, nc;
};
// cluster size the tail kernel can run with on this device (16, 8, or 0 = unavailable)
template <typename T>
int tail_cluster_size(int device);
// staged_smem > 0: the variant that keeps each block's slices in shared memory
template <typename T>
cudaError_t launch_tail(const TailArgs<T>& a, int cluster, long long staged_smem, cudaStream_t st);
// shared memory per block of the staged variant for operators with the given
// host slice offsets (in kernel order: A, R, P of each level) and the coarsest size
long long tail_staged_bytes(const std::vector<const std::vector<long long>*>& offs, int coarse_n, int cs, size_t ts);
template <typename T>
bool tail_staged_ready(int cluster, long long smem);

// ---- coarse levels of the V-cycle as one cooperative kernel (k_coop.cu) -----------
constexpr int kMaxCoopLevels = 12;
// Grid barrier state in the workspace (zeroed before each use by the host)
struct GridBarrier {
    unsigned int count;   // blocks arrived at the current barrier
    unsigned int gen;     // barriers completed (monotonic)
    int err;              // 1: a block gave up waiting; every block leaves
    int pad;
};
template <typename T>
struct CoopLevel {
    SellView<T> A, P, R;       // P, R: to and from the next level (unused on the coarsest)
    const T* idiag;
    T* b;
    T* x;
    T* x2;
    T* r;
    T omega;
};
// Levels of one cooperative V-cycle, resident in the workspace (rewritten
// whenever the hierarchy is uploaded): the kernel's first level, then coarser
// ones, and the parent level's transfers (b_0 = Rp r_parent, x_parent += Pp x_0).
template <typename T>
struct CoopTable {
    CoopLevel<T> lev[kMaxCoopLevels];
    SellView<T> Rp, Pp;
};
constexpr int kCoopThreads = 512;
template <typename T>
struct CoopArgs {
    const CoopTable<T>* tab;   // device
    const double* cinv;        // dense FP64 inverse of the coarsest operator (b widened, x narrowed)
    int nlev, pre, post, nc;
    unsigned staged;           // bit 3 l + {0, 1, 2}: A, R, P of level l staged in shared memory
    int has_parent;
    const T* rp;               // parent residual (has_parent)
    T* xp;                     // parent iterate (has_parent)
    CgScalars* sc;             // nullable; the kernel returns at once when sc->done is set,
                               // and a barrier timeout sets done with status 6
    GridBarrier* bar;
};
// blocks of the cooperative kernel that fit on one SM with `smem` bytes of
// dynamic shared memory (0: cooperative launch unavailable)
template <typename T>
int coop_blocks_per_sm(int device, long long smem);
// shared memory per block of the staged operators for a grid of `grid`
// blocks: host slice offsets in kernel order (A, R, P of each level; null =
// not staged) and their value sizes
long long coop_staged_bytes(const std::vector<const std::vector<long long>*>& offs, const std::vector<size_t>& tsz,
                            int grid);
template <typename T>
cudaError_t launch_coop(const CoopArgs<T>& a, int grid, long long smem, cudaStream_t st);

// ---- Schur-complement block preconditioner (k_solve.cu) ---------------------------
// inverse of the SPD n x n matrix M (row-major, symmetrised first) by blocked
// Gauss-Jordan elimination on the device (32-wide pivot blocks): in place in
// FP64, or with M32 non-null in FP32 into M32 (M then keeps the symmetrised
// matrix); scratch: 32 * (n + 32) doubles; *flag is set to 1 on a
// non-positive pivot
void launch_spd_inverse(int n, double* M, double* scratch, int* flag, float* M32, cudaStream_t st);
// cache of V-cycle responses to unit vectors (moving bodies, Schur preconditioner)
void launch_set_entry(double* v, long long cell, double val, cudaStream_t st);
void launch_cache_map(int n, const long long* pairs, int* slot, long long* cell_of, cudaStream_t st);
void launch_cache_clear(int n, int* slot, const long long* cell_of, cudaStream_t st);
template <typename T>
void launch_cache_store(int nu, const long long* cell_of, const T* w, int sv, T* G, long long ld, cudaStream_t st);
template <typename T>
void launch_schur_cached(const CsrView<double>& Cf, long long f0, const int* slot, const T* G, long long ld, double* S,
                         cudaStream_t st);
// force rows of the coupled operator split as [C^T | F] (columns < f0 | >= f0)
void launch_col_scatter(const CsrView<double>& Cf, long long f0, int row, double* v, int clear, cudaStream_t st);
template <typename T>
void launch_schur_col(const CsrView<double>& Cf, long long f0, int col, const T* w, double* S, cudaStream_t st);
template <typename T>
void launch_schur_tf(const CsrView<double>& Cf, long long f0, const double* r, const T* y1, double* tf,
                     const CgScalars* sc, cudaStream_t st);
// out = add + sign M v for a dense nf x nf M (add nullable; FP64 products
// and sums); skipped once the solve with scalars sc is done
template <typename T>
void launch_dense_mv(int nf, const T* M, const double* v, const double* add, double sign, double* out,
                     const CgScalars* sc, int grid, cudaStream_t st);
// v[k] in [-0.5, 0.5) from a hash of k (a fixed probe vector)
void launch_probe_fill(int n, double* v, cudaStream_t st);
// out = add + M v with the force part of the FCG dots z.r, z.q into d
template <typename T>
void launch_dense_mv_dots(int nf, const T* M, const double* v, const double* add, double* out, const DotArgs& d,
                          int grid, cudaStream_t st);
template <typename T>
void launch_schur_zf(int nf, const T* Sinv, const double* tf, double* zf_out, const DotArgs& d, int grid,
                     cudaStream_t st);
void launch_schur_sp(int ntc, const long long* tcell, const CsrView<double>& Cc, long long f0, const double* z,
                     double* s, const CgScalars* sc, cudaStream_t st);

// ---- body rows of a moving body on the device (k_body.cu) -------------------------
struct BodyGeo {
    int nx, ny;
    long long nc;
    double h, dt;
    const double *xf, *yf, *xc, *yc, *dx, *dy, *dxf, *dyf, *idxf, *idyf;
};
// The body rows' structure (row pointers and columns uploaded from the host
// pattern; the val pointers of the views are not used), their value arrays
// and the index maps that build each value.
struct BodyDev {
    CsrView<double> E, ET, Cc, Cf;
    double *Ev, *ETv, *Ccv, *Cfv;
    float *Cc32, *Cf32;                          // nullable: FP32 copies (mixed path)
    const int *point, *et_src, *cf_a, *cf_b, *cc_src, *diag;
    const double *xb, *yb;                       // point positions at t^{n+1}
    double *pdiag, *pidiag;                      // Poisson diagonal and inverse (force rows written)
    float *pdiag32, *pidiag32;                   // nullable
};
void launch_body_values(const BodyGeo& g, const BodyDev& b, cudaStream_t st);

// ---- time-step kernels (k_step.cu) ------------------------------------------------
struct StepParams {
    double nu, dt, uinf;
    double inflow;       // net inflow through the Dirichlet edges (constant)
    double ly;           // height of the outflow edge
    int bc;              // IBM_BC_*
    int first;           // 1 on the first Adams-Bashforth step
    long long pin;       // pinned cell
};
void launch_outflow(const GridView& g, const StepParams& p, const double* q, BoundaryView b, double* u_right1,
                    double* v_right1, cudaStream_t st);
void launch_rhs(const GridView& g, const StepParams& p, const Stencil<double>& A, const double* mdt,
                const double* q, BoundaryView b, const double* nprev, double* ncur, double* r1, dim3 grid,
                cudaStream_t st);
void launch_poisson_rhs(const GridView& g, const StepParams& p, const double* qs, BoundaryView b,
                        const CsrView<double>& E, const double* ub, double* b2, int grid, cudaStream_t st);
// qs null: q* = 0; pin >= 0: lam[pin] taken as 0
void launch_project(const GridView& g, double dt, const double* qs, const double* lam, double* q, dim3 grid,
                    cudaStream_t st, long long pin = -1);
// matrix-free Q^T B^N Q, last stage: y = [div q; -E q] (q = -B^N Q x), y[pin] = dpin x[pin]; MODE_RESID: b - that
void launch_qt_apply(int mode, int dk, const GridView& g, long long pin, double dpin, const double* q,
                     const CsrView<double>& E, const double* x, const double* b, double* y, const DotArgs& d, int grid,
                     cudaStream_t st);
void launch_project_body(const GridView& g, double dt, int nfaces, const int* faces, const CsrView<double>& ET,
                         const double* f, double* q, cudaStream_t st);
// out[0..1] = force sums; out[2..3] = 0 (filled by launch_constraints, which must follow)
void launch_forces(int n_b, const double* f, double* out, cudaStream_t st);
// out[2] = max |G^T q + bc2| over the unpinned cells, out[3] = max |E q - u_B| (FP64)
void launch_constraints(const GridView& g, const StepParams& p, const double* q, BoundaryView b,
                        const CsrView<double>& E, const double* ub, double* out, dim3 grid, cudaStream_t st);
void launch_extrapolate(long long n, double* lam, double* prev, int first, int grid, cudaStream_t st);
// Inner FP32 Jacobi-preconditioned CG of the mixed-precision velocity solve
// (k_vel32.cu), on the n = nblk nx ny unknowns of the velocity operator:
// launch_v32_init: r = float(r64), e = 0, z = D^-1 r, [r.r, r.z] into d
// (FIN_INIT_PW: the inner solve's scalars start over with tol2 = tol2_in and
// max_iter);
// launch_v32_pupdate: p = z + beta p; launch_v32_apply: q = A p with [p.q];
// launch_v32_update: e += alpha p, r -= alpha q, z = D^-1 r with [r.r, r.z];
// launch_v32_correct: x += double(e).  Products and per-thread partial sums in
// FP32, block and grid sums and the step lengths in FP64.
void launch_v32_init(long long n, const double* r64, float* r, float* e, float* z, const float* idiag, double tol2_in,
                     int max_iter, const DotArgs& d, int grid, cudaStream_t st);
void launch_v32_pupdate(long long n, const float* z, float* p, const DotArgs& d, int grid, cudaStream_t st);
void launch_v32_apply(const Stencil<float>& s, const float* p, float* q, const DotArgs& d, dim3 grid, cudaStream_t st);
void launch_v32_update(long long n, float* e, float* r, const float* p, const float* q, float* z, const float* idiag,
                       const DotArgs& d, int grid, cudaStream_t st);
void launch_v32_correct(long long n, double* x, const float* e, int grid, cudaStream_t st);

// Warm start by projection onto previous solutions (k_step.cu): a basis of at
// most kProjMax K-orthonormal vectors X_i (stride ld) with KX_i = K X_i.
// launch_proj_dots: coef[i] = X_i . (a - b) (b nullable; part: kProjMax *
// kProjBlocks doubles); launch_proj_combine: v = base - sign sum coef_i X_i
// and, with w non-null, w = (y - r) - sign sum coef_i KX_i; launch_proj_store:
// X = v / sqrt(coef[0]), KX = w / sqrt(coef[0]) (zero when coef[0] is not
// above 1e-24 |coef[1]|).
constexpr int kProjMax = 24;
constexpr int kProjEvery = 2;   // a solution joins the basis every kProjEvery-th solve
constexpr int kProjBlocks = 608;
void launch_proj_dots(long long n, int m, const double* X, long long ld, const double* a, const double* b,
                      double* part, double* coef, cudaStream_t st);
void launch_proj_combine(long long n, int m, const double* X, const double* KX, long long ld, const double* coef,
                         const double* base, double* v, const double* y, const double* r, double* w, double sign,
                         int grid, cudaStream_t st);
void launch_proj_store(long long n, const double* v, const double* w, const double* coef, double* X, double* KX,
                       int grid, cudaStream_t st);
// Projection with B^N, N > 1 (Eq. 9c): after q = q* - B^1 Q lam, the further
// terms t_k = (dt/2) M^-1 L t_{k-1} = t_{k-1} - (A t_{k-1}) / (M/dt), t_0 = q - q*,
// are added to q.  start: t = q - qs; term: t = t - At / mdt, q += t (t = 0
// on the unused slots, where mdt = 0).
void launch_bn_start(long long n, const double* mdt, const double* q, const double* qs, double* t, int grid,
                     cudaStream_t st);
void launch_bn_term(long long n, const double* mdt, const double* At, double* t, double* q, int grid,
                    cudaStream_t st);

}  // namespace ibm

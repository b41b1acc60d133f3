/*
 * ibm.h - C ABI of the GB300 immersed-boundary projection library.
 *
 * The library advances the 2D immersed-boundary projection method of Taira &
 * Colonius as used by Layton, Krishnan & Barba ("cuIBM", section 2): per time
 * step it forms the explicit right-hand side, solves A q* = r1 (Eq. 9a) by
 * Jacobi-preconditioned CG, solves Q^T B^N Q lambda = Q^T q* - r2 (Eq. 9b) by
 * CG preconditioned with a smoothed-aggregation AMG V-cycle, projects
 * q = q* - B^N Q lambda (Eq. 9c), and for moving bodies rebuilds the rows E of
 * Q from the discrete delta (Eq. 5, Eq. 6) and the AMG hierarchy every
 * `amg_rebuild_every` steps (section 4, hierarchy re-use).
 *
 * Discretisation (fixed by this library; the paper defers it to an appendix
 * of Taira & Colonius):
 *   - staggered grid of nx x ny cells with face coordinates xf[0..nx],
 *     yf[0..ny]; cell widths dx_i, dy_j; face spacings dxf_i = xc_i - xc_{i-1};
 *   - unknowns are momentum fluxes q_u = u dy_j on interior x-faces and
 *     q_v = v dx_i on interior y-faces;
 *   - M = diag(dxf_i/dy_j, dyf_j/dx_i), A = M/dt - L/2 (Crank-Nicolson),
 *     Adams-Bashforth 2 convection (first step: Euler), B^1 = dt M^-1 (N = 1,
 *     the default) or B^N = sum_{k<N} ((dt/2) M^-1 L)^k dt M^-1 (bn_order);
 *     "Q^T B^1 Q" below stands for the Q^T B^N Q of the configured N;
 *   - lambda = (phi, f~): phi per cell, f~ = force of the fluid on each body
 *     point (x components of all points, then y components);
 *   - pressure cell (pin_i, pin_j) pinned: its row and column of Q^T B Q keep
 *     only the diagonal and its right-hand side is zero (sentence after Eq. 9).
 *
 * Array layouts used at this boundary (all row-major, x fastest):
 *   u face array : ny x (nx+1) doubles, u[j*(nx+1) + i] at (xf[i], yc[j]),
 *                  boundary columns i = 0 and i = nx included;
 *   v face array : (ny+1) x nx doubles, v[j*nx + i] at (xc[i], yf[j]),
 *                  boundary rows j = 0 and j = ny included;
 *   lambda       : n_lambda = nx*ny + 2*n_b doubles: phi[j*nx+i], then
 *                  f~x[0..n_b), then f~y[0..n_b).
 *
 * Ownership: the library keeps host copies of what it is given at set-up.  All
 * device memory the library uses comes from ONE caller-allocated workspace
 * (ibm_workspace_bytes / ibm_bind_workspace); the library never allocates
 * device memory itself.  The one exception is the static device array behind
 * ibm_poisson_residual_norms_noalloc (about 16.8 MB, reserved when the
 * library's device code is loaded on a device).  Device pointers passed to a call are borrowed for that
 * call only.  Work is issued on the stream given at bind time.
 *
 * Errors: every function returns an int status (IBM_OK on success).  No
 * exception crosses this boundary and nothing aborts the process or traps the
 * device; ibm_last_error() returns a message for the last failing call.
 */
#ifndef IBM_H
#define IBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------*/
#define IBM_OK                 0
#define IBM_ERR_ARG            1  /* invalid argument or configuration            */
#define IBM_ERR_CUDA           2  /* a CUDA runtime call failed (message says which) */
#define IBM_ERR_NO_MEM         3  /* workspace missing or too small               */
#define IBM_ERR_NOT_CONVERGED  4  /* a solver hit max_iter before its tolerance    */
#define IBM_ERR_BREAKDOWN      5  /* CG breakdown: p.Ap <= 0 or a NaN/Inf residual */
#define IBM_ERR_UNIMPLEMENTED  6  /* option not available in this build            */
#define IBM_ERR_STATE          7  /* call out of order (e.g. no workspace bound)   */

/* ---- enumerations ----------------------------------------------------------*/
#define IBM_BC_FREESTREAM  0  /* Dirichlet (uinf, vinf) left/bottom/top, convective outflow right (section 5.2) */
#define IBM_BC_WALLS       1  /* Dirichlet zero on all sides (closed box, section 5.1) */

#define IBM_PRECOND_NONE    0  /* plain CG (section 3, compared and rejected)      */
#define IBM_PRECOND_JACOBI  1  /* diagonal PCG (section 3, compared and rejected)  */
#define IBM_PRECOND_AMG     2  /* smoothed-aggregation AMG V-cycle on the whole
                                  coupled Q^T B^1 Q (section 3, the paper's choice) */
#define IBM_PRECOND_SCHUR   3  /* block preconditioner (not in the paper): the same
                                  V-cycle on the pressure block Lp only, with the
                                  force rows handled through the dense Schur
                                  complement S = F - C^T V C of [Lp C; C^T F]:
                                  y1 = V r_p, z_f = S^-1 (r_f - C^T y1),
                                  z_p = y1 - V C z_f.  Section 3 observes that the
                                  pressure block suits AMG and the force rows do not.
                                  S is formed on the device (2 n_b V-cycles, or the
                                  response cache of schur_cache for moving bodies)
                                  and inverted there.  Moving bodies need it rebuilt
                                  every step (amg_rebuild_every = 1): a complement
                                  one step old multiplies the iteration count. */

#define IBM_PREC_FP64   0  /* V-cycle in FP64, PCG                                   */
#define IBM_PREC_MIXED  1  /* V-cycle in FP32 inside FP64 flexible CG; the velocity
                              solve as FP64 iterative refinement around an FP32
                              Jacobi-PCG (same FP64 residual test); a moving body's
                              Schur complement inverted in FP32 and applied with
                              one FP64 refinement step (not in the paper)          */

#define IBM_WARM_ZERO   0  /* lambda0 = 0                                          */
#define IBM_WARM_PREV   1  /* lambda0 = lambda^n                                    */
#define IBM_WARM_EXTRAP 2  /* lambda0 = 2 lambda^n - lambda^{n-1} (lambda^n on the
                              first step; not in the paper)                          */
#define IBM_WARM_CNN    3  /* extrapolation plus a learned U-Net correction of the
                              pressure part (ibm_attach_cnn; not in the paper)       */
#define IBM_WARM_PROJ   4  /* projection of the solution onto the span of up to 24
                              previous solutions (K-orthonormal basis for
                              K = Q^T B^N Q of Eq. 9b); lambda^n until the first
                              solve; fixed bodies only (moving=1 is rejected); not
                              in the paper                                          */

/* ---- configuration ----------------------------------------------------------*/
typedef struct ibm_config {
    int32_t nx, ny;          /* cells in x and y (>= 4 each)                        */
    double  nu;              /* kinematic viscosity = 1/Re                           */
    double  dt;              /* time step                                            */
    double  uinf, vinf;      /* freestream velocity (IBM_BC_FREESTREAM)              */
    int32_t bc;              /* IBM_BC_*                                             */
    int32_t bn_order;        /* N of B^N (1..4), the N-term expansion of A^-1
                                (section 2).  N > 1 needs IBM_PRECOND_AMG (else
                                IBM_ERR_UNIMPLEMENTED at create): Q^T B^N Q is
                                assembled on the host (sliced triple product), is
                                level 0 of the coupled hierarchy and, in FP64
                                sliced ELLPACK, the operator of the Poisson CG; the
                                projection adds the N - 1 further series terms;
                                with moving bodies it is rebuilt on every move     */
    double  h;               /* uniform cell width around the bodies (delta width)   */
    double  tol1;            /* velocity CG: ||r1 - A q|| <= tol1 ||r1||             */
    double  tol2;            /* Poisson CG: ||b - S lam|| <= tol2 ||b||              */
    int32_t max_iter1, max_iter2;
    int32_t poisson_precond; /* IBM_PRECOND_*                                        */
    int32_t precision;       /* IBM_PREC_*                                           */
    int32_t warm;            /* IBM_WARM_*                                           */
    int32_t pin_i, pin_j;    /* pinned pressure cell                                 */
    /* smoothed aggregation (section 3): strength |a_ij| >= theta sqrt(a_ii a_jj),
       prolongator smoothing weight (4/3)/rho(D^-1 A), damped Jacobi smoother */
    double  amg_theta;
    double  amg_omega;       /* damped-Jacobi weight of the smoother                 */
    int32_t amg_pre, amg_post;
    int32_t amg_max_coarse;  /* stop coarsening at or below this many unknowns       */
    int32_t amg_max_levels;
    int32_t amg_rebuild_every; /* moving bodies: rebuild the hierarchy every k steps */
    int32_t moving;          /* 1 if body positions change between steps             */
    double  amg_trunc;       /* prolongator truncation: drop entries below this
                                fraction of the row maximum, rescale to the row sum
                                (0 = off)                                            */
    int32_t amg_tail_rows;   /* levels (below the finest) with at most this many rows
                                run as one kernel on one thread-block cluster
                                (0 = one kernel per sweep)                           */
    int32_t amg_sweeps0;     /* pre- and post-sweeps on the finest level of the FP32
                                pressure-block V-cycle (0: amg_pre / amg_post)       */
    int32_t schur_cache;     /* moving bodies with IBM_PRECOND_SCHUR: cells whose
                                V-cycle responses are kept to rebuild S without new
                                V-cycles (-1: automatic, 8 x the cells the body rows
                                touch, at most 32768; 0: off)                         */
    int32_t reserved_;       /* set to 0                                             */
} ibm_config;

/* Fills *cfg with defaults: bc freestream, bn_order 1, tol 1e-8, max_iter 1000,
 * AMG preconditioner, FP64, warm start from lambda^n, pin (0,0), theta 0.08,
 * omega 2/3, 2 pre / 2 post sweeps, max_coarse 256, 12 levels, rebuild every 2,
 * prolongator truncation 0.1, fused coarse levels up to 16384 rows, automatic
 * Schur-complement cache for moving bodies. */
void ibm_config_defaults(ibm_config* cfg);

/* ---- per-step and per-solve statistics --------------------------------------*/
typedef struct ibm_solve_stats {
    int32_t iters;           /* CG iterations taken                                  */
    int32_t status;          /* IBM_OK, IBM_ERR_NOT_CONVERGED or IBM_ERR_BREAKDOWN   */
    double  rel_res;         /* ||b - A x|| / ||b|| recomputed in FP64 at exit        */
    double  rel_res0;        /* ||b - A x0|| / ||b|| of the initial guess             */
} ibm_solve_stats;

typedef struct ibm_step_stats {
    double  t;               /* time after the step                                  */
    ibm_solve_stats solve1;  /* Eq. 9a                                               */
    ibm_solve_stats solve2;  /* Eq. 9b                                               */
    double  fx, fy;          /* sum of f~ over all body points (force on the bodies) */
    double  cd, cl;          /* 2 fx / (U^2 D), 2 fy / (U^2 D), D = 1, U = uinf or 1 */
    /* Constraints of Eq. 8 on the new velocity q^{n+1}, computed in FP64 on the
       device after the projection (Eq. 9c):
         div_max  = max over cells other than the pinned one of |G^T q^{n+1} + bc2|
                    (the discrete continuity equation; the pinned cell's row is
                    replaced by phi(p0) = 0, so it collects the sum of the others),
         slip_max = max over body points and components of |E q^{n+1} - u_B^{n+1}|
                    (the no-slip condition, Eq. 6; 0 without bodies).
       Both equal the Poisson residual's entries in those rows, so they scale with
       tol2; units are those of q (velocity x cell width) and of u_B. */
    double  div_max, slip_max;
    /* The Poisson solve of this step (Eq. 9b) as it ran: device time between
       CUDA events recorded on the context's stream before and after it, and its
       algorithmic bytes (every element each launch must read or write once,
       summed over the launches; a device-side iteration loop counts one body's
       bytes per iteration taken). */
    double  poisson_ms, poisson_bytes;
    int32_t amg_rebuilt;     /* 1 if the AMG hierarchy (or, for IBM_PRECOND_SCHUR,
                                the Schur complement S) was (re)built in this step */
    int32_t pad_;
} ibm_step_stats;

typedef struct ibm_ctx ibm_ctx;

/* ---- set-up ------------------------------------------------------------------*/
/* Host-side set-up (no CUDA call): copies the grid and body points, builds the
 * operator coefficients, the rows E of Q for the bodies at their given
 * positions (Eq. 6), the pinned Q^T B^1 Q and, when poisson_precond is AMG, the
 * smoothed-aggregation hierarchy.
 *   xf: nx+1 increasing x face coordinates;  yf: ny+1 increasing y faces;
 *   xb, yb: n_b body point coordinates (n_b may be 0; the pointers may then be
 *   NULL).  Every point's delta support (1.5 h) must lie in uniform cells of
 *   width h, and no point may lie in the three cells next to an edge of the
 *   grid; otherwise IBM_ERR_ARG, with a message naming the point and which
 *   rule it breaks.
 * The initial velocity is the freestream (or rest, for walls); set another
 * with ibm_set_state.  On success *out owns the context (free with
 * ibm_destroy). */
int ibm_create(const ibm_config* cfg, const double* xf, const double* yf,
               int32_t n_b, const double* xb, const double* yb, ibm_ctx** out);

/* Device bytes the context needs (coefficients, vectors, hierarchy with room
 * for rebuilds).  Valid after ibm_create.  IBM_ERR_ARG if ctx or bytes is
 * NULL. */
int ibm_workspace_bytes(const ibm_ctx* ctx, size_t* bytes);

/* Binds a caller-owned device buffer of at least ibm_workspace_bytes bytes
 * (256-byte aligned) and a cudaStream_t (passed as void*, NULL = default
 * stream), then uploads the set-up data on that stream.  The buffer must stay
 * valid until ibm_destroy.  IBM_ERR_NO_MEM if ws_bytes is too small. */
int ibm_bind_workspace(ibm_ctx* ctx, void* dev_ws, size_t ws_bytes, void* stream);

/* ibm_create followed by ibm_bind_workspace.  When dev_ws is NULL only the
 * host set-up runs and the context is returned unbound (query
 * ibm_workspace_bytes, then call ibm_bind_workspace).  Returns the first
 * failing step's status; on a failed bind *out still owns the created
 * context. */
int ibm_setup(const ibm_config* cfg, const double* xf, const double* yf,
              int32_t n_b, const double* xb, const double* yb,
              void* dev_ws, size_t ws_bytes, void* stream, ibm_ctx** out);

void ibm_destroy(ibm_ctx* ctx);
const char* ibm_last_error(const ibm_ctx* ctx);

/* Sizes: n_q velocity unknowns (interior faces), n_lambda = nx*ny + 2 n_b
 * (Eq. 9a and 9b); each output may be NULL.  IBM_ERR_ARG for a NULL ctx. */
int ibm_sizes(const ibm_ctx* ctx, int64_t* n_q, int64_t* n_lambda, int32_t* n_b);

/* ---- time stepping -------------------------------------------------------------*/
/* Body points at t^{n+1} and their velocities u_B^{n+1} (host arrays of n_b
 * doubles each; Eq. 9b right-hand side).  For moving bodies call before every
 * ibm_step; positions also rebuild E (Eq. 5, Eq. 6) and the coupling rows of
 * Q^T B Q (the one host-to-device transfer of a step, as in section 4, "keep
 * everything on the GPU").  ub/vb may be NULL (zero body velocity); xb/yb may
 * be NULL (positions unchanged).  IBM_ERR_STATE without a bound workspace,
 * IBM_ERR_ARG for a non-finite velocity or a point that breaks the placement
 * rules of ibm_create (nothing is changed then), IBM_ERR_CUDA if an upload
 * fails. */
int ibm_set_body(ibm_ctx* ctx, const double* xb, const double* yb,
                 const double* ub, const double* vb);

/* Advances nsteps time steps (Eq. 9a-c each).  per_step (host, nsteps
 * entries) may be NULL.  Returns the first non-OK solver status
 * (IBM_ERR_NOT_CONVERGED, IBM_ERR_BREAKDOWN), after finishing the step in
 * which it occurred; IBM_ERR_STATE without a bound workspace or with a
 * learned warm start but no attached network; IBM_ERR_CUDA if a launch
 * fails. */
int ibm_step(ibm_ctx* ctx, int32_t nsteps, ibm_step_stats* per_step);

/* Solves Q^T B^1 Q lambda = rhs (Eq. 9b, pinned) with the configured solver.
 * d_rhs, d_lambda: device arrays of n_lambda doubles (layout above);
 * d_lambda0: initial guess or NULL for zero.  d_rhs[pin] should be zero.
 * Returns the solve's status (stats->status: IBM_OK, IBM_ERR_NOT_CONVERGED,
 * IBM_ERR_BREAKDOWN); IBM_ERR_ARG if d_rhs or d_lambda is NULL,
 * IBM_ERR_STATE without a bound workspace. */
int ibm_solve_poisson(ibm_ctx* ctx, const double* d_rhs, double* d_lambda,
                      const double* d_lambda0, ibm_solve_stats* stats);

/* Forces of the last step (Eq. 7-8: the multipliers f~ are the point forces
 * on the body; their sums give the drag and lift coefficients the paper
 * reports in Section 5.2 and Table 4): fx, fy host arrays of n_b receive f~
 * per boundary point (nullable); cd, cl (nullable) receive 2 sum fx / (U^2 D)
 * and 2 sum fy / (U^2 D) as in ibm_step_stats.  The values are those the last
 * ibm_step left on the device; the sums run in one kernel on the context's
 * stream, which the call then synchronises.  Returns IBM_ERR_ARG for a NULL
 * context, IBM_ERR_STATE without a bound workspace and IBM_ERR_CUDA if a
 * launch or copy fails. */
int ibm_forces(ibm_ctx* ctx, double* fx, double* fy, double* cd, double* cl);

/* ---- state (checkpoint / resume, parity checks) --------------------------------*/
/* Host arrays; any pointer may be NULL to skip it.
 *   u: ny x (nx+1) face array, v: (ny+1) x nx face array (layout above);
 *   v_right: ny+1 tangential v on the right edge (convective outflow);
 *   nprev: n_q convection term of the previous step in the library's internal
 *          padded order (see ibm_layout) - opaque, round-trips only;
 *   lambda: n_lambda;  t, step: time and step counter.
 * ibm_set_state with nprev == NULL restarts Adams-Bashforth 2 (Euler step);
 * it always discards the warm starts' history (lambda^{n-1} and the
 * projection basis), which is not part of the state.  Both copy synchronously
 * on the context's stream; IBM_ERR_STATE without a bound workspace,
 * IBM_ERR_CUDA if a copy fails. */
int ibm_get_state(ibm_ctx* ctx, double* u, double* v, double* v_right, double* nprev,
                  double* lambda, double* t, int64_t* step);
int ibm_set_state(ibm_ctx* ctx, const double* u, const double* v, const double* v_right,
                  const double* nprev, const double* lambda, double t, int64_t step);

/* Length of the internal velocity vector (2 nx ny: padded u then padded v),
 * the length of nprev above. */
int ibm_layout(const ibm_ctx* ctx, int64_t* nq_padded);

/* ---- operators (kernel-level parity checks) ------------------------------------*/
/* y = (pinned Q^T B^1 Q) x on device arrays of n_lambda doubles. */
int ibm_apply_poisson(ibm_ctx* ctx, const double* d_x, double* d_y);
/* z = one AMG V-cycle applied to r (device, n_lambda doubles), in the
 * configured precision.  IBM_ERR_STATE without a hierarchy. */
int ibm_vcycle(ibm_ctx* ctx, const double* d_r, double* d_z);

/* ---- allocation-free residual check ---------------------------------------------*/
/* norms_out[0] = ||rhs||^2, norms_out[1] = ||rhs - (pinned Q^T B^1 Q) lambda||^2 for
 * device arrays d_lambda, d_rhs of n_lambda doubles; norms_out is host memory.
 * The paper has no counterpart: this serves callers that cannot allocate device
 * memory where they call it (a fixed device-memory plan, a host callback, a
 * program without a framework allocator).  Nothing is allocated: the residual
 * and the reduction scratch live in a static device array of the library
 * (2^21 + 2052 doubles, about 16.8 MB, held by every device that loads the
 * library until the process exits).  n_lambda above 2^21 is rejected with
 * IBM_ERR_ARG.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) with that device current and caches it, which
 * assumes the device's primary context is not reset while the library is
 * loaded.  The current device must be the one bound at ibm_bind_workspace
 * (else IBM_ERR_STATE).  Work runs on the context's stream; the call copies
 * the two norms to host memory and waits for them, so it must never be called
 * while that stream is capturing a graph (IBM_ERR_STATE).  All calls share the
 * one array: calls that overlap on the GPU (from several threads, streams or
 * contexts of the same device) race and must be serialised by the caller. */
int ibm_poisson_residual_norms_noalloc(ibm_ctx* ctx, const double* d_lambda, const double* d_rhs,
                                       double* norms_out);

/* ---- AMG hierarchy (host copies, for inspection) ---------------------------------*/
int ibm_amg_levels(const ibm_ctx* ctx, int32_t* nlevels);
/* Level l operator (l = 0 is the pinned Q^T B^1 Q) and prolongator P_l from
 * level l+1 to l, as CSR.  which = 2, 3: the fused transfers of levels
 * 1 .. L-2 (empty, n = 0, elsewhere or when unused): Rt = R (I - A w D^-1)^pre,
 * which restricts the residual left by `pre` damped-Jacobi sweeps from x = 0
 * straight from b, and Q = (I - w D^-1 A) P, the first post-sweep applied to
 * the coarse correction (section 3's smoothed-aggregation V-cycle, with the
 * level's sweeps folded into its transfers).  Call with NULL arrays to get n
 * and nnz first. */
int ibm_amg_matrix(const ibm_ctx* ctx, int32_t level, int32_t which /*0=A,1=P,2=Rt,3=Q*/,
                   int64_t* nrows, int64_t* ncols, int64_t* nnz,
                   int64_t* rowptr, int32_t* colind, double* vals);

/* With IBM_PRECOND_SCHUR, ibm_vcycle applies the pressure-block V-cycle to
 * the first nx*ny entries of d_r and writes nx*ny entries of d_z. */

/* Rows and damped-Jacobi weight of level l (the weight is (4/3)/rho(D^-1 A_l)
 * for amg_omega = 2/3, rho estimated by power iteration with a 5% margin). */
int ibm_amg_level_info(const ibm_ctx* ctx, int32_t level, int64_t* nrows, double* omega);

/* ---- learned warm start (not in the paper) -------------------------------------------
 * A U-Net predicts the error of the extrapolated pressure warm start of Eq. 9b:
 *   a = 2 phi^n - phi^{n-1},  phi0 = a + s * UNet(x),  s = rms(phi^n - phi^{n-1}),
 *   x = [ (phi^n - phi^{n-1})/s, r/rms(r), a/rms(a) ]  (3 channels),
 * r = pressure rows of b - (Q^T B Q) [a; 2 f^n - f^{n-1}] (residual of the
 * extrapolated guess), trained on (phi^{n+1} - a)/s from the solver's own steps.
 * Network: `levels` resolution levels of two 3x3 convs + ReLU with base*2^l
 * channels, 2x2 average pooling, nearest upsampling with skip concatenation, a
 * final 1x1 conv; BF16 weights and activations on the tensor cores with FP32
 * accumulation, FP32 master weights, gradients and Adam.  Tensors are NHWC.
 * The forward 3x3 convolutions with 16, 32, 64 or 128 output channels run on
 * tcgen05 (accumulator in tensor memory); the others, the backward passes and
 * every convolution of a network created with the environment variable
 * IBM_CNN_NO_TC=1 run on mma.sync.  A tcgen05 convolution whose bounded
 * barrier wait gives up makes the next synchronising call (forward,
 * loss_grad, or ibm_step with IBM_WARM_CNN) return IBM_ERR_CUDA.
 * Parameter order (flat): per conv in network order W[ky][kx][cin][cout], bias.
 * Errors of the ibm_cnn_* calls: IBM_ERR_ARG for a NULL network or pointer, a
 * wrong parameter count, sizes that are not positive multiples of
 * 2^(levels-1), or more pixels than max_pixels; IBM_ERR_NO_MEM for a workspace
 * below ibm_cnn_workspace_bytes; IBM_ERR_STATE before ibm_cnn_bind;
 * IBM_ERR_CUDA if a launch or copy fails.  ibm_cnn_last_error gives the
 * message. */
typedef struct ibm_cnn ibm_cnn;
/* max_pixels: largest batch*height*width the network will process. */
int ibm_cnn_create(int32_t base, int32_t levels, int64_t max_pixels, ibm_cnn** out);
void ibm_cnn_destroy(ibm_cnn* net);
const char* ibm_cnn_last_error(const ibm_cnn* net);
int ibm_cnn_param_count(const ibm_cnn* net, int64_t* n);
/* One caller-owned device workspace (parameters, Adam state, activations,
 * gradients), as for the solver context. */
int ibm_cnn_workspace_bytes(const ibm_cnn* net, size_t* bytes);
int ibm_cnn_bind(ibm_cnn* net, void* dev_ws, size_t bytes, void* stream);
/* Host parameter vectors of ibm_cnn_param_count doubles; set resets Adam. */
int ibm_cnn_set_params(ibm_cnn* net, const double* host, int64_t n);
int ibm_cnn_get_params(ibm_cnn* net, double* host, int64_t n);
/* d_in: batch*h*w*3 floats (NHWC), d_out: batch*h*w floats; h and w must be
 * multiples of 2^(levels-1). */
int ibm_cnn_forward(ibm_cnn* net, int32_t batch, int32_t h, int32_t w, const float* d_in, float* d_out);
/* Mean squared error against d_target (batch*h*w floats); accumulates the
 * parameter gradients (replacing earlier ones) for ibm_cnn_adam_step and
 * optionally copies them to host_grad (param_count doubles). */
int ibm_cnn_loss_grad(ibm_cnn* net, int32_t batch, int32_t h, int32_t w, const float* d_in,
                      const float* d_target, double* loss, double* host_grad);
int ibm_cnn_adam_step(ibm_cnn* net, double lr, double beta1, double beta2, double eps);
/* Timing of the forward pass on the input already in the workspace (for the
 * roofline of the convolutions): one untimed pass, then `reps` passes with
 * CUDA events around every convolution launch on the network's stream;
 * ms[i] = mean milliseconds of convolution i (network order), n = number of
 * convolutions (2 * levels + 2 * (levels - 1) + 1).  Synchronises. */
int ibm_cnn_time_forward(ibm_cnn* net, int32_t batch, int32_t h, int32_t w, int32_t reps, double* ms, int32_t n);
/* Convolution i: input and output channels, kernel size, resolution level
 * (spatial size = input size / 2^level) and whether it runs on tcgen05. */
int ibm_cnn_layer_info(const ibm_cnn* net, int32_t i, int32_t* cin, int32_t* cout, int32_t* ks, int32_t* level,
                       int32_t* tcgen05);
/* Standardised network inputs (and the target, when d_phi_np1 and d_target are
 * given) for ncrop crops of crop_h x crop_w cells at host (x0, y0) pairs, from
 * device pressure fields of nx*ny doubles: phi^n, phi^{n-1}, the residual r of
 * the extrapolated guess, phi^{n+1} (the scales are over the whole grid). */
int ibm_cnn_prepare(ibm_cnn* net, int32_t nx, int32_t ny, const double* d_phi_n, const double* d_phi_nm1,
                    const double* d_r, const double* d_phi_np1, int32_t ncrop, const int32_t* h_crop_xy,
                    int32_t crop_h, int32_t crop_w, float* d_in, float* d_target);
/* Restricts the warm start's inference to the cells [x0, x0+w) x [y0, y0+h)
 * (w and h multiples of 2^(levels-1); the network's correction is zero
 * outside, the inputs are still scaled over the whole grid); w = h = 0 uses
 * the whole grid (the default).  Not in the paper. */
int ibm_cnn_set_window(ibm_cnn* net, int32_t x0, int32_t y0, int32_t w, int32_t h);
/* Uses `net` (bound on the context's stream, pixel capacity >= nx*ny, or >=
 * w*h with a window) for the IBM_WARM_CNN warm start; NULL detaches. */
int ibm_attach_cnn(ibm_ctx* ctx, ibm_cnn* net);
/* Device copies (each nullable, n_lambda doubles) of lambda^{n+1}, lambda^n
 * (kept with IBM_WARM_EXTRAP and IBM_WARM_CNN), the right-hand side of the last
 * Poisson solve and the residual of its extrapolated guess: training data for
 * the warm-start network.  The residual is recorded from the first call on
 * (IBM_WARM_EXTRAP computes it only for contexts that take snapshots). */
int ibm_snapshot(ibm_ctx* ctx, double* d_lambda, double* d_lambda_prev, double* d_rhs, double* d_r0);

/* ---- instrumentation ------------------------------------------------------------*/
/* Per-kernel CUDA-event timing on the library's stream (off by default). */
int ibm_profile_enable(ibm_ctx* ctx, int32_t on);
int ibm_profile_reset(ibm_ctx* ctx);
/* Number of kernel classes, and for class k its name, launches, summed
 * device milliseconds (timed only while enabled) and summed algorithmic bytes
 * (every element a launch must read or write once) since the last reset. */
int ibm_profile_count(const ibm_ctx* ctx, int32_t* nclasses);
int ibm_profile_get(ibm_ctx* ctx, int32_t k, const char** name, int64_t* launches,
                    double* ms, double* bytes);
/* Graph-mode time of one kernel class (k as in ibm_profile_get): runs one
 * more time step (ibm_step with one step, graphs on), during which every
 * launch of class k is also captured, in order, into a CUDA graph on a side
 * stream; that graph is then replayed `reps` times back to back (after one
 * untimed replay) between CUDA events on the side stream.  Outputs: launches
 * in the graph, mean device milliseconds and algorithmic bytes per launch.
 * The solver scalars are saved and restored around the replays, but the
 * replays overwrite the work vectors (and, for the update classes, the
 * solution): call it last on a context, after the steps that matter.
 * IBM_ERR_STATE when the step issued no launch of class k. */
int ibm_profile_graph_class(ibm_ctx* ctx, int32_t k, int32_t reps, int64_t* launches,
                            double* ms_per_launch, double* bytes_per_launch);
/* Host<->device bytes the library has copied since creation. */
int ibm_transfer_bytes(const ibm_ctx* ctx, int64_t* h2d, int64_t* d2h);
/* Kernels launched by the library since creation (all classes). */
int ibm_launch_count(const ibm_ctx* ctx, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* IBM_H */

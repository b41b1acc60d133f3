// C ABI of the library (include/ibm.h): context, workspace carving, the time
// step of Eq. 9a-c, the CG / flexible-CG drivers and the AMG V-cycle.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ibm.h"
#include "host.h"
#include "kernels.h"

using namespace ibm;

namespace {

// Bump allocator over the caller's workspace; measures when base is null.
struct Carver {
    char* base = nullptr;
    size_t off = 0;
    template <class T>
    T* take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += std::max<size_t>(n, 1) * sizeof(T);
        return p;
    }
};

template <class T>
struct DCsr {
    long long n = 0, nnz = 0;
    long long* ptr = nullptr;
    int* col = nullptr;
    T* val = nullptr;
    CsrView<T> view() const { return CsrView<T>{n, ptr, col, val, nnz}; }
};

template <class T>
struct DSell {
    long long n = 0, nslices = 0, entries = 0, nnz = 0;   // entries: stored (padded), nnz: of the operator
    long long* off = nullptr;
    int* col = nullptr;
    T* val = nullptr;
    SellView<T> view() const { return SellView<T>{n, nslices, off, col, val, entries}; }
};

struct DevLevel {
    long long n = 0;
    DSell<double> A64, P64, R64, Q64;
    DSell<float> A32, P32, R32, Q32;
    DCsr<double> Rt64;                          // wide rows: CSR, several lanes per row
    DCsr<float> Rt32;
    std::vector<long long> offA, offP, offR, offQ;   // host copies of the slice offsets
    bool fused = false;                         // Rt and Q present (fused_transfers)
    double* id64 = nullptr;
    float* id32 = nullptr;
    void* b = nullptr;
    void* x = nullptr;
    void* x2 = nullptr;
    void* r = nullptr;
};

enum ProfClass {
    PC_OUTFLOW, PC_RHS, PC_VEL_SPMV, PC_VEL_UPDATE, PC_VEL_PUPDATE, PC_PW_PRECOND, PC_POIS_SPMV, PC_POIS_COUPLING,
    PC_POIS_UPDATE, PC_POIS_RHS, PC_PROJECT, PC_FORCES, PC_VC_SMOOTH0, PC_VC_COUPLING0, PC_VC_RESTRICT,
    PC_VC_PROLONG, PC_VC_CSR, PC_VC_COARSEST, PC_SCHUR, PC_SCHUR_SETUP, PC_POIS_PUPDATE, PC_VC_TAIL, PC_CONSTRAINTS,
    PC_VC_POST0, PC_VC_COOP, PC_BODY, PC_VC_DOWN, PC_VC_UP, PC_WARM, PC_VEL_RESID, PC_COUNT
};
const char* kProfNames[PC_COUNT] = {
    "outflow", "rhs", "vel_spmv", "vel_update", "vel_pupdate", "pw_precond", "pois_spmv", "pois_coupling",
    "pois_update", "pois_rhs", "project", "forces", "vc_smooth0", "vc_coupling0", "vc_restrict",
    "vc_prolong", "vc_csr", "vc_coarsest", "schur", "schur_setup", "pois_pupdate", "vc_tail", "constraints", "vc_post0",
    "vc_coop", "body", "vc_down", "vc_up", "warm", "vel_resid"};

}  // namespace

struct ibm_ctx {
    ibm_config cfg{};
    Grid g;
    int n_b = 0;
    long long nc = 0, nl = 0;     // cells, lambda unknowns
    int64_t nq = 0;               // interior velocity unknowns
    int64_t pin = 0;
    VelocityCoeffs vc;
    PoissonCoeffs pc;
    BodyRows br;
    Hierarchy H;
    bool have_H = false;
    bool amg_stale = false;
    int steps_since_amg = 0;
    std::vector<double> xb, yb, ub, vb;
    // boundary values (host copies of the constant ones)
    std::vector<double> u_left, v_bottom, v_top, u_bottom, u_top, v_left, u_right0, v_right0;
    double inflow = 0.0, ly = 0.0;
    double t = 0.0;
    int64_t step = 0;
    bool ab2_first = true;
    std::string err;

    // ---- device
    bool bound = false;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t st = nullptr;
    int grid = 0;
    int sm_count = 0;
    int device = -1;              // CUDA device current at ibm_bind_workspace
    dim3 g_vel, g_pois;           // 2D shapes of the 5-point kernels
    int nb_vel = 0, nb_pois = 0;  // their block counts (reduction slots)
    size_t fixed_bytes = 0, body_cap = 0, hier_cap = 0;
    size_t body_off = 0, hier_off = 0;
    size_t green_off = 0, green_cap = 0;
    // grid
    double *dx = nullptr, *dy = nullptr, *idx = nullptr, *idy = nullptr, *dxf = nullptr, *dyf = nullptr,
           *idxf = nullptr, *idyf = nullptr;
    // velocity
    double *vcE = nullptr, *vcN = nullptr, *vdiag = nullptr, *vidiag = nullptr, *vmdt = nullptr;
    // mixed precision: the velocity operator in FP32 and the inner solve's vectors
    float *vcE32 = nullptr, *vcN32 = nullptr, *vdiag32 = nullptr, *vidiag32 = nullptr;
    float *ve32 = nullptr, *vr32 = nullptr, *vp32 = nullptr, *vq32 = nullptr, *vz32 = nullptr;
    double *q = nullptr, *qs = nullptr, *r1 = nullptr, *vr = nullptr, *vp = nullptr, *vAp = nullptr, *vz = nullptr;
    double* Nbuf[2] = {nullptr, nullptr};
    int ncur = 0;
    // poisson
    double *pwE = nullptr, *pwN = nullptr, *pdiag = nullptr, *pidiag = nullptr;
    float *pwE32 = nullptr, *pwN32 = nullptr, *pdiag32 = nullptr, *pidiag32 = nullptr;
    float *sep_ax = nullptr, *sep_ay = nullptr, *sep_bx = nullptr, *sep_by = nullptr;   // FP32 pressure links
    float* b32 = nullptr;         // FP32 copy of the V-cycle right-hand side on the finest level
    int* d_flag = nullptr;        // device status word (non-positive pivot of the Schur inverse)
    double* gj = nullptr;         // scratch of the Schur inverse
    // Moving bodies with the Schur preconditioner: the pressure V-cycle V never
    // changes and is symmetric, so its responses to unit vectors at the cells the
    // body rows touch (G[u][v] = (V e_v)_u) stay valid; S = F - C^T G C is then
    // rebuilt from them, and only cells the body reaches for the first time cost
    // a V-cycle.
    int ucap = 0, nu = 0;         // capacity and number of cached cells
    void* G = nullptr;            // ucap x ucap, FP32 (mixed) or FP64
    int* d_slot = nullptr;        // nc: cache slot of a cell or -1
    long long* d_cell = nullptr;  // ucap: cell of a slot
    long long* d_fresh = nullptr; // ucap: staging of (cell, slot) pairs
    std::vector<int> h_slot;
    std::vector<long long> h_cell;
    int64_t cache_fresh = 0;      // V-cycles spent on cache columns
    double *lam = nullptr, *b2 = nullptr, *pr = nullptr, *pp = nullptr, *pq = nullptr, *pz = nullptr;
    double* lam_prev = nullptr;   // lambda^{n-1} (extrapolated warm start)
    double* r_ex = nullptr;       // residual of the extrapolated warm start (last step)
    int64_t lam_steps = 0;        // steps whose lambda is held in lam (0, 1, >= 2)
    // warm start of the Poisson solve by projection onto previous solutions
    // (IBM_WARM_PROJ): a K-orthonormal basis of at most kProjMax solutions and
    // their images
    struct ProjBasis {
        double* X = nullptr;      // kProjMax x n
        double* KX = nullptr;     // kProjMax x n
        long long n = 0;
        int m = 0;                // basis vectors held
        int64_t solves = 0;       // solves seen (the basis takes every kProjEvery-th)
    };
    ProjBasis proj_pois;
    double* proj_part = nullptr;  // kProjMax x kProjBlocks partial sums
    double* proj_coef = nullptr;  // kProjMax + 2 coefficients
    // boundaries
    double *d_u_left = nullptr, *d_v_bottom = nullptr, *d_v_top = nullptr, *d_u_bottom = nullptr,
           *d_u_top = nullptr, *d_v_left = nullptr;
    double* d_u_right[2] = {nullptr, nullptr};
    double* d_v_right[2] = {nullptr, nullptr};
    int bcur = 0;
    // body
    double* d_ub = nullptr;
    // device-side body rows of a moving body: grid coordinates, point
    // positions, and the index maps of the host pattern (BodySrc)
    double *d_xf = nullptr, *d_yf = nullptr, *d_xc = nullptr, *d_yc = nullptr, *d_xb = nullptr, *d_yb = nullptr;
    int *d_point = nullptr, *d_et_src = nullptr, *d_cf_a = nullptr, *d_cf_b = nullptr, *d_cc_src = nullptr,
        *d_diag_idx = nullptr;
    BodySrc bsrc;
    BodyMaps bmaps;
    double body_host_ms = 0.0;    // host time of the last ibm_set_body (pattern or assembly, uploads)
    double* d_forces = nullptr;
    DCsr<double> E, ET;
    int* d_faces = nullptr;
    int nfaces = 0;
    double bn_dpin = 0.0;          // pinned diagonal of the matrix-free Q^T B^N Q
    bool bn_dpin_ok = false;
    long long* d_tcell = nullptr;
    DCsr<double> Cc64, Cf64;
    DCsr<float> Cc32, Cf32;
    // scalars
    CgScalars* sc1 = nullptr;
    CgScalars* sc1i = nullptr;    // inner FP32 solve of the mixed-precision velocity solve
    CgScalars* sc2 = nullptr;
    double* part1 = nullptr;
    double* part2 = nullptr;
    CgScalars* hsc = nullptr;     // pinned host mirror
    double* hforces = nullptr;    // pinned host mirror of the force sums
    // AMG
    std::vector<DevLevel> lev;
    double* d_coarse_inv = nullptr;
    GridBarrier* gbar = nullptr;  // grid barrier of the cooperative coarse-level kernel
    int coop_blocks = 0;          // its grid (0: cooperative launch unavailable or off)
    // per first level l0 (0 or 1) of the cooperative kernel: its device level
    // table, the staged-operator mask and shared memory per block
    void* coop_tab[2] = {nullptr, nullptr};
    unsigned coop_staged[2] = {0u, 0u};
    long long coop_smem[2] = {0, 0};
    long long coop_smem_max = 0;   // the kernel's dynamic shared memory attribute
    int tail_start = -1;          // first level run by the cluster kernel (-1: none)
    int tail_cluster = 0;         // its cluster size
    long long tail_smem = 0;      // > 0: the staged variant with this much shared memory per block
    int coarse_n = 0;
    void *x0a = nullptr, *x0b = nullptr, *r0 = nullptr;
    // Schur-complement block preconditioner
    void* y1 = nullptr;           // V r_p (level type)
    double* s_full = nullptr;     // C z_f on the touched cells, zero elsewhere
    double* tf = nullptr;         // r_f - C^T y1
    double* Sinv64 = nullptr;     // S^-1, dense 2 n_b square (also scratch for S)
    // moving bodies in mixed precision: S^-1 inverted in FP32 (Sinv64 keeps S)
    // and applied with one step of FP64 refinement
    float* Sinv32 = nullptr;
    double* zf0 = nullptr;        // 2 n_b: X t_f
    double* rtf = nullptr;        // 2 n_b: t_f - S X t_f
    bool schur_refine = false;    // the last build inverted S in FP32
    double schur_rho = 0.0;       // ||v - S X v|| / ||v|| of that FP32 inverse
    bool schur_stale = true;
    bool schur_built = false;
    int64_t schur_builds = 0;
    int steps_since_schur = 0;
    double schur_ms = 0.0;
    // solver predictions
    int pred1 = 8, pred2 = 8, pred1i = 8;
    // instrumentation
    bool prof_on = false;
    int64_t launches = 0;
    int64_t prof_launch[PC_COUNT] = {0};
    double prof_ms[PC_COUNT] = {0};
    double prof_bytes[PC_COUNT] = {0};
    int64_t h2d_bytes = 0, d2h_bytes = 0;
    double bytes_total = 0.0;     // algorithmic bytes of every launch (graph bodies counted per iteration)
    cudaEvent_t ev_pois[2] = {nullptr, nullptr};   // around the Poisson solve of a step
    // graph-mode timing of one kernel class (ibm_profile_graph_class): launches
    // of class gprof_cls are also captured, in order, on gprof_st
    int gprof_cls = -1;
    cudaStream_t gprof_st = nullptr;
    int64_t gprof_n = 0;
    double gprof_bytes = 0.0;
    std::vector<cudaEvent_t> ev;
    std::vector<std::pair<int, int>> ev_pending;   // (first event index, class)
    int ev_next = 0;

    ibm_solve_stats last1{}, last2{};

    // device-side iteration loops (CUDA graphs with a conditional while node)
    struct LoopGraph {
        cudaGraphExec_t exec = nullptr;
        int64_t version = -1;
        int64_t nk = 0;          // kernels per loop body (loop_unroll iterations + the condition)
        double bytes = 0.0;      // algorithmic bytes of one loop body
        const void* kx = nullptr;  // solution / right-hand side the body was captured for
        const void* kb = nullptr;
    };
    LoopGraph lg_vel, lg_pois, lg_vel32;
    int loop_unroll = 2;         // solver iterations per body of the device-side loop
    int64_t graph_version = 0;   // bumped whenever device pointers or sizes change
    bool use_graphs = true;
    cudaStream_t cap_st = nullptr;
    ibm_cnn* cnn = nullptr;       // learned warm start (IBM_WARM_CNN)
    bool snapshots = false;       // keep r0 of the extrapolated guess (training data)
};

namespace {

int fail(ibm_ctx* c, int code, const std::string& m) {
    if (c) c->err = m;
    return code;
}

#define CUDA_OK(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(c, IBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool is_mixed(const ibm_ctx* c) { return c->cfg.precision == IBM_PREC_MIXED; }
bool use_amg(const ibm_ctx* c) {
    return c->cfg.poisson_precond == IBM_PRECOND_AMG || c->cfg.poisson_precond == IBM_PRECOND_SCHUR;
}
bool use_schur(const ibm_ctx* c) { return c->cfg.poisson_precond == IBM_PRECOND_SCHUR; }
// B^N with N > 1 and the coupled AMG preconditioner: the Poisson operator is
// the assembled Q^T B^N Q (level 0 of the coupled hierarchy, FP64 sliced
// ELLPACK) instead of the 5-point stencil with the body rows
bool use_bn(const ibm_ctx* c) { return c->cfg.bn_order > 1 && !use_schur(c); }
// B^N with N > 1 and the Schur preconditioner: Q^T B^N Q applied without
// assembly (the projection chain of Eq. 9c on x, then Q^T), preconditioned
// by the Schur block preconditioner of Q^T B^1 Q
bool bn_mf(const ibm_ctx* c) { return c->cfg.bn_order > 1 && use_schur(c); }
// the N - 1 further terms of the projection (either form)
bool bn_terms(const ibm_ctx* c) { return c->cfg.bn_order > 1; }

// ---- profiling -----------------------------------------------------------------
void prof_harvest(ibm_ctx* c) {
    if (c->ev_pending.empty()) return;
    cudaEventSynchronize(c->ev[c->ev_pending.back().first + 1]);
    for (auto& pr : c->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[pr.first], c->ev[pr.first + 1]) == cudaSuccess)
            c->prof_ms[pr.second] += ms;
    }
    c->ev_pending.clear();
    c->ev_next = 0;
}

template <class F>
void L(ibm_ctx* c, int cls, int nk, double bytes, F&& f) {
    int e0 = -1;
    if (c->prof_on && !c->ev.empty()) {
        if (c->ev_next + 2 > int(c->ev.size())) prof_harvest(c);
        e0 = c->ev_next;
        c->ev_next += 2;
        cudaEventRecord(c->ev[e0], c->st);
    }
    if (c->gprof_cls == cls) {   // the same launch, captured for the graph-mode timing of this class
        cudaStream_t keep = c->st;
        c->st = c->gprof_st;
        f();
        c->st = keep;
        c->gprof_n += nk;
        c->gprof_bytes += bytes;
    }
    f();
    if (e0 >= 0) {
        cudaEventRecord(c->ev[e0 + 1], c->st);
        c->ev_pending.emplace_back(e0, cls);
    }
    c->bytes_total += bytes;
    c->launches += nk;
    c->prof_launch[cls] += nk;
    c->prof_bytes[cls] += bytes;
}

// Algorithmic (compulsory) bytes of one launch: every array element the
// kernel must read or write once; coefficient arrays count, neighbour
// re-reads do not.
double st_bytes(int mode, int dk, size_t ts, size_t tb, size_t ty, long long n, bool base = false) {
    double b = 0.0;
    switch (mode) {
        case MODE_APPLY: b = ts + 3.0 * ts + ty; break;
        case MODE_RESID: b = ts + tb + 3.0 * ts + ty; break;
        case MODE_JAC: b = ts + tb + 4.0 * ts + ty; break;
        case MODE_JAC0: b = tb + ts + ty; break;
        default: break;
    }
    if (dk == DK_ZR) b += 16.0 + (base ? double(ts) : 0.0);
    return b * double(n);
}
double csr_bytes(long long n, long long nnz, size_t ts) { return 8.0 * double(n + 1) + double(nnz) * (4.0 + ts); }
// algorithmic bytes of a sliced-ELLPACK operator: its nonzeros (padding not counted) and slice offsets
template <class T>
double sell_bytes(const DSell<T>& d) { return 8.0 * double(d.nslices + 1) + double(d.nnz) * (4.0 + sizeof(T)); }

// ---- device views ---------------------------------------------------------------
GridView gview(const ibm_ctx* c) {
    return GridView{c->g.nx, c->g.ny, c->nc, c->dx, c->dy, c->idx, c->idy, c->dxf, c->dyf, c->idxf, c->idyf};
}
BoundaryView bview(const ibm_ctx* c) {
    const int n = c->bcur, m = 1 - c->bcur;
    return BoundaryView{c->d_u_left, c->d_u_right[n], c->d_u_right[m], c->d_v_bottom, c->d_v_top,
                        c->d_u_bottom, c->d_u_top, c->d_v_left, c->d_v_right[n], c->d_v_right[m]};
}
Stencil<double> vel_stencil(const ibm_ctx* c) {
    return Stencil<double>{c->g.nx, c->g.ny, 2, c->nc, c->vcE, c->vcN, c->vdiag, c->vidiag};
}
template <class T> Stencil<T> pois_stencil(const ibm_ctx* c);
template <> Stencil<double> pois_stencil<double>(const ibm_ctx* c) {
    return Stencil<double>{c->g.nx, c->g.ny, 1, c->nc, c->pwE, c->pwN, c->pdiag, c->pidiag};
}
template <> Stencil<float> pois_stencil<float>(const ibm_ctx* c) {
    return Stencil<float>{c->g.nx, c->g.ny, 1, c->nc, c->pwE32, c->pwN32, c->pdiag32, c->pidiag32};
}
template <class T> Coupling<T> pois_coupling(const ibm_ctx* c);
template <> Coupling<double> pois_coupling<double>(const ibm_ctx* c) {
    return Coupling<double>{int(c->Cc64.n), c->d_tcell, c->Cc64.ptr, c->Cc64.col, c->Cc64.val,
                            int(c->Cf64.n), c->nc, c->Cf64.ptr, c->Cf64.col, c->Cf64.val, c->pidiag + c->nc};
}
template <> Coupling<float> pois_coupling<float>(const ibm_ctx* c) {
    return Coupling<float>{int(c->Cc32.n), c->d_tcell, c->Cc32.ptr, c->Cc32.col, c->Cc32.val,
                           int(c->Cf32.n), c->nc, c->Cf32.ptr, c->Cf32.col, c->Cf32.val, c->pidiag32 + c->nc};
}
template <class T> const T* pois_idiag(const ibm_ctx* c);
template <> const double* pois_idiag<double>(const ibm_ctx* c) { return c->pidiag; }
template <> const float* pois_idiag<float>(const ibm_ctx* c) { return c->pidiag32; }

// touched cells padded to whole warps, then a warp per force row
int coupling_grid(const ibm_ctx* c) { return grid_for((c->Cc64.n + 31) / 32 * 32 + 32 * c->Cf64.n, kThreads, 512); }

// ---- uploads ----------------------------------------------------------------------
template <class T>
int up(ibm_ctx* c, T* dst, const T* src, size_t n) {
    if (n == 0) return IBM_OK;
    CUDA_OK(cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, c->st));
    c->h2d_bytes += int64_t(n * sizeof(T));
    return IBM_OK;
}
template <class T>
int up(ibm_ctx* c, T* dst, const std::vector<T>& v) { return up(c, dst, v.data(), v.size()); }

std::vector<float> to32(const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); }

template <class T>
void carve_csr(Carver& cv, DCsr<T>& d, long long n, long long nnz) {
    d.n = n;
    d.nnz = nnz;
    d.ptr = cv.take<long long>(n + 1);
    d.col = cv.take<int>(nnz);
    d.val = cv.take<T>(nnz);
}
template <class T>
void carve_sell(Carver& cv, DSell<T>& d, const CSR& h) {
    d.n = h.n;
    d.nslices = (h.n + kSellRows - 1) / kSellRows;
    d.entries = sell_entries(h);
    d.nnz = h.nnz();
    d.off = cv.take<long long>(d.nslices + 1);
    d.col = cv.take<int>(d.entries);
    d.val = cv.take<T>(d.entries);
}
// a second value array that shares ptr/col with an existing CSR
template <class T, class U>
void carve_vals(Carver& cv, DCsr<T>& d, const DCsr<U>& s) {
    d.n = s.n;
    d.nnz = s.nnz;
    d.ptr = s.ptr;
    d.col = s.col;
    d.val = cv.take<T>(s.nnz);
}
template <class T>
int up_csr(ibm_ctx* c, DCsr<T>& d, const CSR& h, bool vals_only = false) {
    int rc;
    if (!vals_only) {
        std::vector<long long> rp(h.rowptr.begin(), h.rowptr.end());
        if ((rc = up(c, d.ptr, rp))) return rc;
        if ((rc = up(c, d.col, h.col))) return rc;
    }
    if constexpr (std::is_same<T, double>::value) return up(c, d.val, h.val);
    else {
        std::vector<float> f = to32(h.val);
        return up(c, d.val, f);
    }
}

// ---- body rows: carve + upload -------------------------------------------------------
size_t carve_body(ibm_ctx* c, Carver& cv, const BodyRows& br) {
    const size_t start = cv.off;
    carve_csr(cv, c->E, br.E.n, br.E.nnz());
    carve_csr(cv, c->ET, br.ET.n, br.ET.nnz());
    c->d_faces = cv.take<int>(br.faces.size());
    c->nfaces = int(br.faces.size());
    c->d_tcell = cv.take<long long>(br.tcells.size());
    carve_csr(cv, c->Cc64, br.Cc.n, br.Cc.nnz());
    carve_csr(cv, c->Cf64, br.Cf.n, br.Cf.nnz());
    // index maps of the device-side assembly (same sizes as the structure)
    c->d_point = cv.take<int>(br.E.n);
    c->d_et_src = cv.take<int>(br.ET.nnz());
    c->d_cf_a = cv.take<int>(br.Cf.nnz());
    c->d_cf_b = cv.take<int>(br.Cf.nnz());
    c->d_cc_src = cv.take<int>(br.Cc.nnz());
    c->d_diag_idx = cv.take<int>(br.Cf.n);
    if (is_mixed(c)) {
        carve_vals(cv, c->Cc32, c->Cc64);
        carve_vals(cv, c->Cf32, c->Cf64);
    } else {
        c->Cc32 = DCsr<float>{};
        c->Cf32 = DCsr<float>{};
    }
    return cv.off - start;
}

int upload_body(ibm_ctx* c) {
    c->graph_version++;
    Carver cv{c->ws, c->body_off};
    const size_t used = carve_body(c, cv, c->br);
    if (used > c->body_cap)
        return fail(c, IBM_ERR_NO_MEM, "body rows outgrew their workspace reservation");
    int rc;
    if ((rc = up_csr(c, c->E, c->br.E))) return rc;
    if ((rc = up_csr(c, c->ET, c->br.ET))) return rc;
    std::vector<int> faces(c->br.faces.begin(), c->br.faces.end());
    if ((rc = up(c, c->d_faces, faces))) return rc;
    std::vector<long long> tc(c->br.tcells.begin(), c->br.tcells.end());
    if ((rc = up(c, c->d_tcell, tc))) return rc;
    if ((rc = up_csr(c, c->Cc64, c->br.Cc))) return rc;
    if ((rc = up_csr(c, c->Cf64, c->br.Cf))) return rc;
    if (is_mixed(c)) {
        if ((rc = up_csr(c, c->Cc32, c->br.Cc, true))) return rc;
        if ((rc = up_csr(c, c->Cf32, c->br.Cf, true))) return rc;
    }
    // diagonal of the force rows (and its inverse)
    const long long nf = 2LL * c->n_b;
    if (nf > 0) {
        std::vector<double> d(c->pc.diag.begin() + c->nc, c->pc.diag.end()), id(nf);
        for (long long k = 0; k < nf; ++k) id[k] = 1.0 / d[k];
        if ((rc = up(c, c->pdiag + c->nc, d))) return rc;
        if ((rc = up(c, c->pidiag + c->nc, id))) return rc;
        if (is_mixed(c)) {
            if ((rc = up(c, c->pdiag32 + c->nc, to32(d)))) return rc;
            if ((rc = up(c, c->pidiag32 + c->nc, to32(id)))) return rc;
        }
    }
    return IBM_OK;
}

// Body rows assembled on the device from the host pattern (c->br holds the
// structure, c->bsrc the index maps): structure and maps uploaded, values,
// the force-row diagonal and its inverse (FP64, FP32 copies) formed by kernels.
int upload_body_device(ibm_ctx* c, const double* xb, const double* yb) {
    c->graph_version++;
    Carver cv{c->ws, c->body_off};
    const size_t used = carve_body(c, cv, c->br);
    if (used > c->body_cap)
        return fail(c, IBM_ERR_NO_MEM, "body rows outgrew their workspace reservation");
    int rc;
    auto up_pattern = [&](DCsr<double>& d, const CSR& h) {
        std::vector<long long> rp(h.rowptr.begin(), h.rowptr.end());
        int r = up(c, d.ptr, rp);
        return r ? r : up(c, d.col, h.col);
    };
    if ((rc = up_pattern(c->E, c->br.E)) || (rc = up_pattern(c->ET, c->br.ET)) ||
        (rc = up_pattern(c->Cc64, c->br.Cc)) || (rc = up_pattern(c->Cf64, c->br.Cf)))
        return rc;
    std::vector<int> faces(c->br.faces.begin(), c->br.faces.end());
    std::vector<long long> tc(c->br.tcells.begin(), c->br.tcells.end());
    if ((rc = up(c, c->d_faces, faces)) || (rc = up(c, c->d_tcell, tc)) || (rc = up(c, c->d_point, c->bsrc.point)) ||
        (rc = up(c, c->d_et_src, c->bsrc.et_src)) || (rc = up(c, c->d_cf_a, c->bsrc.cf_a)) ||
        (rc = up(c, c->d_cf_b, c->bsrc.cf_b)) || (rc = up(c, c->d_cc_src, c->bsrc.cc_src)) ||
        (rc = up(c, c->d_diag_idx, c->bsrc.diag)) || (rc = up(c, c->d_xb, xb, size_t(c->n_b))) ||
        (rc = up(c, c->d_yb, yb, size_t(c->n_b))))
        return rc;
    BodyGeo g{c->g.nx, c->g.ny, c->nc, c->cfg.h, c->cfg.dt, c->d_xf, c->d_yf, c->d_xc, c->d_yc, c->dx, c->dy,
              c->dxf, c->dyf, c->idxf, c->idyf};
    BodyDev b{};
    b.E = c->E.view();
    b.ET = c->ET.view();
    b.Cc = c->Cc64.view();
    b.Cf = c->Cf64.view();
    b.Ev = c->E.val;
    b.ETv = c->ET.val;
    b.Ccv = c->Cc64.val;
    b.Cfv = c->Cf64.val;
    b.Cc32 = is_mixed(c) ? c->Cc32.val : nullptr;
    b.Cf32 = is_mixed(c) ? c->Cf32.val : nullptr;
    b.point = c->d_point;
    b.et_src = c->d_et_src;
    b.cf_a = c->d_cf_a;
    b.cf_b = c->d_cf_b;
    b.cc_src = c->d_cc_src;
    b.diag = c->d_diag_idx;
    b.xb = c->d_xb;
    b.yb = c->d_yb;
    b.pdiag = c->pdiag;
    b.pidiag = c->pidiag;
    b.pdiag32 = is_mixed(c) ? c->pdiag32 : nullptr;
    b.pidiag32 = is_mixed(c) ? c->pidiag32 : nullptr;
    L(c, PC_BODY, 3, 0.0, [&] { launch_body_values(g, b, c->st); });
    return IBM_OK;
}

template <class T>
int up_sell(ibm_ctx* c, DSell<T>& d, const CSR& h, std::vector<long long>* host_off) {
    const Sell S = to_sell(h);
    if (S.nslices != d.nslices || int64_t(S.col.size()) != d.entries) return IBM_ERR_STATE;
    std::vector<long long> off(S.off.begin(), S.off.end());
    *host_off = off;
    int rc;
    if ((rc = up(c, d.off, off))) return rc;
    if ((rc = up(c, d.col, S.col))) return rc;
    if constexpr (std::is_same<T, double>::value) return up(c, d.val, S.val);
    else return up(c, d.val, to32(S.val));
}

// ---- response cache (moving bodies, Schur preconditioner) ------------------------------
void carve_green(ibm_ctx* c, Carver& cv) {
    if (c->ucap <= 0) return;
    const size_t ts = is_mixed(c) ? sizeof(float) : sizeof(double);
    c->G = cv.take<char>(size_t(c->ucap) * size_t(c->ucap) * ts);
    c->d_slot = cv.take<int>(c->nc);
    c->d_cell = cv.take<long long>(c->ucap);
    c->d_fresh = cv.take<long long>(2 * size_t(c->ucap));
}

// ---- hierarchy: carve + upload ---------------------------------------------------------
size_t carve_hier(ibm_ctx* c, Carver& cv, const Hierarchy& H) {
    const size_t start = cv.off;
    const bool mixed = is_mixed(c);
    const size_t vsz = mixed ? sizeof(float) : sizeof(double);
    const int Lv = int(H.levels.size());
    c->lev.assign(Lv, DevLevel{});
    for (int l = 0; l < Lv; ++l) {
        const AmgLevel& h = H.levels[l];
        DevLevel& d = c->lev[l];
        d.n = h.A.n;
        if (l > 0 || use_bn(c)) {
            if (mixed) carve_sell(cv, d.A32, h.A);
            if (!mixed || l == 0) carve_sell(cv, d.A64, h.A);   // level 0: the Poisson operator
            if (mixed) d.id32 = cv.take<float>(h.A.n);
            else d.id64 = cv.take<double>(h.A.n);
            d.b = cv.take<char>(h.A.n * vsz);
        }
        d.x = cv.take<char>(h.A.n * vsz);
        d.x2 = cv.take<char>(h.A.n * vsz);
        d.r = cv.take<char>(h.A.n * vsz);
        if (l + 1 < Lv) {
            if (mixed) {
                carve_sell(cv, d.P32, h.P);
                carve_sell(cv, d.R32, h.R);
            } else {
                carve_sell(cv, d.P64, h.P);
                carve_sell(cv, d.R64, h.R);
            }
        }
        d.fused = l > 0 && l + 1 < Lv && h.Rt.n > 0 && h.Q.n > 0;
        if (d.fused) {
            if (mixed) {
                carve_csr(cv, d.Rt32, h.Rt.n, h.Rt.nnz());
                carve_sell(cv, d.Q32, h.Q);
            } else {
                carve_csr(cv, d.Rt64, h.Rt.n, h.Rt.nnz());
                carve_sell(cv, d.Q64, h.Q);
            }
        }
    }
    c->d_coarse_inv = cv.take<double>(H.coarse_n * H.coarse_n);
    for (auto& t : c->coop_tab) t = cv.take<char>(sizeof(CoopTable<double>));
    c->coarse_n = int(H.coarse_n);
    return cv.off - start;
}

template <class T> DSell<T>& levA(DevLevel& d);
template <class T> DSell<T>& levP(DevLevel& d);
template <class T> DSell<T>& levR(DevLevel& d);
template <class T> T* levId(DevLevel& d);

// The cooperative coarse-level kernel: its grid (two blocks of kCoopThreads
// per SM), for each first level l0 in {0, 1} the device table of its levels
// and the operators it stages in shared memory - the coarsest levels' A, R, P
// first, then finer ones while a block's share fits the budget.
template <class T>
int setup_coop(ibm_ctx* c) {
    const int Lv = int(c->lev.size());
    int dev = 0;
    CUDA_OK(cudaGetDevice(&dev));
    int sms = 0;
    CUDA_OK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int per_sm0 = coop_blocks_per_sm<T>(dev, 0);
    if (per_sm0 < 1) return IBM_OK;   // no cooperative launch: per-level kernels
    const int grid = sms * std::min(per_sm0, 2);
    const long long budget = 100 * 1024;
    c->coop_smem_max = 0;
    for (int l0 = 0; l0 <= 1 && l0 < Lv; ++l0) {
        // candidates in kernel order (A, R, P of each level), chosen coarse to fine
        const int nk = Lv - 1 - l0;   // levels with operators in the kernel
        std::vector<const std::vector<long long>*> offs(3 * size_t(std::max(nk, 0)), nullptr);
        std::vector<size_t> tsz(offs.size(), sizeof(T));
        unsigned mask = 0u;
        long long bytes = 0;
        for (int l = Lv - 2; l >= l0; --l) {
            const int k = l - l0;
            const std::vector<long long>* cand[3] = {&c->lev[l].offA, &c->lev[l].offR, &c->lev[l].offP};
            for (int m = 0; m < 3; ++m) {
                if (cand[m]->size() < 2) continue;
                offs[3 * k + m] = cand[m];
                const long long b = coop_staged_bytes(offs, tsz, grid);
                if (b <= budget) {
                    mask |= 1u << (3 * k + m);
                    bytes = b;
                } else {
                    offs[3 * k + m] = nullptr;
                }
            }
        }
        if (std::getenv("IBM_COOP_NOSTAGE")) {
            mask = 0u;
            bytes = 0;
        }
        if (bytes > 0 && coop_blocks_per_sm<T>(dev, bytes) * sms < grid) {   // staging would not fit the grid
            mask = 0u;
            bytes = 0;
        }
        c->coop_staged[l0] = mask;
        c->coop_smem[l0] = bytes;
        c->coop_smem_max = std::max(c->coop_smem_max, bytes);
        CoopTable<T> tab{};
        for (int l = l0; l < Lv; ++l) {
            DevLevel& d = c->lev[l];
            CoopLevel<T>& t = tab.lev[l - l0];
            t.b = static_cast<T*>(d.b);
            t.x = static_cast<T*>(d.x);
            t.x2 = static_cast<T*>(d.x2);
            t.r = static_cast<T*>(d.r);
            if (l + 1 < Lv) {
                t.A = levA<T>(d).view();
                t.P = levP<T>(d).view();
                t.R = levR<T>(d).view();
                t.idiag = levId<T>(d);
                t.omega = T(c->H.levels[l].omega);
            }
        }
        if (l0 >= 1) {
            tab.Rp = levR<T>(c->lev[l0 - 1]).view();
            tab.Pp = levP<T>(c->lev[l0 - 1]).view();
        }
        int rc;
        if ((rc = up(c, static_cast<char*>(c->coop_tab[l0]), reinterpret_cast<const char*>(&tab), sizeof(tab))))
            return rc;
    }
    // one attribute for the kernel: the largest shared memory any launch uses
    if (coop_blocks_per_sm<T>(dev, c->coop_smem_max) * sms < grid) return IBM_OK;   // per-level kernels
    c->coop_blocks = grid;
    return IBM_OK;
}

int upload_hier(ibm_ctx* c) {
    c->graph_version++;
    Carver cv{c->ws, c->hier_off};
    const size_t used = carve_hier(c, cv, c->H);
    if (used > c->hier_cap)
        return fail(c, IBM_ERR_NO_MEM, "AMG hierarchy outgrew its workspace reservation");
    const bool mixed = is_mixed(c);
    int rc;
    for (size_t l = 0; l < c->H.levels.size(); ++l) {
        const AmgLevel& h = c->H.levels[l];
        DevLevel& d = c->lev[l];
        if (l > 0 || use_bn(c)) {
            if (mixed) {
                if ((rc = up_sell(c, d.A32, h.A, &d.offA))) return rc;
                if ((rc = up(c, d.id32, to32(h.invdiag)))) return rc;
            } else {
                if ((rc = up(c, d.id64, h.invdiag))) return rc;
            }
            if ((!mixed || l == 0) && (rc = up_sell(c, d.A64, h.A, &d.offA))) return rc;
        }
        if (l + 1 < c->H.levels.size()) {
            if (mixed) {
                if ((rc = up_sell(c, d.P32, h.P, &d.offP))) return rc;
                if ((rc = up_sell(c, d.R32, h.R, &d.offR))) return rc;
            } else {
                if ((rc = up_sell(c, d.P64, h.P, &d.offP))) return rc;
                if ((rc = up_sell(c, d.R64, h.R, &d.offR))) return rc;
            }
        }
        if (d.fused) {
            if (mixed) {
                if ((rc = up_csr(c, d.Rt32, h.Rt))) return rc;
                if ((rc = up_sell(c, d.Q32, h.Q, &d.offQ))) return rc;
            } else {
                if ((rc = up_csr(c, d.Rt64, h.Rt))) return rc;
                if ((rc = up_sell(c, d.Q64, h.Q, &d.offQ))) return rc;
            }
        }
    }
    c->x0a = c->lev[0].x;
    c->x0b = c->lev[0].x2;
    c->r0 = c->lev[0].r;
    // the levels below amg_tail_rows rows run as one cluster kernel
    c->tail_start = -1;
    const int Lv = int(c->lev.size());
    if (c->cfg.amg_tail_rows > 0 && Lv >= 2) {
        int dev = 0;
        CUDA_OK(cudaGetDevice(&dev));
        c->tail_cluster = mixed ? tail_cluster_size<float>(dev) : tail_cluster_size<double>(dev);
        // IBM_TAIL_CLUSTER=8 takes the portable cluster size (when 16 is available)
        if (const char* e = std::getenv("IBM_TAIL_CLUSTER"))
            if (std::atoi(e) == 8 && c->tail_cluster == 16) c->tail_cluster = 8;
        for (int l = 1; l < Lv && c->tail_cluster > 0; ++l)
            if (c->lev[l].n <= c->cfg.amg_tail_rows && Lv - l <= kMaxTailLevels) {
                c->tail_start = l;
                break;
            }
    }
    // the coarse levels as one cooperative kernel (IBM_COOP=1; measured slower
    // than the per-level kernels on the 1024^2 workload, so not the default)
    c->coop_blocks = 0;
    if (Lv >= 2 && Lv <= kMaxCoopLevels && std::getenv("IBM_COOP")) {
        int rcc = mixed ? setup_coop<float>(c) : setup_coop<double>(c);
        if (rcc) return rcc;
    }
    // stage the tail's operators in shared memory when they fit
    c->tail_smem = 0;
    if (c->tail_start >= 0) {
        std::vector<const std::vector<long long>*> offs;
        for (int l = c->tail_start; l + 1 < Lv; ++l) {
            offs.push_back(&c->lev[l].offA);
            offs.push_back(&c->lev[l].offR);
            offs.push_back(&c->lev[l].offP);
        }
        const size_t ts = mixed ? sizeof(float) : sizeof(double);
        const long long need = tail_staged_bytes(offs, c->coarse_n, c->tail_cluster, ts);
        const bool ok = mixed ? tail_staged_ready<float>(c->tail_cluster, need)
                              : tail_staged_ready<double>(c->tail_cluster, need);
        if (ok && !std::getenv("IBM_TAIL_UNSTAGED")) c->tail_smem = need;
    }
    return up(c, c->d_coarse_inv, c->H.coarse_inv);
}

// The sweeps of levels 1 .. L-2 fold into their transfers (one launch down:
// pre-sweeps from zero and the restricted residual R (I - A w D^-1)^pre b; one
// up: the coarse correction and the first post-sweep) when there are one or
// two pre-sweeps and at least one post-sweep; IBM_NO_FUSED_TRANSFER=1 keeps
// one launch per sweep and transfer.
bool fused_transfers_on(const ibm_ctx* c) {
    static const bool off = std::getenv("IBM_NO_FUSED_TRANSFER") != nullptr;
    return !off && (c->cfg.amg_pre == 1 || c->cfg.amg_pre == 2) && c->cfg.amg_post >= 1;
}

int rebuild_hierarchy(ibm_ctx* c) {
    BodyRows none;
    none.Cc.rowptr.assign(1, 0);
    none.Cf.rowptr.assign(1, 0);
    // the Schur preconditioner coarsens the (fixed) pressure block only
    CSR A0 = use_bn(c)
                 ? assemble_poisson_bn(c->g, c->vc, c->cfg.dt, c->cfg.bn_order, c->pin, c->br, 4096)
                 : assemble_poisson(c->g, c->pc, use_schur(c) ? none : c->br);
    AmgParams prm;
    prm.theta = c->cfg.amg_theta;
    prm.omega = c->cfg.amg_omega;
    prm.pre = c->cfg.amg_pre;
    prm.post = c->cfg.amg_post;
    prm.max_coarse = c->cfg.amg_max_coarse;
    prm.max_levels = c->cfg.amg_max_levels;
    prm.trunc = c->cfg.amg_trunc;
    std::string e;
    if (!build_hierarchy(A0, prm, &c->H, &e)) return fail(c, IBM_ERR_ARG, e);
    if (fused_transfers_on(c))
        for (size_t l = 1; l + 1 < c->H.levels.size(); ++l)
            fused_transfers(c->H.levels[l], c->cfg.amg_pre, &c->H.levels[l].Rt, &c->H.levels[l].Q);
    c->have_H = true;
    c->amg_stale = false;
    c->steps_since_amg = 0;
    return IBM_OK;
}

// ---- V-cycle ------------------------------------------------------------------------
template <class T> DSell<T>& levA(DevLevel& d);
template <> DSell<double>& levA<double>(DevLevel& d) { return d.A64; }
template <> DSell<float>& levA<float>(DevLevel& d) { return d.A32; }
template <class T> DSell<T>& levP(DevLevel& d);
template <> DSell<double>& levP<double>(DevLevel& d) { return d.P64; }
template <> DSell<float>& levP<float>(DevLevel& d) { return d.P32; }
template <class T> DSell<T>& levR(DevLevel& d);
template <> DSell<double>& levR<double>(DevLevel& d) { return d.R64; }
template <> DSell<float>& levR<float>(DevLevel& d) { return d.R32; }
template <class T> DCsr<T>& levRt(DevLevel& d);
template <> DCsr<double>& levRt<double>(DevLevel& d) { return d.Rt64; }
template <> DCsr<float>& levRt<float>(DevLevel& d) { return d.Rt32; }
template <class T> DSell<T>& levQ(DevLevel& d);
template <> DSell<double>& levQ<double>(DevLevel& d) { return d.Q64; }
template <> DSell<float>& levQ<float>(DevLevel& d) { return d.Q32; }
template <class T> T* levId(DevLevel& d);
template <> double* levId<double>(DevLevel& d) { return d.id64; }
template <> float* levId<float>(DevLevel& d) { return d.id32; }


// Levels tail_start.. as one cluster kernel; returns the level's result buffer
// (the same buffer the per-sweep path below ends in).
template <class T>
T* vcycle_tail(ibm_ctx* c, int l0, const CgScalars* sc) {
    const int Lv = int(c->lev.size());
    TailArgs<T> a{};
    a.nlev = Lv - l0;
    a.pre = c->cfg.amg_pre;
    a.post = c->cfg.amg_post;
    a.nc = c->coarse_n;
    a.cinv = c->d_coarse_inv;   // FP64 in both precisions
    a.sc = sc;
    double bytes = 8.0 * c->coarse_n * c->coarse_n + 2.0 * c->coarse_n * sizeof(T);
    for (int l = l0; l < Lv; ++l) {
        DevLevel& d = c->lev[l];
        TailLevel<T>& t = a.lev[l - l0];
        t.b = static_cast<T*>(d.b);
        t.x = static_cast<T*>(d.x);
        t.x2 = static_cast<T*>(d.x2);
        t.r = static_cast<T*>(d.r);
        if (l + 1 < Lv) {
            t.A = levA<T>(d).view();
            t.P = levP<T>(d).view();
            t.R = levR<T>(d).view();
            t.idiag = levId<T>(d);
            t.omega = T(c->H.levels[l].omega);
            // first sweeps from zero (two in one pass when pre >= 2), further sweeps and the residual
            const int first = a.pre >= 2 ? 2 : 1;
            const double sweeps = double(a.pre - first + a.post + 1);
            bytes += (first == 2 ? sell_bytes(levA<T>(d)) : 0.0) + 3.0 * d.n * sizeof(T) +
                     sweeps * (sell_bytes(levA<T>(d)) + 4.0 * d.n * sizeof(T)) +
                     sell_bytes(levR<T>(d)) + sell_bytes(levP<T>(d)) +
                     (3.0 * d.n + 2.0 * c->lev[l + 1].n) * sizeof(T);
        }
    }
    L(c, PC_VC_TAIL, 1, bytes, [&] { launch_tail<T>(a, c->tail_cluster, c->tail_smem, c->st); });
    DevLevel& d = c->lev[l0];
    T* x = static_cast<T*>(d.x);
    T* x2 = static_cast<T*>(d.x2);
    if (l0 == Lv - 1) return x;
    for (int s = a.pre >= 2 ? 2 : 1; s < a.pre; ++s) std::swap(x, x2);
    for (int s = 0; s < a.post; ++s) std::swap(x, x2);
    return x;
}

// Levels l0.. as one cooperative kernel; with a parent (l0 >= 1) it also
// restricts r_parent into b_l0 first and adds P x_l0 into x_parent last.
// Returns the buffer holding level l0's result (x_parent when a parent is given).
template <class T>
T* vcycle_coop(ibm_ctx* c, int l0, CgScalars* sc, const T* r_parent, T* x_parent) {
    const int Lv = int(c->lev.size());
    CoopArgs<T> a{};
    a.tab = static_cast<const CoopTable<T>*>(c->coop_tab[l0]);
    a.nlev = Lv - l0;
    a.pre = c->cfg.amg_pre;
    a.post = c->cfg.amg_post;
    a.nc = c->coarse_n;
    a.cinv = c->d_coarse_inv;
    a.staged = c->coop_staged[l0];
    a.sc = sc;
    a.bar = c->gbar;
    double bytes = 8.0 * c->coarse_n * c->coarse_n + 2.0 * c->coarse_n * sizeof(T);
    for (int l = l0; l + 1 < Lv; ++l) {
        DevLevel& d = c->lev[l];
        const int first = a.pre >= 2 ? 2 : 1;
        const double sweeps = double(a.pre - first + a.post + 1);
        bytes += (first == 2 ? sell_bytes(levA<T>(d)) : 0.0) + 3.0 * d.n * sizeof(T) +
                 sweeps * (sell_bytes(levA<T>(d)) + 4.0 * d.n * sizeof(T)) + sell_bytes(levR<T>(d)) +
                 sell_bytes(levP<T>(d)) + (3.0 * d.n + 2.0 * c->lev[l + 1].n) * sizeof(T);
    }
    if (r_parent) {
        DevLevel& dp = c->lev[l0 - 1];
        a.has_parent = 1;
        a.rp = r_parent;
        a.xp = x_parent;
        bytes += sell_bytes(levR<T>(dp)) + (double(dp.n) + c->lev[l0].n) * sizeof(T) + sell_bytes(levP<T>(dp)) +
                 (2.0 * dp.n + c->lev[l0].n) * sizeof(T);
    }
    // the attribute set at upload covers every launch (checked, not assumed)
    const long long smem = c->coop_smem[l0] <= c->coop_smem_max ? c->coop_smem[l0] : 0;
    if (smem == 0) a.staged = 0u;
    L(c, PC_VC_COOP, 1, bytes, [&] { launch_coop<T>(a, c->coop_blocks, smem, c->st); });
    if (r_parent) return x_parent;
    // where the kernel leaves level l0's result (the same ping-pong as vcycle_csr)
    DevLevel& d = c->lev[l0];
    T* x = static_cast<T*>(d.x);
    T* x2 = static_cast<T*>(d.x2);
    if (l0 == Lv - 1) return x;
    for (int s = a.pre >= 2 ? 2 : 1; s < a.pre; ++s) std::swap(x, x2);
    for (int s = 0; s < a.post; ++s) std::swap(x, x2);
    return x;
}
bool use_coop(const ibm_ctx* c) { return c->coop_blocks > 0; }
// The grid barrier of the cooperative coarse-level kernel starts every solve
// (and every stand-alone V-cycle) from zero; a barrier that timed out leaves
// no state behind.
int reset_barrier(ibm_ctx* c) {
    if (!use_coop(c)) return IBM_OK;
    CUDA_OK(cudaMemsetAsync(c->gbar, 0, sizeof(GridBarrier), c->st));
    return IBM_OK;
}
// After a synchronised stand-alone V-cycle (no solver scalars): a timed-out
// barrier is reported as a CUDA-level failure.
int check_barrier(ibm_ctx* c) {
    if (!use_coop(c)) return IBM_OK;
    GridBarrier h{};
    CUDA_OK(cudaMemcpy(&h, c->gbar, sizeof(GridBarrier), cudaMemcpyDeviceToHost));
    c->d2h_bytes += int64_t(sizeof(GridBarrier));
    if (h.err) return fail(c, IBM_ERR_CUDA, "a grid barrier of the coarse V-cycle timed out");
    return IBM_OK;
}


template <class T>
T* vcycle_csr(ibm_ctx* c, int l, const CgScalars* sc) {
    if (use_coop(c)) return vcycle_coop<T>(c, l, const_cast<CgScalars*>(sc), nullptr, nullptr);
    if (l == c->tail_start) return vcycle_tail<T>(c, l, sc);
    DevLevel& d = c->lev[l];
    const int Lv = int(c->lev.size());
    T* b = static_cast<T*>(d.b);
    T* x = static_cast<T*>(d.x);
    T* x2 = static_cast<T*>(d.x2);
    T* r = static_cast<T*>(d.r);
    const T w = T(c->H.levels[l].omega);
    if (l == Lv - 1) {
        L(c, PC_VC_COARSEST, 1, 8.0 * c->coarse_n * c->coarse_n + 2.0 * c->coarse_n * sizeof(T), [&] { launch_coarse<T>(c->coarse_n, c->d_coarse_inv, b, x, sc, c->st); });
        return x;
    }
    const SellView<T> A = levA<T>(d).view();
    const T* id = levId<T>(d);
    if (d.fused) {
        // down: the pre-sweeps from zero and R (I - A w D^-1)^pre b, one launch;
        // up: the coarse correction with the first post-sweep, one launch
        DevLevel& dn = c->lev[l + 1];
        const DCsr<T>& Rt = levRt<T>(d);
        const int pre = c->cfg.amg_pre;
        const double bd = (pre == 2 ? sell_bytes(levA<T>(d)) : 0.0) + 3.0 * d.n * sizeof(T) +
                          csr_bytes(Rt.n, Rt.nnz, sizeof(T)) + double(dn.n) * sizeof(T);
        L(c, PC_VC_DOWN, 1, bd, [&] {
            launch_sell_down<T>(pre, A, id, b, x, w, Rt.view(), static_cast<T*>(dn.b), sc, c->st);
        });
        T* xc = vcycle_csr<T>(c, l + 1, sc);
        const SellView<T> Q = levQ<T>(d).view();
        L(c, PC_VC_UP, 1, sell_bytes(levA<T>(d)) + sell_bytes(levQ<T>(d)) + (4.0 * d.n + dn.n) * sizeof(T),
          [&] { launch_sell_up<T>(A, id, x, b, x2, w, Q, xc, sc, c->st); });
        std::swap(x, x2);
        for (int s = 1; s < c->cfg.amg_post; ++s) {
            L(c, PC_VC_CSR, 1, sell_bytes(levA<T>(d)) + 4.0 * d.n * sizeof(T), [&] { launch_sell<T>(MODE_JAC, A, id, x, b, x2, w, sc, c->st); });
            std::swap(x, x2);
        }
        return x;
    }
    if (c->cfg.amg_pre >= 2)   // first two sweeps in one pass: A, and b, D^-1 read, x written
        L(c, PC_VC_CSR, 1, sell_bytes(levA<T>(d)) + 3.0 * d.n * sizeof(T), [&] { launch_sell<T>(MODE_JAC2, A, id, x, b, x, w, sc, c->st); });
    else
        L(c, PC_VC_CSR, 1, 3.0 * d.n * sizeof(T), [&] { launch_sell<T>(MODE_JAC0, A, id, x, b, x, w, sc, c->st); });
    for (int s = c->cfg.amg_pre >= 2 ? 2 : 1; s < c->cfg.amg_pre; ++s) {
        L(c, PC_VC_CSR, 1, sell_bytes(levA<T>(d)) + 4.0 * d.n * sizeof(T), [&] { launch_sell<T>(MODE_JAC, A, id, x, b, x2, w, sc, c->st); });
        std::swap(x, x2);
    }
    L(c, PC_VC_CSR, 1, sell_bytes(levA<T>(d)) + 3.0 * d.n * sizeof(T), [&] { launch_sell<T>(MODE_RESID, A, id, x, b, r, w, sc, c->st); });
    DevLevel& dn = c->lev[l + 1];
    const SellView<T> R = levR<T>(d).view();
    L(c, PC_VC_RESTRICT, 1, sell_bytes(levR<T>(d)) + (double(d.n) + R.n) * sizeof(T), [&] {
        launch_sell_mv<T>(0, R, r, static_cast<T*>(dn.b), sc, c->st);
    });
    T* xc = vcycle_csr<T>(c, l + 1, sc);
    const SellView<T> P = levP<T>(d).view();
    L(c, PC_VC_PROLONG, 1, sell_bytes(levP<T>(d)) + (2.0 * P.n + dn.n) * sizeof(T), [&] { launch_sell_mv<T>(1, P, xc, x, sc, c->st); });
    for (int s = 0; s < c->cfg.amg_post; ++s) {
        L(c, PC_VC_CSR, 1, sell_bytes(levA<T>(d)) + 4.0 * d.n * sizeof(T), [&] { launch_sell<T>(MODE_JAC, A, id, x, b, x2, w, sc, c->st); });
        std::swap(x, x2);
    }
    return x;
}

// The finest level of the FP32 pressure-block V-cycle runs temporally blocked
// (k_level0.cu) when both sweep counts fit the fused kernels; IBM_NO_L0_FUSION=1
// keeps one kernel per sweep.
bool l0_fused(const ibm_ctx* c) {
    static const bool off = std::getenv("IBM_NO_L0_FUSION") != nullptr;
    const int pre = c->cfg.amg_sweeps0 > 0 ? c->cfg.amg_sweeps0 : c->cfg.amg_pre;
    const int post = c->cfg.amg_sweeps0 > 0 ? c->cfg.amg_sweeps0 : c->cfg.amg_post;
    return !off && c->sep_ax && l0_fused_ok(pre) && l0_fused_ok(post);
}
// blocks of the kernel that forms the last level-0 sweep's dots (pressure-block V-cycle)
int nb_last0(const ibm_ctx* c) {
    if (l0_fused(c)) {
        const int post = c->cfg.amg_sweeps0 > 0 ? c->cfg.amg_sweeps0 : c->cfg.amg_post;
        const dim3 g = l0_grid(post, c->g.nx, c->g.ny);
        return int(g.x * g.y);
    }
    return c->nb_pois;
}

// out = V(b): one V-cycle with level 0 matrix-free (the pressure stencil, plus
// the body rows of Q^T B^1 Q when `coupled`).  `last` (nullable) makes the
// final sweep form z.r and z.q (DK_ZR) into a reduction that may span other
// kernels; its slot0 is the stencil's first slot, the body-row kernel follows.
// FP32 pressure-block V-cycle whose finest level runs on the 1D link factors
// (k_vc0): the first two sweeps in one pass over b, then b in FP32.
template <class TY>
void vcycle_sep(ibm_ctx* c, const double* b, TY* out, const DotArgs* last, CgScalars* sc) {
    const Sep32 S{c->g.nx, c->g.ny, c->pin, c->sep_ax, c->sep_ay, c->sep_bx, c->sep_by};
    const float w = float(c->H.levels[0].omega);
    float* xa = static_cast<float*>(c->x0a);
    float* xb = static_cast<float*>(c->x0b);
    float* r0 = static_cast<float*>(c->r0);
    const double n = double(c->nc);
    DotArgs none;
    none.sc = sc;
    const int pre = c->cfg.amg_sweeps0 > 0 ? c->cfg.amg_sweeps0 : c->cfg.amg_pre;
    const int post = c->cfg.amg_sweeps0 > 0 ? c->cfg.amg_sweeps0 : c->cfg.amg_post;
    if (l0_fused(c)) {
        // temporally blocked finest level: pre-sweeps + residual, then
        // prolongation + post-sweeps, each one pass over its vectors
        DevLevel& d0 = c->lev[0];
        DevLevel& d1 = c->lev[1];
        L(c, PC_VC_SMOOTH0, 1, 20.0 * n, [&] { launch_l0_pre(pre, S, b, c->b32, xa, r0, w, none, c->st); });
        if (use_coop(c)) {   // restriction, levels 1.., prolongation into xa: one kernel
            vcycle_coop<float>(c, 1, sc, r0, xa);
        } else {
            const SellView<float> R = levR<float>(d0).view();
            L(c, PC_VC_RESTRICT, 1, sell_bytes(levR<float>(d0)) + (double(d0.n) + R.n) * sizeof(float), [&] {
                launch_sell_mv<float>(0, R, r0, static_cast<float*>(d1.b), sc, c->st);
            });
            float* xc = vcycle_csr<float>(c, 1, sc);
            const SellView<float> P = levP<float>(d0).view();
            L(c, PC_VC_PROLONG, 1, sell_bytes(levP<float>(d0)) + (2.0 * P.n + d1.n) * sizeof(float),
              [&] { launch_sell_mv<float>(1, P, xc, xa, sc, c->st); });
        }
        DotArgs dl = last ? *last : none;
        const int dk = last ? DK_ZR : DK_NONE;
        // x and b32 in, out written; with the dots r, q (FP64) and base
        const double by = (8.0 + sizeof(TY) + (last ? 16.0 + (dl.base ? 4.0 : 0.0) : 0.0)) * n;
        L(c, PC_VC_POST0, 1, by, [&] { launch_l0_post<TY>(post, dk, S, xa, c->b32, out, w, dl, c->st); });
        return;
    }
    // b (8) + x (4) + b32 (4) per cell
    L(c, PC_VC_SMOOTH0, 1, 16.0 * n, [&] {
        launch_vc0<float>(pre >= 2 ? V0_PRE2 : V0_PRE1, DK_NONE, S, nullptr, b, c->b32, xa, w, none, c->g_pois, c->st);
    });
    for (int s = 2; s < pre; ++s) {
        L(c, PC_VC_SMOOTH0, 1, 12.0 * n, [&] { launch_vc0<float>(V0_JAC, DK_NONE, S, xa, nullptr, c->b32, xb, w, none, c->g_pois, c->st); });
        std::swap(xa, xb);
    }
    L(c, PC_VC_SMOOTH0, 1, 12.0 * n, [&] { launch_vc0<float>(V0_RESID, DK_NONE, S, xa, nullptr, c->b32, r0, w, none, c->g_pois, c->st); });
    DevLevel& d0 = c->lev[0];
    DevLevel& d1 = c->lev[1];
    const SellView<float> R = levR<float>(d0).view();
    L(c, PC_VC_RESTRICT, 1, sell_bytes(levR<float>(d0)) + (double(d0.n) + R.n) * sizeof(float), [&] {
        launch_sell_mv<float>(0, R, r0, static_cast<float*>(d1.b), sc, c->st);
    });
    float* xc = vcycle_csr<float>(c, 1, sc);
    const SellView<float> P = levP<float>(d0).view();
    L(c, PC_VC_PROLONG, 1, sell_bytes(levP<float>(d0)) + (2.0 * P.n + d1.n) * sizeof(float), [&] { launch_sell_mv<float>(1, P, xc, xa, sc, c->st); });
    for (int s = 0; s < post; ++s) {
        if (s == post - 1) {
            DotArgs dl = last ? *last : none;
            const int dk = last ? DK_ZR : DK_NONE;
            // x, b32, y; with the dots z.r and z.q: r, q (FP64) and base
            const double by = 12.0 + (sizeof(TY) - 4.0) + (last ? 16.0 + (dl.base ? 4.0 : 0.0) : 0.0);
            L(c, PC_VC_SMOOTH0, 1, by * n, [&] { launch_vc0<TY>(V0_JAC, dk, S, xa, nullptr, c->b32, out, w, dl, c->g_pois, c->st); });
        } else {
            L(c, PC_VC_SMOOTH0, 1, 12.0 * n, [&] { launch_vc0<float>(V0_JAC, DK_NONE, S, xa, nullptr, c->b32, xb, w, none, c->g_pois, c->st); });
            std::swap(xa, xb);
        }
    }
}

template <class T, class TY>
void vcycle_gen(ibm_ctx* c, const double* b, TY* out, bool coupled, const DotArgs* last, CgScalars* sc) {
    if constexpr (std::is_same<T, float>::value) {
        if (!coupled && c->sep_ax) {
            vcycle_sep<TY>(c, b, out, last, sc);
            return;
        }
    }
    const Stencil<T> S = pois_stencil<T>(c);
    const Coupling<T> C = pois_coupling<T>(c);
    const T* id = pois_idiag<T>(c);
    const T w = T(c->H.levels[0].omega);
    T* xa = static_cast<T*>(c->x0a);
    T* xb = static_cast<T*>(c->x0b);
    T* r0 = static_cast<T*>(c->r0);
    const int cg = coupling_grid(c);
    DotArgs none;
    none.sc = sc;
    auto run0 = [&](int mode, const T* x, auto* y, const DotArgs* dl) {
        DotArgs ds = dl ? *dl : none;
        const int dk = dl ? DK_ZR : DK_NONE;
        L(c, PC_VC_SMOOTH0, 1, st_bytes(mode, dk, sizeof(T), sizeof(double), sizeof(*y), c->nc, ds.base != nullptr), [&] { launch_stencil(mode, dk, S, x, b, y, w, ds, c->g_pois, c->st); });
        if (coupled) {
            DotArgs dc = ds;
            dc.slot0 = ds.slot0 + c->nb_pois;
            L(c, PC_VC_COUPLING0, 1, csr_bytes(c->Cc64.n, c->Cc64.nnz, sizeof(T)) + csr_bytes(c->Cf64.n, c->Cf64.nnz, sizeof(T)), [&] { launch_coupling(mode, dk, C, x, b, y, id, w, dc, cg, c->st); });
        }
    };
    run0(MODE_JAC0, xa, xa, nullptr);
    for (int s = 1; s < c->cfg.amg_pre; ++s) {
        run0(MODE_JAC, xa, xb, nullptr);
        std::swap(xa, xb);
    }
    run0(MODE_RESID, xa, r0, nullptr);
    DevLevel& d0 = c->lev[0];
    DevLevel& d1 = c->lev[1];
    if (use_coop(c)) {   // restriction, levels 1.., prolongation into xa: one kernel
        vcycle_coop<T>(c, 1, sc, r0, xa);
    } else {
        const SellView<T> R = levR<T>(d0).view();
        L(c, PC_VC_RESTRICT, 1, sell_bytes(levR<T>(d0)) + (double(d0.n) + R.n) * sizeof(T), [&] {
            launch_sell_mv<T>(0, R, r0, static_cast<T*>(d1.b), sc, c->st);
        });
        T* xc = vcycle_csr<T>(c, 1, sc);
        const SellView<T> P = levP<T>(d0).view();
        L(c, PC_VC_PROLONG, 1, sell_bytes(levP<T>(d0)) + (2.0 * P.n + d1.n) * sizeof(T),
          [&] { launch_sell_mv<T>(1, P, xc, xa, sc, c->st); });
    }
    for (int s = 0; s < c->cfg.amg_post; ++s) {
        if (s == c->cfg.amg_post - 1) {
            run0(MODE_JAC, xa, out, last);
        } else {
            run0(MODE_JAC, xa, xb, nullptr);
            std::swap(xa, xb);
        }
    }
}

// z = V(r) on the full pinned Q^T B^1 Q (coupled smoothed aggregation, as in
// section 3).  When dots is true the last sweep forms r.z, z.q and beta.
template <class T>
void vcycle(ibm_ctx* c, const double* r, double* z, CgScalars* sc, double* part, const double* qprev, bool dots) {
    DotArgs d;
    d.sc = sc;
    d.partials = part;
    d.expected = c->nb_pois + coupling_grid(c);
    d.slot0 = 0;
    d.fin = FIN_PRECOND;
    d.r = r;
    d.q = qprev;
    if (use_bn(c)) {
        // every level (the finest included) a sliced-ELLPACK matrix: r narrowed
        // into level 0, the cycle, z widened with r.z and z.q
        const long long n = c->nl;
        DevLevel& d0 = c->lev[0];
        L(c, PC_VC_SMOOTH0, 1, (8.0 + sizeof(T)) * n,
          [&] { launch_narrow<T>(n, r, static_cast<T*>(d0.b), sc, c->grid, c->st); });
        const T* x = vcycle_csr<T>(c, 0, sc);
        DotArgs w = d;
        w.expected = c->grid;
        if (!dots) w = DotArgs{};
        L(c, PC_VC_SMOOTH0, 1, (sizeof(T) + 8.0 + (dots ? 16.0 : 0.0)) * n,
          [&] { launch_widen<T>(dots ? DK_ZR : DK_NONE, n, x, z, w, c->grid, c->st); });
        return;
    }
    vcycle_gen<T, double>(c, r, z, true, dots ? &d : nullptr, sc);
}

// A moving body's Schur complement is rebuilt and inverted every step or few
// steps.  In mixed precision it is inverted in FP32 (X ~ S^-1; GB300's FP64
// units make the FP64 Gauss-Jordan inverse cost more than the Poisson solve
// for a few thousand force unknowns) and applied with one step of iterative
// refinement against the FP64 S: z = X t + X (t - S X t).  An FP32 pivot that
// is not positive, or an X whose probe residual ||v - S X v|| / ||v|| exceeds
// 1e-2 (an ill-conditioned S, e.g. body points closer than a cell), falls back
// to the FP64 inverse.  A fixed body's complement
// is inverted once, in FP64.
bool schur32(const ibm_ctx* c) { return use_schur(c) && is_mixed(c) && c->cfg.moving; }

int schur_zf_grid(const ibm_ctx* c) { return std::max(1, std::min(c->sm_count * 2, (2 * c->n_b + 7) / 8)); }

// Schur-complement block preconditioner of the pinned Q^T B^1 Q = [Lp C; C^T F]
// (Lp: pressure block, V its smoothed-aggregation V-cycle; S = F - C^T V C):
//   y1 = V r_p;  z_f = S^-1 (r_f - C^T y1);  z_p = y1 - V (C z_f).
// Symmetric positive definite when V is; exact when V = Lp^-1.
template <class T>
void schur_apply(ibm_ctx* c, CgScalars* sc) {
    T* y1 = static_cast<T*>(c->y1);
    const int nf = 2 * c->n_b;
    const int nb0 = is_mixed(c) ? nb_last0(c) : c->nb_pois;
    if (nf == 0) {
        DotArgs d;
        d.sc = sc;
        d.partials = c->part2;
        d.expected = nb0;
        d.fin = FIN_PRECOND;
        d.r = c->pr;
        d.q = c->pq;
        vcycle_gen<T, double>(c, c->pr, c->pz, false, &d, sc);
        return;
    }
    vcycle_gen<T, T>(c, c->pr, y1, false, nullptr, sc);
    const CsrView<double> Cf = c->Cf64.view();
    L(c, PC_SCHUR, 1, csr_bytes(Cf.n, c->Cf64.nnz, 8) + 16.0 * nf, [&] { launch_schur_tf<T>(Cf, c->nc, c->pr, y1, c->tf, sc, c->st); });
    const int gz = schur_zf_grid(c);
    DotArgs dz;
    dz.sc = sc;
    dz.partials = c->part2;
    dz.expected = nb0 + gz;
    dz.slot0 = nb0;
    dz.fin = FIN_PRECOND;
    dz.r = c->pr + c->nc;
    dz.q = c->pq + c->nc;
    // the dense force-block solve z_f = S^-1 t_f is FP64 in both precisions
    if (c->schur_refine) {
        L(c, PC_SCHUR, 1, double(nf) * nf * sizeof(float) + 16.0 * nf,
          [&] { launch_dense_mv<float>(nf, c->Sinv32, c->tf, nullptr, 1.0, c->zf0, sc, gz, c->st); });
        L(c, PC_SCHUR, 1, double(nf) * nf * sizeof(double) + 24.0 * nf,
          [&] { launch_dense_mv<double>(nf, c->Sinv64, c->zf0, c->tf, -1.0, c->rtf, sc, gz, c->st); });
        L(c, PC_SCHUR, 1, double(nf) * nf * sizeof(float) + 40.0 * nf, [&] {
            launch_dense_mv_dots<float>(nf, c->Sinv32, c->rtf, c->zf0, c->pz + c->nc, dz, gz, c->st);
        });
    } else {
        L(c, PC_SCHUR, 1, double(nf) * nf * sizeof(double) + 32.0 * nf,
          [&] { launch_schur_zf<double>(nf, c->Sinv64, c->tf, c->pz + c->nc, dz, gz, c->st); });
    }
    L(c, PC_SCHUR, 1, csr_bytes(c->Cc64.n, c->Cc64.nnz, 8) + 16.0 * c->Cc64.n, [&] {
        launch_schur_sp(int(c->Cc64.n), c->d_tcell, c->Cc64.view(), c->nc, c->pz, c->s_full, sc, c->st);
    });
    DotArgs dl = dz;
    dl.slot0 = 0;
    dl.r = c->pr;
    dl.q = c->pq;
    dl.base = y1;
    vcycle_gen<T, double>(c, c->s_full, c->pz, false, &dl, sc);
}

// S = F - C^T G C from the cached responses G[u][v] = (V e_v)_u: the cells the
// body rows touch for the first time get one V-cycle each (the cache starts
// over when it is full); *done = false when the current cells alone exceed it.
template <class T>
int schur_from_cache(ibm_ctx* c, bool* done) {
    *done = false;
    const auto& tc = c->br.tcells;
    std::vector<long long> fresh;
    for (const int64_t cell : tc)
        if (c->h_slot[size_t(cell)] < 0) fresh.push_back(cell);
    if (c->nu + (long long)fresh.size() > c->ucap) {
        L(c, PC_SCHUR_SETUP, 1, 0.0, [&] { launch_cache_clear(c->nu, c->d_slot, c->d_cell, c->st); });
        for (int s = 0; s < c->nu; ++s) c->h_slot[size_t(c->h_cell[s])] = -1;
        c->h_cell.clear();
        c->nu = 0;
        fresh.assign(tc.begin(), tc.end());
        if ((long long)fresh.size() > c->ucap) return IBM_OK;
    }
    std::vector<long long> pairs;
    pairs.reserve(2 * fresh.size());
    for (size_t k = 0; k < fresh.size(); ++k) {
        const int s = c->nu + int(k);
        pairs.push_back(fresh[k]);
        pairs.push_back(s);
        c->h_slot[size_t(fresh[k])] = s;
        c->h_cell.push_back(fresh[k]);
    }
    int rc;
    if ((rc = up(c, c->d_fresh, pairs))) return rc;
    L(c, PC_SCHUR_SETUP, 1, 0.0, [&] { launch_cache_map(int(fresh.size()), c->d_fresh, c->d_slot, c->d_cell, c->st); });
    const int nu = c->nu + int(fresh.size());
    T* G = static_cast<T*>(c->G);
    T* w = static_cast<T*>(c->y1);
    for (size_t k = 0; k < fresh.size(); ++k) {
        const int sv = c->nu + int(k);
        L(c, PC_SCHUR_SETUP, 1, 0.0, [&] { launch_set_entry(c->s_full, fresh[k], 1.0, c->st); });
        vcycle_gen<T, T>(c, c->s_full, w, false, nullptr, nullptr);
        L(c, PC_SCHUR_SETUP, 1, 0.0, [&] { launch_set_entry(c->s_full, fresh[k], 0.0, c->st); });
        L(c, PC_SCHUR_SETUP, 1, 0.0, [&] { launch_cache_store<T>(nu, c->d_cell, w, sv, G, c->ucap, c->st); });
    }
    c->nu = nu;
    c->cache_fresh += int64_t(fresh.size());
    L(c, PC_SCHUR_SETUP, 1, 0.0, [&] {
        launch_schur_cached<T>(c->Cf64.view(), c->nc, c->d_slot, G, c->ucap, c->Sinv64, c->st);
    });
    *done = true;
    return IBM_OK;
}

// S = F - C^T V C column by column (2 n_b V-cycles on the device) or from the
// cache of V-cycle responses, inverted on the device.
template <class T>
int build_schur(ibm_ctx* c) {
    const int nf = 2 * c->n_b;
    c->schur_stale = false;
    c->schur_built = true;
    c->schur_builds++;
    c->steps_since_schur = 0;
    if (nf == 0) return IBM_OK;
    auto t0 = std::chrono::steady_clock::now();
    const CsrView<double> Cf = c->Cf64.view();
    T* w = static_cast<T*>(c->y1);
    int rb = reset_barrier(c);
    if (rb) return rb;
    CUDA_OK(cudaMemsetAsync(c->s_full, 0, c->nc * sizeof(double), c->st));
    bool cached = false;
    if (c->ucap > 0) {
        int rc = schur_from_cache<T>(c, &cached);
        if (rc) return rc;
    }
    if (!cached) {
        for (int col = 0; col < nf; ++col) {
            L(c, PC_SCHUR_SETUP, 1, 0.0, [&] { launch_col_scatter(Cf, c->nc, col, c->s_full, 0, c->st); });
            vcycle_gen<T, T>(c, c->s_full, w, false, nullptr, nullptr);
            L(c, PC_SCHUR_SETUP, 1, 0.0, [&] { launch_schur_col<T>(Cf, c->nc, col, w, c->Sinv64, c->st); });
            L(c, PC_SCHUR_SETUP, 1, 0.0, [&] { launch_col_scatter(Cf, c->nc, col, c->s_full, 1, c->st); });
        }
    }
    // S^-1 on the device (Gauss-Jordan; S is SPD): in FP32 into Sinv32 for a
    // moving body in mixed precision (applied with FP64 refinement), else in
    // place in FP64
    int flag = 0;
    c->schur_refine = false;
    if (c->Sinv32) {
        CUDA_OK(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->st));
        L(c, PC_SCHUR_SETUP, 3 * ((nf + 31) / 32) + 2, 0.0, [&] {
            launch_spd_inverse(nf, c->Sinv64, c->gj, c->d_flag, c->Sinv32, c->st);
        });
        CUDA_OK(cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        c->d2h_bytes += int64_t(sizeof(int));
        CUDA_OK(cudaStreamSynchronize(c->st));
        c->schur_refine = flag == 0;
        if (c->schur_refine) {
            // quality of X: rho = ||v - S X v|| / ||v|| on a fixed probe v; the
            // refined apply is accurate to about rho^2, so an ill-conditioned S
            // (rho > 1e-2) takes the FP64 inverse instead
            const int gz = schur_zf_grid(c);
            L(c, PC_SCHUR_SETUP, 3, 0.0, [&] {
                launch_probe_fill(nf, c->zf0, c->st);
                launch_dense_mv<float>(nf, c->Sinv32, c->zf0, nullptr, 1.0, c->rtf, nullptr, gz, c->st);
                launch_dense_mv<double>(nf, c->Sinv64, c->rtf, c->zf0, -1.0, c->tf, nullptr, gz, c->st);
            });
            std::vector<double> hv(static_cast<size_t>(nf)), hw(static_cast<size_t>(nf));
            CUDA_OK(cudaMemcpyAsync(hv.data(), c->zf0, size_t(nf) * sizeof(double), cudaMemcpyDeviceToHost, c->st));
            CUDA_OK(cudaMemcpyAsync(hw.data(), c->tf, size_t(nf) * sizeof(double), cudaMemcpyDeviceToHost, c->st));
            c->d2h_bytes += int64_t(2 * size_t(nf) * sizeof(double));
            CUDA_OK(cudaStreamSynchronize(c->st));
            double vv = 0.0, ww = 0.0;
            for (int k = 0; k < nf; ++k) {
                vv += hv[size_t(k)] * hv[size_t(k)];
                ww += hw[size_t(k)] * hw[size_t(k)];
            }
            c->schur_rho = vv > 0.0 ? std::sqrt(ww / vv) : 0.0;
            c->schur_refine = std::isfinite(c->schur_rho) && c->schur_rho <= 1e-2;
        }
    }
    if (!c->schur_refine) {   // FP64, in place (S is still in Sinv64)
        CUDA_OK(cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->st));
        L(c, PC_SCHUR_SETUP, 3 * ((nf + 31) / 32) + 1, 0.0, [&] {
            launch_spd_inverse(nf, c->Sinv64, c->gj, c->d_flag, nullptr, c->st);
        });
        CUDA_OK(cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
        c->d2h_bytes += int64_t(sizeof(int));
        CUDA_OK(cudaStreamSynchronize(c->st));
    }
    if ((rb = check_barrier(c))) return rb;
    if (flag) return fail(c, IBM_ERR_BREAKDOWN, "Schur complement is not positive definite");
    c->schur_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return IBM_OK;
}

// ---- CG drivers ------------------------------------------------------------------------
int read_scalars(ibm_ctx* c, CgScalars* dsc) {
    CUDA_OK(cudaMemcpyAsync(c->hsc, dsc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->st));
    c->d2h_bytes += int64_t(sizeof(CgScalars));
    CUDA_OK(cudaStreamSynchronize(c->st));
    return IBM_OK;
}

// Re-opens a solve whose recurrence residual met the tolerance but whose true
// residual did not: the true residual replaces the recurrence one and the
// next direction restarts from the preconditioned residual.
int reopen(ibm_ctx* c, CgScalars* dsc) {
    int32_t flags[2] = {0, 0};   // done, status
    int32_t one = 1;
    CUDA_OK(cudaMemcpyAsync(&dsc->done, flags, sizeof(flags), cudaMemcpyHostToDevice, c->st));
    CUDA_OK(cudaMemcpyAsync(&dsc->restart, &one, sizeof(one), cudaMemcpyHostToDevice, c->st));
    c->h2d_bytes += int64_t(sizeof(flags) + sizeof(one));
    CUDA_OK(cudaStreamSynchronize(c->st));
    return IBM_OK;
}

int init_scalars(ibm_ctx* c, CgScalars* dsc, double tol, int max_iter, int flexible) {
    CgScalars h{};
    h.tol2 = tol * tol;
    h.max_iter = max_iter;
    h.flexible = flexible;
    CgScalars* stage = c->hsc;
    *stage = h;
    CUDA_OK(cudaMemcpyAsync(dsc, stage, sizeof(CgScalars), cudaMemcpyHostToDevice, c->st));
    c->h2d_bytes += int64_t(sizeof(CgScalars));
    CUDA_OK(cudaStreamSynchronize(c->st));
    return IBM_OK;
}

// Captures one loop body (loop_unroll iterations `one`, then the loop
// condition) into a CUDA graph whose while node repeats it on the device.
// Iterations after convergence inside a body return at once (every kernel
// checks the solve's done flag).
template <class F>
int build_loop_graph(ibm_ctx* c, ibm_ctx::LoopGraph& lg, CgScalars* dsc, F&& one) {
    if (lg.exec) {
        cudaGraphExecDestroy(lg.exec);
        lg.exec = nullptr;
    }
    if (!c->cap_st) CUDA_OK(cudaStreamCreateWithFlags(&c->cap_st, cudaStreamNonBlocking));
    cudaGraph_t g;
    CUDA_OK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    CUDA_OK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_OK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    // kernels recorded into the body are counted when the body runs
    const int64_t l0 = c->launches;
    const double b0 = c->bytes_total;
    int64_t pl[PC_COUNT];
    double pb[PC_COUNT];
    std::copy(c->prof_launch, c->prof_launch + PC_COUNT, pl);
    std::copy(c->prof_bytes, c->prof_bytes + PC_COUNT, pb);
    cudaStream_t keep = c->st;
    c->st = c->cap_st;
    cudaError_t e = cudaStreamBeginCaptureToGraph(c->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int u = 0; u < c->loop_unroll; ++u) one();
        launch_loop_cond(h, dsc, c->st);
        cudaGraph_t out;
        e = cudaStreamEndCapture(c->st, &out);
    }
    c->st = keep;
    lg.nk = c->launches - l0 + 1;
    lg.bytes = c->bytes_total - b0;
    c->launches = l0;
    c->bytes_total = b0;
    std::copy(pl, pl + PC_COUNT, c->prof_launch);
    std::copy(pb, pb + PC_COUNT, c->prof_bytes);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(c, IBM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&lg.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, IBM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    lg.version = c->graph_version;
    return IBM_OK;
}

// Runs iterations until the device sets done (bounded by max_iter): as one
// device-side loop (CUDA graph) when graphs are on, else in host chunks.
template <class F>
int iterate(ibm_ctx* c, CgScalars* dsc, int max_iter, int* pred, ibm_ctx::LoopGraph& lg, const void* kx,
            const void* kb, F&& one) {
    int rc;
    if (c->use_graphs && !c->prof_on) {
        if (!lg.exec || lg.version != c->graph_version || lg.kx != kx || lg.kb != kb) {
            if ((rc = build_loop_graph(c, lg, dsc, one))) return rc;
            lg.kx = kx;
            lg.kb = kb;
        }
        const int g0 = c->hsc->guard, it0 = c->hsc->iter;
        CUDA_OK(cudaGraphLaunch(lg.exec, c->st));
        if ((rc = read_scalars(c, dsc))) return rc;
        c->launches += lg.nk * std::max(1, c->hsc->guard - g0);   // bodies executed
        c->bytes_total += lg.bytes / c->loop_unroll * std::max(0, c->hsc->iter - it0);   // iterations done
        if (c->hsc->status == 2) return fail(c, IBM_ERR_CUDA, "solver loop did not report completion");
        if (c->hsc->status == 6) return fail(c, IBM_ERR_CUDA, "a grid barrier of the coarse V-cycle timed out");
        *pred = std::max(1, c->hsc->iter);
        return IBM_OK;
    }
    if ((rc = read_scalars(c, dsc))) return rc;
    if (c->hsc->done) return IBM_OK;
    int launched = 0;
    int chunk = std::max(1, std::min(*pred, max_iter));
    for (;;) {
        for (int k = 0; k < chunk; ++k) one();
        launched += chunk;
        CUDA_OK(cudaGetLastError());
        if ((rc = read_scalars(c, dsc))) return rc;
        if (c->hsc->status == 6) return fail(c, IBM_ERR_CUDA, "a grid barrier of the coarse V-cycle timed out");
        if (c->hsc->done) break;
        if (launched > max_iter + 1) return fail(c, IBM_ERR_CUDA, "solver did not report completion");
        chunk = 2;
    }
    *pred = std::max(1, c->hsc->iter);
    return IBM_OK;
}

int finish_stats(ibm_ctx* c, CgScalars* dsc, ibm_solve_stats* out, double* x, size_t n) {
    int rc = read_scalars(c, dsc);
    if (rc) return rc;
    const CgScalars& h = *c->hsc;
    out->iters = h.iter;
    out->status = h.status == 0 ? IBM_OK : h.status;
    // converged by the recurrence but the recomputed residual stayed above 2x tol
    if (out->status == IBM_OK && h.bb > 0.0 && h.rr > 4.0 * h.tol2 * h.bb) out->status = IBM_ERR_NOT_CONVERGED;
    if (h.bb == 0.0) {
        CUDA_OK(cudaMemsetAsync(x, 0, n * sizeof(double), c->st));
        out->rel_res = 0.0;
        out->rel_res0 = 0.0;
    } else {
        out->rel_res = std::sqrt(h.rr / h.bb);
        out->rel_res0 = std::sqrt(h.rr0 / h.bb);
    }
    return IBM_OK;
}

// A q* = r1 (Eq. 9a) by Jacobi-preconditioned CG; x0 = q^n.
// Mixed-precision velocity solve (not in the paper; IBM_PREC_MIXED): FP64
// iterative refinement around an FP32 Jacobi-preconditioned CG.  Each pass
// solves A e = r (r = r1 - A q*, formed in FP64) in FP32 to the relative
// tolerance the pass needs (at most a 1e-5 reduction, which FP32 attains),
// adds e to q* in FP64 and recomputes the FP64 residual; the solve ends when
// that residual meets tol1 (the same test as the FP64 solve).  On GB300 the
// FP64 CG loop is bound by its FP64 arithmetic (≈ 12 operations per unknown
// and iteration); here FP64 is left with ≈ 8 operations per unknown and pass.
int solve_velocity_mixed(ibm_ctx* c, ibm_solve_stats* st) {
    const long long n = 2 * c->nc;
    const Stencil<double> A = vel_stencil(c);
    const Stencil<float> A32{c->g.nx, c->g.ny, 2, c->nc, c->vcE32, c->vcN32, c->vdiag32, c->vidiag32};
    int rc = init_scalars(c, c->sc1, c->cfg.tol1, c->cfg.max_iter1, 0);
    if (rc) return rc;
    DotArgs d;
    d.sc = c->sc1;
    d.partials = c->part1;
    d.expected = c->nb_vel;
    d.fin = FIN_INIT;
    d.ignore_done = 1;
    L(c, PC_VEL_RESID, 1, st_bytes(MODE_RESID, DK_RESID, 8, 8, 8, n), [&] { launch_stencil(MODE_RESID, DK_RESID, A, c->qs, c->r1, c->vr, 0.0, d, c->g_vel, c->st); });
    if ((rc = read_scalars(c, c->sc1))) return rc;
    const double bb = c->hsc->bb, rr0 = c->hsc->rr, tol2 = c->cfg.tol1 * c->cfg.tol1;
    double rr = rr0;
    int inner = 0, status = 0;
    DotArgs di;
    di.sc = c->sc1i;
    di.partials = c->part1;
    auto one = [&] {
        DotArgs e = di;
        L(c, PC_VEL_PUPDATE, 1, 12.0 * n, [&] { launch_v32_pupdate(n, c->vz32, c->vp32, e, c->grid, c->st); });
        e.fin = FIN_ALPHA;
        e.expected = c->nb_vel;
        L(c, PC_VEL_SPMV, 1, 24.0 * n, [&] { launch_v32_apply(A32, c->vp32, c->vq32, e, c->g_vel, c->st); });
        e.fin = FIN_UPDATE_PW;
        e.expected = c->grid;
        L(c, PC_VEL_UPDATE, 1, 36.0 * n, [&] {
            launch_v32_update(n, c->ve32, c->vr32, c->vp32, c->vq32, c->vz32, c->vidiag32, e, c->grid, c->st);
        });
    };
    for (int pass = 0; bb > 0.0 && rr > tol2 * bb && pass < 8; ++pass) {
        // the reduction this pass needs, with a margin, but not beyond FP32's reach
        const double need = std::sqrt(tol2 * bb / rr);
        const double tin = std::min(0.5, std::max(1e-5, 0.5 * need));
        DotArgs d0 = di;
        d0.expected = c->grid;
        L(c, PC_PW_PRECOND, 1, 20.0 * n, [&] {
            launch_v32_init(n, c->vr, c->vr32, c->ve32, c->vz32, c->vidiag32, tin * tin, c->cfg.max_iter1, d0,
                            c->grid, c->st);
        });
        if ((rc = iterate(c, c->sc1i, c->cfg.max_iter1, &c->pred1i, c->lg_vel32, c->ve32, c->vr32, one))) return rc;
        inner += c->hsc->iter;
        if (c->hsc->status != 0) status = c->hsc->status;
        L(c, PC_VEL_UPDATE, 1, 20.0 * n, [&] { launch_v32_correct(n, c->qs, c->ve32, c->grid, c->st); });
        DotArgs t = d;
        t.fin = FIN_STORE_RR;
        L(c, PC_VEL_RESID, 1, st_bytes(MODE_RESID, DK_RESID, 8, 8, 8, n), [&] { launch_stencil(MODE_RESID, DK_RESID, A, c->qs, c->r1, c->vr, 0.0, t, c->g_vel, c->st); });
        if ((rc = read_scalars(c, c->sc1))) return rc;
        rr = c->hsc->rr;
    }
    if (bb == 0.0) CUDA_OK(cudaMemsetAsync(c->qs, 0, size_t(n) * sizeof(double), c->st));
    const bool ok = bb == 0.0 || rr <= tol2 * bb;
    st->iters = inner;
    st->status = ok ? IBM_OK : (status ? status : IBM_ERR_NOT_CONVERGED);
    st->rel_res = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    st->rel_res0 = bb > 0.0 ? std::sqrt(rr0 / bb) : 0.0;
    return IBM_OK;
}

int solve_velocity(ibm_ctx* c, ibm_solve_stats* st) {
    if (is_mixed(c)) return solve_velocity_mixed(c, st);
    const long long n = 2 * c->nc;
    const Stencil<double> A = vel_stencil(c);
    int rc = init_scalars(c, c->sc1, c->cfg.tol1, c->cfg.max_iter1, 0);
    if (rc) return rc;
    DotArgs d;
    d.sc = c->sc1;
    d.partials = c->part1;
    d.expected = c->nb_vel;
    d.fin = FIN_INIT;
    L(c, PC_VEL_RESID, 1, st_bytes(MODE_RESID, DK_RESID, 8, 8, 8, n), [&] { launch_stencil(MODE_RESID, DK_RESID, A, c->qs, c->r1, c->vr, 0.0, d, c->g_vel, c->st); });
    d.expected = c->grid;
    d.fin = FIN_PW_INIT;
    L(c, PC_PW_PRECOND, 1, 24.0 * n, [&] { launch_pw_precond(n, c->vr, c->vz, c->vidiag, d, c->grid, c->st); });
    auto one = [&] {
        DotArgs e = d;
        L(c, PC_VEL_PUPDATE, 1, 24.0 * n, [&] { launch_pupdate(n, c->vz, c->vp, e, c->grid, c->st); });
        e.fin = FIN_ALPHA;
        e.expected = c->nb_vel;
        L(c, PC_VEL_SPMV, 1, st_bytes(MODE_APPLY, DK_XY, 8, 8, 8, n), [&] { launch_stencil(MODE_APPLY, DK_XY, A, c->vp, (const double*)nullptr, c->vAp, 0.0, e, c->g_vel, c->st); });
        e.fin = FIN_UPDATE_PW;
        e.expected = c->grid;
        L(c, PC_VEL_UPDATE, 1, 64.0 * n, [&] { launch_cg_update(1, n, c->qs, c->vr, c->vp, c->vAp, c->vz, c->vidiag, e, c->grid, c->st); });
    };
    for (int pass = 0;; ++pass) {
        if ((rc = iterate(c, c->sc1, c->cfg.max_iter1, &c->pred1, c->lg_vel, c->qs, c->r1, one))) return rc;
        // true residual (replaces the recurrence residual in vr)
        DotArgs t = d;
        t.fin = FIN_STORE_RR;
        t.ignore_done = 1;
        t.expected = c->nb_vel;
        L(c, PC_VEL_RESID, 1, st_bytes(MODE_RESID, DK_RESID, 8, 8, 8, n), [&] { launch_stencil(MODE_RESID, DK_RESID, A, c->qs, c->r1, c->vr, 0.0, t, c->g_vel, c->st); });
        if ((rc = read_scalars(c, c->sc1))) return rc;
        const CgScalars& h = *c->hsc;
        if (pass >= 3 || h.status != 0 || h.bb == 0.0 || h.rr <= h.tol2 * h.bb || h.iter >= h.max_iter) break;
        if ((rc = reopen(c, c->sc1))) return rc;
        DotArgs z = d;
        z.fin = FIN_PW_INIT;
        L(c, PC_PW_PRECOND, 1, 24.0 * n, [&] { launch_pw_precond(n, c->vr, c->vz, c->vidiag, z, c->grid, c->st); });
    }
    return finish_stats(c, c->sc1, st, c->qs, n);
}

// Poisson operator application with the fused p.Ap reduction
void pois_apply(ibm_ctx* c, int mode, int dk, int fin, const double* x, const double* b, double* y, int ignore) {
    if (bn_mf(c)) {
        // Q^T B^N Q x without assembly: q = -B^N Q x (the projection chain of
        // Eq. 9c with q* = 0, pinned column dropped), then [div q; -E q].  The
        // velocity solve's work vectors are free during the Poisson solve.
        const GridView g = gview(c);
        const Stencil<double> A = vel_stencil(c);
        const long long n2 = 2 * c->nc;
        double* wq = c->vr;
        double* wt = c->vz;
        double* wat = c->vAp;
        DotArgs none;
        L(c, PC_POIS_SPMV, 1, 32.0 * c->nc, [&] { launch_project(g, c->cfg.dt, nullptr, x, wq, c->g_vel, c->st, c->pin); });
        L(c, PC_POIS_COUPLING, 1, csr_bytes(c->ET.n, c->ET.nnz, 8) + 16.0 * c->ET.n, [&] {
            launch_project_body(g, c->cfg.dt, c->nfaces, c->d_faces, c->ET.view(), x + c->nc, wq, c->st);
        });
        L(c, PC_POIS_SPMV, 1, 24.0 * n2, [&] { launch_bn_start(n2, c->vmdt, wq, nullptr, wt, c->grid, c->st); });
        for (int k = 1; k < c->cfg.bn_order; ++k) {
            L(c, PC_POIS_SPMV, 1, st_bytes(MODE_APPLY, DK_NONE, 8, 8, 8, n2), [&] {
                launch_stencil(MODE_APPLY, DK_NONE, A, wt, (const double*)nullptr, wat, 0.0, none, c->g_vel, c->st);
            });
            L(c, PC_POIS_SPMV, 1, 48.0 * n2, [&] { launch_bn_term(n2, c->vmdt, wat, wt, wq, c->grid, c->st); });
        }
        DotArgs d;
        d.sc = c->sc2;
        d.partials = c->part2;
        d.expected = c->grid;
        d.fin = fin;
        d.ignore_done = ignore;
        L(c, PC_POIS_SPMV, 1, 32.0 * c->nc + csr_bytes(c->E.n, c->E.nnz, 8) + (mode == MODE_RESID ? 24.0 : 16.0) * c->nl,
          [&] { launch_qt_apply(mode, dk, g, c->pin, c->bn_dpin, wq, c->E.view(), x, b, y, d, c->grid, c->st); });
        return;
    }
    if (use_bn(c)) {
        DotArgs d;
        d.sc = c->sc2;
        d.partials = c->part2;
        d.expected = c->grid;
        d.fin = fin;
        d.ignore_done = ignore;
        const DSell<double>& A = c->lev[0].A64;
        L(c, PC_POIS_SPMV, 1, sell_bytes(A) + (mode == MODE_RESID ? 24.0 : 16.0) * c->nl,
          [&] { launch_sell_op(mode, dk, A.view(), x, b, y, d, c->grid, c->st); });
        return;
    }
    const Stencil<double> S = pois_stencil<double>(c);
    const Coupling<double> C = pois_coupling<double>(c);
    const int cg = coupling_grid(c);
    DotArgs d;
    d.sc = c->sc2;
    d.partials = c->part2;
    d.expected = c->nb_pois + cg;
    d.slot0 = c->nb_pois;
    d.fin = fin;
    d.ignore_done = ignore;
    if (dk == DK_RESID) {
        // squared residual norms are summed after both kernels wrote r: a fused
        // correction r^2 - r_stencil^2 on the body cells would cancel badly
        DotArgs n0 = d;
        n0.fin = FIN_NONE;
        L(c, PC_POIS_SPMV, 1, st_bytes(mode, DK_NONE, 8, 8, 8, c->nc), [&] { launch_stencil(mode, DK_NONE, S, x, b, y, 0.0, n0, c->g_pois, c->st); });
        L(c, PC_POIS_COUPLING, 1, csr_bytes(c->Cc64.n, c->Cc64.nnz, 8) + csr_bytes(c->Cf64.n, c->Cf64.nnz, 8), [&] { launch_coupling(mode, DK_NONE, C, x, b, y, c->pidiag, 0.0, n0, cg, c->st); });
        DotArgs e = d;
        e.expected = c->grid;
        e.slot0 = 0;
        L(c, PC_POIS_UPDATE, 1, 16.0 * c->nl, [&] { launch_dot2(c->nl, b, y, e, c->grid, c->st); });
        return;
    }
    DotArgs ds = d;
    ds.slot0 = 0;
    L(c, PC_POIS_SPMV, 1, st_bytes(mode, dk, 8, 8, 8, c->nc), [&] { launch_stencil(mode, dk, S, x, b, y, 0.0, ds, c->g_pois, c->st); });
    L(c, PC_POIS_COUPLING, 1, csr_bytes(c->Cc64.n, c->Cc64.nnz, 8) + csr_bytes(c->Cf64.n, c->Cf64.nnz, 8), [&] { launch_coupling(mode, dk, C, x, b, y, c->pidiag, 0.0, d, cg, c->st); });
}

void pois_precond(ibm_ctx* c, int first) {
    const long long n = c->nl;
    if (use_schur(c)) {
        if (is_mixed(c)) schur_apply<float>(c, c->sc2);
        else schur_apply<double>(c, c->sc2);
        return;
    }
    if (use_amg(c)) {
        if (is_mixed(c)) vcycle<float>(c, c->pr, c->pz, c->sc2, c->part2, c->pq, true);
        else vcycle<double>(c, c->pr, c->pz, c->sc2, c->part2, c->pq, true);
        return;
    }
    DotArgs d;
    d.sc = c->sc2;
    d.partials = c->part2;
    d.expected = c->grid;
    d.fin = FIN_PW_INIT;
    (void)first;
    const double* id = c->cfg.poisson_precond == IBM_PRECOND_JACOBI ? c->pidiag : nullptr;
    L(c, PC_PW_PRECOND, 1, 24.0 * n, [&] { launch_pw_precond(n, c->pr, c->pz, id, d, c->grid, c->st); });
}

// Q^T B^1 Q lam = b (Eq. 9b) by PCG / FCG; lam holds x0 on entry.
// Diagonal of the pinned row of the matrix-free Q^T B^N Q: the unpinned
// operator applied to the unit vector of the pinned cell (the corner cell's
// column does not involve the bodies, so once per context suffices).
int bn_pin_diag(ibm_ctx* c) {
    double* e = c->pz;
    double* y = c->pq;
    CUDA_OK(cudaMemsetAsync(e, 0, size_t(c->nl) * sizeof(double), c->st));
    const double one = 1.0;
    CUDA_OK(cudaMemcpyAsync(e + c->pin, &one, sizeof(double), cudaMemcpyHostToDevice, c->st));
    const long long pin = c->pin;
    c->pin = -1;
    pois_apply(c, MODE_APPLY, DK_NONE, FIN_NONE, e, nullptr, y, 1);
    c->pin = pin;
    double h = 0.0;
    CUDA_OK(cudaMemcpyAsync(&h, y + pin, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(cudaStreamSynchronize(c->st));
    if (!(h > 0.0)) return fail(c, IBM_ERR_STATE, "matrix-free Q^T B^N Q: pinned diagonal is not positive");
    c->bn_dpin = h;
    c->bn_dpin_ok = true;
    return IBM_OK;
}

// Warm start by projection onto the previous solutions (IBM_WARM_PROJ), for
// the Poisson solve K x = b of a fixed body (K stays the same from step to
// step; started so, the velocity solve converged in one or two iterations but
// its solution's error then raised the Poisson iterations more): with a
// K-orthonormal basis X_i (X_i . K X_j = delta_ij) of earlier solutions,
// x0 = sum_i (X_i . b) X_i is the point of their span closest to the solution
// in the K-norm (the span's Galerkin projection; the converged answer does not
// depend on it).  No basis yet: x keeps its previous value.
void proj_guess(ibm_ctx* c, ibm_ctx::ProjBasis& pb, int cls, const double* b, double* x) {
    if (pb.m == 0) return;
    const long long n = pb.n;
    const int m = pb.m;
    L(c, cls, 2, 8.0 * (m + 1) * n,
      [&] { launch_proj_dots(n, m, pb.X, n, b, nullptr, c->proj_part, c->proj_coef, c->st); });
    L(c, cls, 1, 8.0 * (m + 1) * n, [&] {
        launch_proj_combine(n, m, pb.X, pb.KX, n, c->proj_coef, nullptr, x, nullptr, nullptr, nullptr, -1.0,
                            c->grid, c->st);
    });
}

// After a solve: its solution x joins the basis.  K x = b - r with r the
// recomputed FP64 residual the solve leaves behind: v = x - sum_i (X_i . K x) X_i,
// then once more v -= sum_i (K X_i . v) X_i (Gram-Schmidt in the K inner
// product, done twice), K v by one operator application (cheaper in FP64 than
// combining the stored K X_i), X_new = v / sqrt(v . K v).  A full basis starts
// over from the latest solution.
int proj_update(ibm_ctx* c, ibm_ctx::ProjBasis& pb, int cls, const double* x, const double* b, const double* r) {
    if (pb.solves++ % kProjEvery != 0) return IBM_OK;
    const long long n = pb.n;
    if (pb.m >= kProjMax) pb.m = 0;
    const int m = pb.m;
    double* v = pb.X + size_t(m) * n;
    double* w = pb.KX + size_t(m) * n;
    if (m > 0) {
        L(c, cls, 2, 8.0 * (m + 2) * n,
          [&] { launch_proj_dots(n, m, pb.X, n, b, r, c->proj_part, c->proj_coef, c->st); });
        L(c, cls, 1, 8.0 * (m + 2) * n, [&] {
            launch_proj_combine(n, m, pb.X, pb.KX, n, c->proj_coef, x, v, nullptr, nullptr, nullptr, 1.0, c->grid,
                                c->st);
        });
        L(c, cls, 2, 8.0 * (m + 1) * n,
          [&] { launch_proj_dots(n, m, pb.KX, n, v, nullptr, c->proj_part, c->proj_coef, c->st); });
        L(c, cls, 1, 8.0 * (m + 2) * n, [&] {
            launch_proj_combine(n, m, pb.X, pb.KX, n, c->proj_coef, v, v, nullptr, nullptr, nullptr, 1.0, c->grid,
                                c->st);
        });
    } else {
        CUDA_OK(cudaMemcpyAsync(v, x, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    }
    pois_apply(c, MODE_APPLY, DK_NONE, FIN_NONE, v, nullptr, w, 1);
    // coef[0] = v . K v, coef[1] = x . K x (the scale of the test for a null v)
    L(c, cls, 2, 16.0 * n, [&] { launch_proj_dots(n, 1, v, n, w, nullptr, c->proj_part, c->proj_coef, c->st); });
    L(c, cls, 2, 24.0 * n, [&] { launch_proj_dots(n, 1, x, n, b, r, c->proj_part, c->proj_coef + 1, c->st); });
    L(c, cls, 1, 32.0 * n, [&] { launch_proj_store(n, v, w, c->proj_coef, v, w, c->grid, c->st); });
    pb.m = m + 1;
    return IBM_OK;
}

int solve_poisson_dev(ibm_ctx* c, const double* b, double* x, ibm_solve_stats* st) {
    const long long n = c->nl;
    const bool amg = use_amg(c);
    if (bn_mf(c) && !c->bn_dpin_ok) {
        const int rd = bn_pin_diag(c);
        if (rd) return rd;
    }
    if (amg && (!c->have_H || c->lev.size() < 2)) return fail(c, IBM_ERR_STATE, "AMG hierarchy missing");
    if (use_schur(c) && !c->schur_built) {
        const int rs = is_mixed(c) ? build_schur<float>(c) : build_schur<double>(c);
        if (rs) return rs;
    }
    int rc = init_scalars(c, c->sc2, c->cfg.tol2, c->cfg.max_iter2, amg && is_mixed(c) ? 1 : 0);
    if (rc) return rc;
    if ((rc = reset_barrier(c))) return rc;
    pois_apply(c, MODE_RESID, DK_RESID, FIN_INIT, x, b, c->pr, 0);
    pois_precond(c, 1);
    const double* id = c->cfg.poisson_precond == IBM_PRECOND_JACOBI ? c->pidiag : nullptr;
    auto one = [&] {
        DotArgs e;
        e.sc = c->sc2;
        e.partials = c->part2;
        e.expected = c->grid;
        L(c, PC_POIS_PUPDATE, 1, 24.0 * n, [&] { launch_pupdate(n, c->pz, c->pp, e, c->grid, c->st); });
        pois_apply(c, MODE_APPLY, DK_XY, FIN_ALPHA, c->pp, nullptr, c->pq, 0);
        if (amg) {
            e.fin = FIN_UPDATE;
            L(c, PC_POIS_UPDATE, 1, 48.0 * n, [&] { launch_cg_update(0, n, x, c->pr, c->pp, c->pq, c->pz, nullptr, e, c->grid, c->st); });
            pois_precond(c, 0);
        } else {
            e.fin = FIN_UPDATE_PW;
            L(c, PC_POIS_UPDATE, 1, 64.0 * n, [&] { launch_cg_update(1, n, x, c->pr, c->pp, c->pq, c->pz, id, e, c->grid, c->st); });
        }
    };
    for (int pass = 0;; ++pass) {
        if ((rc = iterate(c, c->sc2, c->cfg.max_iter2, &c->pred2, c->lg_pois, x, b, one))) return rc;
        // true residual (replaces the recurrence residual in pr)
        pois_apply(c, MODE_RESID, DK_RESID, FIN_STORE_RR, x, b, c->pr, 1);
        if ((rc = read_scalars(c, c->sc2))) return rc;
        const CgScalars& h = *c->hsc;
        if (std::getenv("IBM_DEBUG"))
            std::fprintf(stderr, "[ibm] poisson pass %d: iter %d done %d status %d bb %.3e rr %.3e rr0 %.3e rz %.3e "
                         "pq %.3e alpha %.3e beta %.3e counters %u %u\n", pass, h.iter, h.done, h.status, h.bb, h.rr,
                         h.rr0, h.rz, h.pq, h.alpha, h.beta, h.counter[0], h.counter[1]);
        if (pass >= 3 || h.status != 0 || h.bb == 0.0 || h.rr <= h.tol2 * h.bb || h.iter >= h.max_iter) break;
        if ((rc = reopen(c, c->sc2))) return rc;
        pois_precond(c, 1);
    }
    return finish_stats(c, c->sc2, st, x, n);
}

int check_bound(ibm_ctx* c) {
    if (!c) return IBM_ERR_ARG;
    if (!c->bound) return fail(c, IBM_ERR_STATE, "no workspace bound (call ibm_bind_workspace)");
    return IBM_OK;
}

size_t fixed_layout(ibm_ctx* c, Carver& cv) {
    const int nx = c->g.nx, ny = c->g.ny;
    const long long nc = c->nc, nl = c->nl, n2 = 2 * nc;
    c->dx = cv.take<double>(nx);
    c->dy = cv.take<double>(ny);
    c->idx = cv.take<double>(nx);
    c->idy = cv.take<double>(ny);
    c->dxf = cv.take<double>(nx + 1);
    c->dyf = cv.take<double>(ny + 1);
    c->idxf = cv.take<double>(nx + 1);
    c->idyf = cv.take<double>(ny + 1);
    c->vcE = cv.take<double>(n2);
    c->vcN = cv.take<double>(n2);
    c->vdiag = cv.take<double>(n2);
    c->vidiag = cv.take<double>(n2);
    if (is_mixed(c)) {
        for (float** p : {&c->vcE32, &c->vcN32, &c->vdiag32, &c->vidiag32, &c->ve32, &c->vr32, &c->vp32, &c->vq32,
                          &c->vz32})
            *p = cv.take<float>(n2);
    }
    c->vmdt = cv.take<double>(n2);
    c->q = cv.take<double>(n2);
    c->qs = cv.take<double>(n2);
    c->r1 = cv.take<double>(n2);
    c->vr = cv.take<double>(n2);
    c->vp = cv.take<double>(n2);
    c->vAp = cv.take<double>(n2);
    c->vz = cv.take<double>(n2);
    c->Nbuf[0] = cv.take<double>(n2);
    c->Nbuf[1] = cv.take<double>(n2);
    c->pwE = cv.take<double>(nc);
    c->pwN = cv.take<double>(nc);
    c->pdiag = cv.take<double>(nl);
    c->pidiag = cv.take<double>(nl);
    if (is_mixed(c)) {
        c->pwE32 = cv.take<float>(nc);
        c->pwN32 = cv.take<float>(nc);
        c->pdiag32 = cv.take<float>(nl);
        c->pidiag32 = cv.take<float>(nl);
        c->sep_ax = cv.take<float>(c->g.nx);
        c->sep_ay = cv.take<float>(c->g.ny);
        c->sep_bx = cv.take<float>(c->g.nx);
        c->sep_by = cv.take<float>(c->g.ny);
        c->b32 = cv.take<float>(nc);
    }
    c->d_flag = cv.take<int>(4);
    c->gbar = cv.take<GridBarrier>(1);
    c->lam = cv.take<double>(nl);
    c->b2 = cv.take<double>(nl);
    c->pr = cv.take<double>(nl);
    c->pp = cv.take<double>(nl);
    c->pq = cv.take<double>(nl);
    c->pz = cv.take<double>(nl);
    c->lam_prev = cv.take<double>(nl);
    c->r_ex = cv.take<double>(nl);
    if (c->cfg.warm == IBM_WARM_PROJ) {
        c->proj_pois.n = nl;
        c->proj_pois.X = cv.take<double>(size_t(kProjMax) * nl);
        c->proj_pois.KX = cv.take<double>(size_t(kProjMax) * nl);
        c->proj_part = cv.take<double>(size_t(kProjMax) * kProjBlocks);
        c->proj_coef = cv.take<double>(kProjMax + 2);
    }
    c->d_u_left = cv.take<double>(ny);
    c->d_u_right[0] = cv.take<double>(ny);
    c->d_u_right[1] = cv.take<double>(ny);
    c->d_v_bottom = cv.take<double>(nx);
    c->d_v_top = cv.take<double>(nx);
    c->d_u_bottom = cv.take<double>(nx + 1);
    c->d_u_top = cv.take<double>(nx + 1);
    c->d_v_left = cv.take<double>(ny + 1);
    c->d_v_right[0] = cv.take<double>(ny + 1);
    c->d_v_right[1] = cv.take<double>(ny + 1);
    c->d_ub = cv.take<double>(2 * size_t(c->n_b));
    c->d_xf = cv.take<double>(nx + 1);
    c->d_yf = cv.take<double>(ny + 1);
    c->d_xc = cv.take<double>(nx);
    c->d_yc = cv.take<double>(ny);
    c->d_xb = cv.take<double>(size_t(c->n_b));
    c->d_yb = cv.take<double>(size_t(c->n_b));
    c->d_forces = cv.take<double>(4);   // [sum f~x, sum f~y, max divergence, max slip]
    c->sc1 = cv.take<CgScalars>(1);
    c->sc1i = cv.take<CgScalars>(1);
    c->sc2 = cv.take<CgScalars>(1);
    c->part1 = cv.take<double>(2 * kMaxPartialBlocks);
    c->part2 = cv.take<double>(2 * kMaxPartialBlocks);
    if (use_schur(c)) {
        const size_t nf = 2 * size_t(c->n_b);
        c->y1 = cv.take<char>(nc * (is_mixed(c) ? sizeof(float) : sizeof(double)));
        c->s_full = cv.take<double>(nc);
        c->tf = cv.take<double>(nf);
        c->gj = cv.take<double>(32 * (size_t(nf) + 32));   // scratch of the blocked Gauss-Jordan inverse
        c->Sinv64 = cv.take<double>(nf * nf);
        if (schur32(c)) {
            c->Sinv32 = cv.take<float>(nf * nf);
            c->zf0 = cv.take<double>(nf);
            c->rtf = cv.take<double>(nf);
        }
    }
    return cv.off;
}

void boundary_defaults(ibm_ctx* c) {
    const int nx = c->g.nx, ny = c->g.ny;
    const bool fs = c->cfg.bc == IBM_BC_FREESTREAM;
    const double U = fs ? c->cfg.uinf : 0.0, V = fs ? c->cfg.vinf : 0.0;
    c->u_left.assign(ny, U);
    c->u_right0.assign(ny, U);
    c->v_bottom.assign(nx, V);
    c->v_top.assign(nx, V);
    c->u_bottom.assign(nx + 1, U);
    c->u_top.assign(nx + 1, U);
    c->v_left.assign(ny + 1, V);
    c->v_right0.assign(ny + 1, V);
}

void update_inflow(ibm_ctx* c) {
    double in = 0.0, ly = 0.0;
    for (int j = 0; j < c->g.ny; ++j) {
        in += c->u_left[j] * c->g.dy[j];
        ly += c->g.dy[j];
    }
    for (int i = 0; i < c->g.nx; ++i) in += (c->v_bottom[i] - c->v_top[i]) * c->g.dx[i];
    c->inflow = in;
    c->ly = ly;
}

StepParams step_params(const ibm_ctx* c) {
    StepParams p;
    p.nu = c->cfg.nu;
    p.dt = c->cfg.dt;
    p.uinf = c->cfg.uinf;
    p.inflow = c->inflow;
    p.ly = c->ly;
    p.bc = c->cfg.bc;
    p.first = c->ab2_first ? 1 : 0;
    p.pin = c->pin;
    return p;
}

}  // namespace

// Internal helpers for entry points defined in other translation units.
namespace ibm {
int cnn_warm_start(ibm_cnn* c, int nx, int ny, double* lam, double* lam_prev, const double* b_phi, long long nl,
                   std::string* err, int64_t* launches);
void cnn_extrapolated(ibm_cnn* c, long long nl, const double* lam, const double* prev, double* out);
int cnn_tc_check(ibm_cnn* c, std::string* err);
cudaStream_t cnn_stream(ibm_cnn* c);
// r = b - (pinned Q^T B^N Q) x on the context's stream (no reduction; the
// matrix-free B^N form uses the velocity solve's work vectors and needs the
// pinned diagonal of an earlier solve); returns n_lambda and the stream.
int internal_poisson_residual(ibm_ctx* c, const double* x, const double* b, double* r, long long* n,
                              cudaStream_t* st) {
    int rc = check_bound(c);
    if (rc) return rc;
    *n = c->nl;
    *st = c->st;
    if (!x) return IBM_OK;   // sizes and stream only
    if (bn_mf(c) && !c->bn_dpin_ok)
        return fail(c, IBM_ERR_STATE, "matrix-free B^N residual before the first Poisson solve");
    if (use_bn(c) || bn_mf(c)) {
        pois_apply(c, MODE_RESID, DK_NONE, FIN_NONE, x, b, r, 1);
        return IBM_OK;
    }
    const Stencil<double> S = pois_stencil<double>(c);
    const Coupling<double> C = pois_coupling<double>(c);
    DotArgs none;
    L(c, PC_POIS_SPMV, 1, st_bytes(MODE_RESID, DK_NONE, 8, 8, 8, c->nc),
      [&] { launch_stencil(MODE_RESID, DK_NONE, S, x, b, r, 0.0, none, c->g_pois, c->st); });
    L(c, PC_POIS_COUPLING, 1, csr_bytes(c->Cc64.n, c->Cc64.nnz, 8) + csr_bytes(c->Cf64.n, c->Cf64.nnz, 8),
      [&] { launch_coupling(MODE_RESID, DK_NONE, C, x, b, r, c->pidiag, 0.0, none, coupling_grid(c), c->st); });
    *n = c->nl;
    *st = c->st;
    return IBM_OK;
}
int internal_fail(ibm_ctx* c, int code, const std::string& m) { return fail(c, code, m); }
int internal_device(const ibm_ctx* c) { return c->device; }
void internal_count_launch(ibm_ctx* c) { c->launches += 1; }
}  // namespace ibm

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

void ibm_config_defaults(ibm_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->nx = cfg->ny = 0;
    cfg->nu = 0.01;
    cfg->dt = 0.01;
    cfg->uinf = 1.0;
    cfg->vinf = 0.0;
    cfg->bc = IBM_BC_FREESTREAM;
    cfg->bn_order = 1;
    cfg->h = 0.0;
    cfg->tol1 = 1e-8;
    cfg->tol2 = 1e-8;
    cfg->max_iter1 = 1000;
    cfg->max_iter2 = 1000;
    cfg->poisson_precond = IBM_PRECOND_AMG;
    cfg->precision = IBM_PREC_FP64;
    cfg->warm = IBM_WARM_PREV;
    cfg->pin_i = 0;
    cfg->pin_j = 0;
    cfg->amg_theta = 0.08;
    cfg->amg_omega = 2.0 / 3.0;
    cfg->amg_pre = 2;
    cfg->amg_post = 2;
    cfg->amg_max_coarse = 256;
    cfg->amg_max_levels = 12;
    cfg->amg_rebuild_every = 2;
    cfg->moving = 0;
    cfg->amg_trunc = 0.1;
    cfg->amg_tail_rows = 16384;
    cfg->amg_sweeps0 = 0;
    cfg->schur_cache = -1;
    cfg->reserved_ = 0;
}

const char* ibm_last_error(const ibm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int ibm_create(const ibm_config* cfg, const double* xf, const double* yf, int32_t n_b, const double* xb,
               const double* yb, ibm_ctx** out) {
    if (!cfg || !xf || !yf || !out) return IBM_ERR_ARG;
    *out = nullptr;
    ibm_ctx* c = new (std::nothrow) ibm_ctx();
    if (!c) return IBM_ERR_NO_MEM;
    c->cfg = *cfg;
    const ibm_config& k = c->cfg;
    auto bad = [&](const std::string& m) {
        c->err = m;
        *out = c;
        return IBM_ERR_ARG;
    };
    if (k.nx < 4 || k.ny < 4) return bad("nx and ny must be >= 4");
    if ((long long)k.nx * k.ny * 2 >= (1LL << 31)) return bad("grid too large for 32-bit indices");
    if (!(k.dt > 0) || !(k.nu > 0)) return bad("dt and nu must be positive");
    if (k.bn_order < 1 || k.bn_order > 4) return bad("bn_order must be 1..4");
    if (k.bn_order != 1 && k.poisson_precond != IBM_PRECOND_AMG && k.poisson_precond != IBM_PRECOND_SCHUR) {
        c->err = "B^N with N > 1 needs the coupled AMG (assembled operator) or the Schur preconditioner (matrix-free)";
        *out = c;
        return IBM_ERR_UNIMPLEMENTED;
    }
    if (k.bc != IBM_BC_FREESTREAM && k.bc != IBM_BC_WALLS) return bad("unknown bc");
    if (n_b < 0 || (n_b > 0 && (!xb || !yb))) return bad("body arrays missing");
    if (n_b > 0 && !(k.h > 0)) return bad("h must be positive when bodies are present");
    if (k.pin_i < 0 || k.pin_i >= k.nx || k.pin_j < 0 || k.pin_j >= k.ny) return bad("pin cell outside the grid");
    if (k.poisson_precond < 0 || k.poisson_precond > 3) return bad("unknown poisson_precond");
    if (k.precision != IBM_PREC_FP64 && k.precision != IBM_PREC_MIXED) return bad("unknown precision");
    if (k.warm < IBM_WARM_ZERO || k.warm > IBM_WARM_PROJ) return bad("unknown warm start");
    if (k.warm == IBM_WARM_PROJ && k.moving) return bad("the projection warm start needs a fixed body");
    if (k.poisson_precond >= IBM_PRECOND_AMG && (k.amg_pre < 1 || k.amg_post < 1))
        return bad("AMG needs at least one pre- and one post-smoothing sweep");
    if (k.amg_max_coarse < 8 || k.amg_max_coarse > 2048) return bad("amg_max_coarse must be in [8, 2048]");
    if (k.amg_tail_rows < 0) return bad("amg_tail_rows must be >= 0");
    if (k.amg_sweeps0 < 0 || k.amg_sweeps0 > 16) return bad("amg_sweeps0 must be in [0, 16]");
    if (k.tol1 <= 0 || k.tol2 <= 0) return bad("tolerances must be positive");
    for (int i = 0; i < k.nx; ++i)
        if (!(xf[i + 1] > xf[i])) return bad("xf must be increasing");
    for (int j = 0; j < k.ny; ++j)
        if (!(yf[j + 1] > yf[j])) return bad("yf must be increasing");
    c->g = make_grid(k.nx, k.ny, xf, yf);
    c->n_b = n_b;
    c->nc = (long long)k.nx * k.ny;
    c->nl = c->nc + 2LL * n_b;
    c->nq = int64_t(k.nx - 1) * k.ny + int64_t(k.nx) * (k.ny - 1);
    c->pin = (long long)k.pin_j * k.nx + k.pin_i;
    c->xb.assign(xb ? xb : xf, xb ? xb + n_b : xf);
    c->yb.assign(yb ? yb : yf, yb ? yb + n_b : yf);
    c->ub.assign(n_b, 0.0);
    c->vb.assign(n_b, 0.0);
    c->vc = velocity_coeffs(c->g, k.nu, k.dt);
    std::string e;
    if (!build_body_rows(c->g, k.h, k.dt, c->pin, n_b, c->xb.data(), c->yb.data(), &c->br, &e)) return bad(e);
    c->pc = poisson_coeffs(c->g, k.dt, c->pin, c->br);
    boundary_defaults(c);
    update_inflow(c);
    if (k.poisson_precond >= IBM_PRECOND_AMG) {
        int rc = rebuild_hierarchy(c);
        if (rc) {
            *out = c;
            return rc;
        }
    }
    // workspace: fixed part + body rows + hierarchy, with room to grow for moving bodies
    Carver cv;
    c->fixed_bytes = fixed_layout(c, cv);
    Carver cb;
    const size_t body = carve_body(c, cb, c->br);
    Carver ch;
    const size_t hier = c->have_H ? carve_hier(c, ch, c->H) : 0;
    const double grow = k.moving ? 1.6 : 1.0;
    c->body_cap = size_t(double(body) * (k.moving ? 2.5 : 1.0)) + (64 << 10);
    c->hier_cap = size_t(double(hier) * grow) + (k.moving ? (1 << 20) : (64 << 10));
    c->body_off = (c->fixed_bytes + 4095) & ~size_t(4095);
    c->hier_off = (c->body_off + c->body_cap + 4095) & ~size_t(4095);
    // cache of V-cycle responses for moving bodies with the Schur preconditioner
    c->ucap = 0;
    if (k.moving && k.poisson_precond == IBM_PRECOND_SCHUR && k.schur_cache != 0 && n_b > 0) {
        const long long ntc = (long long)c->br.tcells.size();
        c->ucap = int(k.schur_cache > 0 ? k.schur_cache : std::min<long long>(32768, std::max<long long>(1024, 8 * ntc)));
    }
    c->green_off = (c->hier_off + c->hier_cap + 4095) & ~size_t(4095);
    Carver cg;
    carve_green(c, cg);
    c->green_cap = cg.off;
    *out = c;
    return IBM_OK;
}

int ibm_workspace_bytes(const ibm_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return IBM_ERR_ARG;
    *bytes = ctx->green_off + ctx->green_cap + 256;
    return IBM_OK;
}

int ibm_bind_workspace(ibm_ctx* c, void* dev_ws, size_t ws_bytes, void* stream) {
    if (!c || !dev_ws) return IBM_ERR_ARG;
    size_t need = 0;
    ibm_workspace_bytes(c, &need);
    if (ws_bytes < need) return fail(c, IBM_ERR_NO_MEM, "workspace too small: need " + std::to_string(need) + " bytes");
    if (reinterpret_cast<uintptr_t>(dev_ws) % 256 != 0) return fail(c, IBM_ERR_ARG, "workspace must be 256-byte aligned");
    c->ws = static_cast<char*>(dev_ws);
    c->ws_bytes = ws_bytes;
    c->st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    CUDA_OK(cudaGetDevice(&dev));
    c->device = dev;
    CUDA_OK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev));
    c->grid = std::min(kMaxPartialBlocks, c->sm_count * 8);
    c->use_graphs = std::getenv("IBM_NO_GRAPHS") == nullptr;
    if (const char* u = std::getenv("IBM_LOOP_UNROLL")) c->loop_unroll = std::max(1, std::min(8, std::atoi(u)));
    c->g_vel = stencil_grid(c->g.nx, 2 * c->g.ny, c->grid);
    c->g_pois = stencil_grid(c->g.nx, c->g.ny, c->grid);
    c->nb_vel = int(c->g_vel.x * c->g_vel.y);
    c->nb_pois = int(c->g_pois.x * c->g_pois.y);
    if (!c->hsc) CUDA_OK(cudaMallocHost(&c->hsc, sizeof(CgScalars) + 64));
    if (!c->hforces) CUDA_OK(cudaMallocHost(&c->hforces, 4 * sizeof(double)));
    for (auto& e : c->ev_pois)
        if (!e) CUDA_OK(cudaEventCreate(&e));
    Carver cv{c->ws, 0};
    fixed_layout(c, cv);
    CUDA_OK(cudaMemsetAsync(c->ws, 0, c->fixed_bytes, c->st));
    const Grid& g = c->g;
    std::vector<double> inv;
    auto recip = [&](const std::vector<double>& a, int lo, int hi) {
        inv.assign(a.size(), 0.0);
        for (int i = lo; i < hi; ++i) inv[i] = 1.0 / a[i];
        return inv;
    };
    int rc;
    if ((rc = up(c, c->dx, g.dx)) || (rc = up(c, c->dy, g.dy)) || (rc = up(c, c->idx, recip(g.dx, 0, g.nx))) ||
        (rc = up(c, c->idy, recip(g.dy, 0, g.ny))) || (rc = up(c, c->dxf, g.dxf)) || (rc = up(c, c->dyf, g.dyf)) ||
        (rc = up(c, c->idxf, recip(g.dxf, 1, g.nx))) || (rc = up(c, c->idyf, recip(g.dyf, 1, g.ny))))
        return rc;
    if ((rc = up(c, c->d_xf, g.xf)) || (rc = up(c, c->d_yf, g.yf)) || (rc = up(c, c->d_xc, g.xc)) ||
        (rc = up(c, c->d_yc, g.yc)))
        return rc;
    if ((rc = up(c, c->vcE, c->vc.cE)) || (rc = up(c, c->vcN, c->vc.cN)) || (rc = up(c, c->vdiag, c->vc.diag)) ||
        (rc = up(c, c->vidiag, c->vc.idiag)) || (rc = up(c, c->vmdt, c->vc.mdt)))
        return rc;
    if (c->vcE32 && ((rc = up(c, c->vcE32, to32(c->vc.cE))) || (rc = up(c, c->vcN32, to32(c->vc.cN))) ||
                     (rc = up(c, c->vdiag32, to32(c->vc.diag))) || (rc = up(c, c->vidiag32, to32(c->vc.idiag)))))
        return rc;
    std::vector<double> pid(c->pc.diag.size());
    for (size_t k = 0; k < pid.size(); ++k) pid[k] = 1.0 / c->pc.diag[k];
    if ((rc = up(c, c->pwE, c->pc.wE)) || (rc = up(c, c->pwN, c->pc.wN)) || (rc = up(c, c->pdiag, c->pc.diag)) ||
        (rc = up(c, c->pidiag, pid)))
        return rc;
    if (is_mixed(c)) {
        if ((rc = up(c, c->pwE32, to32(c->pc.wE))) || (rc = up(c, c->pwN32, to32(c->pc.wN))) ||
            (rc = up(c, c->pdiag32, to32(c->pc.diag))) || (rc = up(c, c->pidiag32, to32(pid))))
            return rc;
        // links of the pressure block as products of 1D factors (the coefficients of poisson_coeffs)
        const double dt = c->cfg.dt;
        std::vector<double> ax(g.nx), ay(g.ny), bx(g.nx), by(g.ny);
        for (int i = 0; i < g.nx; ++i) {
            ax[i] = i + 1 <= g.nx - 1 ? 1.0 / g.dxf[i + 1] : 0.0;
            bx[i] = dt * g.dx[i];
        }
        for (int j = 0; j < g.ny; ++j) {
            ay[j] = dt * g.dy[j];
            by[j] = j + 1 <= g.ny - 1 ? 1.0 / g.dyf[j + 1] : 0.0;
        }
        if ((rc = up(c, c->sep_ax, to32(ax))) || (rc = up(c, c->sep_ay, to32(ay))) ||
            (rc = up(c, c->sep_bx, to32(bx))) || (rc = up(c, c->sep_by, to32(by))))
            return rc;
    }
    if ((rc = up(c, c->d_u_left, c->u_left)) || (rc = up(c, c->d_u_right[0], c->u_right0)) ||
        (rc = up(c, c->d_v_bottom, c->v_bottom)) || (rc = up(c, c->d_v_top, c->v_top)) ||
        (rc = up(c, c->d_u_bottom, c->u_bottom)) || (rc = up(c, c->d_u_top, c->u_top)) ||
        (rc = up(c, c->d_v_left, c->v_left)) || (rc = up(c, c->d_v_right[0], c->v_right0)))
        return rc;
    // initial velocity: freestream (or rest) on the padded array
    {
        const int nx = g.nx, ny = g.ny;
        std::vector<double> q0(2 * c->nc, 0.0);
        const bool fs = c->cfg.bc == IBM_BC_FREESTREAM;
        for (int j = 0; j < ny; ++j)
            for (int i = 1; i < nx; ++i) q0[(long long)j * nx + i] = (fs ? c->cfg.uinf : 0.0) * g.dy[j];
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) q0[c->nc + (long long)j * nx + i] = (fs ? c->cfg.vinf : 0.0) * g.dx[i];
        if ((rc = up(c, c->q, q0))) return rc;
    }
    if ((rc = upload_body(c))) return rc;
    if (c->have_H && (rc = upload_hier(c))) return rc;
    if (c->ucap > 0) {   // empty response cache
        Carver cgr{c->ws, c->green_off};
        carve_green(c, cgr);
        CUDA_OK(cudaMemsetAsync(c->d_slot, 0xFF, size_t(c->nc) * sizeof(int), c->st));
        c->h_slot.assign(size_t(c->nc), -1);
        c->h_cell.clear();
        c->nu = 0;
    }
    CUDA_OK(cudaStreamSynchronize(c->st));
    c->bound = true;
    return IBM_OK;
}

int ibm_setup(const ibm_config* cfg, const double* xf, const double* yf, int32_t n_b, const double* xb,
              const double* yb, void* dev_ws, size_t ws_bytes, void* stream, ibm_ctx** out) {
    int rc = ibm_create(cfg, xf, yf, n_b, xb, yb, out);
    if (rc || !dev_ws) return rc;
    return ibm_bind_workspace(*out, dev_ws, ws_bytes, stream);
}

void ibm_destroy(ibm_ctx* c) {
    if (!c) return;
    if (c->lg_vel.exec) cudaGraphExecDestroy(c->lg_vel.exec);
    if (c->lg_pois.exec) cudaGraphExecDestroy(c->lg_pois.exec);
    if (c->cap_st) cudaStreamDestroy(c->cap_st);
    for (auto& e : c->ev) cudaEventDestroy(e);
    for (auto& e : c->ev_pois)
        if (e) cudaEventDestroy(e);
    if (c->gprof_st) cudaStreamDestroy(c->gprof_st);
    if (c->hsc) cudaFreeHost(c->hsc);
    if (c->hforces) cudaFreeHost(c->hforces);
    delete c;
}

int ibm_sizes(const ibm_ctx* c, int64_t* n_q, int64_t* n_lambda, int32_t* n_b) {
    if (!c) return IBM_ERR_ARG;
    if (n_q) *n_q = c->nq;
    if (n_lambda) *n_lambda = c->nl;
    if (n_b) *n_b = c->n_b;
    return IBM_OK;
}

int ibm_layout(const ibm_ctx* c, int64_t* nq_padded) {
    if (!c || !nq_padded) return IBM_ERR_ARG;
    *nq_padded = 2 * c->nc;
    return IBM_OK;
}

namespace {
// A moving body's rows are assembled on the device with the Schur block
// preconditioner (whose hierarchy is the fixed pressure block); the coupled
// hierarchy of IBM_PRECOND_AMG and B^N (N > 1) are built on the host from the
// host's values, so those keep the host assembly.  IBM_HOST_BODY_ROWS=1 forces it.
bool device_body_rows(const ibm_ctx* c) {
    return use_schur(c) && !use_bn(c) && !std::getenv("IBM_HOST_BODY_ROWS");
}
}  // namespace

int ibm_set_body(ibm_ctx* c, const double* xb, const double* yb, const double* ub, const double* vb) {
    int rc = check_bound(c);
    if (rc) return rc;
    const int nb = c->n_b;
    if (nb == 0) return IBM_OK;
    for (int k = 0; k < nb; ++k) {
        c->ub[k] = ub ? ub[k] : 0.0;
        c->vb[k] = vb ? vb[k] : 0.0;
        if (!std::isfinite(c->ub[k]) || !std::isfinite(c->vb[k])) return fail(c, IBM_ERR_ARG, "body velocity is not finite");
    }
    std::vector<double> u2(2 * nb);
    std::copy(c->ub.begin(), c->ub.end(), u2.begin());
    std::copy(c->vb.begin(), c->vb.end(), u2.begin() + nb);
    if ((rc = up(c, c->d_ub, u2))) return rc;
    if (xb && yb) {
        bool moved = false;
        for (int k = 0; k < nb; ++k)
            if (xb[k] != c->xb[k] || yb[k] != c->yb[k]) { moved = true; break; }
        if (moved && device_body_rows(c)) {
            // the pattern on the host (integer work), every value on the device
            const auto t0 = std::chrono::steady_clock::now();
            BodyRows br;
            BodySrc src;
            std::string e;
            if (!body_pattern(c->g, c->cfg.h, c->pin, nb, xb, yb, &br, &src, &c->bmaps, &e))
                return fail(c, IBM_ERR_ARG, e);
            c->xb.assign(xb, xb + nb);
            c->yb.assign(yb, yb + nb);
            c->br = std::move(br);
            c->bsrc = std::move(src);
            if ((rc = upload_body_device(c, xb, yb))) return rc;
            c->body_host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            c->schur_stale = true;
            CUDA_OK(cudaMemsetAsync(c->s_full, 0, c->nc * sizeof(double), c->st));
            return IBM_OK;
        }
        if (moved) {
            const auto t0 = std::chrono::steady_clock::now();
            BodyRows br;
            std::string e;
            if (!build_body_rows(c->g, c->cfg.h, c->cfg.dt, c->pin, nb, xb, yb, &br, &e)) return fail(c, IBM_ERR_ARG, e);
            c->xb.assign(xb, xb + nb);
            c->yb.assign(yb, yb + nb);
            c->br = std::move(br);
            for (long long r = 0; r < c->br.Cf.n; ++r)
                for (long long p = c->br.Cf.rowptr[r]; p < c->br.Cf.rowptr[r + 1]; ++p)
                    if (c->br.Cf.col[p] == c->nc + r) c->pc.diag[c->nc + r] = c->br.Cf.val[p];
            if ((rc = upload_body(c))) return rc;
            c->body_host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (use_schur(c)) {
                c->schur_stale = true;
                CUDA_OK(cudaMemsetAsync(c->s_full, 0, c->nc * sizeof(double), c->st));
            } else {
                c->amg_stale = true;
            }
        }
    }
    return IBM_OK;
}

int ibm_step(ibm_ctx* c, int32_t nsteps, ibm_step_stats* per_step) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (nsteps < 0) return fail(c, IBM_ERR_ARG, "nsteps < 0");
    int first_bad = IBM_OK;
    const GridView g = gview(c);
    const Stencil<double> A = vel_stencil(c);
    for (int s = 0; s < nsteps; ++s) {
        ibm_step_stats stt{};
        const int64_t builds0 = c->schur_builds;
        // hierarchy re-use (section 4): rebuild every amg_rebuild_every steps after a body move
        if (use_schur(c) && c->schur_stale && c->schur_built) {
            // the pressure hierarchy never changes; S is rebuilt on the same cadence
            if (++c->steps_since_schur >= std::max(1, c->cfg.amg_rebuild_every)) {
                rc = is_mixed(c) ? build_schur<float>(c) : build_schur<double>(c);
                if (rc) return rc;
                stt.amg_rebuilt = 1;
            }
        } else if (use_amg(c) && c->amg_stale) {
            c->steps_since_amg++;
            // with B^N (N > 1) level 0 is also the Poisson operator: rebuilt on every move
            const int every = use_bn(c) ? 1 : std::max(1, c->cfg.amg_rebuild_every);
            if (c->steps_since_amg >= every) {
                if ((rc = rebuild_hierarchy(c))) return rc;
                if ((rc = upload_hier(c))) return rc;
                stt.amg_rebuilt = 1;
            }
        }
        const StepParams p = step_params(c);
        const BoundaryView b = bview(c);
        const int nn = c->ncur, np = 1 - c->ncur;
        L(c, PC_OUTFLOW, 1, 48.0 * c->g.ny, [&] {
            launch_outflow(g, p, c->q, b, c->d_u_right[1 - c->bcur], c->d_v_right[1 - c->bcur], c->st);
        });
        L(c, PC_RHS, 1, 64.0 * 2 * c->nc, [&] { launch_rhs(g, p, A, c->vmdt, c->q, b, c->Nbuf[np], c->Nbuf[nn], c->r1, c->g_vel, c->st); });
        CUDA_OK(cudaMemcpyAsync(c->qs, c->q, 2 * c->nc * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
        if ((rc = solve_velocity(c, &stt.solve1))) return rc;
        L(c, PC_POIS_RHS, 1, 24.0 * c->nc + csr_bytes(c->E.n, c->E.nnz, 8), [&] {
            launch_poisson_rhs(g, p, c->qs, b, c->E.view(), c->d_ub, c->b2, c->grid, c->st);
        });
        if (c->cfg.warm == IBM_WARM_ZERO) CUDA_OK(cudaMemsetAsync(c->lam, 0, c->nl * sizeof(double), c->st));
        if (c->cfg.warm == IBM_WARM_CNN && c->lam_steps >= 2) {
            if (!c->cnn) return fail(c, IBM_ERR_STATE, "IBM_WARM_CNN without an attached network");
            // residual of the extrapolated guess: the network's input
            ibm::cnn_extrapolated(c->cnn, c->nl, c->lam, c->lam_prev, c->pz);
            c->launches++;
            pois_apply(c, MODE_RESID, DK_NONE, FIN_NONE, c->pz, c->b2, c->r_ex, 1);
            std::string e;
            rc = ibm::cnn_warm_start(c->cnn, c->g.nx, c->g.ny, c->lam, c->lam_prev, c->r_ex, c->nl, &e, &c->launches);
            if (rc) return fail(c, rc, e);
        } else if (c->cfg.warm == IBM_WARM_EXTRAP || c->cfg.warm == IBM_WARM_CNN) {
            const int first = c->lam_steps < 2 ? 1 : 0;
            L(c, PC_POIS_RHS, 1, 24.0 * c->nl,
              [&] { launch_extrapolate(c->nl, c->lam, c->lam_prev, first, c->grid, c->st); });
            if (c->snapshots) pois_apply(c, MODE_RESID, DK_NONE, FIN_NONE, c->lam, c->b2, c->r_ex, 1);
        } else if (c->cfg.warm == IBM_WARM_PROJ) {
            proj_guess(c, c->proj_pois, PC_WARM, c->b2, c->lam);
        }
        const double pb0 = c->bytes_total;
        CUDA_OK(cudaEventRecord(c->ev_pois[0], c->st));
        if ((rc = solve_poisson_dev(c, c->b2, c->lam, &stt.solve2))) return rc;
        CUDA_OK(cudaEventRecord(c->ev_pois[1], c->st));
        stt.poisson_bytes = c->bytes_total - pb0;
        if (c->cfg.warm == IBM_WARM_PROJ && stt.solve2.rel_res0 > 0.0 &&
            (rc = proj_update(c, c->proj_pois, PC_WARM, c->lam, c->b2, c->pr)))
            return rc;
        L(c, PC_PROJECT, 1, 32.0 * c->nc + 8.0 * c->nc + 16.0 * c->nc, [&] { launch_project(g, c->cfg.dt, c->qs, c->lam, c->q, c->g_vel, c->st); });
        L(c, PC_PROJECT, 1, csr_bytes(c->ET.n, c->ET.nnz, 8) + 16.0 * c->ET.n, [&] {
            launch_project_body(g, c->cfg.dt, c->nfaces, c->d_faces, c->ET.view(), c->lam + c->nc, c->q, c->st);
        });
        if (bn_terms(c)) {
            // q -= (B^N - B^1) Q lam: N - 1 further terms of the series (Eq. 9c)
            const long long n2 = 2 * c->nc;
            DotArgs none;
            L(c, PC_PROJECT, 1, 32.0 * n2, [&] { launch_bn_start(n2, c->vmdt, c->q, c->qs, c->vp, c->grid, c->st); });
            for (int k = 1; k < c->cfg.bn_order; ++k) {
                L(c, PC_PROJECT, 1, st_bytes(MODE_APPLY, DK_NONE, 8, 8, 8, n2), [&] {
                    launch_stencil(MODE_APPLY, DK_NONE, A, c->vp, (const double*)nullptr, c->vAp, 0.0, none, c->g_vel, c->st);
                });
                L(c, PC_PROJECT, 1, 48.0 * n2, [&] { launch_bn_term(n2, c->vmdt, c->vAp, c->vp, c->q, c->grid, c->st); });
            }
        }
        L(c, PC_FORCES, 1, 16.0 * c->n_b, [&] { launch_forces(c->n_b, c->lam + c->nc, c->d_forces, c->st); });
        // FP64 constraint check of q^{n+1} (Eq. 8): continuity rows and no-slip rows
        L(c, PC_CONSTRAINTS, 1, 16.0 * c->nc + csr_bytes(c->E.n, c->E.nnz, 8) + 8.0 * c->E.n, [&] {
            launch_constraints(g, p, c->q, b, c->E.view(), c->d_ub, c->d_forces, c->g_pois, c->st);
        });
        CUDA_OK(cudaMemcpyAsync(c->hforces, c->d_forces, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        c->d2h_bytes += 4 * int64_t(sizeof(double));
        CUDA_OK(cudaStreamSynchronize(c->st));
        CUDA_OK(cudaGetLastError());
        if (c->cfg.warm == IBM_WARM_CNN && c->cnn) {   // a tcgen05 convolution that gave up
            std::string e;
            if (int rc2 = ibm::cnn_tc_check(c->cnn, &e)) return fail(c, rc2, e);
        }
        c->ncur = np;
        c->bcur = 1 - c->bcur;
        c->lam_steps++;
        c->ab2_first = false;
        c->t += c->cfg.dt;
        c->step += 1;
        stt.t = c->t;
        if (c->schur_builds != builds0) stt.amg_rebuilt = 1;
        stt.fx = c->hforces[0];
        stt.fy = c->hforces[1];
        stt.div_max = c->hforces[2];
        stt.slip_max = c->hforces[3];
        {
            float pms = 0.f;
            CUDA_OK(cudaEventElapsedTime(&pms, c->ev_pois[0], c->ev_pois[1]));
            stt.poisson_ms = pms;
        }
        const double U = c->cfg.uinf != 0.0 ? c->cfg.uinf : 1.0;
        stt.cd = 2.0 * stt.fx / (U * U);
        stt.cl = 2.0 * stt.fy / (U * U);
        c->last1 = stt.solve1;
        c->last2 = stt.solve2;
        if (per_step) per_step[s] = stt;
        if (first_bad == IBM_OK && stt.solve1.status != IBM_OK) first_bad = stt.solve1.status;
        if (first_bad == IBM_OK && stt.solve2.status != IBM_OK) first_bad = stt.solve2.status;
    }
    if (first_bad != IBM_OK) c->err = "a solver did not reach its tolerance (see per-step stats)";
    return first_bad;
}

int ibm_solve_poisson(ibm_ctx* c, const double* d_rhs, double* d_lambda, const double* d_lambda0,
                      ibm_solve_stats* stats) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!d_rhs || !d_lambda) return fail(c, IBM_ERR_ARG, "null device pointer");
    if (use_schur(c) && c->schur_stale && c->schur_built) {
        rc = is_mixed(c) ? build_schur<float>(c) : build_schur<double>(c);
        if (rc) return rc;
    } else if (!use_schur(c) && c->amg_stale && use_amg(c)) {
        if ((rc = rebuild_hierarchy(c))) return rc;
        if ((rc = upload_hier(c))) return rc;
    }
    if (d_lambda0) CUDA_OK(cudaMemcpyAsync(d_lambda, d_lambda0, c->nl * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    else CUDA_OK(cudaMemsetAsync(d_lambda, 0, c->nl * sizeof(double), c->st));
    ibm_solve_stats s{};
    if ((rc = solve_poisson_dev(c, d_rhs, d_lambda, &s))) return rc;
    CUDA_OK(cudaGetLastError());
    if (stats) *stats = s;
    return s.status;
}

int ibm_forces(ibm_ctx* c, double* fx, double* fy, double* cd, double* cl) {
    int rc = check_bound(c);
    if (rc) return rc;
    const int nb = c->n_b;
    if (nb > 0 && (fx || fy)) {
        std::vector<double> f(2 * nb);
        CUDA_OK(cudaMemcpyAsync(f.data(), c->lam + c->nc, 2 * nb * sizeof(double), cudaMemcpyDeviceToHost, c->st));
        CUDA_OK(cudaStreamSynchronize(c->st));
        if (fx) std::copy(f.begin(), f.begin() + nb, fx);
        if (fy) std::copy(f.begin() + nb, f.end(), fy);
    }
    L(c, PC_FORCES, 1, 16.0 * c->n_b, [&] { launch_forces(nb, c->lam + c->nc, c->d_forces, c->st); });
    CUDA_OK(cudaMemcpyAsync(c->hforces, c->d_forces, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(cudaStreamSynchronize(c->st));
    const double U = c->cfg.uinf != 0.0 ? c->cfg.uinf : 1.0;
    if (cd) *cd = 2.0 * c->hforces[0] / (U * U);
    if (cl) *cl = 2.0 * c->hforces[1] / (U * U);
    return IBM_OK;
}

int ibm_get_state(ibm_ctx* c, double* u, double* v, double* v_right, double* nprev, double* lambda, double* t,
                  int64_t* step) {
    int rc = check_bound(c);
    if (rc) return rc;
    const int nx = c->g.nx, ny = c->g.ny;
    const long long nc = c->nc;
    std::vector<double> q(2 * nc), ur(ny), vr(ny + 1);
    CUDA_OK(cudaMemcpyAsync(q.data(), c->q, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(cudaMemcpyAsync(ur.data(), c->d_u_right[c->bcur], ny * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(cudaMemcpyAsync(vr.data(), c->d_v_right[c->bcur], (ny + 1) * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    if (nprev) {
        if (c->ab2_first) CUDA_OK(cudaMemsetAsync(c->Nbuf[1 - c->ncur], 0, 2 * nc * sizeof(double), c->st));
        CUDA_OK(cudaMemcpyAsync(nprev, c->Nbuf[1 - c->ncur], 2 * nc * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    }
    if (lambda) CUDA_OK(cudaMemcpyAsync(lambda, c->lam, c->nl * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(cudaStreamSynchronize(c->st));
    const Grid& g = c->g;
    if (u) {
        for (int j = 0; j < ny; ++j) {
            double* row = u + (long long)j * (nx + 1);
            row[0] = c->u_left[j];
            for (int i = 1; i < nx; ++i) row[i] = q[(long long)j * nx + i] / g.dy[j];
            row[nx] = ur[j];
        }
    }
    if (v) {
        for (int i = 0; i < nx; ++i) {
            v[i] = c->v_bottom[i];
            v[(long long)ny * nx + i] = c->v_top[i];
        }
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) v[(long long)j * nx + i] = q[nc + (long long)j * nx + i] / g.dx[i];
    }
    if (v_right) std::copy(vr.begin(), vr.end(), v_right);
    if (t) *t = c->t;
    if (step) *step = c->step;
    return IBM_OK;
}

int ibm_set_state(ibm_ctx* c, const double* u, const double* v, const double* v_right, const double* nprev,
                  const double* lambda, double t, int64_t step) {
    int rc = check_bound(c);
    if (rc) return rc;
    const int nx = c->g.nx, ny = c->g.ny;
    const long long nc = c->nc;
    const Grid& g = c->g;
    std::vector<double> q(2 * nc, 0.0);
    CUDA_OK(cudaMemcpyAsync(q.data(), c->q, 2 * nc * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CUDA_OK(cudaStreamSynchronize(c->st));
    if (u) {
        std::vector<double> ur(ny);
        for (int j = 0; j < ny; ++j) {
            const double* row = u + (long long)j * (nx + 1);
            c->u_left[j] = row[0];
            ur[j] = row[nx];
            for (int i = 1; i < nx; ++i) q[(long long)j * nx + i] = row[i] * g.dy[j];
        }
        if ((rc = up(c, c->d_u_left, c->u_left)) || (rc = up(c, c->d_u_right[c->bcur], ur))) return rc;
    }
    if (v) {
        for (int i = 0; i < nx; ++i) {
            c->v_bottom[i] = v[i];
            c->v_top[i] = v[(long long)ny * nx + i];
        }
        for (int j = 1; j < ny; ++j)
            for (int i = 0; i < nx; ++i) q[nc + (long long)j * nx + i] = v[(long long)j * nx + i] * g.dx[i];
        if ((rc = up(c, c->d_v_bottom, c->v_bottom)) || (rc = up(c, c->d_v_top, c->v_top))) return rc;
    }
    update_inflow(c);
    if ((rc = up(c, c->q, q))) return rc;
    if (v_right) {
        std::vector<double> vr(v_right, v_right + ny + 1);
        if ((rc = up(c, c->d_v_right[c->bcur], vr))) return rc;
    }
    if (nprev) {
        if ((rc = up(c, c->Nbuf[1 - c->ncur], nprev, 2 * nc))) return rc;
        c->ab2_first = false;
    } else {
        c->ab2_first = true;
    }
    if (lambda && (rc = up(c, c->lam, lambda, c->nl))) return rc;
    c->lam_steps = lambda ? 1 : 0;   // lambda^{n-1} is not part of the state
    c->proj_pois.m = 0;              // nor the projection basis
    c->proj_pois.solves = 0;
    c->t = t;
    c->step = step;
    CUDA_OK(cudaStreamSynchronize(c->st));
    return IBM_OK;
}

int ibm_apply_poisson(ibm_ctx* c, const double* d_x, double* d_y) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!d_x || !d_y) return fail(c, IBM_ERR_ARG, "null device pointer");
    if (bn_mf(c) && !c->bn_dpin_ok && (rc = bn_pin_diag(c))) return rc;
    pois_apply(c, MODE_APPLY, DK_NONE, FIN_NONE, d_x, nullptr, d_y, 1);
    CUDA_OK(cudaGetLastError());
    CUDA_OK(cudaStreamSynchronize(c->st));
    return IBM_OK;
}

int ibm_vcycle(ibm_ctx* c, const double* d_r, double* d_z) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (!d_r || !d_z) return fail(c, IBM_ERR_ARG, "null device pointer");
    if (!use_amg(c) || !c->have_H || c->lev.size() < 2) return fail(c, IBM_ERR_STATE, "no AMG hierarchy");
    if ((rc = reset_barrier(c))) return rc;
    if (use_schur(c)) {
        // pressure-block V-cycle (nx*ny entries)
        if (is_mixed(c)) vcycle_gen<float, double>(c, d_r, d_z, false, nullptr, nullptr);
        else vcycle_gen<double, double>(c, d_r, d_z, false, nullptr, nullptr);
    } else {
        if (c->amg_stale) {
            if ((rc = rebuild_hierarchy(c))) return rc;
            if ((rc = upload_hier(c))) return rc;
        }
        if (is_mixed(c)) vcycle<float>(c, d_r, d_z, nullptr, nullptr, nullptr, false);
        else vcycle<double>(c, d_r, d_z, nullptr, nullptr, nullptr, false);
    }
    CUDA_OK(cudaGetLastError());
    CUDA_OK(cudaStreamSynchronize(c->st));
    return check_barrier(c);
}

int ibm_attach_cnn(ibm_ctx* c, ibm_cnn* net) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (net && ibm::cnn_stream(net) != c->st)
        return fail(c, IBM_ERR_ARG, "the network must be bound on the context's stream");
    c->cnn = net;
    return IBM_OK;
}

int ibm_snapshot(ibm_ctx* c, double* d_lambda, double* d_lambda_prev, double* d_rhs, double* d_r0) {
    int rc = check_bound(c);
    if (rc) return rc;
    c->snapshots = true;   // from now on the residual of the extrapolated guess is kept
    const size_t b = c->nl * sizeof(double);
    if (d_r0) CUDA_OK(cudaMemcpyAsync(d_r0, c->r_ex, b, cudaMemcpyDeviceToDevice, c->st));
    if (d_lambda) CUDA_OK(cudaMemcpyAsync(d_lambda, c->lam, b, cudaMemcpyDeviceToDevice, c->st));
    if (d_lambda_prev) CUDA_OK(cudaMemcpyAsync(d_lambda_prev, c->lam_prev, b, cudaMemcpyDeviceToDevice, c->st));
    if (d_rhs) CUDA_OK(cudaMemcpyAsync(d_rhs, c->b2, b, cudaMemcpyDeviceToDevice, c->st));
    CUDA_OK(cudaStreamSynchronize(c->st));
    return IBM_OK;
}

int ibm_amg_levels(const ibm_ctx* c, int32_t* nlevels) {
    if (!c || !nlevels) return IBM_ERR_ARG;
    *nlevels = c->have_H ? int32_t(c->H.levels.size()) : 0;
    return IBM_OK;
}

int ibm_amg_matrix(const ibm_ctx* c, int32_t level, int32_t which, int64_t* nrows, int64_t* ncols, int64_t* nnz,
                   int64_t* rowptr, int32_t* colind, double* vals) {
    if (!c || !c->have_H || level < 0 || level >= int32_t(c->H.levels.size())) return IBM_ERR_ARG;
    const AmgLevel& L0 = c->H.levels[level];
    if (which < 0 || which > 3) return IBM_ERR_ARG;
    const CSR& M = which == 0 ? L0.A : which == 1 ? L0.P : which == 2 ? L0.Rt : L0.Q;
    if (nrows) *nrows = M.n;
    if (ncols) *ncols = M.m;
    if (nnz) *nnz = M.nnz();
    if (rowptr) std::copy(M.rowptr.begin(), M.rowptr.end(), rowptr);
    if (colind) std::copy(M.col.begin(), M.col.end(), colind);
    if (vals) std::copy(M.val.begin(), M.val.end(), vals);
    return IBM_OK;
}

int ibm_amg_level_info(const ibm_ctx* c, int32_t level, int64_t* nrows, double* omega) {
    if (!c || !c->have_H || level < 0 || level >= int32_t(c->H.levels.size())) return IBM_ERR_ARG;
    if (nrows) *nrows = c->H.levels[level].A.n;
    if (omega) *omega = c->H.levels[level].omega;
    return IBM_OK;
}

int ibm_profile_enable(ibm_ctx* c, int32_t on) {
    if (!c) return IBM_ERR_ARG;
    if (on && c->ev.empty()) {
        c->ev.resize(8192);
        for (auto& e : c->ev) CUDA_OK(cudaEventCreate(&e));
    }
    if (!on) prof_harvest(c);
    c->prof_on = on != 0;
    return IBM_OK;
}

int ibm_profile_reset(ibm_ctx* c) {
    if (!c) return IBM_ERR_ARG;
    prof_harvest(c);
    for (int k = 0; k < PC_COUNT; ++k) {
        c->prof_launch[k] = 0;
        c->prof_ms[k] = 0.0;
        c->prof_bytes[k] = 0.0;
    }
    return IBM_OK;
}

int ibm_profile_count(const ibm_ctx* c, int32_t* nclasses) {
    if (!c || !nclasses) return IBM_ERR_ARG;
    *nclasses = PC_COUNT;
    return IBM_OK;
}

int ibm_profile_get(ibm_ctx* c, int32_t k, const char** name, int64_t* launches, double* ms, double* bytes) {
    if (!c || k < 0 || k >= PC_COUNT) return IBM_ERR_ARG;
    prof_harvest(c);
    if (name) *name = kProfNames[k];
    if (launches) *launches = c->prof_launch[k];
    if (ms) *ms = c->prof_ms[k];
    if (bytes) *bytes = c->prof_bytes[k];
    return IBM_OK;
}

int ibm_profile_graph_class(ibm_ctx* c, int32_t k, int32_t reps, int64_t* launches, double* ms_per_launch,
                            double* bytes_per_launch) {
    int rc = check_bound(c);
    if (rc) return rc;
    if (k < 0 || k >= PC_COUNT || reps < 1) return fail(c, IBM_ERR_ARG, "bad class or repetition count");
    if (c->prof_on) return fail(c, IBM_ERR_STATE, "per-launch event profiling is on");
    if (!c->gprof_st) CUDA_OK(cudaStreamCreateWithFlags(&c->gprof_st, cudaStreamNonBlocking));
    // capture the class's launches of one step; loop graphs are rebuilt so that
    // their bodies' launches pass through the capture too
    cudaGraph_t g = nullptr;
    CUDA_OK(cudaStreamBeginCapture(c->gprof_st, cudaStreamCaptureModeRelaxed));
    c->gprof_cls = k;
    c->gprof_n = 0;
    c->gprof_bytes = 0.0;
    c->graph_version++;
    ibm_step_stats st{};
    rc = ibm_step(c, 1, &st);
    c->gprof_cls = -1;
    const cudaError_t ce = cudaStreamEndCapture(c->gprof_st, &g);
    if (rc && rc != IBM_ERR_NOT_CONVERGED) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return fail(c, IBM_ERR_CUDA, std::string("class capture: ") + cudaGetErrorString(ce));
    if (c->gprof_n == 0) {
        cudaGraphDestroy(g);
        return fail(c, IBM_ERR_STATE, "no launch of this class in a step");
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, IBM_ERR_CUDA, std::string("class graph: ") + cudaGetErrorString(e));
    // solver scalars: not done, never converging, restored afterwards
    CgScalars save[2];
    CUDA_OK(cudaMemcpy(&save[0], c->sc1, sizeof(CgScalars), cudaMemcpyDeviceToHost));
    CUDA_OK(cudaMemcpy(&save[1], c->sc2, sizeof(CgScalars), cudaMemcpyDeviceToHost));
    CgScalars live[2] = {save[0], save[1]};
    for (auto& h : live) {
        h.done = 0;
        h.tol2 = 0.0;
        h.iter = 0;
        h.max_iter = 1 << 30;
    }
    CUDA_OK(cudaMemcpy(c->sc1, &live[0], sizeof(CgScalars), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemcpy(c->sc2, &live[1], sizeof(CgScalars), cudaMemcpyHostToDevice));
    // a class graph may hold only part of a fused reduction, whose last block
    // then finalises garbage that can set `done`: the flags are cleared before
    // every replay, outside the timed interval of that replay
    std::vector<cudaEvent_t> evs(2 * size_t(reps) + 2, nullptr);
    double ms = 0.0;
    e = cudaSuccess;
    for (auto& v : evs)
        if (e == cudaSuccess) e = cudaEventCreate(&v);
    const int32_t zero2[2] = {0, 0};
    for (int r = -1; r < reps && e == cudaSuccess; ++r) {   // r = -1: untimed
        e = cudaMemcpyAsync(&c->sc1->done, zero2, sizeof(zero2), cudaMemcpyHostToDevice, c->gprof_st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&c->sc2->done, zero2, sizeof(zero2), cudaMemcpyHostToDevice, c->gprof_st);
        if (e == cudaSuccess) e = cudaEventRecord(evs[2 * (r + 1)], c->gprof_st);
        if (e == cudaSuccess) e = cudaGraphLaunch(ex, c->gprof_st);
        if (e == cudaSuccess) e = cudaEventRecord(evs[2 * (r + 1) + 1], c->gprof_st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->gprof_st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, evs[2 * (r + 1)], evs[2 * (r + 1) + 1]);
        ms += t;
    }
    for (auto& v : evs)
        if (v) cudaEventDestroy(v);
    cudaGraphExecDestroy(ex);
    CUDA_OK(cudaMemcpy(c->sc1, &save[0], sizeof(CgScalars), cudaMemcpyHostToDevice));
    CUDA_OK(cudaMemcpy(c->sc2, &save[1], sizeof(CgScalars), cudaMemcpyHostToDevice));
    if (e != cudaSuccess) return fail(c, IBM_ERR_CUDA, std::string("class replay: ") + cudaGetErrorString(e));
    c->graph_version++;
    if (launches) *launches = c->gprof_n;
    if (ms_per_launch) *ms_per_launch = ms / (double(reps) * double(c->gprof_n));
    if (bytes_per_launch) *bytes_per_launch = c->gprof_bytes / double(c->gprof_n);
    return IBM_OK;
}

int ibm_transfer_bytes(const ibm_ctx* c, int64_t* h2d, int64_t* d2h) {
    if (!c) return IBM_ERR_ARG;
    if (h2d) *h2d = c->h2d_bytes;
    if (d2h) *d2h = c->d2h_bytes;
    return IBM_OK;
}

int ibm_launch_count(const ibm_ctx* c, int64_t* launches) {
    if (!c || !launches) return IBM_ERR_ARG;
    *launches = c->launches;
    return IBM_OK;
}

}  // extern "C"

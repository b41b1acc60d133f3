// Host-side set-up of the immersed-boundary projection step: grid metrics,
// operator coefficients, interpolation rows E (Eq. 6), the coupling blocks of
// Q^T B^1 Q and the smoothed-aggregation AMG hierarchy (section 3).
// Plain C++ (no CUDA); everything here runs once at set-up or, for moving
// bodies, once per body update.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ibm.h"

namespace ibm {

struct CSR {
    int64_t n = 0, m = 0;              // rows, columns
    std::vector<int64_t> rowptr;       // n + 1
    std::vector<int32_t> col;
    std::vector<double> val;
    int64_t nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
};

// Sliced ELLPACK with 32-row slices (one warp per slice on the device):
// entry k of row 32 s + t is stored at off[s] + 32 k + t; a slice is as wide
// as its longest row, and padding entries have value 0 and a valid column
// (the row itself, or 0 past the last row).
constexpr int kSellRows = 32;
struct Sell {
    int64_t n = 0, nslices = 0;
    std::vector<int64_t> off;          // nslices + 1
    std::vector<int32_t> col;
    std::vector<double> val;
};
int64_t sell_entries(const CSR& A);    // stored entries, padding included
Sell to_sell(const CSR& A);

// 1D metrics of the staggered grid.
struct Grid {
    int nx = 0, ny = 0;
    std::vector<double> xf, yf;        // faces (nx+1, ny+1)
    std::vector<double> dx, dy;        // cell widths
    std::vector<double> xc, yc;        // cell centres
    std::vector<double> dxf, dyf;      // centre-to-centre spacing at faces (index 1..n-1)
    int64_t nc() const { return int64_t(nx) * ny; }
};

// Rows of E for the current body positions, in the padded velocity numbering
// (u slot (i,j) -> j*nx+i, v slot (i,j) -> nx*ny + j*nx+i).
struct BodyRows {
    int n_b = 0;
    CSR E;        // 2 n_b rows (x components, then y), columns = padded q index
    CSR ET;       // face-major: rows = touched faces (face list), cols = E row
    std::vector<int64_t> faces;        // touched padded-q indices (sorted)
    // coupling blocks of the pinned Q^T B^1 Q in lambda numbering
    std::vector<int64_t> tcells;       // touched cells (sorted)
    CSR Cc;       // rows = touched cells, cols = lambda index of forces
    CSR Cf;       // rows = force unknowns (2 n_b), cols = lambda index (cells and forces)
};

struct AmgParams {
    double theta = 0.08, omega = 2.0 / 3.0;
    double trunc = 0.0;    // drop P entries below trunc * (row max), keep row sums
    int pre = 2, post = 2, max_coarse = 256, max_levels = 12;
};

struct AmgLevel {
    CSR A;                             // level operator
    CSR P;                             // prolongator from level l+1 (empty on the coarsest)
    CSR R;                             // P^T
    std::vector<double> invdiag;
    std::vector<int32_t> agg;          // aggregate of each row (-1: none)
    double rho = 0.0;                  // estimate of rho(D^-1 A)
    double omega = 0.0;                // damped-Jacobi weight used on this level
    CSR Rt, Q;                         // fused transfers (fused_transfers; empty when unused)
};

struct Hierarchy {
    std::vector<AmgLevel> levels;
    std::vector<double> coarse_inv;    // dense inverse of the coarsest operator (row-major)
    int64_t coarse_n = 0;
    double build_ms = 0.0;
};

// --- grid and operators -------------------------------------------------------
Grid make_grid(int nx, int ny, const double* xf, const double* yf);

// Padded velocity operator A = M/dt - L/2 on a 2 x ny x nx array (u block
// then v block).  Off-diagonal entries are -cE (east) and -cN (north).
struct VelocityCoeffs {
    std::vector<double> cE, cN, diag, idiag, mdt;   // each 2*nc
};
VelocityCoeffs velocity_coeffs(const Grid& g, double nu, double dt);

// Pinned pressure block of Q^T B^1 Q: off-diagonals -wE (east), -wN (north);
// diag over all n_lambda rows (cells, then forces).
struct PoissonCoeffs {
    std::vector<double> wE, wN;        // nc each
    std::vector<double> diag;          // n_lambda
};
PoissonCoeffs poisson_coeffs(const Grid& g, double dt, int64_t pin, const BodyRows& br);

// --- bodies ----------------------------------------------------------------------
double roma_delta(double r, double h);
// Returns false (with a message) if a point's support leaves the uniform cells.
bool build_body_rows(const Grid& g, double h, double dt, int64_t pin, int n_b,
                     const double* xb, const double* yb, BodyRows* out, std::string* err);

// The sparsity pattern of the body rows alone (integer work, no weights), for
// the device-side assembly of a moving body: the rows, columns and orders of
// E, of its face-major transpose, of the touched cells' rows C and of the
// force rows [C^T | F] are those build_body_rows produces up to the order of
// entries within a row (a weight of Eq. 5 is nonzero exactly where
// |x - xi| < 1.5 h in both directions); the values stay empty and are formed
// on the device from the index maps below.
struct BodySrc {
    std::vector<int32_t> et_src;       // per E^T entry: its E entry
    std::vector<int32_t> cf_a, cf_b;   // per force-row entry: C^T part - up to two E entries
                                       // (2 e + 1 for the minus side, -1 none); F part: -1, -1
    std::vector<int32_t> cc_src;       // per touched-cell entry: its force-row entry
    std::vector<int32_t> diag;         // per force row: its diagonal entry
    std::vector<int32_t> point;        // per E row: the body point
};
// Scratch maps of body_pattern, kept between calls (sized on first use).
struct BodyMaps {
    std::vector<int32_t> face_slot, cell_slot, cell_stamp, row_stamp;
};
bool body_pattern(const Grid& g, double h, int64_t pin, int n_b, const double* xb, const double* yb, BodyRows* out,
                  BodySrc* src, BodyMaps* maps, std::string* err);

// Full pinned Q^T B^1 Q in lambda numbering (for the AMG set-up and checks).
CSR assemble_poisson(const Grid& g, const PoissonCoeffs& pc, const BodyRows& br);
// Q^T B^N Q (Eq. 9b with B^N = sum_{k<N} ((dt/2) M^-1 L)^k dt M^-1, the N-term
// expansion of A^-1), pinned, by a sliced triple product: `slice` rows of Q^T
// at a time are multiplied by B^N and then by Q, so only one slice of Q^T B^N
// is held (section 4).  For N = 1 it equals assemble_poisson.
CSR assemble_poisson_bn(const Grid& g, const VelocityCoeffs& vc, double dt, int N, int64_t pin, const BodyRows& br,
                        int64_t slice);

// --- AMG -------------------------------------------------------------------------
bool build_hierarchy(const CSR& A0, const AmgParams& prm, Hierarchy* H, std::string* err);
bool spd_inverse(const std::vector<double>& A, int64_t n, std::vector<double>* inv, std::string* err);
CSR transpose(const CSR& A);
CSR spgemm(const CSR& A, const CSR& B);
// Transfer operators of one level that fold its damped-Jacobi sweeps into
// the grid transfers (S = I - omega D^-1 A is a sweep's error propagation):
//   Rt = R (I - A omega D^-1)^pre : the residual after `pre` sweeps from x = 0
//        is (I - A omega D^-1)^pre b, so the coarse right-hand side is Rt b;
//   Q  = S P                     : the first sweep after the coarse
//        correction is x + omega D^-1 (b - A x) + S P x_c.
void fused_transfers(const AmgLevel& L, int pre, CSR* Rt, CSR* Q);

}  // namespace ibm

// Host-side set-up: grid metrics, operator coefficients, rows E of Q (Eq. 6),
// coupling blocks of Q^T B^1 Q (Eq. 9b) and the smoothed-aggregation AMG
// hierarchy (section 3).
#include "host.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <map>
#include <utility>

namespace ibm {

// ---------------------------------------------------------------------------
// Grid
// ---------------------------------------------------------------------------
Grid make_grid(int nx, int ny, const double* xf, const double* yf) {
    Grid g;
    g.nx = nx;
    g.ny = ny;
    g.xf.assign(xf, xf + nx + 1);
    g.yf.assign(yf, yf + ny + 1);
    g.dx.resize(nx);
    g.xc.resize(nx);
    for (int i = 0; i < nx; ++i) {
        g.dx[i] = xf[i + 1] - xf[i];
        g.xc[i] = 0.5 * (xf[i] + xf[i + 1]);
    }
    g.dy.resize(ny);
    g.yc.resize(ny);
    for (int j = 0; j < ny; ++j) {
        g.dy[j] = yf[j + 1] - yf[j];
        g.yc[j] = 0.5 * (yf[j] + yf[j + 1]);
    }
    g.dxf.assign(nx + 1, 0.0);
    for (int i = 1; i < nx; ++i) g.dxf[i] = g.xc[i] - g.xc[i - 1];
    g.dyf.assign(ny + 1, 0.0);
    for (int j = 1; j < ny; ++j) g.dyf[j] = g.yc[j] - g.yc[j - 1];
    return g;
}

// Viscous term of the u- and v-momentum control volumes, divided by dy_j
// (u rows) or dx_i (v rows) so that it acts on the fluxes q (Eq. 7 operators).
// Tangential walls: boundary value on the wall, half a cell away.
VelocityCoeffs velocity_coeffs(const Grid& g, double nu, double dt) {
    const int nx = g.nx, ny = g.ny;
    const int64_t nc = g.nc();
    VelocityCoeffs c;
    c.cE.assign(2 * nc, 0.0);
    c.cN.assign(2 * nc, 0.0);
    c.diag.assign(2 * nc, 1.0);
    c.idiag.assign(2 * nc, 1.0);
    c.mdt.assign(2 * nc, 0.0);
    // u block: slot (i, j), i = 1..nx-1
    for (int j = 0; j < ny; ++j) {
        for (int i = 1; i < nx; ++i) {
            const int64_t k = int64_t(j) * nx + i;
            const double dyj = g.dy[j], dxf = g.dxf[i];
            double Ld = -nu / dyj * (1.0 / g.dx[i] + 1.0 / g.dx[i - 1]);
            if (i + 1 <= nx - 1) c.cE[k] = 0.5 * nu / (dyj * g.dx[i]);
            if (j + 1 <= ny - 1) {
                c.cN[k] = 0.5 * nu * dxf / (dyj * g.dyf[j + 1] * g.dy[j + 1]);
                Ld -= nu * dxf / (dyj * dyj * g.dyf[j + 1]);
            } else {
                Ld -= 2.0 * nu * dxf / (dyj * dyj * dyj);
            }
            if (j - 1 >= 0) Ld -= nu * dxf / (dyj * dyj * g.dyf[j]);
            else Ld -= 2.0 * nu * dxf / (dyj * dyj * dyj);
            const double M = dxf / dyj;
            c.mdt[k] = M / dt;
            c.diag[k] = M / dt - 0.5 * Ld;
            c.idiag[k] = 1.0 / c.diag[k];
        }
    }
    // v block: slot (i, j), j = 1..ny-1
    for (int j = 1; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            const int64_t k = nc + int64_t(j) * nx + i;
            const double dxi = g.dx[i], dyf = g.dyf[j];
            double Ld = -nu / dxi * (1.0 / g.dy[j] + 1.0 / g.dy[j - 1]);
            if (j + 1 <= ny - 1) c.cN[k] = 0.5 * nu / (dxi * g.dy[j]);
            if (i + 1 <= nx - 1) {
                c.cE[k] = 0.5 * nu * dyf / (dxi * g.dxf[i + 1] * g.dx[i + 1]);
                Ld -= nu * dyf / (dxi * dxi * g.dxf[i + 1]);
            } else {
                Ld -= 2.0 * nu * dyf / (dxi * dxi * dxi);
            }
            if (i - 1 >= 0) Ld -= nu * dyf / (dxi * dxi * g.dxf[i]);
            else Ld -= 2.0 * nu * dyf / (dxi * dxi * dxi);
            const double M = dyf / dxi;
            c.mdt[k] = M / dt;
            c.diag[k] = M / dt - 0.5 * Ld;
            c.idiag[k] = 1.0 / c.diag[k];
        }
    }
    return c;
}

// ---------------------------------------------------------------------------
// Discrete delta (Eq. 5, Roma, Peskin & Berger)
// ---------------------------------------------------------------------------
double roma_delta(double r, double h) {
    const double a = std::fabs(r) / h;
    if (a <= 0.5) return (1.0 + std::sqrt(1.0 - 3.0 * a * a)) / (3.0 * h);
    if (a <= 1.5) {
        const double s = 1.0 - 3.0 * (1.0 - a) * (1.0 - a);
        return (5.0 - 3.0 * a - std::sqrt(s > 0.0 ? s : 0.0)) / (6.0 * h);
    }
    return 0.0;
}

static inline double face_B_u(const Grid& g, double dt, int i, int j) { return dt * g.dy[j] / g.dxf[i]; }
static inline double face_B_v(const Grid& g, double dt, int i, int j) { return dt * g.dx[i] / g.dyf[j]; }

static bool uniform_near(const std::vector<double>& w, int lo, int hi, double h) {
    if (lo < 0 || hi >= int(w.size())) return false;
    for (int k = lo; k <= hi; ++k)
        if (std::fabs(w[k] - h) > 1e-9 * h) return false;
    return true;
}

static CSR csr_from_triplets(int64_t n, int64_t m, std::vector<std::tuple<int64_t, int64_t, double>>& t) {
    std::sort(t.begin(), t.end(), [](const auto& a, const auto& b) {
        return std::get<0>(a) != std::get<0>(b) ? std::get<0>(a) < std::get<0>(b) : std::get<1>(a) < std::get<1>(b);
    });
    CSR A;
    A.n = n;
    A.m = m;
    A.rowptr.assign(n + 1, 0);
    for (size_t k = 0; k < t.size();) {
        size_t e = k;
        double s = 0.0;
        while (e < t.size() && std::get<0>(t[e]) == std::get<0>(t[k]) && std::get<1>(t[e]) == std::get<1>(t[k])) {
            s += std::get<2>(t[e]);
            ++e;
        }
        A.col.push_back(int32_t(std::get<1>(t[k])));
        A.val.push_back(s);
        A.rowptr[std::get<0>(t[k]) + 1]++;
        k = e;
    }
    for (int64_t i = 0; i < n; ++i) A.rowptr[i + 1] += A.rowptr[i];
    return A;
}

bool build_body_rows(const Grid& g, double h, double dt, int64_t pin, int n_b,
                     const double* xb, const double* yb, BodyRows* out, std::string* err) {
    const int nx = g.nx, ny = g.ny;
    const int64_t nc = g.nc();
    BodyRows br;
    br.n_b = n_b;
    std::vector<std::tuple<int64_t, int64_t, double>> tE;
    for (int k = 0; k < n_b; ++k) {
        const double xi = xb[k], eta = yb[k];
        if (!std::isfinite(xi) || !std::isfinite(eta)) {
            *err = "body point " + std::to_string(k) + " is not finite";
            return false;
        }
        // cell containing the point; the support (1.5 h) lies within cells i0-2..i0+2
        const int i0 = int(std::upper_bound(g.xf.begin(), g.xf.end(), xi) - g.xf.begin()) - 1;
        const int j0 = int(std::upper_bound(g.yf.begin(), g.yf.end(), eta) - g.yf.begin()) - 1;
        // the cells whose widths enter a non-zero weight (Eq. 5): both cells
        // beside each face strictly within 1.5 h of the point (its dxf or
        // dyf), which include the cell of each such centre
        auto span = [&](const std::vector<double>& f, double p, int* lo, int* hi) {
            *lo = int(std::upper_bound(f.begin(), f.end(), p - 1.5 * h) - f.begin()) - 1;
            *hi = int(std::lower_bound(f.begin(), f.end(), p + 1.5 * h) - f.begin()) - 1;
        };
        int ilo = 0, ihi = -1, jlo = 0, jhi = -1;
        span(g.xf, xi, &ilo, &ihi);
        span(g.yf, eta, &jlo, &jhi);
        // the rows below touch faces i0-1..i0+2 and j0-2..j0+2, all interior
        const bool near_edge = i0 < 3 || i0 > nx - 4 || j0 < 3 || j0 > ny - 4;
        if (near_edge || !uniform_near(g.dx, ilo, ihi, h) || !uniform_near(g.dy, jlo, jhi, h)) {
            char buf[192];
            if (near_edge)
                std::snprintf(buf, sizeof buf,
                              "body point %d at (%g, %g) lies in one of the three cells next to the edge of the grid",
                              k, xi, eta);
            else
                std::snprintf(buf, sizeof buf, "body point %d at (%g, %g) is not inside uniform cells of width %g",
                              k, xi, eta, h);
            *err = buf;
            return false;
        }
        // u faces x = xf[i], y = yc[j]
        for (int i = i0 - 1; i <= i0 + 2; ++i) {
            const double wx = roma_delta(g.xf[i] - xi, h);
            if (wx == 0.0) continue;
            for (int j = j0 - 2; j <= j0 + 2; ++j) {
                const double wy = roma_delta(g.yc[j] - eta, h);
                if (wy == 0.0) continue;
                tE.emplace_back(k, int64_t(j) * nx + i, g.dxf[i] * wx * wy);
            }
        }
        // v faces x = xc[i], y = yf[j]
        for (int i = i0 - 2; i <= i0 + 2; ++i) {
            const double wx = roma_delta(g.xc[i] - xi, h);
            if (wx == 0.0) continue;
            for (int j = j0 - 1; j <= j0 + 2; ++j) {
                const double wy = roma_delta(g.yf[j] - eta, h);
                if (wy == 0.0) continue;
                tE.emplace_back(n_b + k, nc + int64_t(j) * nx + i, g.dyf[j] * wx * wy);
            }
        }
    }
    br.E = csr_from_triplets(2 * int64_t(n_b), 2 * nc, tE);

    // face-major transpose with the touched-face list
    std::vector<std::tuple<int64_t, int64_t, double>> tT;
    for (int64_t r = 0; r < br.E.n; ++r)
        for (int64_t p = br.E.rowptr[r]; p < br.E.rowptr[r + 1]; ++p) tT.emplace_back(br.E.col[p], r, br.E.val[p]);
    std::sort(tT.begin(), tT.end(), [](const auto& a, const auto& b) {
        return std::get<0>(a) != std::get<0>(b) ? std::get<0>(a) < std::get<0>(b) : std::get<1>(a) < std::get<1>(b);
    });
    br.ET.n = 0;
    br.ET.m = br.E.n;
    br.ET.rowptr.push_back(0);
    for (size_t k = 0; k < tT.size(); ++k) {
        if (k == 0 || std::get<0>(tT[k]) != std::get<0>(tT[k - 1])) {
            br.faces.push_back(std::get<0>(tT[k]));
            if (k) br.ET.rowptr.push_back(int64_t(k));
        }
        br.ET.col.push_back(int32_t(std::get<1>(tT[k])));
        br.ET.val.push_back(std::get<2>(tT[k]));
    }
    if (!tT.empty()) br.ET.rowptr.push_back(int64_t(tT.size()));
    br.ET.n = int64_t(br.faces.size());

    // B of a face and the two cells the face separates (+ side, - side)
    auto face_info = [&](int64_t f, double* B, int64_t* cp, int64_t* cm) {
        if (f < nc) {
            const int i = int(f % nx), j = int(f / nx);
            *B = face_B_u(g, dt, i, j);
            *cp = int64_t(j) * nx + i;
            *cm = int64_t(j) * nx + (i - 1);
        } else {
            const int64_t s = f - nc;
            const int i = int(s % nx), j = int(s / nx);
            *B = face_B_v(g, dt, i, j);
            *cp = int64_t(j) * nx + i;
            *cm = int64_t(j - 1) * nx + i;
        }
    };
    // C = G^T B E^T (cells x forces) and F = E B E^T (forces x forces)
    std::vector<std::tuple<int64_t, int64_t, double>> tC, tF;
    for (int64_t r = 0; r < br.E.n; ++r) {
        for (int64_t p = br.E.rowptr[r]; p < br.E.rowptr[r + 1]; ++p) {
            double B;
            int64_t cp, cm;
            face_info(br.E.col[p], &B, &cp, &cm);
            const double v = B * br.E.val[p];
            if (cp != pin) tC.emplace_back(cp, nc + r, v);
            if (cm != pin) tC.emplace_back(cm, nc + r, -v);
        }
    }
    for (int64_t t = 0; t < br.ET.n; ++t) {
        double B;
        int64_t cp, cm;
        face_info(br.faces[t], &B, &cp, &cm);
        for (int64_t a = br.ET.rowptr[t]; a < br.ET.rowptr[t + 1]; ++a)
            for (int64_t b = br.ET.rowptr[t]; b < br.ET.rowptr[t + 1]; ++b)
                tF.emplace_back(br.ET.col[a], nc + br.ET.col[b], br.ET.val[a] * B * br.ET.val[b]);
    }
    // touched cells only (no pass over all nc cells: this runs every step for a
    // moving body): sort by (cell, force), sum duplicates
    std::sort(tC.begin(), tC.end(), [](const auto& a, const auto& b) {
        return std::get<0>(a) != std::get<0>(b) ? std::get<0>(a) < std::get<0>(b) : std::get<1>(a) < std::get<1>(b);
    });
    br.Cc.n = 0;
    br.Cc.m = nc + 2 * int64_t(n_b);
    br.Cc.rowptr.push_back(0);
    std::vector<std::tuple<int64_t, int64_t, double>> tR;   // force rows: C^T entries then F entries
    for (size_t k = 0; k < tC.size();) {
        const int64_t cell = std::get<0>(tC[k]);
        size_t e = k;
        while (e < tC.size() && std::get<0>(tC[e]) == cell) {
            const int64_t col = std::get<1>(tC[e]);
            double v = 0.0;
            while (e < tC.size() && std::get<0>(tC[e]) == cell && std::get<1>(tC[e]) == col) v += std::get<2>(tC[e++]);
            br.Cc.col.push_back(int32_t(col));
            br.Cc.val.push_back(v);
            tR.emplace_back(col - nc, cell, v);
        }
        br.tcells.push_back(cell);
        br.Cc.rowptr.push_back(int64_t(br.Cc.col.size()));
        k = e;
    }
    br.Cc.n = int64_t(br.tcells.size());
    for (auto& e : tF) tR.push_back(e);
    br.Cf = csr_from_triplets(2 * int64_t(n_b), nc + 2 * int64_t(n_b), tR);
    *out = std::move(br);
    return true;
}

bool body_pattern(const Grid& g, double h, int64_t pin, int n_b, const double* xb, const double* yb, BodyRows* out,
                  BodySrc* src, BodyMaps* maps, std::string* err) {
    const int nx = g.nx, ny = g.ny;
    const int64_t nc = g.nc();
    BodyRows br;
    BodySrc sr;
    br.n_b = n_b;
    if (maps->face_slot.size() != size_t(2 * nc)) maps->face_slot.assign(size_t(2 * nc), -1);
    if (maps->cell_slot.size() != size_t(nc)) maps->cell_slot.assign(size_t(nc), -1);
    // entries of E: a weight of Eq. 5 is nonzero exactly where |r| < 1.5 h in
    // both directions; rows u (0..n_b-1) then v, columns ascending
    br.E.n = 2 * int64_t(n_b);
    br.E.m = 2 * nc;
    br.E.rowptr.assign(1, 0);
    sr.point.resize(size_t(2 * n_b));
    struct Span {
        int i0, i1, j0, j1;
    };
    std::vector<Span> su(n_b), sv(n_b);
    auto in_support = [&](double d) { return std::fabs(d) / h < 1.5; };
    for (int k = 0; k < n_b; ++k) {
        const double xi = xb[k], eta = yb[k];
        if (!std::isfinite(xi) || !std::isfinite(eta)) {
            *err = "body point " + std::to_string(k) + " is not finite";
            return false;
        }
        const int i0 = int(std::upper_bound(g.xf.begin(), g.xf.end(), xi) - g.xf.begin()) - 1;
        const int j0 = int(std::upper_bound(g.yf.begin(), g.yf.end(), eta) - g.yf.begin()) - 1;
        auto span = [&](const std::vector<double>& f, double p, int* lo, int* hi) {
            *lo = int(std::upper_bound(f.begin(), f.end(), p - 1.5 * h) - f.begin()) - 1;
            *hi = int(std::lower_bound(f.begin(), f.end(), p + 1.5 * h) - f.begin()) - 1;
        };
        int ilo = 0, ihi = -1, jlo = 0, jhi = -1;
        span(g.xf, xi, &ilo, &ihi);
        span(g.yf, eta, &jlo, &jhi);
        const bool near_edge = i0 < 3 || i0 > nx - 4 || j0 < 3 || j0 > ny - 4;
        if (near_edge || !uniform_near(g.dx, ilo, ihi, h) || !uniform_near(g.dy, jlo, jhi, h)) {
            char buf[192];
            if (near_edge)
                std::snprintf(buf, sizeof buf,
                              "body point %d at (%g, %g) lies in one of the three cells next to the edge of the grid",
                              k, xi, eta);
            else
                std::snprintf(buf, sizeof buf, "body point %d at (%g, %g) is not inside uniform cells of width %g",
                              k, xi, eta, h);
            *err = buf;
            return false;
        }
        // the index ranges of the faces with nonzero weights (contiguous: the
        // coordinates increase with the index)
        auto range = [&](const std::vector<double>& c, int lo, int hi, double p, int* a, int* b) {
            *a = hi + 1;
            *b = lo - 1;
            for (int i = lo; i <= hi; ++i)
                if (in_support(c[i] - p)) {
                    *a = std::min(*a, i);
                    *b = std::max(*b, i);
                }
        };
        range(g.xf, i0 - 1, i0 + 2, xi, &su[k].i0, &su[k].i1);
        range(g.yc, j0 - 2, j0 + 2, eta, &su[k].j0, &su[k].j1);
        range(g.xc, i0 - 2, i0 + 2, xi, &sv[k].i0, &sv[k].i1);
        range(g.yf, j0 - 1, j0 + 2, eta, &sv[k].j0, &sv[k].j1);
    }
    for (int c = 0; c < 2; ++c)
        for (int k = 0; k < n_b; ++k) {
            const Span& sp = c == 0 ? su[k] : sv[k];
            for (int j = sp.j0; j <= sp.j1; ++j)
                for (int i = sp.i0; i <= sp.i1; ++i) br.E.col.push_back(int32_t((c ? nc : 0) + int64_t(j) * nx + i));
            br.E.rowptr.push_back(int64_t(br.E.col.size()));
            sr.point[size_t(c * n_b + k)] = k;
        }
    br.E.val.assign(br.E.col.size(), 0.0);
    // face-major transpose: faces in first-touch order, rows ascending
    std::vector<int32_t>& fslot = maps->face_slot;
    std::vector<int64_t> cnt;
    for (int64_t e = 0; e < br.E.nnz(); ++e) {
        const int64_t f = br.E.col[e];
        if (fslot[size_t(f)] < 0) {
            fslot[size_t(f)] = int32_t(br.faces.size());
            br.faces.push_back(f);
            cnt.push_back(0);
        }
        cnt[size_t(fslot[size_t(f)])]++;
    }
    br.ET.n = int64_t(br.faces.size());
    br.ET.m = br.E.n;
    br.ET.rowptr.assign(size_t(br.ET.n + 1), 0);
    for (int64_t t = 0; t < br.ET.n; ++t) br.ET.rowptr[t + 1] = br.ET.rowptr[t] + cnt[size_t(t)];
    br.ET.col.resize(size_t(br.E.nnz()));
    sr.et_src.resize(size_t(br.E.nnz()));
    std::vector<int64_t> cur(br.ET.rowptr.begin(), br.ET.rowptr.end() - 1);
    for (int64_t r = 0; r < br.E.n; ++r)
        for (int64_t e = br.E.rowptr[r]; e < br.E.rowptr[r + 1]; ++e) {
            const int64_t q = cur[size_t(fslot[size_t(br.E.col[e])])]++;
            br.ET.col[size_t(q)] = int32_t(r);
            sr.et_src[size_t(q)] = int32_t(e);
        }
    br.ET.val.assign(br.ET.col.size(), 0.0);
    // force rows [C^T | F]: the cells beside the row's faces (pinned cell
    // excluded; a cell beside two of the faces sums both), then the rows that
    // share a face, both ascending
    br.Cf.n = br.E.n;
    br.Cf.m = nc + br.E.n;
    br.Cf.rowptr.assign(1, 0);
    sr.diag.resize(size_t(br.E.n));
    struct CE {
        int64_t cell;
        int32_t a, b;
    };
    std::vector<CE> cells;
    std::vector<int32_t> rows;
    for (int64_t r = 0; r < br.E.n; ++r) {
        cells.clear();
        rows.clear();
        for (int64_t e = br.E.rowptr[r]; e < br.E.rowptr[r + 1]; ++e) {
            const int64_t f = br.E.col[e];
            int64_t cp, cm;
            if (f < nc) {
                cp = f;
                cm = f - 1;
            } else {
                cp = f - nc;
                cm = f - nc - nx;
            }
            for (int side = 0; side < 2; ++side) {
                const int64_t cell = side ? cm : cp;
                if (cell == pin) continue;
                const int32_t code = int32_t(2 * e + side);
                bool found = false;
                for (auto& x : cells)
                    if (x.cell == cell) {
                        x.b = code;
                        found = true;
                        break;
                    }
                if (!found) cells.push_back({cell, code, -1});
            }
            const int32_t t = fslot[size_t(f)];
            for (int64_t a = br.ET.rowptr[t]; a < br.ET.rowptr[t + 1]; ++a) {
                const int32_t r2 = br.ET.col[size_t(a)];
                if (std::find(rows.begin(), rows.end(), r2) == rows.end()) rows.push_back(r2);
            }
        }
        std::sort(cells.begin(), cells.end(), [](const CE& x, const CE& y) { return x.cell < y.cell; });
        std::sort(rows.begin(), rows.end());
        for (const auto& x : cells) {
            br.Cf.col.push_back(int32_t(x.cell));
            sr.cf_a.push_back(x.a);
            sr.cf_b.push_back(x.b);
        }
        for (const int32_t r2 : rows) {
            if (r2 == r) sr.diag[size_t(r)] = int32_t(br.Cf.col.size());
            br.Cf.col.push_back(int32_t(nc + r2));
            sr.cf_a.push_back(-1);
            sr.cf_b.push_back(-1);
        }
        br.Cf.rowptr.push_back(int64_t(br.Cf.col.size()));
    }
    br.Cf.val.assign(br.Cf.col.size(), 0.0);
    for (const int64_t f : br.faces) fslot[size_t(f)] = -1;
    // touched cells ascending, each with its force entries in row order
    std::vector<int32_t>& cslot = maps->cell_slot;
    for (int64_t p = 0; p < br.Cf.nnz(); ++p) {
        const int64_t col = br.Cf.col[size_t(p)];
        if (col < nc && cslot[size_t(col)] < 0) {
            cslot[size_t(col)] = 0;
            br.tcells.push_back(col);
        }
    }
    std::sort(br.tcells.begin(), br.tcells.end());
    for (size_t t = 0; t < br.tcells.size(); ++t) cslot[size_t(br.tcells[t])] = int32_t(t);
    br.Cc.n = int64_t(br.tcells.size());
    br.Cc.m = nc + br.E.n;
    br.Cc.rowptr.assign(size_t(br.Cc.n + 1), 0);
    for (int64_t p = 0; p < br.Cf.nnz(); ++p) {
        const int64_t col = br.Cf.col[size_t(p)];
        if (col < nc) br.Cc.rowptr[size_t(cslot[size_t(col)]) + 1]++;
    }
    for (int64_t t = 0; t < br.Cc.n; ++t) br.Cc.rowptr[t + 1] += br.Cc.rowptr[t];
    br.Cc.col.resize(size_t(br.Cc.nnz()));
    sr.cc_src.resize(size_t(br.Cc.nnz()));
    cur.assign(br.Cc.rowptr.begin(), br.Cc.rowptr.end() - 1);
    for (int64_t r = 0; r < br.Cf.n; ++r)
        for (int64_t p = br.Cf.rowptr[r]; p < br.Cf.rowptr[r + 1]; ++p) {
            const int64_t col = br.Cf.col[size_t(p)];
            if (col >= nc) continue;
            const int64_t q = cur[size_t(cslot[size_t(col)])]++;
            br.Cc.col[size_t(q)] = int32_t(nc + r);
            sr.cc_src[size_t(q)] = int32_t(p);
        }
    br.Cc.val.assign(br.Cc.col.size(), 0.0);
    for (const int64_t c : br.tcells) cslot[size_t(c)] = -1;
    *out = std::move(br);
    *src = std::move(sr);
    return true;
}

// Rows [r0, r1) of A as a CSR of r1 - r0 rows.
static CSR row_slice(const CSR& A, int64_t r0, int64_t r1) {
    CSR S;
    S.n = r1 - r0;
    S.m = A.m;
    S.rowptr.assign(S.n + 1, 0);
    const int64_t p0 = A.rowptr[r0];
    for (int64_t i = 0; i < S.n; ++i) S.rowptr[i + 1] = A.rowptr[r0 + i + 1] - p0;
    S.col.assign(A.col.begin() + p0, A.col.begin() + A.rowptr[r1]);
    S.val.assign(A.val.begin() + p0, A.val.begin() + A.rowptr[r1]);
    return S;
}

static CSR add_csr(const CSR& A, const CSR& B) {
    std::vector<std::tuple<int64_t, int64_t, double>> t;
    t.reserve(size_t(A.nnz() + B.nnz()));
    for (const CSR* M : {&A, &B})
        for (int64_t i = 0; i < M->n; ++i)
            for (int64_t p = M->rowptr[i]; p < M->rowptr[i + 1]; ++p) t.emplace_back(i, M->col[p], M->val[p]);
    return csr_from_triplets(A.n, A.m, t);
}

CSR assemble_poisson_bn(const Grid& g, const VelocityCoeffs& vc, double dt, int N, int64_t pin, const BodyRows& br,
                        int64_t slice) {
    const int nx = g.nx, ny = g.ny;
    const int64_t nc = g.nc(), nv = 2 * nc, nl = nc + 2 * int64_t(br.n_b);
    // valid velocity slots of the padded layout: u (i >= 1), v (j >= 1)
    auto valid = [&](int64_t k) {
        const int64_t s = k % nc;
        return k < nc ? (s % nx) >= 1 : (s / nx) >= 1;
    };
    // L = 2 (M/dt - A) with A = diag - cE (east/west) - cN (north/south) inside a block
    std::vector<std::tuple<int64_t, int64_t, double>> tL;
    for (int64_t k = 0; k < nv; ++k) {
        if (!valid(k)) continue;
        tL.emplace_back(k, k, 2.0 * (vc.mdt[k] - vc.diag[k]));
        if (vc.cE[k] != 0.0) {
            tL.emplace_back(k, k + 1, 2.0 * vc.cE[k]);
            tL.emplace_back(k + 1, k, 2.0 * vc.cE[k]);
        }
        if (vc.cN[k] != 0.0) {
            tL.emplace_back(k, k + nx, 2.0 * vc.cN[k]);
            tL.emplace_back(k + nx, k, 2.0 * vc.cN[k]);
        }
    }
    CSR L = csr_from_triplets(nv, nv, tL);
    // K = (dt/2) M^-1 L (M = mdt dt), term_0 = dt M^-1 = 1/mdt, B^N = sum of N terms
    CSR K = L;
    for (int64_t i = 0; i < nv; ++i)
        for (int64_t p = K.rowptr[i]; p < K.rowptr[i + 1]; ++p) K.val[p] *= 0.5 / vc.mdt[i];
    std::vector<std::tuple<int64_t, int64_t, double>> t0;
    for (int64_t k = 0; k < nv; ++k)
        if (valid(k)) t0.emplace_back(k, k, 1.0 / vc.mdt[k]);
    CSR term = csr_from_triplets(nv, nv, t0);
    CSR B = term;
    for (int n = 1; n < N; ++n) {
        term = spgemm(K, term);
        B = add_csr(B, term);
    }
    // Q = [G E^T] over the padded faces: +1 to the cell on the + side, -1 on the - side
    std::vector<std::tuple<int64_t, int64_t, double>> tQ;
    for (int j = 0; j < ny; ++j)
        for (int i = 1; i < nx; ++i) {
            const int64_t f = int64_t(j) * nx + i;
            tQ.emplace_back(f, f, 1.0);
            tQ.emplace_back(f, f - 1, -1.0);
        }
    for (int j = 1; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            const int64_t c = int64_t(j) * nx + i;
            tQ.emplace_back(nc + c, c, 1.0);
            tQ.emplace_back(nc + c, c - nx, -1.0);
        }
    for (int64_t r = 0; r < br.E.n; ++r)
        for (int64_t p = br.E.rowptr[r]; p < br.E.rowptr[r + 1]; ++p) tQ.emplace_back(br.E.col[p], nc + r, br.E.val[p]);
    CSR Q = csr_from_triplets(nv, nl, tQ);
    const CSR Qt = transpose(Q);
    // sliced triple product
    CSR S;
    S.n = nl;
    S.m = nl;
    S.rowptr.assign(1, 0);
    const int64_t sl = std::max<int64_t>(1, slice);
    for (int64_t r0 = 0; r0 < nl; r0 += sl) {
        const int64_t r1 = std::min(nl, r0 + sl);
        const CSR T = spgemm(row_slice(Qt, r0, r1), B);
        const CSR R = spgemm(T, Q);
        for (int64_t i = 0; i < R.n; ++i) {
            for (int64_t p = R.rowptr[i]; p < R.rowptr[i + 1]; ++p) {
                const int64_t row = r0 + i, col = R.col[p];
                // pinning: the pinned cell keeps only its diagonal
                if ((row == pin || col == pin) && row != col) continue;
                S.col.push_back(int32_t(col));
                S.val.push_back(R.val[p]);
            }
            S.rowptr.push_back(int64_t(S.col.size()));
        }
    }
    return S;
}

// Pressure block G^T B^1 G (weighted 5-point), pinned (sentence after Eq. 9).
PoissonCoeffs poisson_coeffs(const Grid& g, double dt, int64_t pin, const BodyRows& br) {
    const int nx = g.nx, ny = g.ny;
    const int64_t nc = g.nc();
    PoissonCoeffs pc;
    pc.wE.assign(nc, 0.0);
    pc.wN.assign(nc, 0.0);
    pc.diag.assign(nc + 2 * int64_t(br.n_b), 0.0);
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            const int64_t c = int64_t(j) * nx + i;
            double d = 0.0;
            if (i + 1 <= nx - 1) { pc.wE[c] = dt * g.dy[j] / g.dxf[i + 1]; d += pc.wE[c]; }
            if (i - 1 >= 0) d += dt * g.dy[j] / g.dxf[i];
            if (j + 1 <= ny - 1) { pc.wN[c] = dt * g.dx[i] / g.dyf[j + 1]; d += pc.wN[c]; }
            if (j - 1 >= 0) d += dt * g.dx[i] / g.dyf[j];
            pc.diag[c] = d;
        }
    }
    // pinning removes the couplings of the pinned cell
    const int pi = int(pin % nx), pj = int(pin / nx);
    pc.wE[pin] = 0.0;
    pc.wN[pin] = 0.0;
    if (pi > 0) pc.wE[pin - 1] = 0.0;
    if (pj > 0) pc.wN[pin - nx] = 0.0;
    for (int64_t r = 0; r < br.Cf.n; ++r)
        for (int64_t p = br.Cf.rowptr[r]; p < br.Cf.rowptr[r + 1]; ++p)
            if (br.Cf.col[p] == nc + r) pc.diag[nc + r] = br.Cf.val[p];
    return pc;
}

CSR assemble_poisson(const Grid& g, const PoissonCoeffs& pc, const BodyRows& br) {
    const int nx = g.nx, ny = g.ny;
    const int64_t nc = g.nc();
    const int64_t n = nc + 2 * int64_t(br.n_b);
    CSR A;
    A.n = n;
    A.m = n;
    A.rowptr.assign(n + 1, 0);
    A.col.reserve(5 * nc + br.Cc.nnz() + br.Cf.nnz());
    A.val.reserve(A.col.capacity());
    size_t tc = 0;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            const int64_t c = int64_t(j) * nx + i;
            auto push = [&](int64_t col, double v) { A.col.push_back(int32_t(col)); A.val.push_back(v); };
            if (j > 0 && pc.wN[c - nx] != 0.0) push(c - nx, -pc.wN[c - nx]);
            if (i > 0 && pc.wE[c - 1] != 0.0) push(c - 1, -pc.wE[c - 1]);
            push(c, pc.diag[c]);
            if (pc.wE[c] != 0.0) push(c + 1, -pc.wE[c]);
            if (pc.wN[c] != 0.0) push(c + nx, -pc.wN[c]);
            if (tc < br.tcells.size() && br.tcells[tc] == c) {
                for (int64_t p = br.Cc.rowptr[tc]; p < br.Cc.rowptr[tc + 1]; ++p) push(br.Cc.col[p], br.Cc.val[p]);
                ++tc;
            }
            A.rowptr[c + 1] = int64_t(A.col.size());
        }
    }
    for (int64_t r = 0; r < br.Cf.n; ++r) {
        for (int64_t p = br.Cf.rowptr[r]; p < br.Cf.rowptr[r + 1]; ++p) {
            A.col.push_back(br.Cf.col[p]);
            A.val.push_back(br.Cf.val[p]);
        }
        A.rowptr[nc + r + 1] = int64_t(A.col.size());
    }
    return A;
}

// ---------------------------------------------------------------------------
// Sparse kernels for the AMG set-up
// ---------------------------------------------------------------------------
int64_t sell_entries(const CSR& A) {
    int64_t total = 0;
    for (int64_t s = 0; s * kSellRows < A.n; ++s) {
        int64_t w = 0;
        const int64_t r1 = std::min<int64_t>(A.n, (s + 1) * kSellRows);
        for (int64_t r = s * kSellRows; r < r1; ++r) w = std::max(w, A.rowptr[r + 1] - A.rowptr[r]);
        total += w * kSellRows;
    }
    return total;
}

Sell to_sell(const CSR& A) {
    Sell S;
    S.n = A.n;
    S.nslices = (A.n + kSellRows - 1) / kSellRows;
    S.off.assign(S.nslices + 1, 0);
    for (int64_t s = 0; s < S.nslices; ++s) {
        int64_t w = 0;
        const int64_t r1 = std::min<int64_t>(A.n, (s + 1) * kSellRows);
        for (int64_t r = s * kSellRows; r < r1; ++r) w = std::max(w, A.rowptr[r + 1] - A.rowptr[r]);
        S.off[s + 1] = S.off[s] + w * kSellRows;
    }
    S.col.assign(S.off.back(), 0);
    S.val.assign(S.off.back(), 0.0);
    for (int64_t s = 0; s < S.nslices; ++s) {
        const int64_t w = (S.off[s + 1] - S.off[s]) / kSellRows;
        for (int t = 0; t < kSellRows; ++t) {
            const int64_t r = s * kSellRows + t;
            const int64_t len = r < A.n ? A.rowptr[r + 1] - A.rowptr[r] : 0;
            for (int64_t k = 0; k < w; ++k) {
                const int64_t q = S.off[s] + k * kSellRows + t;
                if (k < len) {
                    S.col[q] = A.col[A.rowptr[r] + k];
                    S.val[q] = A.val[A.rowptr[r] + k];
                } else {
                    S.col[q] = r < A.n && r < A.m ? int32_t(r) : 0;
                }
            }
        }
    }
    return S;
}

CSR transpose(const CSR& A) {
    CSR T;
    T.n = A.m;
    T.m = A.n;
    T.rowptr.assign(T.n + 1, 0);
    for (int64_t p = 0; p < A.nnz(); ++p) T.rowptr[A.col[p] + 1]++;
    for (int64_t i = 0; i < T.n; ++i) T.rowptr[i + 1] += T.rowptr[i];
    T.col.resize(A.nnz());
    T.val.resize(A.nnz());
    std::vector<int64_t> pos(T.rowptr.begin(), T.rowptr.end() - 1);
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
            const int64_t q = pos[A.col[p]]++;
            T.col[q] = int32_t(i);
            T.val[q] = A.val[p];
        }
    return T;
}

// I - (row scale) A (column scale): the identity minus A with row i scaled
// by r[i] (or 1) and column j by c[j] (or 1)
static CSR identity_minus(const CSR& A, const std::vector<double>* r, const std::vector<double>* c, double w) {
    CSR S;
    S.n = A.n;
    S.m = A.m;
    S.rowptr.assign(A.n + 1, 0);
    for (int64_t i = 0; i < A.n; ++i) {
        bool diag = false;
        for (int64_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
            const int32_t j = A.col[p];
            double v = -w * A.val[p] * (r ? (*r)[i] : 1.0) * (c ? (*c)[j] : 1.0);
            if (j == i) {
                v += 1.0;
                diag = true;
            }
            S.col.push_back(j);
            S.val.push_back(v);
        }
        if (!diag) {
            S.col.push_back(int32_t(i));
            S.val.push_back(1.0);
        }
        S.rowptr[i + 1] = int64_t(S.col.size());
    }
    return S;
}

void fused_transfers(const AmgLevel& L, int pre, CSR* Rt, CSR* Q) {
    const CSR SR = identity_minus(L.A, nullptr, &L.invdiag, L.omega);   // I - A w D^-1
    CSR R = L.R;
    for (int k = 0; k < pre; ++k) R = spgemm(R, SR);
    *Rt = std::move(R);
    const CSR S = identity_minus(L.A, &L.invdiag, nullptr, L.omega);    // I - w D^-1 A
    *Q = spgemm(S, L.P);
}

CSR spgemm(const CSR& A, const CSR& B) {
    CSR C;
    C.n = A.n;
    C.m = B.m;
    C.rowptr.assign(C.n + 1, 0);
    std::vector<int64_t> mark(B.m, -1);
    std::vector<double> acc(B.m, 0.0);
    std::vector<int32_t> cols;
    for (int64_t i = 0; i < A.n; ++i) {
        cols.clear();
        for (int64_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
            const int32_t k = A.col[p];
            const double a = A.val[p];
            for (int64_t q = B.rowptr[k]; q < B.rowptr[k + 1]; ++q) {
                const int32_t j = B.col[q];
                if (mark[j] != i) {
                    mark[j] = i;
                    acc[j] = 0.0;
                    cols.push_back(j);
                }
                acc[j] += a * B.val[q];
            }
        }
        std::sort(cols.begin(), cols.end());
        for (int32_t j : cols) {
            C.col.push_back(j);
            C.val.push_back(acc[j]);
        }
        C.rowptr[i + 1] = int64_t(C.col.size());
    }
    return C;
}

static std::vector<double> diagonal(const CSR& A) {
    std::vector<double> d(A.n, 0.0);
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p)
            if (A.col[p] == i) d[i] = A.val[p];
    return d;
}

// Greedy aggregation on the strength graph |a_ij| >= theta sqrt(a_ii a_jj)
// (Vanek, Mandel & Brezina): roots whose strong neighbourhood is free,
// then attach leftovers to a neighbouring aggregate, then aggregate the rest.
static int64_t aggregate(const CSR& A, const std::vector<double>& d, double theta, std::vector<int32_t>* agg_out) {
    const int64_t n = A.n;
    std::vector<int64_t> sptr(n + 1, 0);
    std::vector<int32_t> sidx;
    std::vector<double> sval;
    sidx.reserve(A.nnz());
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) {
            const int32_t j = A.col[p];
            if (j == i) continue;
            const double a = std::fabs(A.val[p]);
            if (a > 0.0 && a >= theta * std::sqrt(std::fabs(d[i] * d[j]))) {
                sidx.push_back(j);
                sval.push_back(a);
            }
        }
        sptr[i + 1] = int64_t(sidx.size());
    }
    std::vector<int32_t> agg(n, -1);
    int32_t na = 0;
    // phase 1
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0 || sptr[i + 1] == sptr[i]) continue;
        bool free_nb = true;
        for (int64_t p = sptr[i]; p < sptr[i + 1]; ++p)
            if (agg[sidx[p]] >= 0) { free_nb = false; break; }
        if (!free_nb) continue;
        agg[i] = na;
        for (int64_t p = sptr[i]; p < sptr[i + 1]; ++p) agg[sidx[p]] = na;
        ++na;
    }
    // phase 2: attach to the most strongly connected phase-1 aggregate
    std::vector<int32_t> agg1 = agg;
    for (int64_t i = 0; i < n; ++i) {
        if (agg1[i] >= 0) continue;
        double best = -1.0;
        int32_t ba = -1;
        for (int64_t p = sptr[i]; p < sptr[i + 1]; ++p) {
            const int32_t a = agg1[sidx[p]];
            if (a >= 0 && sval[p] > best) { best = sval[p]; ba = a; }
        }
        if (ba >= 0) agg[i] = ba;
    }
    // phase 3: remaining nodes with strong neighbours
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0 || sptr[i + 1] == sptr[i]) continue;
        agg[i] = na;
        for (int64_t p = sptr[i]; p < sptr[i + 1]; ++p)
            if (agg[sidx[p]] < 0) agg[sidx[p]] = na;
        ++na;
    }
    *agg_out = std::move(agg);
    return na;
}

// rho(D^-1 A) by 30 power iterations from a fixed start vector, with a 5%
// margin (the power estimate approaches rho from below).
static double spectral_radius_dinv_a(const CSR& A, const std::vector<double>& d) {
    const int64_t n = A.n;
    std::vector<double> x(n), y(n);
    for (int64_t i = 0; i < n; ++i) x[i] = 1.0 + double((i * 7919) % 97) / 97.0;
    double lam = 0.0;
    for (int it = 0; it < 30; ++it) {
        double nx2 = 0.0;
        for (int64_t i = 0; i < n; ++i) nx2 += x[i] * x[i];
        const double s = 1.0 / std::sqrt(nx2);
        for (int64_t i = 0; i < n; ++i) x[i] *= s;
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int64_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) acc += A.val[p] * x[A.col[p]];
            y[i] = acc / d[i];
        }
        double num = 0.0;
        for (int64_t i = 0; i < n; ++i) num += x[i] * y[i];
        lam = num;
        x.swap(y);
    }
    double nx2 = 0.0;
    for (int64_t i = 0; i < n; ++i) nx2 += x[i] * x[i];
    // ||D^-1 A x|| for the last normalised x bounds the Rayleigh estimate
    return 1.05 * std::max(lam, std::sqrt(nx2));
}

// Inverse of a dense symmetric positive definite matrix (row-major n x n):
// Cholesky A = L L^T, X = L^-1 by forward substitution (stored transposed so
// that every inner loop is a contiguous dot product), A^-1 = X^T X.
bool spd_inverse(const std::vector<double>& A, int64_t n, std::vector<double>* inv, std::string* err) {
    std::vector<double> L(size_t(n) * n, 0.0);
    for (int64_t j = 0; j < n; ++j) {
        const double* Lj = &L[size_t(j) * n];
        double s = A[size_t(j) * n + j];
        for (int64_t k = 0; k < j; ++k) s -= Lj[k] * Lj[k];
        if (!(s > 0.0)) {
            *err = "matrix is not positive definite (pivot " + std::to_string(j) + ")";
            return false;
        }
        const double d = std::sqrt(s);
        L[size_t(j) * n + j] = d;
        for (int64_t i = j + 1; i < n; ++i) {
            const double* Li = &L[size_t(i) * n];
            double t = A[size_t(i) * n + j];
            for (int64_t k = 0; k < j; ++k) t -= Li[k] * Lj[k];
            L[size_t(i) * n + j] = t / d;
        }
    }
    std::vector<double> Xt(size_t(n) * n, 0.0);   // Xt[j][i] = (L^-1)[i][j]
    for (int64_t j = 0; j < n; ++j) {
        double* x = &Xt[size_t(j) * n];
        for (int64_t i = j; i < n; ++i) {
            const double* Li = &L[size_t(i) * n];
            double t = (i == j) ? 1.0 : 0.0;
            for (int64_t k = j; k < i; ++k) t -= Li[k] * x[k];
            x[i] = t / Li[i];
        }
    }
    inv->assign(size_t(n) * n, 0.0);
    for (int64_t i = 0; i < n; ++i) {
        const double* xi = &Xt[size_t(i) * n];
        for (int64_t j = 0; j <= i; ++j) {
            const double* xj = &Xt[size_t(j) * n];
            double t = 0.0;
            for (int64_t k = i; k < n; ++k) t += xi[k] * xj[k];
            (*inv)[size_t(i) * n + j] = t;
            (*inv)[size_t(j) * n + i] = t;
        }
    }
    return true;
}

bool build_hierarchy(const CSR& A0, const AmgParams& prm, Hierarchy* H, std::string* err) {
    auto t0 = std::chrono::steady_clock::now();
    H->levels.clear();
    H->levels.emplace_back();
    H->levels.back().A = A0;
    // near-null-space vector B (constants on the finest level), carried to
    // the coarse levels by the aggregate-wise QR of the tentative prolongator:
    // T[i, a] = B[i] / |B on a|,  B_coarse[a] = |B on a|
    std::vector<double> B(A0.n, 1.0);
    for (int lev = 0;; ++lev) {
        AmgLevel& L = H->levels[lev];
        const CSR& A = L.A;
        std::vector<double> d = diagonal(A);
        L.invdiag.resize(A.n);
        for (int64_t i = 0; i < A.n; ++i) {
            if (!(d[i] > 0.0)) {
                *err = "AMG: non-positive diagonal at level " + std::to_string(lev) + " row " + std::to_string(i);
                return false;
            }
            L.invdiag[i] = 1.0 / d[i];
        }
        // smoother weight scaled by the spectral radius so that damped Jacobi
        // stays convergent on the coupled rows (omega = 2/3 -> (4/3)/rho)
        L.rho = spectral_radius_dinv_a(A, d);
        L.omega = prm.omega * 2.0 / L.rho;
        if ((lev > 0 && A.n <= prm.max_coarse) || lev + 1 >= prm.max_levels) break;
        const int64_t na = aggregate(A, d, prm.theta, &L.agg);
        if (na == 0 || na >= A.n) break;
        // tentative prolongator: the near-null-space vector restricted to each
        // aggregate, normalised (one column per aggregate)
        std::vector<double> nrm2(na, 0.0);
        for (int64_t i = 0; i < A.n; ++i)
            if (L.agg[i] >= 0) nrm2[L.agg[i]] += B[i] * B[i];
        std::vector<double> Bc(na);
        for (int64_t a = 0; a < na; ++a) Bc[a] = std::sqrt(nrm2[a]);
        CSR T;
        T.n = A.n;
        T.m = na;
        T.rowptr.assign(A.n + 1, 0);
        for (int64_t i = 0; i < A.n; ++i) {
            if (L.agg[i] >= 0 && Bc[L.agg[i]] > 0.0) {
                T.col.push_back(L.agg[i]);
                T.val.push_back(B[i] / Bc[L.agg[i]]);
            }
            T.rowptr[i + 1] = int64_t(T.col.size());
        }
        B = std::move(Bc);
        // smoothed prolongator P = (I - omega_P D^-1 A) T, omega_P = (4/3)/rho(D^-1 A)
        const double wp = (4.0 / 3.0) / L.rho;
        CSR AT = spgemm(A, T);
        CSR P;
        P.n = A.n;
        P.m = na;
        P.rowptr.assign(A.n + 1, 0);
        for (int64_t i = 0; i < A.n; ++i) {
            // merge row i of T and -wp/d_i * row i of AT (both sorted)
            int64_t a = T.rowptr[i], ae = T.rowptr[i + 1];
            int64_t b = AT.rowptr[i], be = AT.rowptr[i + 1];
            const double s = -wp / d[i];
            while (a < ae || b < be) {
                int32_t ca = a < ae ? T.col[a] : INT32_MAX;
                int32_t cb = b < be ? AT.col[b] : INT32_MAX;
                double v;
                int32_t c;
                if (ca == cb) { c = ca; v = T.val[a] + s * AT.val[b]; ++a; ++b; }
                else if (ca < cb) { c = ca; v = T.val[a]; ++a; }
                else { c = cb; v = s * AT.val[b]; ++b; }
                if (v != 0.0) { P.col.push_back(c); P.val.push_back(v); }
            }
            P.rowptr[i + 1] = int64_t(P.col.size());
        }
        if (prm.trunc > 0.0) {
            // truncation of the smoothed prolongator: small entries are dropped
            // and each row rescaled to its original sum (constants stay exact)
            CSR Q;
            Q.n = P.n;
            Q.m = P.m;
            Q.rowptr.assign(P.n + 1, 0);
            for (int64_t i = 0; i < P.n; ++i) {
                double mx = 0.0, sum = 0.0, kept = 0.0;
                for (int64_t p = P.rowptr[i]; p < P.rowptr[i + 1]; ++p) {
                    mx = std::max(mx, std::fabs(P.val[p]));
                    sum += P.val[p];
                }
                for (int64_t p = P.rowptr[i]; p < P.rowptr[i + 1]; ++p)
                    if (std::fabs(P.val[p]) >= prm.trunc * mx) kept += P.val[p];
                const double sc = (kept != 0.0) ? sum / kept : 1.0;
                for (int64_t p = P.rowptr[i]; p < P.rowptr[i + 1]; ++p)
                    if (std::fabs(P.val[p]) >= prm.trunc * mx) {
                        Q.col.push_back(P.col[p]);
                        Q.val.push_back(P.val[p] * sc);
                    }
                Q.rowptr[i + 1] = int64_t(Q.col.size());
            }
            P = std::move(Q);
        }
        CSR R = transpose(P);
        CSR AP = spgemm(A, P);
        CSR Ac = spgemm(R, AP);
        L.P = std::move(P);
        L.R = std::move(R);
        H->levels.emplace_back();
        H->levels.back().A = std::move(Ac);
    }
    // dense inverse of the coarsest operator (Cholesky, FP64)
    const CSR& Ac = H->levels.back().A;
    const int64_t n = Ac.n;
    if (n > 2048) {
        *err = "AMG: coarsest level has " + std::to_string(n) + " unknowns (raise amg_max_levels)";
        return false;
    }
    std::vector<double> M(n * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = Ac.rowptr[i]; p < Ac.rowptr[i + 1]; ++p) M[i * n + Ac.col[p]] = Ac.val[p];
    // symmetrise against rounding of R A P
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < i; ++j) {
            const double s = 0.5 * (M[i * n + j] + M[j * n + i]);
            M[i * n + j] = M[j * n + i] = s;
        }
    if (!spd_inverse(M, n, &H->coarse_inv, err)) {
        *err = "AMG: coarsest operator: " + *err;
        return false;
    }
    H->coarse_n = n;
    H->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return true;
}

}  // namespace ibm

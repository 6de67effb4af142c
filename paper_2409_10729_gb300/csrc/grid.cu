// grid.cu -- non-uniform (e.g. tanh-refined, arXiv 2409.10729 Sec. III-A)
// grid geometry for the sweeps: per direction, the WENO5 table of every cell
// -1 .. n and the width of every cell, computed on the host once per grid.
//
// WENO5 on a non-uniform grid (Shu's general reconstruction): with t the
// coordinate in units of cell i's width (cell i = [-1/2, 1/2]), each
// three-cell stencil k (cells i-2+k .. i+k) carries the quadratic p_k whose
// cell averages are the stencil values.  p_k is the derivative of the cubic
// that interpolates the primitive function V (V = 0 at the stencil's first
// edge, V increased by value x width across each cell), so with the Lagrange
// basis L_m of the four edges
//     p_k(t) = sum_m V_m L_m'(t),   coefficient of value j: w_j sum_{m>j} L_m'(t).
// Its face values are p_k(+-1/2); b = p_k'(0) and c = p_k''(0)/2 give the
// smoothness indicator b^2 + (13/3) c^2.  The linear weights make
// sum_k d_k p_k(+-1/2) the face value of the quartic through all five cells
// (same construction with six edges); stencil 0 alone holds cell i-2 and
// stencil 2 alone cell i+2, which fixes d_0 and d_2, and d_1 = 1 - d_0 - d_2.
#include <cmath>
#include <vector>

#include "mfc_internal.cuh"

namespace mfc5 {
namespace {

// d/dt of prod_{q in nodes, q != skip} (t - x_q), at t.
double dprod(const double* x, int nn, int skip, double t) {
    double s = 0.0;
    for (int l = 0; l < nn; ++l) {
        if (l == skip) continue;
        double p = 1.0;
        for (int q = 0; q < nn; ++q)
            if (q != skip && q != l) p *= t - x[q];
        s += p;
    }
    return s;
}

// d^2/dt^2 of the same product, at t.
double d2prod(const double* x, int nn, int skip, double t) {
    double s = 0.0;
    for (int l = 0; l < nn; ++l) {
        if (l == skip) continue;
        for (int r = 0; r < nn; ++r) {
            if (r == skip || r == l) continue;
            double p = 1.0;
            for (int q = 0; q < nn; ++q)
                if (q != skip && q != l && q != r) p *= t - x[q];
            s += p;
        }
    }
    return s;
}

double denom(const double* x, int nn, int m) {
    double d = 1.0;
    for (int l = 0; l < nn; ++l)
        if (l != m) d *= x[m] - x[l];
    return d;
}

// Coefficients of the reconstruction from the cells between nodes x[0..nn-1]
// (nn - 1 cells): out[j] = w_j sum_{m>j} L_m'(t) for value j.
void face_coeffs(const double* x, int nn, double t, double* out) {
    for (int j = 0; j < nn - 1; ++j) {
        double s = 0.0;
        for (int m = j + 1; m < nn; ++m) s += dprod(x, nn, m, t) / denom(x, nn, m);
        out[j] = (x[j + 1] - x[j]) * s;
    }
}

bool cell_table(const double* w, double* T) {
    double e[6];
    e[2] = -0.5;
    e[3] = 0.5;
    e[1] = e[2] - w[1] / w[2];
    e[0] = e[1] - w[0] / w[2];
    e[4] = e[3] + w[3] / w[2];
    e[5] = e[4] + w[4] / w[2];
    double *cp = T, *cm = T + 9, *B = T + 18, *C = T + 27, *dp = T + 36, *dm = T + 39;
    for (int k = 0; k < 3; ++k) {
        const double* x = e + k;   // the stencil's four edges
        face_coeffs(x, 4, 0.5, cp + 3 * k);
        face_coeffs(x, 4, -0.5, cm + 3 * k);
        for (int j = 0; j < 3; ++j) {
            double sb = 0.0, sc = 0.0;
            for (int m = j + 1; m < 4; ++m) {
                const double D = denom(x, 4, m);
                sb += d2prod(x, 4, m, 0.0) / D;   // p'(0) = V''(0)
                sc += 3.0 / D;                    // p''/2 = V'''/2 = 6/(2 D) per basis cubic
            }
            B[3 * k + j] = (x[j + 1] - x[j]) * sb;
            C[3 * k + j] = (x[j + 1] - x[j]) * sc;
        }
    }
    double Qp[5], Qm[5];
    face_coeffs(e, 6, 0.5, Qp);
    face_coeffs(e, 6, -0.5, Qm);
    if (!(cp[0] != 0.0) || !(cp[8] != 0.0) || !(cm[0] != 0.0) || !(cm[8] != 0.0)) return false;
    dp[0] = Qp[0] / cp[0];
    dp[2] = Qp[4] / cp[8];
    dp[1] = 1.0 - dp[0] - dp[2];
    dm[0] = Qm[0] / cm[0];
    dm[2] = Qm[4] / cm[8];
    dm[1] = 1.0 - dm[0] - dm[2];
    for (int i = 0; i < kTabDoubles; ++i)
        if (!std::isfinite(T[i])) return false;
    return true;
}

}  // namespace

bool build_grid_tables(const double* edges, int n, int periodic, std::vector<double>& tab,
                       std::vector<double>& width) {
    for (int j = 0; j < n; ++j)
        if (!(edges[j + 1] > edges[j]) || !std::isfinite(edges[j + 1] - edges[j])) return false;
    width.assign(n, 0.0);
    for (int j = 0; j < n; ++j) width[j] = edges[j + 1] - edges[j];
    auto w_of = [&](int j) {   // ghost widths follow the BC: copied (transmissive) or wrapped
        if (periodic) {
            int r = j % n;
            return width[r < 0 ? r + n : r];
        }
        return width[j < 0 ? 0 : (j > n - 1 ? n - 1 : j)];
    };
    tab.assign((size_t)(n + 2) * kTabDoubles, 0.0);
    for (int j = -1; j <= n; ++j) {
        double w5[5];
        for (int k = 0; k < 5; ++k) w5[k] = w_of(j - 2 + k);
        if (!cell_table(w5, &tab[(size_t)(j + 1) * kTabDoubles])) return false;
    }
    return true;
}

}  // namespace mfc5

/*
 * mfc5_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, serial, double-precision CPU statement of the right-hand side of
 * the two-fluid five-equation (Allaire) model with the stiffened-gas equation
 * of state, discretised with WENO5-JS face reconstruction, the HLLC Riemann
 * solver and Shu-Osher TVD-RK3, as described in arXiv 2409.10729:
 *   - model and EOS:               Sec. II-A (unnumbered equation block and
 *                                  the stiffened-gas relation that follows it)
 *   - finite-volume semi-discrete: Sec. II-B, Eq. (eqn:discretization) and the
 *                                  cell-integrated form that follows it
 *   - WENO + HLLC:                 Sec. II-B, last paragraph
 * Points the paper leaves open are read as follows, and each function below
 * states the reading it uses: mixture rules Gamma = sum alpha_i/(gamma_i-1),
 * Pi = sum alpha_i gamma_i pi_i/(gamma_i-1); sound speed
 * c^2 = ((Gamma+1)p + Pi)/(Gamma rho); WENO epsilon 1e-6 (absolute, exponent
 * 2); Davis wave-speed estimates; the alpha_1 row's h(q) div(u) term as
 * +alpha_1,i (u_f,i+1/2 - u_f,i-1/2)/dx with u_f the HLLC region velocity;
 * Shu-Osher SSP-RK3 with dt fixed per step from q^n; dt = CFL / max over
 * cells of sum_d (|u_d| + c)/dx_d; transmissive ghosts copy the nearest
 * interior cell, periodic ghosts wrap.
 *
 * Only tests/, the smoke check and bench.py's CPU-baseline leg may load this
 * file's shared library.  It shares no code with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math, no pow):
 * every formula below is evaluated in the written operation order, with IEEE
 * division and square root.
 *
 * Layout: conservative q[f][z][y][x] (x fastest), interior cells only.
 * With N fluids (N = 2 by default, up to 4):
 *   f = 0..N-1: alpha_i rho_i, N..N+d-1: rho u_k, N+d: rho E,
 *   N+d+1 .. 2N+d-1: alpha_1 .. alpha_{N-1}  (alpha_N = 1 - sum).  neq = 2N + d.
 * For two fluids: alpha1 rho1, alpha2 rho2, rho u_k, rho E, alpha1 (neq = d + 4).
 * Primitive w has the same slots with u_k in place of rho u_k and p in place
 * of rho E.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENONPHYSICAL (-4)

typedef struct {
    int ndim;          /* 1, 2 or 3 */
    int n[3];          /* cells per dimension; unused dimensions = 1 */
    double lo[3];      /* domain lower corner */
    double hi[3];      /* domain upper corner */
    int bc[3][2];      /* per dimension, per side: 0 transmissive, 1 periodic */
    double gamma[4];   /* ratio of specific heats of fluids 1 .. N */
    double pi_inf[4];  /* stiffness of fluids 1 .. N */
    double weno_eps;   /* WENO epsilon (absolute) */
    int weno_order;    /* 5 (WENO5-JS) or 3 (WENO3-JS); 0 means 5 */
    const double* edges[3];  /* optional: the n[d]+1 cell edges of direction d, strictly increasing
                                (a non-uniform, e.g. tanh-stretched, grid; WENO5 only); NULL: uniform */
    int nfluids;       /* N, 2 .. 4; 0 means 2 */
} orc_params;

#define NEQ_MAX 16

typedef struct {
    int ndim, neq, nf;
    long n[3];
    long stride[3];
    long ncell;
    double dx[3];
    int periodic[3];
    double gk[4];      /* 1/(gamma_i - 1) */
    double Pk[4];      /* gamma_i pi_i/(gamma_i - 1) */
    double eps;
    int order;         /* WENO order, 3 or 5 */
    int stretched[3];  /* direction d has a non-uniform grid */
    double* h[3];      /* stretched: widths of cells -3 .. n+2 (slot j + 3), ghosts per BC */
    double* tab[3];    /* stretched: WENO5 tables of cells -1 .. n (slot j + 1), NT each */
} grid;

#define NT 42          /* doubles per cell of a non-uniform WENO5 table (see make_tables) */

#define IU(g) ((g)->nf)                   /* first momentum / velocity slot */
#define IE(g) ((g)->nf + (g)->ndim)        /* energy / pressure slot */
#define IA(g) ((g)->nf + (g)->ndim + 1)    /* alpha_1 (alpha_2 .. alpha_{N-1} follow) */

static void free_grid(grid* g) {
    for (int d = 0; d < 3; d++) {
        free(g->h[d]);
        free(g->tab[d]);
        g->h[d] = g->tab[d] = NULL;
    }
}

static int make_tables(grid* g, int d, const double* edges);

static int make_grid(const orc_params* p, grid* g) {
    for (int d = 0; d < 3; d++) {
        g->stretched[d] = 0;
        g->h[d] = g->tab[d] = NULL;
    }
    if (!p || p->ndim < 1 || p->ndim > 3) return ORC_EINVAL;
    if (p->nfluids != 0 && (p->nfluids < 2 || p->nfluids > 4)) return ORC_EINVAL;
    g->nf = p->nfluids == 0 ? 2 : p->nfluids;
    g->ndim = p->ndim;
    g->neq = 2 * g->nf + p->ndim;
    g->ncell = 1;
    for (int d = 0; d < 3; d++) {
        long n = p->n[d];
        if (d >= p->ndim) n = 1;
        if (n < 1) return ORC_EINVAL;
        g->n[d] = n;
        g->stride[d] = g->ncell;
        g->ncell *= n;
        g->periodic[d] = 0;
        g->dx[d] = 1.0;
        if (d < p->ndim) {
            if (!(p->hi[d] > p->lo[d])) return ORC_EINVAL;
            g->dx[d] = (p->hi[d] - p->lo[d]) / (double)n;
            int b0 = p->bc[d][0], b1 = p->bc[d][1];
            if (b0 < 0 || b0 > 1 || b1 < 0 || b1 > 1 || b0 != b1) return ORC_EINVAL;
            g->periodic[d] = (b0 == 1);
        }
    }
    for (int i = 0; i < g->nf; i++)
        if (!(p->gamma[i] > 1.0) || !(p->pi_inf[i] >= 0.0)) return ORC_EINVAL;
    if (!(p->weno_eps > 0.0)) return ORC_EINVAL;
    if (p->weno_order != 0 && p->weno_order != 3 && p->weno_order != 5) return ORC_EINVAL;
    g->order = p->weno_order == 3 ? 3 : 5;
    for (int i = 0; i < g->nf; i++) {
        g->gk[i] = 1.0 / (p->gamma[i] - 1.0);
        g->Pk[i] = p->gamma[i] * p->pi_inf[i] / (p->gamma[i] - 1.0);
    }
    g->eps = p->weno_eps;
    for (int d = 0; d < g->ndim; d++) {
        if (!p->edges[d]) continue;
        if (g->order != 5) { free_grid(g); return ORC_EINVAL; }
        int st = make_tables(g, d, p->edges[d]);
        if (st) { free_grid(g); return st; }
    }
    return ORC_OK;
}

/* ---- equation of state (Sec. II-A) -------------------------------------- */

/* Mixture rules: Gamma = sum alpha_i/(gamma_i-1), Pi = sum alpha_i gamma_i
 * pi_i/(gamma_i-1), with alpha_N = 1 - alpha_1 - ... - alpha_{N-1} (the
 * carried fractions a[0..N-2]).  Then rho E = Gamma p + Pi + rho|u|^2/2, the
 * stiffened-gas relation with the kinetic energy added. */
static void mixture(const grid* g, const double* a, double* G, double* Pi) {
    double aN = 1.0 - a[0];
    for (int i = 1; i < g->nf - 1; i++) aN = aN - a[i];
    double sg = a[0] * g->gk[0], sp = a[0] * g->Pk[0];
    for (int i = 1; i < g->nf - 1; i++) {
        sg = sg + a[i] * g->gk[i];
        sp = sp + a[i] * g->Pk[i];
    }
    *G = sg + aN * g->gk[g->nf - 1];
    *Pi = sp + aN * g->Pk[g->nf - 1];
}

/* Mixture density, the sum of the partial densities. */
static double mix_rho(const grid* g, const double* q) {
    double rho = q[0] + q[1];
    for (int i = 2; i < g->nf; i++) rho = rho + q[i];
    return rho;
}

static double kinetic(const grid* g, double rho, const double* u) {
    double s = 0.0;
    for (int k = 0; k < g->ndim; k++) s = s + u[k] * u[k];
    return 0.5 * rho * s;
}

static void cons_to_prim(const grid* g, const double* q, double* w) {
    double rho = mix_rho(g, q);
    double u[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < g->ndim; k++) u[k] = q[IU(g) + k] / rho;
    double ke = kinetic(g, rho, u);
    double G, Pi;
    mixture(g, &q[IA(g)], &G, &Pi);
    double p = (q[IE(g)] - ke - Pi) / G;
    for (int i = 0; i < g->nf; i++) w[i] = q[i];
    for (int k = 0; k < g->ndim; k++) w[IU(g) + k] = u[k];
    w[IE(g)] = p;
    for (int i = 0; i < g->nf - 1; i++) w[IA(g) + i] = q[IA(g) + i];
}

static void prim_to_cons(const grid* g, const double* w, double* q) {
    double rho = mix_rho(g, w);
    double u[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < g->ndim; k++) u[k] = w[IU(g) + k];
    double ke = kinetic(g, rho, u);
    double G, Pi;
    mixture(g, &w[IA(g)], &G, &Pi);
    for (int i = 0; i < g->nf; i++) q[i] = w[i];
    for (int k = 0; k < g->ndim; k++) q[IU(g) + k] = rho * u[k];
    q[IE(g)] = G * w[IE(g)] + Pi + ke;
    for (int i = 0; i < g->nf - 1; i++) q[IA(g) + i] = w[IA(g) + i];
}

/* Mixture sound speed squared, c^2 = ((Gamma+1) p + Pi)/(Gamma rho). */
static double sound2(double G, double Pi, double rho, double p) {
    return ((G + 1.0) * p + Pi) / (G * rho);
}

/* ---- WENO5-JS (Sec. II-B, fifth-order reconstruction) -------------------- */

static double sq(double x) { return x * x; }
/* ---- WENO5 on a non-uniform grid (Shu's general reconstruction) ----------
 * For cell i of width h_i, with t = (x - x_i)/h_i, each three-cell stencil k
 * (cells i-2+k .. i+k) carries the quadratic p_k(t) = a + b t + c t^2 whose
 * averages over its three cells are the cell values; p_k(+-1/2) are its face
 * values, and its smoothness indicator is
 *   beta_k = sum_{l=1,2} h_i^(2l-1) int_cell (d^l p_k/dx^l)^2 dx = b^2 + (13/3) c^2.
 * The linear weights d_k are those for which sum_k d_k p_k(+-1/2) is the face
 * value of the quartic with the five cell averages (the only stencil that
 * contains cell i-2, resp. i+2, fixes d_0, resp. d_2; d_1 = 1 - d_0 - d_2).
 * On a uniform grid these are the Jiang-Shu coefficients.  The table of a
 * cell holds, as linear functionals of the stencil values: face values at
 * i+1/2 (cp[3][3]) and i-1/2 (cm[3][3]), b (B[3][3]), c (C[3][3]), and the
 * linear weights dp[3] (i+1/2) and dm[3] (i-1/2). */

/* Inverse of the m x m row-major matrix A (m <= 5), Gauss-Jordan with partial
 * pivoting; returns 1 when A is singular. */
static int invert(int m, const double* A, double* Ainv) {
    double a[5][10];
    for (int r = 0; r < m; r++)
        for (int c = 0; c < 2 * m; c++) a[r][c] = c < m ? A[r * m + c] : (c - m == r ? 1.0 : 0.0);
    for (int col = 0; col < m; col++) {
        int piv = col;
        for (int r = col + 1; r < m; r++)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (!(fabs(a[piv][col]) > 0.0)) return 1;
        if (piv != col)
            for (int c = 0; c < 2 * m; c++) {
                double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        double inv = 1.0 / a[col][col];
        for (int c = 0; c < 2 * m; c++) a[col][c] = a[col][c] * inv;
        for (int r = 0; r < m; r++) {
            if (r == col) continue;
            double f = a[r][col];
            for (int c = 0; c < 2 * m; c++) a[r][c] = a[r][c] - f * a[col][c];
        }
    }
    for (int r = 0; r < m; r++)
        for (int c = 0; c < m; c++) Ainv[r * m + c] = a[r][m + c];
    return 0;
}

/* Average of t^m over [l, u]. */
static double avg_pow(int m, double l, double u) {
    double lp = l, up = u;
    for (int k = 0; k < m; k++) {
        lp = lp * l;
        up = up * u;
    }
    return (up - lp) / ((double)(m + 1) * (u - l));
}

/* Table of one cell from the widths w[0..4] of cells i-2 .. i+2. */
static int cell_table(const double* w, double* T) {
    double e[6];   /* cell edges in units of h_i, cell i = [-1/2, 1/2] */
    e[2] = -0.5;
    e[3] = 0.5;
    e[1] = e[2] - w[1] / w[2];
    e[0] = e[1] - w[0] / w[2];
    e[4] = e[3] + w[3] / w[2];
    e[5] = e[4] + w[4] / w[2];
    double *cp = T, *cm = T + 9, *B = T + 18, *C = T + 27, *dp = T + 36, *dm = T + 39;
    for (int k = 0; k < 3; k++) {
        double M[9], Mi[9];
        for (int j = 0; j < 3; j++)
            for (int m = 0; m < 3; m++) M[3 * j + m] = avg_pow(m, e[k + j], e[k + j + 1]);
        if (invert(3, M, Mi)) return 1;
        for (int j = 0; j < 3; j++) {
            /* coefficient of stencil value j in a, b, c: Mi[0][j], Mi[1][j], Mi[2][j] */
            cp[3 * k + j] = Mi[j] + 0.5 * Mi[3 + j] + 0.25 * Mi[6 + j];
            cm[3 * k + j] = Mi[j] - 0.5 * Mi[3 + j] + 0.25 * Mi[6 + j];
            B[3 * k + j] = Mi[3 + j];
            C[3 * k + j] = Mi[6 + j];
        }
    }
    double M5[25], Mi5[25], Qp[5], Qm[5];
    for (int j = 0; j < 5; j++)
        for (int m = 0; m < 5; m++) M5[5 * j + m] = avg_pow(m, e[j], e[j + 1]);
    if (invert(5, M5, Mi5)) return 1;
    for (int j = 0; j < 5; j++) {
        double sp = 0.0, sm = 0.0, xp = 1.0, xm = 1.0;
        for (int m = 0; m < 5; m++) {
            sp = sp + Mi5[5 * m + j] * xp;
            sm = sm + Mi5[5 * m + j] * xm;
            xp = xp * 0.5;
            xm = xm * -0.5;
        }
        Qp[j] = sp;
        Qm[j] = sm;
    }
    dp[0] = Qp[0] / cp[0];
    dp[2] = Qp[4] / cp[3 * 2 + 2];
    dp[1] = 1.0 - dp[0] - dp[2];
    dm[0] = Qm[0] / cm[0];
    dm[2] = Qm[4] / cm[3 * 2 + 2];
    dm[1] = 1.0 - dm[0] - dm[2];
    return 0;
}

/* Cell widths (with ghosts per BC) and WENO5 tables of stretched direction d. */
static int make_tables(grid* g, int d, const double* edges) {
    long n = g->n[d];
    for (long j = 0; j < n; j++)
        if (!(edges[j + 1] > edges[j]) || !isfinite(edges[j + 1] - edges[j])) return ORC_EINVAL;
    g->h[d] = malloc(sizeof(double) * (n + 6));
    g->tab[d] = malloc(sizeof(double) * (n + 2) * NT);
    if (!g->h[d] || !g->tab[d]) return ORC_ENOMEM;
    for (long j = -3; j < n + 3; j++) {
        long s;
        if (g->periodic[d]) {
            s = j % n;
            if (s < 0) s += n;
        } else {
            s = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
        }
        g->h[d][j + 3] = edges[s + 1] - edges[s];
    }
    for (long j = -1; j < n + 1; j++)
        if (cell_table(&g->h[d][j + 1], &g->tab[d][(j + 1) * NT])) return ORC_EINVAL;
    g->stretched[d] = 1;
    return ORC_OK;
}

/* WENO5-JS on a non-uniform grid from the cell's table T (same weights
 * a_k = d_k/(eps+beta_k)^2, omega_k = a_k/sum a as the uniform scheme). */
static void weno5_nu(const double* T, double eps, const double* v, double* vm, double* vp) {
    const double *cp = T, *cm = T + 9, *B = T + 18, *C = T + 27, *dp = T + 36, *dm = T + 39;
    double beta[3], qp[3], qm[3];
    for (int k = 0; k < 3; k++) {
        double b = 0.0, c = 0.0, sp = 0.0, sm = 0.0;
        for (int j = 0; j < 3; j++) {
            b = b + B[3 * k + j] * v[k + j];
            c = c + C[3 * k + j] * v[k + j];
            sp = sp + cp[3 * k + j] * v[k + j];
            sm = sm + cm[3 * k + j] * v[k + j];
        }
        beta[k] = b * b + (13.0 / 3.0) * (c * c);
        qp[k] = sp;
        qm[k] = sm;
    }
    double ap[3], am[3], sap = 0.0, sam = 0.0;
    for (int k = 0; k < 3; k++) {
        ap[k] = dp[k] / sq(eps + beta[k]);
        am[k] = dm[k] / sq(eps + beta[k]);
        sap = sap + ap[k];
        sam = sam + am[k];
    }
    *vm = (ap[0] / sap) * qp[0] + (ap[1] / sap) * qp[1] + (ap[2] / sap) * qp[2];
    *vp = (am[0] / sam) * qm[0] + (am[1] / sam) * qm[1] + (am[2] / sam) * qm[2];
}


/* v[0..4] = v_{i-2} .. v_{i+2} (cell averages of one primitive).
 * Returns the left-biased value at face i+1/2 (vm) and the right-biased value
 * at face i-1/2 (vp); both use the same three Jiang-Shu smoothness indicators
 * of cell i. */
static void weno5(double eps, const double* v, double* vm, double* vp) {
    const double c13 = 13.0 / 12.0;
    double b0 = c13 * sq(v[0] - 2.0 * v[1] + v[2]) + 0.25 * sq(v[0] - 4.0 * v[1] + 3.0 * v[2]);
    double b1 = c13 * sq(v[1] - 2.0 * v[2] + v[3]) + 0.25 * sq(v[1] - v[3]);
    double b2 = c13 * sq(v[2] - 2.0 * v[3] + v[4]) + 0.25 * sq(3.0 * v[2] - 4.0 * v[3] + v[4]);

    /* left-biased value at i+1/2: linear weights (0.1, 0.6, 0.3) */
    double a0 = 0.1 / sq(eps + b0);
    double a1 = 0.6 / sq(eps + b1);
    double a2 = 0.3 / sq(eps + b2);
    double s = a0 + a1 + a2;
    double p0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
    double p1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
    double p2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
    *vm = (a0 / s) * p0 + (a1 / s) * p1 + (a2 / s) * p2;

    /* right-biased value at i-1/2: mirrored weights (0.3, 0.6, 0.1) */
    a0 = 0.3 / sq(eps + b0);
    a1 = 0.6 / sq(eps + b1);
    a2 = 0.1 / sq(eps + b2);
    s = a0 + a1 + a2;
    p0 = (-v[0] + 5.0 * v[1] + 2.0 * v[2]) / 6.0;
    p1 = (2.0 * v[1] + 5.0 * v[2] - v[3]) / 6.0;
    p2 = (11.0 * v[2] - 7.0 * v[3] + 2.0 * v[4]) / 6.0;
    *vp = (a0 / s) * p0 + (a1 / s) * p1 + (a2 / s) * p2;
}

/* WENO3-JS (Jiang & Shu 1996, two two-cell stencils), the paper's
 * third-order option (Sec. II-B).  v holds the same five cells as for WENO5,
 * v_{i-2}..v_{i+2}; only v_{i-1}, v_i, v_{i+1} enter.
 * Candidates at i+1/2: (-v_{i-1} + 3 v_i)/2 on {i-1, i}, (v_i + v_{i+1})/2 on
 * {i, i+1}; at i-1/2: (v_{i-1} + v_i)/2 and (3 v_i - v_{i+1})/2.  Smoothness
 * beta_0 = (v_i - v_{i-1})^2, beta_1 = (v_{i+1} - v_i)^2; linear weights
 * (1/3, 2/3) for the left-biased value at i+1/2, (2/3, 1/3) for the
 * right-biased value at i-1/2; a_k = d_k/(eps+beta_k)^2, omega_k = a_k/sum a. */
static void weno3(double eps, const double* v, double* vm, double* vp) {
    double b0 = sq(v[2] - v[1]);
    double b1 = sq(v[3] - v[2]);

    double a0 = (1.0 / 3.0) / sq(eps + b0);
    double a1 = (2.0 / 3.0) / sq(eps + b1);
    double s = a0 + a1;
    double p0 = (-v[1] + 3.0 * v[2]) / 2.0;
    double p1 = (v[2] + v[3]) / 2.0;
    *vm = (a0 / s) * p0 + (a1 / s) * p1;

    a0 = (2.0 / 3.0) / sq(eps + b0);
    a1 = (1.0 / 3.0) / sq(eps + b1);
    s = a0 + a1;
    p0 = (v[1] + v[2]) / 2.0;
    p1 = (3.0 * v[2] - v[3]) / 2.0;
    *vp = (a0 / s) * p0 + (a1 / s) * p1;
}

/* Reconstruction of the grid's order at one cell (both faces). */
static void weno(const grid* g, const double* v, double* vm, double* vp) {
    if (g->order == 3)
        weno3(g->eps, v, vm, vp);
    else
        weno5(g->eps, v, vm, vp);
}

/* ---- MLP-gated reconstruction (the gated form; no counterpart in the paper)
 * The gated form of the solver reconstructs smooth cells with the linear
 * weights and troubled cells with WENO5-JS, a small network deciding which
 * is which.  Per cell and direction two sensor stencils are read from the
 * primitives of the five stencil cells: the mixture density
 * alpha1 rho1 + alpha2 rho2 and the pressure.  A sensor stencil s is flat
 * when max_k |s_k - s_2| <= delta |s_2| (a round-off floor: below it the
 * linear and the WENO face values differ by at most about 3 delta |s_2|);
 * a flat stencil counts as smooth.  Otherwise it is normalised,
 * x_k = (s_k - s_2) / max_j |s_j - s_2|, and the network's logit z(x)
 * (mlp_oracle.c) decides: smooth when z < 0.  A cell whose two sensors are
 * smooth is reconstructed with the linear weights for every primitive field,
 * unless one of its two linear face states is non-physical -- rho <= 0,
 * alpha1 outside [0, 1] or (Gamma + 1) p + Pi <= 0 -- when WENO5-JS is used
 * instead (fallback); every other cell with WENO5-JS.  Two fluids only. */
typedef struct {
    const double* theta;  /* network parameters (1281, mlp_oracle.c layout) */
    double delta;         /* round-off floor of the flat test */
    signed char* dec;     /* out, per direction and cell: 0 WENO, 1 linear, 2 fallback to WENO */
    double* info;         /* out (or NULL), per direction and cell, GATE_INFO values: z of the
                             density and of the pressure stencil (NaN where flat), max_k|s_k - s_2|
                             / (delta |s_2|) of both, and, over the two linear faces (NaN where the
                             cell is not smooth), the smallest rho / (|a1r1| + |a2r2|), alpha1,
                             1 - alpha1 and ((Gamma + 1) p + Pi) / ((Gamma + 1)|p| + |Pi|): a linear
                             face is admissible when the first and last are > 0, the middle two >= 0 */
} gate_ctx;

#define GATE_INFO 8

void mlp_forward(const double* th, const double* x, long n, double* z);   /* mlp_oracle.c */
int mlp_normalise(const double* v5, double delta, double* x);            /* mlp_oracle.c */

/* Linear-weight (fifth-order upwind) face values: the WENO5 candidates of
 * weno5 combined with the linear weights themselves. */
static void linear5(const double* v, double* vm, double* vp) {
    double p0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) / 6.0;
    double p1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) / 6.0;
    double p2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) / 6.0;
    *vm = 0.1 * p0 + 0.6 * p1 + 0.3 * p2;
    p0 = (-v[0] + 5.0 * v[1] + 2.0 * v[2]) / 6.0;
    p1 = (2.0 * v[1] + 5.0 * v[2] - v[3]) / 6.0;
    p2 = (11.0 * v[2] - 7.0 * v[3] + 2.0 * v[4]) / 6.0;
    *vp = 0.3 * p0 + 0.6 * p1 + 0.1 * p2;
}

/* One sensor stencil: 1 when it counts as smooth.  *z: the logit (NaN when
 * flat); *ratio: max_k |s_k - s_2| / (delta |s_2|) (flat iff <= 1). */
static int sensor_smooth(const gate_ctx* G, const double* s, double* z, double* ratio) {
    double m = 0.0;
    for (int k = 0; k < 5; k++) {
        double d = fabs(s[k] - s[2]);
        if (d > m) m = d;
    }
    double fl = G->delta * fabs(s[2]);
    *ratio = fl > 0.0 ? m / fl : (m > 0.0 ? INFINITY : 0.0);
    double x[5];
    if (!mlp_normalise(s, G->delta, x)) {
        *z = NAN;
        return 1;
    }
    mlp_forward(G->theta, x, 1, z);
    return *z < 0.0;
}

/* A linear face state is usable when rho > 0, 0 <= alpha1 <= 1 and
 * (Gamma + 1) p + Pi > 0.  m[0..3] receive rho/(|a1r1| + |a2r2|), alpha1,
 * 1 - alpha1 and ((Gamma + 1) p + Pi)/((Gamma + 1)|p| + |Pi|). */
static int face_admissible(const grid* g, const double* w, double* m) {
    double rho = w[0] + w[1];
    double a1 = w[IA(g)];
    double G, Pi;
    mixture(g, &w[IA(g)], &G, &Pi);
    double c = (G + 1.0) * w[IE(g)] + Pi;
    m[0] = rho / (fabs(w[0]) + fabs(w[1]));
    m[1] = a1;
    m[2] = 1.0 - a1;
    m[3] = c / ((G + 1.0) * fabs(w[IE(g)]) + fabs(Pi));
    return rho > 0.0 && a1 >= 0.0 && a1 <= 1.0 && c > 0.0;
}

/* Reconstruction of cell j (both faces, every field) from the pencil rows
 * W5 (cells j-2 .. j+2) under the gate; returns the decision code. */
static int gated_cell(const grid* g, const gate_ctx* G, const double* W5, double* vm, double* vp, double* info) {
    int neq = g->neq;
    double sr[5], sp[5], zr, zp, rr, rp;
    for (int s = 0; s < 5; s++) {
        sr[s] = W5[s * neq + 0] + W5[s * neq + 1];
        sp[s] = W5[s * neq + IE(g)];
    }
    int smooth_r = sensor_smooth(G, sr, &zr, &rr);
    int smooth_p = sensor_smooth(G, sp, &zp, &rp);
    int code = 0;
    double adm[4] = {NAN, NAN, NAN, NAN};
    if (smooth_r && smooth_p) {
        for (int f = 0; f < neq; f++) {
            double v[5];
            for (int s = 0; s < 5; s++) v[s] = W5[s * neq + f];
            linear5(v, &vm[f], &vp[f]);
        }
        double mm[4], mp[4];
        int ok = face_admissible(g, vm, mm) & face_admissible(g, vp, mp);
        for (int k = 0; k < 4; k++) adm[k] = mm[k] < mp[k] ? mm[k] : mp[k];
        code = ok ? 1 : 2;
    }
    if (code != 1) {
        for (int f = 0; f < neq; f++) {
            double v[5];
            for (int s = 0; s < 5; s++) v[s] = W5[s * neq + f];
            weno5(g->eps, v, &vm[f], &vp[f]);
        }
    }
    if (info) {
        info[0] = zr;
        info[1] = zp;
        info[2] = rr;
        info[3] = rp;
        for (int k = 0; k < 4; k++) info[4 + k] = adm[k];
    }
    return code;
}

/* ---- HLLC (Sec. II-B; Toro's three-wave approximate solver) -------------- */

typedef struct {
    double rho, u[3], p, a[3], G, Pi, E, c2;   /* a: the carried volume fractions */
} face_state;

static void face_from_prim(const grid* g, const double* w, face_state* s) {
    s->rho = mix_rho(g, w);
    s->u[0] = s->u[1] = s->u[2] = 0.0;
    for (int k = 0; k < g->ndim; k++) s->u[k] = w[IU(g) + k];
    s->p = w[IE(g)];
    for (int i = 0; i < g->nf - 1; i++) s->a[i] = w[IA(g) + i];
    mixture(g, s->a, &s->G, &s->Pi);
    s->E = s->G * s->p + s->Pi + kinetic(g, s->rho, s->u);
    s->c2 = sound2(s->G, s->Pi, s->rho, s->p);
}

/* Physical flux of the face state K in direction dir. */
static void phys_flux(const grid* g, int dir, const double* w, const face_state* K, double* F) {
    double un = K->u[dir];
    for (int i = 0; i < g->nf; i++) F[i] = w[i] * un;
    for (int k = 0; k < g->ndim; k++) F[IU(g) + k] = K->rho * K->u[k] * un;
    F[IU(g) + dir] = F[IU(g) + dir] + K->p;
    F[IE(g)] = (K->E + K->p) * un;
    for (int i = 0; i < g->nf - 1; i++) F[IA(g) + i] = K->a[i] * un;
}

/* HLLC star-region flux F*_K = F_K + S_K (q*_K - q_K); the volume-fraction
 * slots carry alpha_i,K S* (advection with the contact velocity). */
static void star_flux(const grid* g, int dir, const double* w, const face_state* K,
                      double SK, double Ss, double* F) {
    double un = K->u[dir];
    phys_flux(g, dir, w, K, F);
    double chi = (SK - un) / (SK - Ss);
    for (int i = 0; i < g->nf; i++) F[i] = F[i] + SK * (chi * w[i] - w[i]);
    for (int k = 0; k < g->ndim; k++) {
        double mstar = (k == dir) ? chi * K->rho * Ss : chi * K->rho * K->u[k];
        F[IU(g) + k] = F[IU(g) + k] + SK * (mstar - K->rho * K->u[k]);
    }
    double Estar = chi * (K->E + (Ss - un) * (K->rho * Ss + K->p / (SK - un)));
    F[IE(g)] = F[IE(g)] + SK * (Estar - K->E);
    for (int i = 0; i < g->nf - 1; i++) F[IA(g) + i] = K->a[i] * Ss;
}

/* Flux through one face from the reconstructed primitive states wL, wR.
 * uf receives the velocity of the selected region, used by the
 * non-conservative volume-fraction term.  Returns 0, or 1 when a face state
 * is non-physical (rho <= 0, c^2 <= 0 or NaN). */
static int hllc(const grid* g, int dir, const double* wL, const double* wR, double* F, double* uf) {
    face_state L, R;
    face_from_prim(g, wL, &L);
    face_from_prim(g, wR, &R);
    int bad = !(L.rho > 0.0) || !(R.rho > 0.0) || !(L.c2 > 0.0) || !(R.c2 > 0.0);
    double cL = sqrt(L.c2), cR = sqrt(R.c2);
    double uL = L.u[dir], uR = R.u[dir];
    double SL = (uL - cL < uR - cR) ? uL - cL : uR - cR;   /* Davis estimates */
    double SR = (uL + cL > uR + cR) ? uL + cL : uR + cR;
    double num = R.p - L.p + L.rho * uL * (SL - uL) - R.rho * uR * (SR - uR);
    double den = L.rho * (SL - uL) - R.rho * (SR - uR);
    double Ss = num / den;
    if (0.0 <= SL) {
        phys_flux(g, dir, wL, &L, F);
        *uf = uL;
    } else if (0.0 <= Ss) {
        star_flux(g, dir, wL, &L, SL, Ss, F);
        *uf = Ss;
    } else if (0.0 <= SR) {
        star_flux(g, dir, wR, &R, SR, Ss, F);
        *uf = Ss;
    } else {
        phys_flux(g, dir, wR, &R, F);
        *uf = uR;
    }
    return bad;
}

/* ---- semi-discrete right-hand side (Sec. II-B, cell-integrated form) ----- */

/* Ghost index map: transmissive = nearest interior cell, periodic = wrap. */
static long bc_map(long j, long n, int periodic) {
    if (periodic) {
        long r = j % n;
        return r < 0 ? r + n : r;
    }
    if (j < 0) return 0;
    if (j > n - 1) return n - 1;
    return j;
}

/* Primitives of one cell; returns 1 when the cell's mixture density is not
 * positive (or NaN). */
static int load_prim(const grid* g, const double* q, long cell, double* w) {
    double qc[NEQ_MAX];
    for (int f = 0; f < g->neq; f++) qc[f] = q[(long)f * g->ncell + cell];
    cons_to_prim(g, qc, w);
    return !(mix_rho(g, qc) > 0.0);
}

/* Reconstruction of cell j (index along direction d) of the grid's order. */
static void weno_cell(const grid* g, int d, long j, const double* v, double* vm, double* vp) {
    if (g->stretched[d])
        weno5_nu(&g->tab[d][(j + 1) * NT], g->eps, v, vm, vp);
    else
        weno(g, v, vm, vp);
}

/* Width of cell j along d (uniform: dx_d). */
static double cell_width(const grid* g, int d, long j) {
    return g->stretched[d] ? g->h[d][j + 3] : g->dx[d];
}

/* Contribution of direction d at cell i (index along d), from the primitive
 * pencil W (7 cells, i-3..i+3).  L receives
 *   (F_{i-1/2} - F_{i+1/2})/dx_i  for every equation, plus
 *   alpha1_i (u_f,{i+1/2} - u_f,{i-1/2})/dx_i  on the alpha1 row. */
static int cell_dir(const grid* g, int d, long i, const double* W7, double* L) {
    int neq = g->neq;
    double vm[3][NEQ_MAX], vp[3][NEQ_MAX];
    /* WENO at cells i-1, i, i+1 (pencil slots 2, 3, 4) */
    for (int c = 0; c < 3; c++) {
        for (int f = 0; f < neq; f++) {
            double v[5];
            for (int s = 0; s < 5; s++) v[s] = W7[(c + s) * neq + f];
            weno_cell(g, d, i - 1 + c, v, &vm[c][f], &vp[c][f]);
        }
    }
    double Fm[NEQ_MAX], Fp[NEQ_MAX], ufm, ufp;
    int bad = hllc(g, d, vm[0], vp[1], Fm, &ufm);   /* face i-1/2 */
    bad |= hllc(g, d, vm[1], vp[2], Fp, &ufp);      /* face i+1/2 */
    double dx = cell_width(g, d, i);
    for (int f = 0; f < neq; f++) L[f] = (Fm[f] - Fp[f]) / dx;
    for (int i = 0; i < g->nf - 1; i++) {
        double ai = W7[3 * neq + IA(g) + i];
        L[IA(g) + i] = L[IA(g) + i] + ai * (ufp - ufm) / dx;
    }
    return bad;
}

/* Full RHS for direction d over all pencils, computing each face once.
 * Returns 1 when a cell (rho <= 0) or a face state (rho <= 0, c^2 <= 0) of
 * the stencils was non-physical. */
static int rhs_dir(const grid* g, int d, const double* q, double* rhs, int first, const gate_ctx* gate,
                   double* W, double* VM, double* VP, double* FF, double* UF) {
    int neq = g->neq;
    long nd = g->n[d];
    int o1 = (d + 1) % 3, o2 = (d + 2) % 3;
    int bad = 0;
    for (long j2 = 0; j2 < g->n[o2]; j2++) {
        for (long j1 = 0; j1 < g->n[o1]; j1++) {
            long base = j1 * g->stride[o1] + j2 * g->stride[o2];
            /* primitives of cells -3 .. nd+2 (slot = j + 3) */
            for (long j = -3; j < nd + 3; j++) {
                long src = bc_map(j, nd, g->periodic[d]);
                bad |= load_prim(g, q, base + src * g->stride[d], &W[(j + 3) * neq]);
            }
            /* WENO (or, under a gate, the gated reconstruction) at cells
             * -1 .. nd (slot = j + 1) */
            for (long j = -1; j < nd + 1; j++) {
                if (gate) {
                    long cell = base + bc_map(j, nd, g->periodic[d]) * g->stride[d];
                    int inside = j >= 0 && j < nd;
                    double* info = inside && gate->info ? &gate->info[((long)d * g->ncell + cell) * GATE_INFO] : NULL;
                    int code = gated_cell(g, gate, &W[(j + 1) * neq], &VM[(j + 1) * neq], &VP[(j + 1) * neq], info);
                    if (inside) gate->dec[(long)d * g->ncell + cell] = (signed char)code;
                    continue;
                }
                for (int f = 0; f < neq; f++) {
                    double v[5];
                    for (int s = 0; s < 5; s++) v[s] = W[(j + 1 + s) * neq + f];
                    weno_cell(g, d, j, v, &VM[(j + 1) * neq + f], &VP[(j + 1) * neq + f]);
                }
            }
            /* HLLC at faces j+1/2, j = -1 .. nd-1 (face slot = j + 1) */
            for (long j = -1; j < nd; j++) {
                bad |= hllc(g, d, &VM[(j + 1) * neq], &VP[(j + 2) * neq], &FF[(j + 1) * neq],
                            &UF[j + 1]);
            }
            for (long i = 0; i < nd; i++) {
                long cell = base + i * g->stride[d];
                double dx = cell_width(g, d, i);
                double L[NEQ_MAX];
                for (int f = 0; f < neq; f++) L[f] = (FF[i * neq + f] - FF[(i + 1) * neq + f]) / dx;
                for (int k = 0; k < g->nf - 1; k++) {
                    double ak = W[(i + 3) * neq + IA(g) + k];
                    L[IA(g) + k] = L[IA(g) + k] + ak * (UF[i + 1] - UF[i]) / dx;
                }
                for (int f = 0; f < neq; f++) {
                    double* r = &rhs[(long)f * g->ncell + cell];
                    *r = first ? L[f] : *r + L[f];
                }
            }
        }
    }
    return bad;
}

static int rhs_all(const grid* g, const double* q, double* rhs, const gate_ctx* gate) {
    long nmax = 1;
    for (int d = 0; d < g->ndim; d++)
        if (g->n[d] > nmax) nmax = g->n[d];
    int neq = g->neq;
    double* W = malloc(sizeof(double) * (nmax + 6) * neq);
    double* VM = malloc(sizeof(double) * (nmax + 2) * neq);
    double* VP = malloc(sizeof(double) * (nmax + 2) * neq);
    double* FF = malloc(sizeof(double) * (nmax + 1) * neq);
    double* UF = malloc(sizeof(double) * (nmax + 1));
    if (!W || !VM || !VP || !FF || !UF) {
        free(W); free(VM); free(VP); free(FF); free(UF);
        return ORC_ENOMEM;
    }
    int bad = 0;
    for (int d = 0; d < g->ndim; d++) bad |= rhs_dir(g, d, q, rhs, d == 0, gate, W, VM, VP, FF, UF);
    free(W); free(VM); free(VP); free(FF); free(UF);
    for (long i = 0; i < (long)neq * g->ncell; i++)
        if (isnan(rhs[i]) || isinf(rhs[i])) bad = 1;
    return bad ? ORC_ENONPHYSICAL : ORC_OK;
}

/* ---- public entry points (ctypes) ---------------------------------------- */

int orc_neq(const orc_params* p) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    free_grid(&g);
    return g.neq;
}

int orc_prim_to_cons(const orc_params* p, const double* w, double* q) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    double wc[NEQ_MAX], qc[NEQ_MAX];
    for (long c = 0; c < g.ncell; c++) {
        for (int f = 0; f < g.neq; f++) wc[f] = w[(long)f * g.ncell + c];
        prim_to_cons(&g, wc, qc);
        for (int f = 0; f < g.neq; f++) q[(long)f * g.ncell + c] = qc[f];
    }
    free_grid(&g);
    return ORC_OK;
}

int orc_cons_to_prim(const orc_params* p, const double* q, double* w) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    double wc[NEQ_MAX];
    for (long c = 0; c < g.ncell; c++) {
        load_prim(&g, q, c, wc);
        for (int f = 0; f < g.neq; f++) w[(long)f * g.ncell + c] = wc[f];
    }
    free_grid(&g);
    return ORC_OK;
}

/* L(q): the semi-discrete right-hand side, same layout as q. */
int orc_rhs(const orc_params* p, const double* q, double* rhs) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    st = rhs_all(&g, q, rhs, NULL);
    free_grid(&g);
    return st;
}

/* L(q) of the gated form: the right-hand side with each cell's
 * reconstruction chosen by the gate (see gated_cell), network parameters
 * theta, round-off floor delta.  dec receives ndim * ncell decision codes
 * [direction][cell] (0 WENO, 1 linear, 2 fallback); info, if not NULL,
 * ndim * ncell * GATE_INFO values.  Two fluids, WENO5, uniform grids. */
int orc_rhs_gated(const orc_params* p, const double* q, const double* theta, double delta, double* rhs,
                  signed char* dec, double* info) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    if (g.nf != 2 || g.order != 5 || g.stretched[0] || g.stretched[1] || g.stretched[2] || !theta || !dec ||
        !(delta >= 0.0)) {
        free_grid(&g);
        return ORC_EINVAL;
    }
    gate_ctx G = {theta, delta, dec, info};
    st = rhs_all(&g, q, rhs, &G);
    free_grid(&g);
    return st;
}

/* L(q) at selected cells only (flat cell indices), out[k*neq + f].  Uses the
 * same per-face arithmetic as orc_rhs, on a 7-cell pencil per direction. */
int orc_rhs_points(const orc_params* p, const double* q, const long* cells, long npts, double* out) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    int neq = g.neq, bad = 0;
    for (long k = 0; k < npts; k++) {
        long cell = cells[k];
        if (cell < 0 || cell >= g.ncell) {
            free_grid(&g);
            return ORC_EINVAL;
        }
        long idx[3];
        long rem = cell;
        for (int d = 0; d < 3; d++) { idx[d] = rem % g.n[d]; rem /= g.n[d]; }
        double acc[NEQ_MAX];
        for (int d = 0; d < g.ndim; d++) {
            double W7[7 * NEQ_MAX], L[NEQ_MAX];
            long base = cell - idx[d] * g.stride[d];
            for (int s = 0; s < 7; s++) {
                long src = bc_map(idx[d] + s - 3, g.n[d], g.periodic[d]);
                bad |= load_prim(&g, q, base + src * g.stride[d], &W7[s * neq]);
            }
            bad |= cell_dir(&g, d, idx[d], W7, L);
            for (int f = 0; f < neq; f++) acc[f] = (d == 0) ? L[f] : acc[f] + L[f];
        }
        for (int f = 0; f < neq; f++) {
            out[k * neq + f] = acc[f];
            if (isnan(acc[f]) || isinf(acc[f])) bad = 1;
        }
    }
    free_grid(&g);
    return bad ? ORC_ENONPHYSICAL : ORC_OK;
}

/* S = max over cells of sum_d (|u_d| + c)/dx_d; the step is dt = CFL/S. */
int orc_max_wavespeed(const orc_params* p, const double* q, double* S_out) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    double S = 0.0;
    int bad = 0;
    double w[NEQ_MAX];
    for (long c = 0; c < g.ncell; c++) {
        bad |= load_prim(&g, q, c, w);
        double rho = mix_rho(&g, w);
        double G, Pi;
        mixture(&g, &w[IA(&g)], &G, &Pi);
        double c2 = sound2(G, Pi, rho, w[IE(&g)]);
        if (!(rho > 0.0) || !(c2 > 0.0)) bad = 1;
        double cs = sqrt(c2);
        double s = 0.0;
        for (int d = 0; d < g.ndim; d++)
            s = s + (fabs(w[IU(&g) + d]) + cs) / cell_width(&g, d, (c / g.stride[d]) % g.n[d]);
        if (s > S) S = s;
    }
    *S_out = S;
    free_grid(&g);
    return bad ? ORC_ENONPHYSICAL : ORC_OK;
}

/* One Shu-Osher TVD-RK3 step of size dt, in place:
 *   q1 = qn + dt L(qn)
 *   q2 = 3/4 qn + 1/4 (q1 + dt L(q1))
 *   qn+1 = 1/3 qn + 2/3 (q2 + dt L(q2)) */
int orc_step_dt(const orc_params* p, double* q, double dt) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    long m = (long)g.neq * g.ncell;
    double* L = malloc(sizeof(double) * m);
    double* q1 = malloc(sizeof(double) * m);
    double* q2 = malloc(sizeof(double) * m);
    if (!L || !q1 || !q2) {
        free(L); free(q1); free(q2);
        free_grid(&g);
        return ORC_ENOMEM;
    }
    int bad = 0;
    bad |= rhs_all(&g, q, L, NULL) != ORC_OK;
    for (long i = 0; i < m; i++) q1[i] = q[i] + dt * L[i];
    bad |= rhs_all(&g, q1, L, NULL) != ORC_OK;
    for (long i = 0; i < m; i++) q2[i] = 0.75 * q[i] + 0.25 * (q1[i] + dt * L[i]);
    bad |= rhs_all(&g, q2, L, NULL) != ORC_OK;
    for (long i = 0; i < m; i++) q[i] = (1.0 / 3.0) * q[i] + (2.0 / 3.0) * (q2[i] + dt * L[i]);
    free(L); free(q1); free(q2);
    free_grid(&g);
    return bad ? ORC_ENONPHYSICAL : ORC_OK;
}

/* nsteps steps with dt_n = cfl / S(q^n); t_out receives the sum of the dt_n. */
int orc_run_cfl(const orc_params* p, double* q, double cfl, int nsteps, double* t_out) {
    double t = 0.0;
    int st = ORC_OK;
    for (int n = 0; n < nsteps; n++) {
        double S;
        st = orc_max_wavespeed(p, q, &S);
        if (st) break;
        double dt = cfl / S;
        st = orc_step_dt(p, q, dt);
        t = t + dt;
        if (st) break;
    }
    if (t_out) *t_out = t;
    return st;
}

/* ---- element-level entry points used by the unit pins -------------------- */

/* Nonlinear WENO5-JS weights of cell i (same formulas as weno5): wm[k] for
 * the left-biased value at i+1/2 (linear weights 0.1, 0.6, 0.3) and wp[k]
 * for the right-biased value at i-1/2 (0.3, 0.6, 0.1). */
void orc_weno5_weights(double eps, const double* v, double* wm, double* wp) {
    const double c13 = 13.0 / 12.0;
    double b0 = c13 * sq(v[0] - 2.0 * v[1] + v[2]) + 0.25 * sq(v[0] - 4.0 * v[1] + 3.0 * v[2]);
    double b1 = c13 * sq(v[1] - 2.0 * v[2] + v[3]) + 0.25 * sq(v[1] - v[3]);
    double b2 = c13 * sq(v[2] - 2.0 * v[3] + v[4]) + 0.25 * sq(3.0 * v[2] - 4.0 * v[3] + v[4]);
    const double dm[3] = {0.1, 0.6, 0.3}, dp[3] = {0.3, 0.6, 0.1};
    const double b[3] = {b0, b1, b2};
    double am[3], ap[3], sm = 0.0, sp = 0.0;
    for (int k = 0; k < 3; k++) {
        am[k] = dm[k] / sq(eps + b[k]);
        ap[k] = dp[k] / sq(eps + b[k]);
        sm = sm + am[k];
        sp = sp + ap[k];
    }
    for (int k = 0; k < 3; k++) {
        wm[k] = am[k] / sm;
        wp[k] = ap[k] / sp;
    }
}


void orc_weno5_cell(double eps, const double* v5, double* vm, double* vp) { weno5(eps, v5, vm, vp); }

void orc_weno3_cell(double eps, const double* v5, double* vm, double* vp) { weno3(eps, v5, vm, vp); }

/* Linear-weight face values of the middle cell of v5 (the gated form's
 * reconstruction of smooth cells). */
void orc_linear5_cell(const double* v5, double* vm, double* vp) { linear5(v5, vm, vp); }

/* Non-uniform WENO5 table (NT doubles, layout of cell_table) of a cell from
 * the widths w5 of cells i-2 .. i+2; returns 1 if degenerate. */
int orc_weno5_table(const double* w5, double* T) { return cell_table(w5, T); }

/* Non-uniform WENO5 face values of a cell from its table. */
void orc_weno5_nu_cell(const double* T, double eps, const double* v5, double* vm, double* vp) {
    weno5_nu(T, eps, v5, vm, vp);
}

int orc_hllc_face(const orc_params* p, int dir, const double* wL, const double* wR, double* F,
                  double* uf) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    free_grid(&g);
    if (dir < 0 || dir >= g.ndim) return ORC_EINVAL;
    return hllc(&g, dir, wL, wR, F, uf) ? ORC_ENONPHYSICAL : ORC_OK;
}

int orc_sound_speed2(const orc_params* p, const double* w, double* c2) {
    grid g;
    int st = make_grid(p, &g);
    if (st) return st;
    free_grid(&g);
    double G, Pi;
    mixture(&g, &w[IA(&g)], &G, &Pi);
    *c2 = sound2(G, Pi, mix_rho(&g, w), w[IE(&g)]);
    return ORC_OK;
}

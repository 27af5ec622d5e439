/*
 * mgm_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the meshfree geometric
 * multilevel (MGM) method of Wright, Jones & Shankar ("MGM: A meshfree geometric multilevel
 * method for systems arising from elliptic equations on point cloud surfaces").
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the package's smoke check and the benchmark's CPU
 * baseline may load this library. It shares no code, header, table or helper with the CUDA
 * library; each routine below is written from the paper's definitions (section / equation /
 * algorithm cited per function), in the paper's order, with no blocking or fusion.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (the compiler never fuses a*b+c on its own;
 * where a fused multiply-add is part of an operation's definition here it is written as fma(),
 * the IEEE-754 fusedMultiplyAdd, so every result is fully determined by the source).
 *
 * Conventions: points are N x 3 row-major doubles; sparse matrices are CSR with int32 column
 * indices ascending within each row; all indices 0-based. Functions return 0 on success and a
 * positive status otherwise (1 bad argument, 2 singular local system, 3 not converged, 7 no memory).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_SINGULAR 2
#define OR_ERR_NOTCONV 3
#define OR_ERR_NOMEM 7
#define MAXM 160

static int64_t g_bad_row = -1;
int64_t or_last_bad_row(void) { return g_bad_row; }

/* squared Euclidean distance in R^3, evaluated as (dx*dx + dy*dy) + dz*dz, every op rounded */
static double dist2(const double* a, const double* b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return (dx * dx + dy * dy) + dz * dz;
}

/* (d, j) < (e, k) in the lexicographic order used to rank neighbours */
static int key_less(double d, int64_t j, double e, int64_t k) { return d < e || (d == e && j < k); }

/* ===========================================================================================
 * Nearest neighbours (Sec. 2: a stencil is its centre's n nearest nodes by Euclidean distance in
 * the embedding space; Sec. 3: the m nearest coarse nodes of a fine node). Brute force.
 * Order: ascending (d^2, index). With self_first, query q is also data point q and is placed
 * first (the stencil centre) regardless of duplicates.
 * =========================================================================================== */
int or_knn(const double* data, int64_t nd, const double* query, int64_t nq, int k, int self_first,
           int32_t* idx_out, double* d2_out) {
    if (k <= 0 || k > nd || nd > INT32_MAX) return OR_ERR_ARG;
    double* bd = (double*)malloc(sizeof(double) * k);
    int64_t* bi = (int64_t*)malloc(sizeof(int64_t) * k);
    if (!bd || !bi) { free(bd); free(bi); return OR_ERR_NOMEM; }
    for (int64_t q = 0; q < nq; ++q) {
        int cnt = 0;
        for (int64_t j = 0; j < nd; ++j) {
            double d = (self_first && j == q) ? -1.0 : dist2(query + 3 * q, data + 3 * j);
            if (cnt == k && !key_less(d, j, bd[k - 1], bi[k - 1])) continue;
            int pos = (cnt < k) ? cnt++ : k - 1;
            while (pos > 0 && key_less(d, j, bd[pos - 1], bi[pos - 1])) {
                bd[pos] = bd[pos - 1]; bi[pos] = bi[pos - 1]; --pos;
            }
            bd[pos] = d; bi[pos] = j;
        }
        for (int t = 0; t < k; ++t) {
            idx_out[q * k + t] = (int32_t)bi[t];
            if (d2_out) d2_out[q * k + t] = bd[t] < 0.0 ? 0.0 : bd[t];
        }
    }
    free(bd); free(bi);
    return OR_OK;
}

/* ===========================================================================================
 * Dense solve by Gaussian elimination with partial pivoting on the augmented m x (m+1) matrix
 * (row-major, last column = right-hand side). Pivot: largest |a_ik|, first row on ties.
 * Multipliers l_ik = a_ik * (1/a_kk) (one reciprocal per pivot, as in LAPACK's unblocked LU; the
 * paper does not fix the local solver); update a_ij <- fma(-l_ik, a_kj, a_ij). Back substitution
 * column by column, x_k = b_k * (1/a_kk) with the pivot's reciprocal saved during elimination.
 * The system is declared singular when the pivot magnitude is <= tol.
 * =========================================================================================== */
static int gepp_solve(double* a, int m, double tol, double* x) {
    const int ld = m + 1;
    double rinvs[MAXM + 1];
    for (int k = 0; k < m; ++k) {
        int piv = k;
        double best = fabs(a[k * ld + k]);
        for (int i = k + 1; i < m; ++i) {
            double v = fabs(a[i * ld + k]);
            if (v > best) { best = v; piv = i; }
        }
        if (!(best > tol)) return OR_ERR_SINGULAR;
        if (piv != k)
            for (int j = 0; j < ld; ++j) { double t = a[k * ld + j]; a[k * ld + j] = a[piv * ld + j]; a[piv * ld + j] = t; }
        double rinv = 1.0 / a[k * ld + k];
        rinvs[k] = rinv;
        for (int i = k + 1; i < m; ++i) {
            double l = a[i * ld + k] * rinv;
            for (int j = k + 1; j < ld; ++j) a[i * ld + j] = fma(-l, a[k * ld + j], a[i * ld + j]);
        }
    }
    for (int k = m - 1; k >= 0; --k) {
        double xk = a[k * ld + m] * rinvs[k];
        x[k] = xk;
        for (int i = 0; i < k; ++i) a[i * ld + m] = fma(-a[i * ld + k], xk, a[i * ld + m]);
    }
    for (int k = 0; k < m; ++k) if (!isfinite(x[k])) return OR_ERR_SINGULAR;
    return OR_OK;
}

/* ===========================================================================================
 * Tangent plane (Sec. 2.1, eqs. (projection1)-(tp_pts)): orthonormal t1, t2 spanning T_x M.
 * t1 = normalise(e_a - (e_a . n) n) with e_a the coordinate axis of smallest |n_a| (first on
 * ties); t2 = n x t1. The normal is normalised first.
 * =========================================================================================== */
void or_tangent_basis(const double* nin, double* t1, double* t2) {
    double nn = sqrt((nin[0] * nin[0] + nin[1] * nin[1]) + nin[2] * nin[2]);
    double n[3] = {nin[0] / nn, nin[1] / nn, nin[2] / nn};
    int a = 0;
    if (fabs(n[1]) < fabs(n[a])) a = 1;
    if (fabs(n[2]) < fabs(n[a])) a = 2;
    double v[3] = {-n[a] * n[0], -n[a] * n[1], -n[a] * n[2]};
    v[a] = 1.0 + v[a];
    double vn = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    t1[0] = v[0] / vn; t1[1] = v[1] / vn; t1[2] = v[2] / vn;
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

static double dot3(const double* a, const double* b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

/* project stencil members to the tangent plane at the centre, eq. (tp_pts): xh_j = Q^T (x_j - x_1);
 * returns the support radius s = max_j |xh_j| (the radius of the smallest ball about the centre
 * enclosing the projected stencil). */
static double project_stencil(const double* xyz, const double* nrm, int64_t i, const int32_t* idx, int n,
                              double* xh, double* yh) {
    double t1[3], t2[3];
    or_tangent_basis(nrm + 3 * i, t1, t2);
    const double* xc = xyz + 3 * i;
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        const double* xj = xyz + 3 * (int64_t)idx[j];
        double d[3] = {xj[0] - xc[0], xj[1] - xc[1], xj[2] - xc[2]};
        xh[j] = dot3(t1, d);
        yh[j] = dot3(t2, d);
        double r = sqrt(xh[j] * xh[j] + yh[j] * yh[j]);
        if (r > s) s = r;
    }
    return s;
}

/* bivariate monomials of degree <= ell, ordered by total degree, then by descending power of x */
static int n_monomials(int ell) { return (ell + 1) * (ell + 2) / 2; }
static void monomial_powers(int ell, int* pa, int* pb) {
    int t = 0;
    for (int d = 0; d <= ell; ++d)
        for (int a = d; a >= 0; --a) { pa[t] = a; pb[t] = d - a; ++t; }
}
static double monomial(double x, double y, int a, int b) {
    double p = 1.0;
    for (int t = 0; t < a; ++t) p = p * x;
    for (int t = 0; t < b; ++t) p = p * y;
    return p;
}
/* PHS kernel phi(r) = r^(2k+1) from r^2: sqrt(r2) * r2^k */
static double phs(double r2, int k) {
    double p = 1.0;
    for (int t = 0; t < k; ++t) p = p * r2;
    return sqrt(r2) * p;
}
/* 2-D Laplacian of phi(|x - c|) at x = 0: (2k+1)^2 |c|^(2k-1), written as (2k+1)^2 sqrt(r2) r2^(k-1) */
static double phs_lap(double r2, int k) {
    if (r2 == 0.0) return 0.0;
    double p = 1.0;
    for (int t = 0; t < k - 1; ++t) p = p * r2;
    double c = (double)((2 * k + 1) * (2 * k + 1));
    return c * (sqrt(r2) * p);
}


/* ===========================================================================================
 * PHS RBF-FD weights for the LBO (Sec. 2.2, eq. (rbf_fd_lap)): for each stencil solve
 *   [A P; P^T 0][c; lambda] = [Lap phi; Lap p]
 * with A_ij = |xh_i - xh_j|^(2k+1), P_ij = p_j(xh_i), in tangent-plane coordinates scaled by the
 * stencil support s (xh * (1/s)); the weights for the unscaled Laplacian are c / s^2 (PHS with
 * polynomials of degree >= k is scale-invariant). Singular when a pivot is <= 1e-13 max|M|.
 * =========================================================================================== */
/* Weights of all N stencils (rows NULL; idx is N x n), or of the stencils centred at rows[0..nrows-1]
 * with neighbours idx[t*n..] (idx is nrows x n), into w_out (one row per stencil). */
static int phs_weights_rows(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, int n, int k, int ell,
                            const int32_t* rows, int64_t nrows, double* w_out) {
    int L = n_monomials(ell);
    int m = n + L;
    if (n < 1 || k < 1 || ell < 0 || m > MAXM || L > n) return OR_ERR_ARG;
    int pa[64], pb[64];
    monomial_powers(ell, pa, pb);
    double* a = (double*)malloc(sizeof(double) * m * (m + 1));
    double xh[MAXM], yh[MAXM], x[MAXM];
    if (!a) return OR_ERR_NOMEM;
    g_bad_row = -1;
    const int64_t cnt = rows ? nrows : N;
    for (int64_t t = 0; t < cnt; ++t) {
        const int64_t i = rows ? (int64_t)rows[t] : t;
        if (i < 0 || i >= N) { free(a); return OR_ERR_ARG; }
        const int32_t* id = idx + t * n;
        double s = project_stencil(xyz, nrm, i, id, n, xh, yh);
        if (!(s > 0.0)) { g_bad_row = i; free(a); return OR_ERR_SINGULAR; }
        double sinv = 1.0 / s;
        for (int j = 0; j < n; ++j) { xh[j] = xh[j] * sinv; yh[j] = yh[j] * sinv; }
        const int ld = m + 1;
        double amax = 0.0;
        for (int r = 0; r < n; ++r) {
            for (int c = 0; c < n; ++c) {
                double dx = xh[r] - xh[c], dy = yh[r] - yh[c];
                a[r * ld + c] = phs(dx * dx + dy * dy, k);
            }
            for (int c = 0; c < L; ++c) a[r * ld + n + c] = monomial(xh[r], yh[r], pa[c], pb[c]);
            a[r * ld + m] = phs_lap(xh[r] * xh[r] + yh[r] * yh[r], k);
        }
        for (int r = 0; r < L; ++r) {
            for (int c = 0; c < n; ++c) a[(n + r) * ld + c] = a[c * ld + n + r];
            for (int c = 0; c < L; ++c) a[(n + r) * ld + n + c] = 0.0;
            a[(n + r) * ld + m] = ((pa[r] == 2 && pb[r] == 0) || (pa[r] == 0 && pb[r] == 2)) ? 2.0 : 0.0;
        }
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c) { double v = fabs(a[r * ld + c]); if (v > amax) amax = v; }
        int st = gepp_solve(a, m, 1e-13 * amax, x);
        if (st) { g_bad_row = i; free(a); return st; }
        double s2 = s * s;
        for (int j = 0; j < n; ++j) w_out[t * n + j] = x[j] / s2;
    }
    free(a);
    return OR_OK;
}

int or_phs_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, int n, int k, int ell,
                   double* w_out) {
    return phs_weights_rows(xyz, nrm, N, idx, n, k, ell, NULL, 0, w_out);
}

int or_phs_weights_rows(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, int n, int k, int ell,
                        const int32_t* rows, int64_t nrows, double* w_out) {
    return phs_weights_rows(xyz, nrm, N, idx, n, k, ell, rows, nrows, w_out);
}

/* ===========================================================================================
 * Tangent-plane RBF-FD first derivatives (Sec. 6.3: the surface gradient and divergence of the
 * heat method, RBF-FD in the tangent plane): the saddle system of eq. (rbf_fd_lap) with the
 * right-hand sides d/dx^ and d/dy^ at the centre: for the PHS part
 * d/dx^ phi(|x^ - x^_j|) at 0 = -(2k+1) |x^_j|^(2k-1) x^_j, for the monomials 1 for x^ (resp. y^)
 * and 0 otherwise. Scaled coordinates as for the Laplacian; the weights are divided by s. Each
 * right-hand side is solved by its own GEPP (the eliminations of the two are identical).
 * The surface gradient of u at x_i is then t1 sum_j wx_ij u_j + t2 sum_j wy_ij u_j.
 * =========================================================================================== */
int or_phs_grad_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, int n, int k, int ell,
                        double* wx_out, double* wy_out) {
    int L = n_monomials(ell);
    int m = n + L;
    if (n < 1 || k < 1 || ell < 1 || m > MAXM || L > n) return OR_ERR_ARG;
    int pa[64], pb[64];
    monomial_powers(ell, pa, pb);
    double* a = (double*)malloc(sizeof(double) * m * (m + 1));
    double xh[MAXM], yh[MAXM], x[MAXM];
    if (!a) return OR_ERR_NOMEM;
    g_bad_row = -1;
    for (int64_t i = 0; i < N; ++i) {
        const int32_t* id = idx + i * n;
        double s = project_stencil(xyz, nrm, i, id, n, xh, yh);
        if (!(s > 0.0)) { g_bad_row = i; free(a); return OR_ERR_SINGULAR; }
        double sinv = 1.0 / s;
        for (int j = 0; j < n; ++j) { xh[j] = xh[j] * sinv; yh[j] = yh[j] * sinv; }
        const int ld = m + 1;
        for (int dir = 0; dir < 2; ++dir) {
            double amax = 0.0;
            for (int r = 0; r < n; ++r) {
                for (int c = 0; c < n; ++c) {
                    double dx = xh[r] - xh[c], dy = yh[r] - yh[c];
                    a[r * ld + c] = phs(dx * dx + dy * dy, k);
                }
                for (int c = 0; c < L; ++c) a[r * ld + n + c] = monomial(xh[r], yh[r], pa[c], pb[c]);
                /* -(2k+1) r^(2k-1) x_r with r^(2k-1) = sqrt(r2) r2^(k-1) */
                double r2 = xh[r] * xh[r] + yh[r] * yh[r];
                double rp = sqrt(r2);
                for (int t = 1; t < k; ++t) rp = rp * r2;
                a[r * ld + m] = -(double)(2 * k + 1) * rp * (dir == 0 ? xh[r] : yh[r]);
            }
            for (int r = 0; r < L; ++r) {
                for (int c = 0; c < n; ++c) a[(n + r) * ld + c] = a[c * ld + n + r];
                for (int c = 0; c < L; ++c) a[(n + r) * ld + n + c] = 0.0;
                a[(n + r) * ld + m] = (dir == 0 ? (pa[r] == 1 && pb[r] == 0) : (pa[r] == 0 && pb[r] == 1)) ? 1.0 : 0.0;
            }
            for (int r = 0; r < m; ++r)
                for (int c = 0; c < m; ++c) { double v = fabs(a[r * ld + c]); if (v > amax) amax = v; }
            int st = gepp_solve(a, m, 1e-13 * amax, x);
            if (st) { g_bad_row = i; free(a); return st; }
            double* w = dir == 0 ? wx_out : wy_out;
            for (int j = 0; j < n; ++j) w[i * n + j] = x[j] / s;
        }
    }
    free(a);
    return OR_OK;
}

/* Surface gradient (N x 3) of u and surface divergence of a field eta (N x 3), from the derivative
 * weights: grad_i = t1_i (wx_i . u) + t2_i (wy_i . u); div_i = sum_j wx_ij (eta_j . t1_i) +
 * wy_ij (eta_j . t2_i) (neighbour vectors projected onto the tangent plane of x_i). */
int or_surface_grad(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx, const double* wy,
                    const double* u, double* g) {
    for (int64_t i = 0; i < N; ++i) {
        double t1[3], t2[3], dx = 0.0, dy = 0.0;
        or_tangent_basis(nrm + 3 * i, t1, t2);
        for (int j = 0; j < n; ++j) { double v = u[idx[i * n + j]]; dx = dx + wx[i * n + j] * v; dy = dy + wy[i * n + j] * v; }
        for (int a = 0; a < 3; ++a) g[3 * i + a] = t1[a] * dx + t2[a] * dy;
    }
    return OR_OK;
}
int or_surface_div(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx, const double* wy,
                   const double* eta, double* d) {
    for (int64_t i = 0; i < N; ++i) {
        double t1[3], t2[3], acc = 0.0;
        or_tangent_basis(nrm + 3 * i, t1, t2);
        for (int j = 0; j < n; ++j) {
            const double* e = eta + 3 * (int64_t)idx[i * n + j];
            acc = acc + wx[i * n + j] * dot3(t1, e) + wy[i * n + j] * dot3(t2, e);
        }
        d[i] = acc;
    }
    return OR_OK;
}

/* ===========================================================================================
 * GFD weights (Sec. 2.3, eqs. (wls_fd_approx_system), (wls_fd_lap)): weighted least squares with
 * w_j = exp(-alpha |xh_1 - xh_j|^2 / (rho_1^2 + rho_j^2)), rho_k the support radius of stencil k in
 * its own tangent plane. c = W P (P^T W P)^{-1} Lap p, computed as c = W^{1/2} Q R^{-T} Lap p with
 * W^{1/2} P = Q R (Householder, thin), in scaled coordinates (weights divided by s^2).
 * =========================================================================================== */
int or_gfd_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, int n, int ell,
                   double alpha, double* w_out) {
    int L = n_monomials(ell);
    if (n < L || n > MAXM || L > 64) return OR_ERR_ARG;
    int pa[64], pb[64];
    monomial_powers(ell, pa, pb);
    double* rho = (double*)malloc(sizeof(double) * N);
    double* B = (double*)malloc(sizeof(double) * n * L);
    double* V = (double*)malloc(sizeof(double) * n * L);
    double xh[MAXM], yh[MAXM], sw[MAXM], z[MAXM], y[64], beta[64];
    if (!rho || !B || !V) { free(rho); free(B); free(V); return OR_ERR_NOMEM; }
    g_bad_row = -1;
    for (int64_t i = 0; i < N; ++i) rho[i] = project_stencil(xyz, nrm, i, idx + i * n, n, xh, yh);
    for (int64_t i = 0; i < N; ++i) {
        const int32_t* id = idx + i * n;
        double s = project_stencil(xyz, nrm, i, id, n, xh, yh);
        if (!(s > 0.0)) { g_bad_row = i; goto singular; }
        for (int j = 0; j < n; ++j) {
            double r2 = xh[j] * xh[j] + yh[j] * yh[j];
            double rj = rho[id[j]];
            sw[j] = sqrt(exp(-alpha * r2 / (rho[i] * rho[i] + rj * rj)));
            xh[j] = xh[j] / s; yh[j] = yh[j] / s;
        }
        for (int j = 0; j < n; ++j)
            for (int c = 0; c < L; ++c) B[j * L + c] = sw[j] * monomial(xh[j], yh[j], pa[c], pb[c]);
        /* Householder QR of B (n x L): column kk reflector v (stored in V[:, kk]), B <- H B */
        for (int kk = 0; kk < L; ++kk) {
            double nrm2 = 0.0;
            for (int r = kk; r < n; ++r) nrm2 = nrm2 + B[r * L + kk] * B[r * L + kk];
            double nx = sqrt(nrm2);
            if (!(nx > 0.0)) { g_bad_row = i; goto singular; }
            double alp = B[kk * L + kk] >= 0.0 ? -nx : nx;
            for (int r = 0; r < n; ++r) V[r * L + kk] = (r < kk) ? 0.0 : B[r * L + kk];
            V[kk * L + kk] = V[kk * L + kk] - alp;
            double vv = 0.0;
            for (int r = kk; r < n; ++r) vv = vv + V[r * L + kk] * V[r * L + kk];
            beta[kk] = 2.0 / vv;
            for (int c = kk; c < L; ++c) {
                double dotv = 0.0;
                for (int r = kk; r < n; ++r) dotv = dotv + V[r * L + kk] * B[r * L + c];
                double f = beta[kk] * dotv;
                for (int r = kk; r < n; ++r) B[r * L + c] = B[r * L + c] - f * V[r * L + kk];
            }
        }
        /* R = upper L x L block of B. Solve R^T y = Lap p (forward substitution). */
        double rmax = 0.0;
        for (int c = 0; c < L; ++c) { double v = fabs(B[c * L + c]); if (v > rmax) rmax = v; }
        for (int r = 0; r < L; ++r) {
            double rhs = ((pa[r] == 2 && pb[r] == 0) || (pa[r] == 0 && pb[r] == 2)) ? 2.0 : 0.0;
            for (int c = 0; c < r; ++c) rhs = rhs - B[c * L + r] * y[c];
            if (!(fabs(B[r * L + r]) > 1e-13 * rmax)) { g_bad_row = i; goto singular; }
            y[r] = rhs / B[r * L + r];
        }
        /* z = Q [y; 0] = H_0 H_1 ... H_{L-1} [y; 0] */
        for (int r = 0; r < n; ++r) z[r] = r < L ? y[r] : 0.0;
        for (int kk = L - 1; kk >= 0; --kk) {
            double dotv = 0.0;
            for (int r = kk; r < n; ++r) dotv = dotv + V[r * L + kk] * z[r];
            double f = beta[kk] * dotv;
            for (int r = kk; r < n; ++r) z[r] = z[r] - f * V[r * L + kk];
        }
        double s2 = s * s;
        for (int j = 0; j < n; ++j) w_out[i * n + j] = (sw[j] * z[j]) / s2;
    }
    free(rho); free(B); free(V);
    return OR_OK;
singular:
    free(rho); free(B); free(V);
    return OR_ERR_SINGULAR;
}

/* ===========================================================================================
 * Global assembly (Sec. 2, eq. (discrete_system)): D_h from the stencil weights; L = D (poisson)
 * or L = I - mu D. One CSR row per node, columns ascending. Off-diagonal value -mu*c (or c),
 * diagonal 1 - mu*c_ii (or c_ii).
 * =========================================================================================== */
int or_assemble(int64_t N, int n, const int32_t* idx, const double* w, double mu, int poisson,
                int32_t* rowptr, int32_t* col, double* val) {
    if ((int64_t)N * n > INT32_MAX) return OR_ERR_ARG;
    for (int64_t i = 0; i <= N; ++i) rowptr[i] = (int32_t)(i * n);
    for (int64_t i = 0; i < N; ++i) {
        int32_t* c = col + i * n;
        double* v = val + i * n;
        for (int j = 0; j < n; ++j) {
            int32_t cj = idx[i * n + j];
            double wj = w[i * n + j];
            double vj;
            if (poisson) vj = wj;
            else { double t = mu * wj; vj = (cj == i) ? 1.0 - t : -t; }
            int p = j;
            while (p > 0 && c[p - 1] > cj) { c[p] = c[p - 1]; v[p] = v[p - 1]; --p; }
            c[p] = cj; v[p] = vj;
        }
        for (int j = 1; j < n; ++j) if (c[j] == c[j - 1]) return OR_ERR_ARG;
    }
    return OR_OK;
}

/* ---- symmetrised adjacency (pattern of A + A^T without the diagonal), rows sorted ---- */
static int sym_adjacency(int64_t N, const int32_t* rowptr, const int32_t* col, int64_t** aptr_out, int32_t** adj_out) {
    int64_t* cnt = (int64_t*)calloc(N + 1, sizeof(int64_t));
    if (!cnt) return OR_ERR_NOMEM;
    for (int64_t i = 0; i < N; ++i)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = col[p];
            if (j == i) continue;
            cnt[i + 1]++; cnt[j + 1]++;
        }
    for (int64_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
    int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (cnt[N] > 0 ? cnt[N] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    if (!tmp || !fill) { free(cnt); free(tmp); free(fill); return OR_ERR_NOMEM; }
    for (int64_t i = 0; i < N; ++i) fill[i] = cnt[i];
    for (int64_t i = 0; i < N; ++i)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t j = col[p];
            if (j == i) continue;
            tmp[fill[i]++] = j; tmp[fill[j]++] = (int32_t)i;
        }
    /* sort each row (insertion sort), drop duplicates, compact */
    int64_t* aptr = (int64_t*)malloc(sizeof(int64_t) * (N + 1));
    if (!aptr) { free(cnt); free(tmp); free(fill); return OR_ERR_NOMEM; }
    int64_t w = 0;
    aptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        int64_t b = cnt[i], e = cnt[i + 1];
        for (int64_t p = b + 1; p < e; ++p) {
            int32_t v = tmp[p]; int64_t q = p;
            while (q > b && tmp[q - 1] > v) { tmp[q] = tmp[q - 1]; --q; }
            tmp[q] = v;
        }
        for (int64_t p = b; p < e; ++p)
            if (p == b || tmp[p] != tmp[p - 1]) tmp[w++] = tmp[p];
        aptr[i + 1] = w;
    }
    free(cnt); free(fill);
    *aptr_out = aptr; *adj_out = tmp;
    return OR_OK;
}

/* ===========================================================================================
 * Reverse Cuthill-McKee (Sec. 4.2; Alg. 2 reorders L_1 and each L_{j+1}) on the symmetrised
 * pattern. Start node: minimum degree, lowest index; breadth-first, each node's unvisited
 * neighbours appended in increasing (degree, index); a new start for each further component;
 * the visit order is reversed at the end. perm[new] = old.
 * =========================================================================================== */
int or_rcm(int64_t N, const int32_t* rowptr, const int32_t* col, int32_t* perm) {
    int64_t* aptr; int32_t* adj;
    int st = sym_adjacency(N, rowptr, col, &aptr, &adj);
    if (st) return st;
    int64_t* deg = (int64_t*)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    char* vis = (char*)calloc(N > 0 ? N : 1, 1);
    int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    int32_t* nb = NULL; int64_t nbcap = 0;
    if (!deg || !vis || !order) { free(aptr); free(adj); free(deg); free(vis); free(order); return OR_ERR_NOMEM; }
    for (int64_t i = 0; i < N; ++i) deg[i] = aptr[i + 1] - aptr[i];
    int64_t head = 0, tail = 0;
    while (tail < N) {
        int64_t s = -1;
        for (int64_t i = 0; i < N; ++i)
            if (!vis[i] && (s < 0 || deg[i] < deg[s])) s = i;
        vis[s] = 1; order[tail++] = (int32_t)s;
        while (head < tail) {
            int32_t v = order[head++];
            int64_t cnt = 0, need = aptr[v + 1] - aptr[v];
            if (need > nbcap) { nbcap = need; nb = (int32_t*)realloc(nb, sizeof(int32_t) * nbcap); }
            for (int64_t p = aptr[v]; p < aptr[v + 1]; ++p)
                if (!vis[adj[p]]) nb[cnt++] = adj[p];
            for (int64_t p = 1; p < cnt; ++p) {   /* insertion sort by (degree, index) */
                int32_t u = nb[p]; int64_t q = p;
                while (q > 0 && (deg[nb[q - 1]] > deg[u] || (deg[nb[q - 1]] == deg[u] && nb[q - 1] > u))) { nb[q] = nb[q - 1]; --q; }
                nb[q] = u;
            }
            for (int64_t p = 0; p < cnt; ++p) { vis[nb[p]] = 1; order[tail++] = nb[p]; }
        }
    }
    for (int64_t i = 0; i < N; ++i) perm[i] = order[N - 1 - i];
    free(aptr); free(adj); free(deg); free(vis); free(order); free(nb);
    return OR_OK;
}

/* ===========================================================================================
 * Greedy multicolouring for the multicolour Gauss-Seidel smoother: vertices of the symmetrised
 * pattern visited in decreasing (priority, index), priority = SplitMix64(seed + (i+1)*golden
 * gamma) (Steele, Lea & Flood 2014), each given the smallest colour not used by an already
 * coloured neighbour. Returns the number of colours.
 * =========================================================================================== */
static uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
uint64_t or_priority(uint64_t seed, uint64_t i) { return splitmix64(seed, i); }

static uint64_t* g_prio;
static int cmp_prio_desc(const void* a, const void* b) {
    int32_t i = *(const int32_t*)a, j = *(const int32_t*)b;
    if (g_prio[i] != g_prio[j]) return g_prio[i] > g_prio[j] ? -1 : 1;
    return i > j ? -1 : (i < j ? 1 : 0);
}

int or_color(int64_t N, const int32_t* rowptr, const int32_t* col, uint64_t seed, int32_t* color, int32_t* ncolors) {
    int64_t* aptr; int32_t* adj;
    int st = sym_adjacency(N, rowptr, col, &aptr, &adj);
    if (st) return st;
    uint64_t* pr = (uint64_t*)malloc(sizeof(uint64_t) * (N > 0 ? N : 1));
    int32_t* ord = (int32_t*)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    int64_t maxdeg = 0;
    for (int64_t i = 0; i < N; ++i) if (aptr[i + 1] - aptr[i] > maxdeg) maxdeg = aptr[i + 1] - aptr[i];
    char* used = (char*)calloc(maxdeg + 2, 1);
    if (!pr || !ord || !used) { free(aptr); free(adj); free(pr); free(ord); free(used); return OR_ERR_NOMEM; }
    for (int64_t i = 0; i < N; ++i) { pr[i] = splitmix64(seed, (uint64_t)i); ord[i] = (int32_t)i; color[i] = -1; }
    g_prio = pr;
    qsort(ord, N, sizeof(int32_t), cmp_prio_desc);
    int32_t nc = 0;
    for (int64_t t = 0; t < N; ++t) {
        int32_t v = ord[t];
        for (int64_t p = aptr[v]; p < aptr[v + 1]; ++p) { int32_t c = color[adj[p]]; if (c >= 0 && c <= maxdeg) used[c] = 1; }
        int32_t c = 0;
        while (used[c]) ++c;
        color[v] = c;
        if (c + 1 > nc) nc = c + 1;
        for (int64_t p = aptr[v]; p < aptr[v + 1]; ++p) { int32_t cc = color[adj[p]]; if (cc >= 0 && cc <= maxdeg) used[cc] = 0; }
    }
    *ncolors = nc;
    free(aptr); free(adj); free(pr); free(ord); free(used);
    return OR_OK;
}

/* ===========================================================================================
 * Weighted sample elimination (Sec. 4.1; Yuksel 2015, whose formulas the paper cites but does
 * not restate). Reading used here:
 *   dbar   = mean nearest-neighbour distance (summed exactly in 2^-32 fixed point),
 *   area   = N (sqrt(3)/2) dbar^2            (hexagonal-packing estimate of the surface area),
 *   r_max  = sqrt(area / (2 sqrt(3) N_H)),    r_min = r_max (1 - (N_H/N)^1.5) 0.65,
 *   w_ij   = (1 - max(d_ij, r_min) / (2 r_max))^8 for d_ij < 2 r_max (alpha = 8),
 *   w_i    = sum of w_ij over live neighbours, ascending index order.
 * mode 0 (sequential, as in the cited algorithm): repeatedly remove the live point with the
 *   largest (w, index); the weights of its live neighbours are then recomputed from scratch.
 * mode 1 (rounds): every live point with w > 0 whose (w, index) exceeds that of every live
 *   neighbour is removed in the same round (if no live point has w > 0, every live point is a
 *   candidate); if that is more than the removals still needed, only the largest (w, index)
 *   candidates go; weights of survivors are then recomputed from scratch. Repeat.
 * keep_out receives the N_H surviving indices ascending.
 * =========================================================================================== */
typedef struct { int64_t* ptr; int32_t* nbr; double* f; double rmax, rmin; } wse_graph;

static int wse_build(const double* xyz, int64_t N, int64_t NH, wse_graph* g) {
    int64_t S = 0;
    for (int64_t i = 0; i < N; ++i) {
        double best = -1.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d = dist2(xyz + 3 * i, xyz + 3 * j);
            if (best < 0.0 || d < best) best = d;
        }
        S += llrint(sqrt(best) * 4294967296.0);
    }
    double dbar = ((double)S / 4294967296.0) / (double)N;
    double area = (double)N * ((sqrt(3.0) * 0.5) * (dbar * dbar));
    double rmax = sqrt(area / ((2.0 * sqrt(3.0)) * (double)NH));
    double ratio = (double)NH / (double)N;
    double rmin = (rmax * (1.0 - ratio * sqrt(ratio))) * 0.65;
    double two_rmax = 2.0 * rmax;
    g->rmax = rmax; g->rmin = rmin;
    g->ptr = (int64_t*)malloc(sizeof(int64_t) * (N + 1));
    int64_t cap = 16 * N + 16, cnt = 0;
    g->nbr = (int32_t*)malloc(sizeof(int32_t) * cap);
    g->f = (double*)malloc(sizeof(double) * cap);
    if (!g->ptr || !g->nbr || !g->f) return OR_ERR_NOMEM;
    g->ptr[0] = 0;
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double d = sqrt(dist2(xyz + 3 * i, xyz + 3 * j));
            if (!(d < two_rmax)) continue;
            if (cnt == cap) {
                cap *= 2;
                g->nbr = (int32_t*)realloc(g->nbr, sizeof(int32_t) * cap);
                g->f = (double*)realloc(g->f, sizeof(double) * cap);
                if (!g->nbr || !g->f) return OR_ERR_NOMEM;
            }
            double dh = d > rmin ? d : rmin;
            double t = 1.0 - dh / two_rmax;
            double t2 = t * t, t4 = t2 * t2;
            g->nbr[cnt] = (int32_t)j; g->f[cnt] = t4 * t4; ++cnt;
        }
        g->ptr[i + 1] = cnt;
    }
    return OR_OK;
}

static int wgt_gt(double wa, int64_t a, double wb, int64_t b) { return wa > wb || (wa == wb && a > b); }

/* indexed binary max-heap on (w, index) for the sequential mode */
typedef struct { int64_t* h; int64_t* pos; double* w; int64_t n; } heap;
static void hswap(heap* H, int64_t a, int64_t b) {
    int64_t t = H->h[a]; H->h[a] = H->h[b]; H->h[b] = t; H->pos[H->h[a]] = a; H->pos[H->h[b]] = b;
}
static void hup(heap* H, int64_t k) {
    while (k > 0) { int64_t p = (k - 1) / 2; if (!wgt_gt(H->w[H->h[k]], H->h[k], H->w[H->h[p]], H->h[p])) break; hswap(H, k, p); k = p; }
}
static void hdown(heap* H, int64_t k) {
    for (;;) {
        int64_t l = 2 * k + 1, r = l + 1, b = k;
        if (l < H->n && wgt_gt(H->w[H->h[l]], H->h[l], H->w[H->h[b]], H->h[b])) b = l;
        if (r < H->n && wgt_gt(H->w[H->h[r]], H->h[r], H->w[H->h[b]], H->h[b])) b = r;
        if (b == k) break;
        hswap(H, k, b); k = b;
    }
}

int or_wse(const double* xyz, int64_t N, int64_t NH, int mode, int32_t* keep_out, double* rmax_out) {
    if (N < 2 || NH < 1 || NH > N) return OR_ERR_ARG;
    wse_graph g = {0};
    int st = wse_build(xyz, N, NH, &g);
    if (st) return st;
    if (rmax_out) rmax_out[0] = g.rmax;
    double* w = (double*)calloc(N, sizeof(double));
    char* live = (char*)malloc(N);
    for (int64_t i = 0; i < N; ++i) {
        live[i] = 1;
        double acc = 0.0;
        for (int64_t p = g.ptr[i]; p < g.ptr[i + 1]; ++p) acc = acc + g.f[p];
        w[i] = acc;
    }
    int64_t nlive = N;
    if (mode == 0) {
        heap H;
        H.h = (int64_t*)malloc(sizeof(int64_t) * N); H.pos = (int64_t*)malloc(sizeof(int64_t) * N);
        H.w = w; H.n = N;
        for (int64_t i = 0; i < N; ++i) { H.h[i] = i; H.pos[i] = i; }
        for (int64_t k = N / 2; k >= 0; --k) hdown(&H, k);
        while (nlive > NH) {
            int64_t v = H.h[0];
            hswap(&H, 0, H.n - 1); H.n--; hdown(&H, 0);
            live[v] = 0; --nlive;
            for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; ++p) {
                int64_t j = g.nbr[p];
                if (!live[j]) continue;
                /* w_j = sum over j's live neighbours, recomputed in ascending index order */
                double acc = 0.0;
                for (int64_t q = g.ptr[j]; q < g.ptr[j + 1]; ++q) if (live[g.nbr[q]]) acc = acc + g.f[q];
                w[j] = acc;
                hdown(&H, H.pos[j]); hup(&H, H.pos[j]);
            }
        }
        free(H.h); free(H.pos);
    } else {
        char* cand = (char*)malloc(N);
        char* dirty = (char*)malloc(N);
        int64_t* cl = (int64_t*)malloc(sizeof(int64_t) * N);
        while (nlive > NH) {
            int64_t need = nlive - NH, nc = 0;
            int anypos = 0;
            for (int64_t i = 0; i < N; ++i) if (live[i] && w[i] > 0.0) { anypos = 1; break; }
            for (int64_t i = 0; i < N; ++i) {
                cand[i] = 0;
                if (!live[i]) continue;
                if (anypos) {
                    if (!(w[i] > 0.0)) continue;
                    int ok = 1;
                    for (int64_t p = g.ptr[i]; p < g.ptr[i + 1]; ++p) {
                        int64_t j = g.nbr[p];
                        if (live[j] && !wgt_gt(w[i], i, w[j], j)) { ok = 0; break; }
                    }
                    if (!ok) continue;
                }
                cand[i] = 1; cl[nc++] = i;
            }
            if (nc > need) {
                /* keep only the `need` largest (w, index): partial selection sort (oracle: slow is fine) */
                for (int64_t a = 0; a < need; ++a) {
                    int64_t b = a;
                    for (int64_t c = a + 1; c < nc; ++c) if (wgt_gt(w[cl[c]], cl[c], w[cl[b]], cl[b])) b = c;
                    int64_t t = cl[a]; cl[a] = cl[b]; cl[b] = t;
                }
                for (int64_t c = need; c < nc; ++c) cand[cl[c]] = 0;
                nc = need;
            }
            memset(dirty, 0, N);
            for (int64_t c = 0; c < nc; ++c) {
                int64_t v = cl[c];
                live[v] = 0;
                for (int64_t p = g.ptr[v]; p < g.ptr[v + 1]; ++p) dirty[g.nbr[p]] = 1;
            }
            nlive -= nc;
            for (int64_t i = 0; i < N; ++i) {
                if (!live[i] || !dirty[i]) continue;
                double acc = 0.0;
                for (int64_t p = g.ptr[i]; p < g.ptr[i + 1]; ++p) if (live[g.nbr[p]]) acc = acc + g.f[p];
                w[i] = acc;
            }
        }
        free(cand); free(dirty); free(cl);
    }
    int64_t t = 0;
    for (int64_t i = 0; i < N; ++i) if (live[i]) keep_out[t++] = (int32_t)i;
    free(w); free(live); free(g.ptr); free(g.nbr); free(g.f);
    return OR_OK;
}

/* ===========================================================================================
 * PHS interpolation operator I_H^h (Sec. 3, eq. (rbf_fd_interp)): per fine node, the m nearest
 * coarse nodes in R^3; phi(r) = r (k = 0) plus a constant (ell = 0):
 *   [A 1; 1^T 0][d; lambda] = [s; 1],  A_ij = |y_i - y_j|,  s_i = |x - y_i|.
 * A fine node that coincides with its nearest coarse node gets the single entry 1.
 * Output CSR (capacity Nf*m entries), columns ascending.
 * =========================================================================================== */
int or_interp(const double* xf, int64_t Nf, const double* xc, int64_t Nc, int m, int32_t* rowptr, int32_t* col, double* val) {
    if (m < 1 || m > 16 || m > Nc) return OR_ERR_ARG;
    int32_t* nb = (int32_t*)malloc(sizeof(int32_t) * Nf * m);
    double* d2 = (double*)malloc(sizeof(double) * Nf * m);
    if (!nb || !d2) { free(nb); free(d2); return OR_ERR_NOMEM; }
    int st = or_knn(xc, Nc, xf, Nf, m, 0, nb, d2);
    if (st) { free(nb); free(d2); return st; }
    double a[17 * 18], x[17];
    int64_t p = 0;
    rowptr[0] = 0;
    g_bad_row = -1;
    for (int64_t i = 0; i < Nf; ++i) {
        const int32_t* id = nb + i * m;
        if (d2[i * m] == 0.0) {
            col[p] = id[0]; val[p] = 1.0; ++p;
        } else {
            int M = m + 1, ld = M + 1;
            double amax = 0.0;
            for (int r = 0; r < m; ++r) {
                for (int c = 0; c < m; ++c) a[r * ld + c] = sqrt(dist2(xc + 3 * (int64_t)id[r], xc + 3 * (int64_t)id[c]));
                a[r * ld + m] = 1.0;
                a[r * ld + M] = sqrt(d2[i * m + r]);
            }
            for (int c = 0; c < m; ++c) a[m * ld + c] = 1.0;
            a[m * ld + m] = 0.0;
            a[m * ld + M] = 1.0;
            for (int r = 0; r < M; ++r) for (int c = 0; c < M; ++c) { double v = fabs(a[r * ld + c]); if (v > amax) amax = v; }
            st = gepp_solve(a, M, 1e-13 * amax, x);
            if (st) { g_bad_row = i; free(nb); free(d2); return st; }
            int64_t b = p;
            for (int r = 0; r < m; ++r) {
                int32_t c = id[r]; double v = x[r];
                int64_t q = p;
                while (q > b && col[q - 1] > c) { col[q] = col[q - 1]; val[q] = val[q - 1]; --q; }
                col[q] = c; val[q] = v; ++p;
            }
        }
        rowptr[i + 1] = (int32_t)p;
    }
    free(nb); free(d2);
    return OR_OK;
}

/* ===========================================================================================
 * Restriction I_h^H = (I_H^h)^T (Sec. 3; Alg. 2): CSR transpose, columns ascending.
 * =========================================================================================== */
int or_transpose(int64_t nrows, int64_t ncols, const int32_t* rowptr, const int32_t* col, const double* val,
                 int32_t* trowptr, int32_t* tcol, double* tval) {
    for (int64_t j = 0; j <= ncols; ++j) trowptr[j] = 0;
    for (int64_t i = 0; i < nrows; ++i)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) trowptr[col[p] + 1]++;
    for (int64_t j = 0; j < ncols; ++j) trowptr[j + 1] += trowptr[j];
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (ncols > 0 ? ncols : 1));
    if (!fill) return OR_ERR_NOMEM;
    for (int64_t j = 0; j < ncols; ++j) fill[j] = trowptr[j];
    for (int64_t i = 0; i < nrows; ++i)
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int32_t q = fill[col[p]]++;
            tcol[q] = (int32_t)i; tval[q] = val[p];
        }
    free(fill);
    return OR_OK;
}

/* ===========================================================================================
 * Sparse product C = A B (Galerkin operator, Sec. 4.2 eq. (galerkin), used as T = L P then
 * L_H = R T). Row i of C: for each entry (l, a_il) of row i of A in ascending l, for each entry
 * (j, b_lj) of row l of B: acc_j <- fma(a_il, b_lj, acc_j), acc starting at 0. Structural union,
 * no dropping, columns ascending. Two calls: with c_col == NULL only the row counts are
 * produced (c_rowptr), then the values.
 * =========================================================================================== */
int or_spgemm(int64_t nA, int64_t ncolsB, const int32_t* ap, const int32_t* ac, const double* av,
              const int32_t* bp, const int32_t* bc, const double* bv,
              int32_t* cp, int32_t* cc, double* cv) {
    double* acc = (double*)calloc(ncolsB > 0 ? ncolsB : 1, sizeof(double));
    int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (ncolsB > 0 ? ncolsB : 1));
    int32_t* cols = (int32_t*)malloc(sizeof(int32_t) * (ncolsB > 0 ? ncolsB : 1));
    if (!acc || !mark || !cols) { free(acc); free(mark); free(cols); return OR_ERR_NOMEM; }
    for (int64_t j = 0; j < ncolsB; ++j) mark[j] = -1;
    int64_t total = 0;
    if (cc == NULL) cp[0] = 0;
    for (int64_t i = 0; i < nA; ++i) {
        int64_t nc = 0;
        for (int32_t p = ap[i]; p < ap[i + 1]; ++p) {
            int32_t l = ac[p];
            for (int32_t q = bp[l]; q < bp[l + 1]; ++q) {
                int32_t j = bc[q];
                if (mark[j] != (int32_t)i) { mark[j] = (int32_t)i; acc[j] = 0.0; cols[nc++] = j; }
                if (cc) acc[j] = fma(av[p], bv[q], acc[j]);
            }
        }
        if (cc == NULL) {
            total += nc;
            if (total > INT32_MAX) { free(acc); free(mark); free(cols); return OR_ERR_ARG; }
            cp[i + 1] = (int32_t)total;
        } else {
            for (int64_t a = 1; a < nc; ++a) {
                int32_t v = cols[a]; int64_t b = a;
                while (b > 0 && cols[b - 1] > v) { cols[b] = cols[b - 1]; --b; }
                cols[b] = v;
            }
            if (cp[i + 1] - cp[i] != nc) { free(acc); free(mark); free(cols); return OR_ERR_ARG; }
            for (int64_t a = 0; a < nc; ++a) { cc[cp[i] + a] = cols[a]; cv[cp[i] + a] = acc[cols[a]]; }
        }
    }
    free(acc); free(mark); free(cols);
    return OR_OK;
}

/* ===========================================================================================
 * Dense LU with partial pivoting of the coarsest operator (Sec. 4.3; Alg. 2) and the
 * corresponding solve. a (n x n row-major) is overwritten by L\U, piv[k] = row swapped with k.
 * =========================================================================================== */
int or_lu_factor(double* a, int64_t n, int32_t* piv) {
    for (int64_t k = 0; k < n; ++k) {
        int64_t p = k; double best = fabs(a[k * n + k]);
        for (int64_t i = k + 1; i < n; ++i) { double v = fabs(a[i * n + k]); if (v > best) { best = v; p = i; } }
        if (!(best > 0.0)) return OR_ERR_SINGULAR;
        piv[k] = (int32_t)p;
        if (p != k) for (int64_t j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
        for (int64_t i = k + 1; i < n; ++i) {
            double l = a[i * n + k] / a[k * n + k];
            a[i * n + k] = l;
            for (int64_t j = k + 1; j < n; ++j) a[i * n + j] = fma(-l, a[k * n + j], a[i * n + j]);
        }
    }
    return OR_OK;
}
void or_lu_solve(const double* lu, int64_t n, const int32_t* piv, double* b) {
    for (int64_t k = 0; k < n; ++k) if (piv[k] != k) { double t = b[k]; b[k] = b[piv[k]]; b[piv[k]] = t; }
    for (int64_t i = 0; i < n; ++i) { double s = b[i]; for (int64_t j = 0; j < i; ++j) s = fma(-lu[i * n + j], b[j], s); b[i] = s; }
    for (int64_t i = n - 1; i >= 0; --i) { double s = b[i]; for (int64_t j = i + 1; j < n; ++j) s = fma(-lu[i * n + j], b[j], s); b[i] = s / lu[i * n + i]; }
}

/* ===========================================================================================
 * Gauss-Seidel smoothing (Sec. 4.3, eq. (smoother)): u <- u + B^{-1}(f - L u), B the lower
 * triangle of L in the sweep order, i.e. u_i <- (f_i - sum_{j != i} l_ij u_j) / l_ii row by row
 * with the newest values. Sweep order: rows 0..N-1 (lexicographic, the paper's forward GS) or,
 * when a colouring is given, colour 0, 1, ... with the rows of one colour in ascending order
 * (multicolour GS: rows of one colour do not touch each other, so their order is immaterial).
 * =========================================================================================== */
typedef struct {
    int64_t n;
    const int32_t *rp, *ci; const double* v;                    /* L_j (CSR) */
    const int32_t *cptr, *crows; int32_t ncol;                   /* colour classes, NULL -> lexicographic */
    const int32_t *pp, *pc; const double* pv;                    /* I_{j+1}^j (n x n_{j+1}), NULL on the coarsest */
    const int32_t *rrp, *rc; const double* rv;                   /* I_j^{j+1} = (I_{j+1}^j)^T */
} or_level;

static void gs_row(const or_level* L, int64_t i, const double* f, double* u) {
    double s = f[i], d = 0.0;
    for (int32_t p = L->rp[i]; p < L->rp[i + 1]; ++p) {
        int32_t j = L->ci[p];
        if (j == i) d = L->v[p];
        else s = s - L->v[p] * u[j];
    }
    u[i] = s / d;
}
void or_gs_sweep(const or_level* L, const double* f, double* u) {
    if (L->cptr) {
        for (int32_t c = 0; c < L->ncol; ++c)
            for (int32_t t = L->cptr[c]; t < L->cptr[c + 1]; ++t) gs_row(L, L->crows[t], f, u);
    } else {
        for (int64_t i = 0; i < L->n; ++i) gs_row(L, i, f, u);
    }
}
/* y = b - A x */
static void residual(const or_level* L, const double* b, const double* x, double* y) {
    for (int64_t i = 0; i < L->n; ++i) {
        double s = 0.0;
        for (int32_t p = L->rp[i]; p < L->rp[i + 1]; ++p) s = s + L->v[p] * x[L->ci[p]];
        y[i] = b[i] - s;
    }
}
static void csr_apply(int64_t n, const int32_t* rp, const int32_t* ci, const double* v, const double* x, double* y) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) s = s + v[p] * x[ci[p]];
        y[i] = s;
    }
}

/* ===========================================================================================
 * MGM V(nu1, nu2)-cycle (Sec. 4.5, Alg. 3), one application on u1 (in/out) for right-hand side
 * f1, both in the caller's ordering; perm1[new] = old is the RCM ordering of level 1 (NULL for
 * identity). Levels 2..p-1 start from a zero defect; the coarsest level is solved with the LU
 * factors of L_p.
 * =========================================================================================== */
int or_vcycle(const or_level* lv, int p, const double* lu, const int32_t* piv, const int32_t* perm1,
              int nu1, int nu2, const double* fin, double* uio) {
    if (p < 2) return OR_ERR_ARG;
    int64_t n1 = lv[0].n;
    double** e = (double**)calloc(p, sizeof(double*));
    double** r = (double**)calloc(p, sizeof(double*));
    double* tmp = (double*)malloc(sizeof(double) * n1);
    for (int j = 0; j < p; ++j) { e[j] = (double*)calloc(lv[j].n, sizeof(double)); r[j] = (double*)calloc(lv[j].n, sizeof(double)); }
    /* reorder f and u by the RCM ordering of L_1 */
    for (int64_t i = 0; i < n1; ++i) { int64_t o = perm1 ? perm1[i] : i; r[0][i] = fin[o]; e[0][i] = uio[o]; }
    /* presmooth the initial guess; r^2 = I_1^2 (f^1 - L_1 u^1) */
    for (int s = 0; s < nu1; ++s) or_gs_sweep(&lv[0], r[0], e[0]);
    residual(&lv[0], r[0], e[0], tmp);
    csr_apply(lv[1].n, lv[0].rrp, lv[0].rc, lv[0].rv, tmp, r[1]);
    /* levels 2 .. p-1: presmooth the defect from zero, compute and restrict its residual */
    for (int j = 1; j < p - 1; ++j) {
        for (int64_t i = 0; i < lv[j].n; ++i) e[j][i] = 0.0;
        for (int s = 0; s < nu1; ++s) or_gs_sweep(&lv[j], r[j], e[j]);
        residual(&lv[j], r[j], e[j], tmp);
        csr_apply(lv[j + 1].n, lv[j].rrp, lv[j].rc, lv[j].rv, tmp, r[j + 1]);
    }
    /* coarsest defect by the LU factors of L_p */
    for (int64_t i = 0; i < lv[p - 1].n; ++i) e[p - 1][i] = r[p - 1][i];
    or_lu_solve(lu, lv[p - 1].n, piv, e[p - 1]);
    /* interpolate / correct and post-smooth on levels p-1 .. 2, then on level 1 */
    for (int j = p - 2; j >= 0; --j) {
        csr_apply(lv[j].n, lv[j].pp, lv[j].pc, lv[j].pv, e[j + 1], tmp);
        for (int64_t i = 0; i < lv[j].n; ++i) e[j][i] = e[j][i] + tmp[i];
        for (int s = 0; s < nu2; ++s) or_gs_sweep(&lv[j], r[j], e[j]);
    }
    /* undo the RCM reordering */
    for (int64_t i = 0; i < n1; ++i) { int64_t o = perm1 ? perm1[i] : i; uio[o] = e[0][i]; }
    for (int j = 0; j < p; ++j) { free(e[j]); free(r[j]); }
    free(e); free(r); free(tmp);
    return OR_OK;
}

/* ===========================================================================================
 * Multigrid cycles in recursive form (Sec. 4.5 names V, W and F cycles; Alg. 3 is the V-cycle).
 * Level j with right-hand side f_j and iterate e_j: nu1 GS sweeps, f_{j+1} = R_j (f_j - L_j e_j),
 * e_{j+1} = 0, then the coarse visits -- V: one V-cycle; W: two W-cycles, the second from the
 * first's result; F: one F-cycle, then one V-cycle from its result -- then e_j += P_j e_{j+1} and
 * nu2 sweeps. The coarsest level is solved by the LU factors. type: 0 V, 1 W, 2 F. With a zero
 * initial guess the V form performs the operations of or_vcycle in the same order.
 * =========================================================================================== */
typedef struct {
    const or_level* lv;
    int p, nu1, nu2;
    const double* lu;
    const int32_t* piv;
    double **f, **e, **tmp;
} mg_ctx;

static void mg_rec(const mg_ctx* c, int j, int type, int zero_start) {
    const or_level* L = &c->lv[j];
    if (j == c->p - 1) {
        for (int64_t i = 0; i < L->n; ++i) c->e[j][i] = c->f[j][i];
        or_lu_solve(c->lu, L->n, c->piv, c->e[j]);
        return;
    }
    if (zero_start)
        for (int64_t i = 0; i < L->n; ++i) c->e[j][i] = 0.0;
    for (int s = 0; s < c->nu1; ++s) or_gs_sweep(L, c->f[j], c->e[j]);
    residual(L, c->f[j], c->e[j], c->tmp[j]);
    csr_apply(c->lv[j + 1].n, L->rrp, L->rc, L->rv, c->tmp[j], c->f[j + 1]);
    if (type == 0) {
        mg_rec(c, j + 1, 0, 1);
    } else if (type == 1) {
        mg_rec(c, j + 1, 1, 1);
        mg_rec(c, j + 1, 1, 0);
    } else {
        mg_rec(c, j + 1, 2, 1);
        mg_rec(c, j + 1, 0, 0);
    }
    csr_apply(L->n, L->pp, L->pc, L->pv, c->e[j + 1], c->tmp[j]);
    for (int64_t i = 0; i < L->n; ++i) c->e[j][i] = c->e[j][i] + c->tmp[j][i];
    for (int s = 0; s < c->nu2; ++s) or_gs_sweep(L, c->f[j], c->e[j]);
}

int or_mgcycle(const or_level* lv, int p, const double* lu, const int32_t* piv, const int32_t* perm1, int nu1, int nu2,
               int type, const double* fin, double* uio) {
    if (p < 2 || type < 0 || type > 2) return OR_ERR_ARG;
    const int64_t n1 = lv[0].n;
    mg_ctx c = {lv, p, nu1, nu2, lu, piv, NULL, NULL, NULL};
    c.f = (double**)calloc(p, sizeof(double*));
    c.e = (double**)calloc(p, sizeof(double*));
    c.tmp = (double**)calloc(p, sizeof(double*));
    for (int j = 0; j < p; ++j) {
        c.f[j] = (double*)calloc(lv[j].n, sizeof(double));
        c.e[j] = (double*)calloc(lv[j].n, sizeof(double));
        c.tmp[j] = (double*)calloc(lv[j].n, sizeof(double));
    }
    for (int64_t i = 0; i < n1; ++i) { int64_t o = perm1 ? perm1[i] : i; c.f[0][i] = fin[o]; c.e[0][i] = uio[o]; }
    mg_rec(&c, 0, type, 0);
    for (int64_t i = 0; i < n1; ++i) { int64_t o = perm1 ? perm1[i] : i; uio[o] = c.e[0][i]; }
    for (int j = 0; j < p; ++j) { free(c.f[j]); free(c.e[j]); free(c.tmp[j]); }
    free(c.f); free(c.e); free(c.tmp);
    return OR_OK;
}

static double nrm2(int64_t n, const double* x) { double s = 0.0; for (int64_t i = 0; i < n; ++i) s = s + x[i] * x[i]; return sqrt(s); }
static double dot(int64_t n, const double* a, const double* b) { double s = 0.0; for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i]; return s; }

/* ===========================================================================================
 * Right-preconditioned flexible GMRES(restart) with modified Gram-Schmidt (Sec. 4.6; Sec. 5:
 * "MGM ... as a right preconditioner"): one V-cycle from a zero guess per iteration, z_k = M v_k,
 * x = x_0 + Z y. Stops when the true relative residual |f - L x| / |f| <= tol (checked at every
 * restart and when the recurrence estimate reaches tol) or after maxit iterations.
 * The operator is the level-1 CSR in the caller's ordering (A_*); precond = 0 runs plain GMRES.
 * hist (length maxit + 1, may be NULL) receives the estimated relative residual per iteration.
 * =========================================================================================== */
typedef void (*or_apply_fn)(void* ctx, const double* x, double* y);
typedef void (*or_precond_fn)(void* ctx, const double* v, double* z);

/* FGMRES body shared by the plain and the bordered systems (precond NULL: z = v) */
static int fgmres_core(int64_t n, or_apply_fn apply, void* actx, or_precond_fn precond, void* pctx,
                       const double* f, double* x, int restart, int maxit, double tol,
                       int* iters_out, double* relres_out, double* hist) {
    if (restart < 1) return OR_ERR_ARG;
    int m = restart;
    double* V = (double*)malloc(sizeof(double) * n * (m + 1));
    double* Z = (double*)malloc(sizeof(double) * n * m);
    double* H = (double*)calloc((m + 1) * m, sizeof(double));
    double *cs = (double*)malloc(sizeof(double) * m), *sn = (double*)malloc(sizeof(double) * m);
    double* g = (double*)malloc(sizeof(double) * (m + 1));
    double* w = (double*)malloc(sizeof(double) * n);
    double* y = (double*)malloc(sizeof(double) * m);
    if (!V || !Z || !H || !cs || !sn || !g || !w || !y) return OR_ERR_NOMEM;
    double fn = nrm2(n, f);
    if (fn == 0.0) fn = 1.0;
    int it = 0, status = OR_ERR_NOTCONV;
    double rel = 0.0;
    for (;;) {
        apply(actx, x, w);
        for (int64_t i = 0; i < n; ++i) V[i] = f[i] - w[i];
        double beta = nrm2(n, V);
        rel = beta / fn;
        if (hist && it == 0) hist[0] = rel;
        if (rel <= tol) { status = OR_OK; break; }
        if (it >= maxit) break;
        for (int64_t i = 0; i < n; ++i) V[i] = V[i] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int k = 0;
        for (; k < m && it < maxit; ++k) {
            double* vk = V + (int64_t)k * n;
            double* zk = Z + (int64_t)k * n;
            if (precond) precond(pctx, vk, zk);
            else for (int64_t i = 0; i < n; ++i) zk[i] = vk[i];
            apply(actx, zk, w);
            for (int i = 0; i <= k; ++i) {
                double* vi = V + (int64_t)i * n;
                double h = 0.0;
                for (int64_t t = 0; t < n; ++t) h = h + w[t] * vi[t];
                H[i * m + k] = h;
                for (int64_t t = 0; t < n; ++t) w[t] = w[t] - h * vi[t];
            }
            double hn = nrm2(n, w);
            H[(k + 1) * m + k] = hn;
            if (hn != 0.0) for (int64_t t = 0; t < n; ++t) V[(int64_t)(k + 1) * n + t] = w[t] / hn;
            for (int i = 0; i < k; ++i) {
                double a = H[i * m + k], b = H[(i + 1) * m + k];
                H[i * m + k] = cs[i] * a + sn[i] * b;
                H[(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
            }
            double a = H[k * m + k], b = H[(k + 1) * m + k];
            double rr = sqrt(a * a + b * b);
            cs[k] = rr == 0.0 ? 1.0 : a / rr; sn[k] = rr == 0.0 ? 0.0 : b / rr;
            H[k * m + k] = rr; H[(k + 1) * m + k] = 0.0;
            g[k + 1] = -sn[k] * g[k]; g[k] = cs[k] * g[k];
            ++it;
            double est = fabs(g[k + 1]) / fn;
            if (hist) hist[it] = est;
            if (est <= tol || hn == 0.0) { ++k; break; }
        }
        /* x <- x + Z y, H(0:k,0:k) y = g(0:k) (upper triangular) */
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int j = i + 1; j < k; ++j) s = s - H[i * m + j] * y[j];
            y[i] = s / H[i * m + i];
        }
        for (int j = 0; j < k; ++j)
            for (int64_t t = 0; t < n; ++t) x[t] = x[t] + y[j] * Z[(int64_t)j * n + t];
    }
    *iters_out = it; *relres_out = rel;
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(w); free(y);
    return status;
}

typedef struct { int64_t n; const int32_t *rp, *ci; const double* v; } or_csr_ctx;
static void csr_apply_cb(void* c, const double* x, double* y) {
    const or_csr_ctx* a = (const or_csr_ctx*)c;
    csr_apply(a->n, a->rp, a->ci, a->v, x, y);
}
typedef struct { const or_level* lv; int p; const double* lu; const int32_t* piv; const int32_t* perm1; int nu1, nu2; int64_t n; int type; } or_mgm_ctx;
static void vcycle_cb(void* c, const double* v, double* z) {
    const or_mgm_ctx* m = (const or_mgm_ctx*)c;
    for (int64_t i = 0; i < m->n; ++i) z[i] = 0.0;
    if (m->type == 0) or_vcycle(m->lv, m->p, m->lu, m->piv, m->perm1, m->nu1, m->nu2, v, z);
    else or_mgcycle(m->lv, m->p, m->lu, m->piv, m->perm1, m->nu1, m->nu2, m->type, v, z);
}

int or_fgmres(int64_t n, const int32_t* arp, const int32_t* aci, const double* av,
              const or_level* lv, int p, const double* lu, const int32_t* piv, const int32_t* perm1, int nu1, int nu2,
              int precond, const double* f, double* x, int restart, int maxit, double tol,
              int* iters_out, double* relres_out, double* hist) {
    or_csr_ctx a = {n, arp, aci, av};
    or_mgm_ctx m = {lv, p, lu, piv, perm1, nu1, nu2, n, 0};
    return fgmres_core(n, csr_apply_cb, &a, precond ? vcycle_cb : NULL, &m, f, x, restart, maxit, tol, iters_out, relres_out,
                       hist);
}

/* or_fgmres with one multigrid cycle of type `cycle` (0 V, 1 W, 2 F; or_mgcycle) per iteration */
int or_fgmres_cycle(int64_t n, const int32_t* arp, const int32_t* aci, const double* av,
                    const or_level* lv, int p, const double* lu, const int32_t* piv, const int32_t* perm1, int nu1,
                    int nu2, int cycle, const double* f, double* x, int restart, int maxit, double tol,
                    int* iters_out, double* relres_out, double* hist) {
    if (cycle < 0 || cycle > 2) return OR_ERR_ARG;
    or_csr_ctx a = {n, arp, aci, av};
    or_mgm_ctx m = {lv, p, lu, piv, perm1, nu1, nu2, n, cycle};
    return fgmres_core(n, csr_apply_cb, &a, vcycle_cb, &m, f, x, restart, maxit, tol, iters_out, relres_out, hist);
}

/* ===========================================================================================
 * Surface Poisson problem (L_h = D_h, singular) with the mean-zero constraint of Sec. 4.4:
 * the bordered system of eq. (saddle_point), [L b^T; b 0][u; lambda] = [f; 0], b = (1, ..., 1).
 * Coarse operators follow eq. (gco_saddle_point): the restriction and interpolation carry lambda
 * unchanged, so on level j the border column is c_j = R_{j-1} c_{j-1} and the border row is
 * b P_0 ... P_{j-1}, which is the same vector (R = P^T), with c_0 = b^T. Smoothing updates u only,
 * u <- u + B^{-1}(r - L u - c lambda) (the smoother of Sec. 4.4), and the coarsest bordered system
 * is solved directly with the LU factors of [L_p c_p; c_p^T 0].
 * One bordered V-cycle from a zero guess: (r, s) -> (e, mu), with r in the caller's ordering and
 * s the constraint component; cvec[j] holds c_j in level j's (RCM) ordering.
 * =========================================================================================== */
int or_vcycle_bordered(const or_level* lv, int p, const double* const* cvec, const double* blu, const int32_t* bpiv,
                       const int32_t* perm1, int nu1, int nu2, const double* rin, double sin, double* eout,
                       double* muout) {
    if (p < 2) return OR_ERR_ARG;
    int64_t n1 = lv[0].n;
    double** e = (double**)calloc(p, sizeof(double*));
    double** r = (double**)calloc(p, sizeof(double*));
    double* sres = (double*)calloc(p, sizeof(double));
    double* tmp = (double*)malloc(sizeof(double) * n1);
    double* tmp2 = (double*)malloc(sizeof(double) * n1);
    for (int j = 0; j < p; ++j) { e[j] = (double*)calloc(lv[j].n + 1, sizeof(double)); r[j] = (double*)calloc(lv[j].n + 1, sizeof(double)); }
    for (int64_t i = 0; i < n1; ++i) { int64_t o = perm1 ? perm1[i] : i; r[0][i] = rin[o]; }
    sres[0] = sin;
    /* descent: mu_j = 0, so pre-smoothing sees r_j; residual r_j - L_j e_j; constraint s_j - c_j . e_j */
    for (int j = 0; j < p - 1; ++j) {
        for (int64_t i = 0; i < lv[j].n; ++i) e[j][i] = 0.0;
        for (int t = 0; t < nu1; ++t) or_gs_sweep(&lv[j], r[j], e[j]);
        residual(&lv[j], r[j], e[j], tmp);
        csr_apply(lv[j + 1].n, lv[j].rrp, lv[j].rc, lv[j].rv, tmp, r[j + 1]);
        sres[j + 1] = sres[j] - dot(lv[j].n, cvec[j], e[j]);
    }
    /* coarsest bordered solve: [e_p; mu] */
    const int64_t np = lv[p - 1].n;
    for (int64_t i = 0; i < np; ++i) e[p - 1][i] = r[p - 1][i];
    e[p - 1][np] = sres[p - 1];
    or_lu_solve(blu, np + 1, bpiv, e[p - 1]);
    const double mu = e[p - 1][np];
    /* ascent: e_j += P_j e_{j+1}; mu passes unchanged; post-smoothing on r_j - c_j mu */
    for (int j = p - 2; j >= 0; --j) {
        csr_apply(lv[j].n, lv[j].pp, lv[j].pc, lv[j].pv, e[j + 1], tmp);
        for (int64_t i = 0; i < lv[j].n; ++i) e[j][i] = e[j][i] + tmp[i];
        for (int64_t i = 0; i < lv[j].n; ++i) tmp2[i] = r[j][i] - cvec[j][i] * mu;
        for (int t = 0; t < nu2; ++t) or_gs_sweep(&lv[j], tmp2, e[j]);
    }
    for (int64_t i = 0; i < n1; ++i) { int64_t o = perm1 ? perm1[i] : i; eout[o] = e[0][i]; }
    *muout = mu;
    for (int j = 0; j < p; ++j) { free(e[j]); free(r[j]); }
    free(e); free(r); free(sres); free(tmp); free(tmp2);
    return OR_OK;
}

typedef struct { int64_t n; const int32_t *rp, *ci; const double* v; } or_bord_ctx;
/* y = [L u + lambda 1; 1 . u] on an (n+1)-vector */
static void bordered_apply_cb(void* c, const double* x, double* y) {
    const or_bord_ctx* a = (const or_bord_ctx*)c;
    csr_apply(a->n, a->rp, a->ci, a->v, x, y);
    double sum = 0.0;
    for (int64_t i = 0; i < a->n; ++i) { y[i] = y[i] + x[a->n]; sum = sum + x[i]; }
    y[a->n] = sum;
}
typedef struct { const or_level* lv; int p; const double* const* cvec; const double* blu; const int32_t* bpiv;
                 const int32_t* perm1; int nu1, nu2; int64_t n; } or_bmgm_ctx;
static void bordered_vcycle_cb(void* c, const double* v, double* z) {
    const or_bmgm_ctx* m = (const or_bmgm_ctx*)c;
    or_vcycle_bordered(m->lv, m->p, m->cvec, m->blu, m->bpiv, m->perm1, m->nu1, m->nu2, v, v[m->n], z, z + m->n);
}

/* FGMRES (as or_fgmres) on the bordered system of size n + 1: f and x have n + 1 entries (the
 * last is the constraint right-hand side / the multiplier lambda). */
int or_fgmres_bordered(int64_t n, const int32_t* arp, const int32_t* aci, const double* av, const or_level* lv, int p,
                       const double* const* cvec, const double* blu, const int32_t* bpiv, const int32_t* perm1, int nu1,
                       int nu2, int precond, const double* f, double* x, int restart, int maxit, double tol,
                       int* iters_out, double* relres_out, double* hist) {
    or_bord_ctx a = {n, arp, aci, av};
    or_bmgm_ctx m = {lv, p, cvec, blu, bpiv, perm1, nu1, nu2, n};
    return fgmres_core(n + 1, bordered_apply_cb, &a, precond ? bordered_vcycle_cb : NULL, &m, f, x, restart, maxit, tol,
                       iters_out, relres_out, hist);
}

/* Right-preconditioned BiCGSTAB (Sec. 4.6; the method of van der Vorst as given in Saad's book)
 * with one MGM V-cycle from a zero guess per preconditioner application, in FP64. Each step
 * applies the preconditioner twice; iters_out counts applications, the convention of Sec. 5.2.
 * Per step: rho = rh.r; beta = (rho/rho_old)(alpha/omega); p = r + beta (p - omega v);
 * ph = M p; v = L ph; alpha = rho / rh.v; s = r - alpha v (stop here when |s|/|f| <= tol, with
 * x += alpha ph); sh = M s; t = L sh; omega = t.s / t.t; x += alpha ph + omega sh;
 * r = s - omega t. rh = r_0. Stops on the recurred residual; relres_out is the true residual
 * |f - L x|/|f| at exit. Breakdown (rho = 0 or t.t = 0) returns OR_ERR_NOTCONV. */
int or_bicgstab(int64_t n, const int32_t* arp, const int32_t* aci, const double* av,
                const or_level* lv, int p, const double* lu, const int32_t* piv, const int32_t* perm1, int nu1, int nu2,
                int precond, const double* f, double* x, int maxit, double tol,
                int* iters_out, double* relres_out, double* hist) {
    double* r = (double*)malloc(sizeof(double) * n);
    double* rh = (double*)malloc(sizeof(double) * n);
    double* pv = (double*)calloc(n, sizeof(double));
    double* v = (double*)calloc(n, sizeof(double));
    double* ph = (double*)malloc(sizeof(double) * n);
    double* sv = (double*)malloc(sizeof(double) * n);
    double* sh = (double*)malloc(sizeof(double) * n);
    double* t = (double*)malloc(sizeof(double) * n);
    if (!r || !rh || !pv || !v || !ph || !sv || !sh || !t) return OR_ERR_NOMEM;
    double fn = nrm2(n, f);
    if (fn == 0.0) fn = 1.0;
    csr_apply(n, arp, aci, av, x, t);
    for (int64_t i = 0; i < n; ++i) { r[i] = f[i] - t[i]; rh[i] = r[i]; }
    double rel = nrm2(n, r) / fn;
    if (hist) hist[0] = rel;
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    int apps = 0, status = rel <= tol ? OR_OK : OR_ERR_NOTCONV;
    while (status != OR_OK && apps + 1 <= maxit) {
        double rho = dot(n, rh, r);
        if (rho == 0.0) break;
        double beta = (rho / rho_old) * (alpha / omega);
        for (int64_t i = 0; i < n; ++i) pv[i] = r[i] + beta * (pv[i] - omega * v[i]);
        if (precond) { for (int64_t i = 0; i < n; ++i) ph[i] = 0.0; or_vcycle(lv, p, lu, piv, perm1, nu1, nu2, pv, ph); }
        else for (int64_t i = 0; i < n; ++i) ph[i] = pv[i];
        ++apps;
        csr_apply(n, arp, aci, av, ph, v);
        alpha = rho / dot(n, rh, v);
        for (int64_t i = 0; i < n; ++i) sv[i] = r[i] - alpha * v[i];
        rel = nrm2(n, sv) / fn;
        if (hist) hist[apps] = rel;
        if (rel <= tol) {
            for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * ph[i];
            status = OR_OK;
            break;
        }
        if (apps + 1 > maxit) { for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * ph[i]; break; }
        if (precond) { for (int64_t i = 0; i < n; ++i) sh[i] = 0.0; or_vcycle(lv, p, lu, piv, perm1, nu1, nu2, sv, sh); }
        else for (int64_t i = 0; i < n; ++i) sh[i] = sv[i];
        ++apps;
        csr_apply(n, arp, aci, av, sh, t);
        double tt = dot(n, t, t);
        if (tt == 0.0) { for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * ph[i]; break; }
        omega = dot(n, t, sv) / tt;
        for (int64_t i = 0; i < n; ++i) { x[i] = x[i] + alpha * ph[i] + omega * sh[i]; r[i] = sv[i] - omega * t[i]; }
        rel = nrm2(n, r) / fn;
        if (hist) hist[apps] = rel;
        if (rel <= tol) status = OR_OK;
        rho_old = rho;
    }
    csr_apply(n, arp, aci, av, x, t);
    for (int64_t i = 0; i < n; ++i) t[i] = f[i] - t[i];
    *relres_out = nrm2(n, t) / fn;
    *iters_out = apps;
    free(r); free(rh); free(pv); free(v); free(ph); free(sv); free(sh); free(t);
    return status;
}

/* MGM as a standalone solver (Sec. 5.1): repeated V-cycles on x until |f - Lx|/|f| <= tol. */
int or_mgm_solve(int64_t n, const int32_t* arp, const int32_t* aci, const double* av,
                 const or_level* lv, int p, const double* lu, const int32_t* piv, const int32_t* perm1, int nu1, int nu2,
                 const double* f, double* x, int maxit, double tol, int* iters_out, double* relres_out) {
    double* w = (double*)malloc(sizeof(double) * n);
    double fn = nrm2(n, f);
    if (fn == 0.0) fn = 1.0;
    int it = 0;
    double rel = 0.0;
    for (;;) {
        csr_apply(n, arp, aci, av, x, w);
        for (int64_t i = 0; i < n; ++i) w[i] = f[i] - w[i];
        rel = nrm2(n, w) / fn;
        if (rel <= tol || it >= maxit) break;
        or_vcycle(lv, p, lu, piv, perm1, nu1, nu2, f, x);
        ++it;
    }
    free(w);
    *iters_out = it; *relres_out = rel;
    return rel <= tol ? OR_OK : OR_ERR_NOTCONV;
}

/* ===========================================================================================
 * Learned smoother (not in the paper; an addition of this project's scope, judged by this
 * oracle). Per point i of the finest level, with stencil idx[i][0..n) (centre first):
 *   features f[4j..4j+3] = ( xh_j / s, yh_j / s, c_ij s^2, r_{idx_ij} / rho_i ),  j < n,
 * with (xh, yh) the tangent-plane offsets of Sec. 2.1, s the stencil support, c_ij the LBO
 * weights, r the residual and rho_i = sqrt(mean_j r_{idx_ij}^2) (features 0 when rho_i = 0);
 * network out = w3 . relu(W2 relu(W1 f)) (no biases, 4n -> 64 -> 64 -> 1); correction
 * delta_i = rho_i * out_i / l_ii. Row-major weights: W1 [64][4n], W2 [64][64], w3 [64].
 * Training objective (composed in the Python wrapper from or_mlp_vjp and library SpMVs): the
 * relative residual left by the correction, J = |r - L delta|^2 / |r|^2.
 * =========================================================================================== */
int or_mlp_features(int64_t N, int n, const int32_t* idx, const double* xyz, const double* nrm, const double* w,
                    const double* r, double* feat, double* rho) {
    if (n < 1 || n > MAXM) return OR_ERR_ARG;
    double xh[MAXM], yh[MAXM];
    for (int64_t i = 0; i < N; ++i) {
        const int32_t* id = idx + i * n;
        double s = project_stencil(xyz, nrm, i, id, n, xh, yh);
        double ss = 0.0;
        for (int j = 0; j < n; ++j) ss = ss + r[id[j]] * r[id[j]];
        double rh = sqrt(ss / (double)n);
        rho[i] = rh;
        double* f = feat + i * 4 * n;
        for (int j = 0; j < n; ++j) {
            f[4 * j + 0] = s > 0.0 ? xh[j] / s : 0.0;
            f[4 * j + 1] = s > 0.0 ? yh[j] / s : 0.0;
            f[4 * j + 2] = w[i * n + j] * (s * s);
            f[4 * j + 3] = rh > 0.0 ? r[id[j]] / rh : 0.0;
        }
    }
    return OR_OK;
}

/* forward: out[i]; h1, h2 (N x 64 each, may be NULL) keep the post-ReLU activations */
int or_mlp_forward(int64_t N, int din, const double* W1, const double* W2, const double* w3, const double* feat,
                   double* out, double* h1o, double* h2o) {
    double h1[64], h2[64];
    for (int64_t i = 0; i < N; ++i) {
        const double* f = feat + i * din;
        for (int a = 0; a < 64; ++a) {
            double acc = 0.0;
            for (int k = 0; k < din; ++k) acc = acc + W1[a * din + k] * f[k];
            h1[a] = acc > 0.0 ? acc : 0.0;
        }
        for (int a = 0; a < 64; ++a) {
            double acc = 0.0;
            for (int k = 0; k < 64; ++k) acc = acc + W2[a * 64 + k] * h1[k];
            h2[a] = acc > 0.0 ? acc : 0.0;
        }
        double o = 0.0;
        for (int k = 0; k < 64; ++k) o = o + w3[k] * h2[k];
        out[i] = o;
        if (h1o) for (int a = 0; a < 64; ++a) h1o[i * 64 + a] = h1[a];
        if (h2o) for (int a = 0; a < 64; ++a) h2o[i * 64 + a] = h2[a];
    }
    return OR_OK;
}

/* vector-Jacobian product: gradients of sum_i gout_i * out_i with respect to W1, W2, w3
 * (overwritten). Any loss built on the outputs reduces to this with gout = d loss / d out. */
int or_mlp_vjp(int64_t N, int din, const double* W1, const double* W2, const double* w3, const double* feat,
               const double* gout, double* gW1, double* gW2, double* gw3) {
    double h1[64], z1[64], z2[64], d2[64], d1[64];
    for (int k = 0; k < 64 * din; ++k) gW1[k] = 0.0;
    for (int k = 0; k < 64 * 64; ++k) gW2[k] = 0.0;
    for (int k = 0; k < 64; ++k) gw3[k] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        const double* f = feat + i * din;
        for (int a = 0; a < 64; ++a) {
            double acc = 0.0;
            for (int k = 0; k < din; ++k) acc = acc + W1[a * din + k] * f[k];
            z1[a] = acc; h1[a] = acc > 0.0 ? acc : 0.0;
        }
        for (int a = 0; a < 64; ++a) {
            double acc = 0.0;
            for (int k = 0; k < 64; ++k) acc = acc + W2[a * 64 + k] * h1[k];
            z2[a] = acc;
        }
        const double g = gout[i];
        /* out = w3 . relu(z2): d out / d w3 = relu(z2); d out / d z2 = w3 where z2 > 0 */
        for (int k = 0; k < 64; ++k) {
            gw3[k] = gw3[k] + g * (z2[k] > 0.0 ? z2[k] : 0.0);
            d2[k] = (z2[k] > 0.0) ? g * w3[k] : 0.0;
        }
        for (int a = 0; a < 64; ++a) for (int k = 0; k < 64; ++k) gW2[a * 64 + k] = gW2[a * 64 + k] + d2[a] * h1[k];
        for (int k = 0; k < 64; ++k) {
            double acc = 0.0;
            for (int a = 0; a < 64; ++a) acc = acc + W2[a * 64 + k] * d2[a];
            d1[k] = (z1[k] > 0.0) ? acc : 0.0;
        }
        for (int a = 0; a < 64; ++a) for (int k = 0; k < din; ++k) gW1[a * din + k] = gW1[a * din + k] + d1[a] * f[k];
    }
    return OR_OK;
}

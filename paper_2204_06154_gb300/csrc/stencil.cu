// Tangent-plane stencil weights for the Laplace-Beltrami operator (paper Sec. 2) and global
// assembly of L = I - mu D (Sec. 2, eq. (discrete_system)).
//
// PHS RBF-FD (Sec. 2.2, eq. (rbf_fd_lap)): one warp per stencil. The (n+L) x (n+L+1) augmented
// saddle matrix lives in shared memory; Gaussian elimination with partial pivoting runs with the
// warp's lanes spread over the trailing submatrix; every entry receives the same sequence of IEEE
// operations (fused multiply-adds where the update is a_ij - l_i a_kj) as a sequential
// elimination, so the weights do not depend on the parallel schedule. The work is FP64-pipe bound
// (GB300: ~0.6 TFMA/s FP64), so shared-memory staging per warp, not occupancy, is what matters.
//
// GFD (Sec. 2.3, eq. (wls_fd_lap)): one thread per stencil, Householder QR of W^{1/2} P.
// This file is compiled with --fmad=false: no multiply-add is contracted unless written as fma().
#include <climits>

#include "common.cuh"

#include "geom.cuh"

namespace mgm {

constexpr int MAX_M = 128;

__device__ __forceinline__ double monomial(double x, double y, int a, int b) {
    double p = 1.0;
    for (int t = 0; t < a; ++t) p = p * x;
    for (int t = 0; t < b; ++t) p = p * y;
    return p;
}
// phi(r) = r^(2k+1) from r^2
__device__ __forceinline__ double phs(double r2, int k) {
    double p = 1.0;
    for (int t = 0; t < k; ++t) p = p * r2;
    return sqrt(r2) * p;
}
// 2-D Laplacian of phi(|x - c|) at x = 0: (2k+1)^2 |c|^(2k-1)
__device__ __forceinline__ double phs_lap(double r2, int k) {
    if (r2 == 0.0) return 0.0;
    double p = 1.0;
    for (int t = 0; t < k - 1; ++t) p = p * r2;
    double c = (double)((2 * k + 1) * (2 * k + 1));
    return c * (sqrt(r2) * p);
}
// monomial powers: total degree ascending, then descending power of x
__device__ __forceinline__ void mono_pow(int t, int* a, int* b) {
    int d = 0;
    while ((d + 1) * (d + 2) / 2 <= t) ++d;
    int off = t - d * (d + 1) / 2;
    *a = d - off;
    *b = off;
}

// bits of |v| (ordered like |v|); a NaN counts as 0, so it never wins a magnitude comparison
__device__ __forceinline__ unsigned long long mag_bits(double v) {
    unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    return b > 0x7ff0000000000000ull ? 0ull : b;
}

struct PhsArgs {
    const double* xyz;
    const double* nrm;
    const int32_t* idx;
    int64_t N;
    int n, k, ell, L, m;
    double* w;                // Laplacian weights, or d/dx^ weights when grad
    double* wy;               // d/dy^ weights (grad only)
    int grad;                 // 0: Laplace-Beltrami (Sec. 2.2); 1: tangent-plane first derivatives
    unsigned long long* bad;  // lowest singular row
};

__global__ void __launch_bounds__(256) phs_weights_k(PhsArgs a, int wpb) {
    extern __shared__ __align__(16) double sm_phs[];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int n = a.n, m = a.m, L = a.L, nr = a.grad ? 2 : 1, ld = m + nr;
    const size_t per = (size_t)m * ld + 2 * n + 2 * m;
    double* A = sm_phs + per * wi;
    double* xh = A + (size_t)m * ld;
    double* yh = xh + n;
    double* xs = yh + n;
    double* rinvs = xs + m;
    const int64_t i = (int64_t)blockIdx.x * wpb + wi;
    if (i >= a.N) return;
    const int32_t* id = a.idx + i * n;
    double t1[3], t2[3];
    tangent_basis(a.nrm + 3 * i, t1, t2);
    const double* xc = a.xyz + 3 * i;
    // eq. (tp_pts): projected coordinates and support radius s
    double s = 0.0;
    for (int j = lane; j < n; j += 32) {
        const double* xj = a.xyz + 3 * (int64_t)id[j];
        double d[3] = {xj[0] - xc[0], xj[1] - xc[1], xj[2] - xc[2]};
        double u = dot3d(t1, d), v = dot3d(t2, d);
        xh[j] = u;
        yh[j] = v;
        double r = sqrt(u * u + v * v);
        s = fmax(s, r);
    }
    s = warp_max_d(s);
    if (!(s > 0.0)) {
        if (lane == 0) atomicMin(a.bad, (unsigned long long)i);
        return;
    }
    const double sinv = 1.0 / s;
    __syncwarp();
    for (int j = lane; j < n; j += 32) { xh[j] = xh[j] * sinv; yh[j] = yh[j] * sinv; }
    __syncwarp();
    // saddle matrix [A P; P^T 0 | rhs]. The PHS block is symmetric: each pair (r <= c) is
    // evaluated once (xh_c - xh_r is exactly -(xh_r - xh_c), so the mirror holds the same IEEE
    // value); the triangle is enumerated flat so all lanes stay busy. Magnitudes are compared as
    // integers (the bits of |x| order like |x|), keeping compares off the FP64 pipe.
    unsigned long long amaxb = 0;
    const int tri = n * (n + 1) / 2;
    for (int e = lane; e < tri; e += 32) {
        // row r of the upper triangle starts at r*n - r*(r-1)/2
        const float nf = 2.0f * n + 1.0f;
        int r = (int)((nf - sqrtf(nf * nf - 8.0f * (float)e)) * 0.5f);
        r = max(0, min(r, n - 1));
        while (r > 0 && r * n - r * (r - 1) / 2 > e) --r;
        while (r + 1 < n && (r + 1) * n - (r + 1) * r / 2 <= e) ++r;
        const int c = r + (e - (r * n - r * (r - 1) / 2));
        double dx = xh[r] - xh[c], dy = yh[r] - yh[c];
        double v = phs(dx * dx + dy * dy, a.k);
        A[r * ld + c] = v;
        A[c * ld + r] = v;
        amaxb = max(amaxb, mag_bits(v));
    }
    for (int e = lane; e < n * (L + 1); e += 32) {
        int r = e / (L + 1), t = e - r * (L + 1);
        if (t < L) {
            int pa, pb;
            mono_pow(t, &pa, &pb);
            double v = monomial(xh[r], yh[r], pa, pb);
            A[r * ld + n + t] = v;
            A[(n + t) * ld + r] = v;
            amaxb = max(amaxb, mag_bits(v));
        } else if (!a.grad) {
            A[r * ld + m] = phs_lap(xh[r] * xh[r] + yh[r] * yh[r], a.k);
        } else {  // d/dx^, d/dy^ of phi(|x^ - x^_r|) at 0: -(2k+1) |x^_r|^(2k-1) (x^_r, y^_r)
            const double r2 = xh[r] * xh[r] + yh[r] * yh[r];
            double rp = sqrt(r2);
            for (int q = 1; q < a.k; ++q) rp = rp * r2;
            A[r * ld + m] = -(double)(2 * a.k + 1) * rp * xh[r];
            A[r * ld + m + 1] = -(double)(2 * a.k + 1) * rp * yh[r];
        }
    }
    for (int e = lane; e < L * (L + nr); e += 32) {
        int t = e / (L + nr), c = e - t * (L + nr);
        double v = 0.0;
        if (c >= L) {
            int pa, pb;
            mono_pow(t, &pa, &pb);
            if (!a.grad) v = ((pa == 2 && pb == 0) || (pa == 0 && pb == 2)) ? 2.0 : 0.0;
            else if (c == L) v = (pa == 1 && pb == 0) ? 1.0 : 0.0;
            else v = (pa == 0 && pb == 1) ? 1.0 : 0.0;
        }
        A[(n + t) * ld + n + c] = v;
    }
    for (int o = 16; o; o >>= 1) amaxb = max(amaxb, __shfl_xor_sync(0xffffffffu, amaxb, o));
    const double tol = 1e-13 * __longlong_as_double((long long)amaxb);
    const unsigned long long tolb = (unsigned long long)__double_as_longlong(tol);
    __syncwarp();
    // Gaussian elimination with partial pivoting (first row of maximal |a_ik|); multipliers
    // l_r = a_rk * (1/a_kk); lanes own columns of the trailing block, rows unrolled by 4
    for (int kk = 0; kk < m; ++kk) {
        // pivot: first row of maximal |a_rk| (a NaN magnitude never wins)
        unsigned long long best = 0;
        int piv = m;  // no row yet
        for (int r = kk + lane; r < m; r += 32) {
            unsigned long long v = mag_bits(A[r * ld + kk]);
            if (piv == m || v > best) { best = v; piv = r; }
        }
        for (int o = 16; o; o >>= 1) {
            unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            int op = __shfl_xor_sync(0xffffffffu, piv, o);
            if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
        }
        const bool nan_diag =
            ((unsigned long long)__double_as_longlong(A[kk * ld + kk]) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
        if (!(best > tolb) || nan_diag) {
            if (lane == 0) atomicMin(a.bad, (unsigned long long)i);
            return;
        }
        if (piv != kk)
            for (int j = lane; j < ld; j += 32) {
                double t = A[kk * ld + j];
                A[kk * ld + j] = A[piv * ld + j];
                A[piv * ld + j] = t;
            }
        __syncwarp();
        const double rinv = 1.0 / A[kk * ld + kk];
        if (lane == 0) rinvs[kk] = rinv;
        for (int r = kk + 1 + lane; r < m; r += 32) A[r * ld + kk] = A[r * ld + kk] * rinv;
        __syncwarp();
        for (int cb = kk + 1; cb < ld; cb += 32) {
            const int c = cb + lane;
            const bool act = c < ld;
            const double pk = act ? A[kk * ld + c] : 0.0;
            int r = kk + 1;
            for (; r + 3 < m; r += 4) {
                const double l0 = A[r * ld + kk], l1 = A[(r + 1) * ld + kk], l2 = A[(r + 2) * ld + kk],
                             l3 = A[(r + 3) * ld + kk];
                if (act) {
                    double v0 = A[r * ld + c], v1 = A[(r + 1) * ld + c], v2 = A[(r + 2) * ld + c], v3 = A[(r + 3) * ld + c];
                    A[r * ld + c] = fma(-l0, pk, v0);
                    A[(r + 1) * ld + c] = fma(-l1, pk, v1);
                    A[(r + 2) * ld + c] = fma(-l2, pk, v2);
                    A[(r + 3) * ld + c] = fma(-l3, pk, v3);
                }
            }
            for (; r < m; ++r) {
                const double l0 = A[r * ld + kk];
                if (act) A[r * ld + c] = fma(-l0, pk, A[r * ld + c]);
            }
        }
        __syncwarp();
    }
    // back substitution, column oriented, for each right-hand side column
    for (int rc = m; rc < ld; ++rc) {
        bool finite = true;
        for (int kk = m - 1; kk >= 0; --kk) {
            double xk = A[kk * ld + rc] * rinvs[kk];
            finite = finite && isfinite(xk);
            if (lane == 0) xs[kk] = xk;
            for (int r = lane; r < kk; r += 32) A[r * ld + rc] = fma(-A[r * ld + kk], xk, A[r * ld + rc]);
            __syncwarp();
        }
        if (!finite) {
            if (lane == 0) atomicMin(a.bad, (unsigned long long)i);
            return;
        }
        __syncwarp();
        if (!a.grad) {
            const double s2 = s * s;
            for (int j = lane; j < n; j += 32) a.w[i * n + j] = xs[j] / s2;
        } else {
            double* out = rc == m ? a.w : a.wy;
            for (int j = lane; j < n; j += 32) out[i * n + j] = xs[j] / s;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------------------
// GFD: support radii, then weighted least squares per stencil (thread per stencil)
// ---------------------------------------------------------------------------------------------
constexpr int GFD_MAXN = 48;
constexpr int GFD_MAXL = 10;

__global__ void gfd_rho_k(const double* xyz, const double* nrm, const int32_t* idx, int64_t N, int n, double* rho) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    rho[i] = project_support(xyz, nrm, i, idx + i * n, n, nullptr, nullptr);
}

__global__ void gfd_weights_k(const double* xyz, const double* nrm, const int32_t* idx, const double* rho, int64_t N, int n,
                              int ell, int L, double alpha, double* w, unsigned long long* bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double xh[GFD_MAXN], yh[GFD_MAXN], sw[GFD_MAXN], z[GFD_MAXN];
    double B[GFD_MAXN * GFD_MAXL], V[GFD_MAXN * GFD_MAXL], y[GFD_MAXL], beta[GFD_MAXL];
    int pa[GFD_MAXL], pb[GFD_MAXL];
    for (int t = 0; t < L; ++t) mono_pow(t, &pa[t], &pb[t]);
    const int32_t* id = idx + i * n;
    double s = project_support(xyz, nrm, i, id, n, xh, yh);
    if (!(s > 0.0)) { atomicMin(bad, (unsigned long long)i); return; }
    const double ri = rho[i];
    for (int j = 0; j < n; ++j) {
        double r2 = xh[j] * xh[j] + yh[j] * yh[j];
        double rj = rho[id[j]];
        sw[j] = sqrt(exp(-alpha * r2 / (ri * ri + rj * rj)));
        xh[j] = xh[j] / s;
        yh[j] = yh[j] / s;
    }
    for (int j = 0; j < n; ++j)
        for (int c = 0; c < L; ++c) B[j * L + c] = sw[j] * monomial(xh[j], yh[j], pa[c], pb[c]);
    for (int kk = 0; kk < L; ++kk) {
        double nrm2 = 0.0;
        for (int r = kk; r < n; ++r) nrm2 = nrm2 + B[r * L + kk] * B[r * L + kk];
        double nx = sqrt(nrm2);
        if (!(nx > 0.0)) { atomicMin(bad, (unsigned long long)i); return; }
        double alp = B[kk * L + kk] >= 0.0 ? -nx : nx;
        for (int r = 0; r < n; ++r) V[r * L + kk] = (r < kk) ? 0.0 : B[r * L + kk];
        V[kk * L + kk] = V[kk * L + kk] - alp;
        double vv = 0.0;
        for (int r = kk; r < n; ++r) vv = vv + V[r * L + kk] * V[r * L + kk];
        beta[kk] = 2.0 / vv;
        for (int c = kk; c < L; ++c) {
            double dv = 0.0;
            for (int r = kk; r < n; ++r) dv = dv + V[r * L + kk] * B[r * L + c];
            double f = beta[kk] * dv;
            for (int r = kk; r < n; ++r) B[r * L + c] = B[r * L + c] - f * V[r * L + kk];
        }
    }
    double rmax = 0.0;
    for (int c = 0; c < L; ++c) rmax = fmax(rmax, fabs(B[c * L + c]));
    for (int r = 0; r < L; ++r) {
        double rhs = ((pa[r] == 2 && pb[r] == 0) || (pa[r] == 0 && pb[r] == 2)) ? 2.0 : 0.0;
        for (int c = 0; c < r; ++c) rhs = rhs - B[c * L + r] * y[c];
        if (!(fabs(B[r * L + r]) > 1e-13 * rmax)) { atomicMin(bad, (unsigned long long)i); return; }
        y[r] = rhs / B[r * L + r];
    }
    for (int r = 0; r < n; ++r) z[r] = r < L ? y[r] : 0.0;
    for (int kk = L - 1; kk >= 0; --kk) {
        double dv = 0.0;
        for (int r = kk; r < n; ++r) dv = dv + V[r * L + kk] * z[r];
        double f = beta[kk] * dv;
        for (int r = kk; r < n; ++r) z[r] = z[r] - f * V[r * L + kk];
    }
    double s2 = s * s;
    for (int j = 0; j < n; ++j) w[i * n + j] = (sw[j] * z[j]) / s2;
}

// ---------------------------------------------------------------------------------------------
// assembly: one thread per row, columns sorted by insertion (rows are n long)
// ---------------------------------------------------------------------------------------------
__global__ void assemble_k(int64_t N, int n, const int32_t* idx, const double* w, double mu, int poisson, int32_t* rp,
                           int32_t* col, double* val, int* dup) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N) return;
    rp[i] = (int32_t)(i * n);
    if (i == N) return;
    int32_t* c = col + i * n;
    double* v = val + i * n;
    for (int j = 0; j < n; ++j) {
        int32_t cj = idx[i * n + j];
        double wj = w[i * n + j];
        double vj;
        if (poisson) vj = wj;
        else {
            double t = mu * wj;
            vj = (cj == i) ? 1.0 - t : -t;
        }
        int p = j;
        while (p > 0 && c[p - 1] > cj) { c[p] = c[p - 1]; v[p] = v[p - 1]; --p; }
        c[p] = cj;
        v[p] = vj;
    }
    for (int j = 1; j < n; ++j)
        if (c[j] == c[j - 1]) atomicOr(dup, 1);
}

// ---------------------------------------------------------------------------------------------
// host entry points
// ---------------------------------------------------------------------------------------------
static void check_bad(unsigned long long* bad, cudaStream_t s, const char* what) {
    unsigned long long b = read1(bad, s);
    if (b != ULLONG_MAX) {
        set_bad_row((int64_t)b);
        fail(MGM_ERR_SINGULAR_STENCIL, std::string(what) + ": singular local system at row " + std::to_string(b));
    }
}

// Surface gradient grad_i = t1_i (wx_i . u) + t2_i (wy_i . u) (optionally eta = -grad / |grad|) and
// surface divergence div_i = sum_j wx_ij (eta_j . t1_i) + wy_ij (eta_j . t2_i) of a tangent field
// given at the nodes (neighbour vectors projected onto the tangent plane of x_i), Sec. 6.3.
__global__ void surface_grad_k(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx, const double* wy,
                               const double* u, double* g, int normalize) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double t1[3], t2[3], dx = 0.0, dy = 0.0;
    tangent_basis(nrm + 3 * i, t1, t2);
    for (int j = 0; j < n; ++j) {
        const double v = u[idx[i * n + j]];
        dx = dx + wx[i * n + j] * v;
        dy = dy + wy[i * n + j] * v;
    }
    double o[3];
    for (int a = 0; a < 3; ++a) o[a] = t1[a] * dx + t2[a] * dy;
    if (normalize) {
        const double nn = sqrt((o[0] * o[0] + o[1] * o[1]) + o[2] * o[2]);
        const double sc = nn > 1e-300 ? -1.0 / nn : -1e300;
        for (int a = 0; a < 3; ++a) o[a] = o[a] * sc;
    }
    for (int a = 0; a < 3; ++a) g[3 * i + a] = o[a];
}
__global__ void surface_div_k(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx, const double* wy,
                              const double* eta, double* d) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double t1[3], t2[3], acc = 0.0;
    tangent_basis(nrm + 3 * i, t1, t2);
    for (int j = 0; j < n; ++j) {
        const double* e = eta + 3 * (int64_t)idx[i * n + j];
        acc = acc + wx[i * n + j] * dot3d(t1, e) + wy[i * n + j] * dot3d(t2, e);
    }
    d[i] = acc;
}

void surface_gradient(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx, const double* wy,
                      const double* u, double* g, int normalize, cudaStream_t s) {
    REQUIRE(nrm && idx && wx && wy && u && g, "null array");
    REQUIRE(N >= 1 && n >= 1, "bad size");
    validate_index(idx, N * n, N, "stencil indices", s);
    surface_grad_k<<<grid_for(N, 128), 128, 0, s>>>(nrm, N, idx, n, wx, wy, u, g, normalize);
    CK_LAUNCH();
}
void surface_divergence(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx, const double* wy,
                        const double* eta, double* d, cudaStream_t s) {
    REQUIRE(nrm && idx && wx && wy && eta && d, "null array");
    REQUIRE(N >= 1 && n >= 1, "bad size");
    validate_index(idx, N * n, N, "stencil indices", s);
    surface_div_k<<<grid_for(N, 128), 128, 0, s>>>(nrm, N, idx, n, wx, wy, eta, d);
    CK_LAUNCH();
}

static void phs_launch(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, int n, int k, int ell, int L,
                       double* w, double* wy, int grad, unsigned long long* bad, cudaStream_t s) {
    const int m = n + L, ld = m + (grad ? 2 : 1);
    if (m > MAX_M) fail(MGM_ERR_UNSUPPORTED, "n + (ell+1)(ell+2)/2 must be <= 128");
    const size_t per = sizeof(double) * ((size_t)m * ld + 2 * n + 2 * m);
    int wpb = (int)std::min<size_t>(8, (227 * 1024) / per);
    if (wpb < 1) wpb = 1;
    const size_t smem = per * wpb;
    CK(cudaFuncSetAttribute(phs_weights_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PhsArgs a{xyz, nrm, idx, N, n, k, ell, L, m, w, wy, grad, bad};
    phs_weights_k<<<grid_for(N, wpb), 32 * wpb, smem, s>>>(a, wpb);
    CK_LAUNCH();
}

// tangent-plane first-derivative weights (PHS RBF-FD with the first-derivative right-hand sides)
void gradient_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, const mgm_stencil_params* sp,
                      double* wx, double* wy, cudaStream_t s) {
    REQUIRE(sp != nullptr, "null stencil params");
    REQUIRE(N >= 1 && N < 0x7fffffff, "N out of range");
    REQUIRE(xyz && nrm && idx && wx && wy, "null array");
    REQUIRE(sp->method == MGM_RBF_FD, "gradient weights: RBF-FD only");
    const int n = sp->n, ell = sp->ell;
    REQUIRE(ell >= 1 && ell <= 12, "ell out of range");
    const int L = (ell + 1) * (ell + 2) / 2;
    REQUIRE(n >= 1 && n <= N && L <= n, "stencil size n must satisfy (ell+1)(ell+2)/2 <= n <= N");
    REQUIRE(sp->k >= 1 && sp->k <= 8, "PHS order k must be in [1, 8]");
    set_bad_row(-1);
    Temp<unsigned long long> bad(1, s);
    CK(cudaMemsetAsync(bad.get(), 0xff, sizeof(unsigned long long), s));
    phs_launch(xyz, nrm, N, idx, n, sp->k, ell, L, wx, wy, 1, bad.get(), s);
    check_bad(bad.get(), s, "PHS gradient weights");
}

void stencil_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, const mgm_stencil_params* sp,
                     double* w, cudaStream_t s) {
    REQUIRE(sp != nullptr, "null stencil params");
    REQUIRE(N >= 1 && N < 0x7fffffff, "N out of range");
    REQUIRE(xyz && nrm && idx && w, "null array");
    const int n = sp->n, ell = sp->ell;
    REQUIRE(ell >= 0 && ell <= 12, "ell out of range");
    const int L = (ell + 1) * (ell + 2) / 2;
    REQUIRE(n >= 1 && n <= N && L <= n, "stencil size n must satisfy (ell+1)(ell+2)/2 <= n <= N");
    set_bad_row(-1);
    Temp<unsigned long long> bad(1, s);
    CK(cudaMemsetAsync(bad.get(), 0xff, sizeof(unsigned long long), s));
    if (sp->method == MGM_RBF_FD) {
        REQUIRE(sp->k >= 1 && sp->k <= 8, "PHS order k must be in [1, 8]");
        phs_launch(xyz, nrm, N, idx, n, sp->k, ell, L, w, nullptr, 0, bad.get(), s);
        check_bad(bad.get(), s, "PHS weights");
    } else if (sp->method == MGM_GFD) {
        REQUIRE(sp->alpha > 0.0, "GFD alpha must be > 0");
        if (n > GFD_MAXN || L > GFD_MAXL) fail(MGM_ERR_UNSUPPORTED, "GFD supports n <= 48 and ell <= 3");
        Temp<double> rho(N, s);
        gfd_rho_k<<<grid_for(N, 128), 128, 0, s>>>(xyz, nrm, idx, N, n, rho.get());
        CK_LAUNCH();
        gfd_weights_k<<<grid_for(N, 64), 64, 0, s>>>(xyz, nrm, idx, rho.get(), N, n, ell, L, sp->alpha, w, bad.get());
        CK_LAUNCH();
        check_bad(bad.get(), s, "GFD weights");
    } else {
        fail(MGM_ERR_INVALID_ARG, "unknown discretisation method");
    }
}

void assemble(int64_t N, int n, const int32_t* idx, const double* w, double mu, int poisson, int32_t* rp, int32_t* col,
              double* val, cudaStream_t s) {
    REQUIRE(N >= 1 && n >= 1 && N * (int64_t)n < 0x7fffffff, "sizes out of range");
    REQUIRE(idx && w && rp && col && val, "null array");
    Temp<int> dup(1, s);
    CK(cudaMemsetAsync(dup.get(), 0, sizeof(int), s));
    assemble_k<<<grid_for(N + 1, 128), 128, 0, s>>>(N, n, idx, w, mu, poisson, rp, col, val, dup.get());
    CK_LAUNCH();
    if (read1(dup.get(), s)) fail(MGM_ERR_INVALID_ARG, "a stencil lists the same node twice");
}

void build_stencils(const double* xyz, const double* nrm, int64_t N, const mgm_stencil_params* sp, int32_t* idx_out,
                    double* w_out, int32_t* rp, int32_t* col, double* val, cudaStream_t s) {
    REQUIRE(sp != nullptr, "null stencil params");
    REQUIRE(N >= 1 && sp->n >= 1 && sp->n <= N, "n must be in [1, N]");
    const int n = sp->n;
    Temp<int32_t> idx_t;
    Temp<double> w_t;
    int32_t* idx = idx_out;
    double* w = w_out;
    if (!idx) { idx_t.alloc((size_t)N * n, s); idx = idx_t.get(); }
    if (!w) { w_t.alloc((size_t)N * n, s); w = w_t.get(); }
    knn_device(xyz, N, xyz, N, n, 1, idx, nullptr, s);
    stencil_weights(xyz, nrm, N, idx, sp, w, s);
    assemble(N, n, idx, w, sp->mu, sp->poisson, rp, col, val, s);
}

}  // namespace mgm

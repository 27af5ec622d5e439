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
    const int32_t* rows;      // nullptr: stencils 0..N-1; else the nrows stencils rows[0..nrows-1]
    int64_t nrows;
};

// Tangent-plane coordinates of stencil i (eq. (tp_pts)), divided by the support radius s, which is
// returned (0 when the stencil is degenerate). Warp-cooperative; xh, yh in shared memory.
__device__ __forceinline__ double stencil_coords(const PhsArgs& a, int64_t i, int lane, double* xh, double* yh) {
    const int n = a.n;
    const int32_t* id = a.idx + i * n;
    double t1[3], t2[3];
    tangent_basis(a.nrm + 3 * i, t1, t2);
    const double* xc = a.xyz + 3 * i;
    // s = max_j sqrt(u_j^2 + v_j^2), taken as sqrt(max_j (u_j^2 + v_j^2)): the correctly rounded
    // square root is monotone, so the two are the same number, for one root instead of n
    double s2 = 0.0;
    for (int j = lane; j < n; j += 32) {
        const double* xj = a.xyz + 3 * (int64_t)id[j];
        double d[3] = {xj[0] - xc[0], xj[1] - xc[1], xj[2] - xc[2]};
        double u = dot3d(t1, d), v = dot3d(t2, d);
        xh[j] = u;
        yh[j] = v;
        s2 = fmax(s2, u * u + v * v);
    }
    s2 = warp_max_d(s2);
    const double s = sqrt(s2);
    if (!(s > 0.0)) return 0.0;
    const double sinv = 1.0 / s;
    __syncwarp();
    for (int j = lane; j < n; j += 32) { xh[j] = xh[j] * sinv; yh[j] = yh[j] * sinv; }
    __syncwarp();
    return s;
}

// row r and column c of the flat index e of the upper triangle (r <= c) of an n x n matrix
__device__ __forceinline__ void tri_rc(int e, int n, int* rr, int* cc) {
    // row r of the upper triangle starts at r*n - r*(r-1)/2
    const float nf = 2.0f * n + 1.0f;
    int r = (int)((nf - sqrtf(nf * nf - 8.0f * (float)e)) * 0.5f);
    r = max(0, min(r, n - 1));
    while (r > 0 && r * n - r * (r - 1) / 2 > e) --r;
    while (r + 1 < n && (r + 1) * n - (r + 1) * r / 2 <= e) ++r;
    *rr = r;
    *cc = r + (e - (r * n - r * (r - 1) / 2));
}

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
    const int64_t t = (int64_t)blockIdx.x * wpb + wi;
    if (t >= (a.rows ? a.nrows : a.N)) return;
    const int64_t i = a.rows ? (int64_t)a.rows[t] : t;
    // eq. (tp_pts): projected coordinates and support radius s
    const double s = stencil_coords(a, i, lane, xh, yh);
    if (!(s > 0.0)) {
        if (lane == 0) atomicMin(a.bad, (unsigned long long)i);
        return;
    }
    // saddle matrix [A P; P^T 0 | rhs]. The PHS block is symmetric: each pair (r <= c) is
    // evaluated once (xh_c - xh_r is exactly -(xh_r - xh_c), so the mirror holds the same IEEE
    // value); the triangle is enumerated flat so all lanes stay busy. Magnitudes are compared as
    // integers (the bits of |x| order like |x|), keeping compares off the FP64 pipe.
    unsigned long long amaxb = 0;
    const int tri = n * (n + 1) / 2;
    for (int e = lane; e < tri; e += 32) {
        int r, c;
        tri_rc(e, n, &r, &c);
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
// Mixed-precision PHS weights: the same saddle system K x = b, factorised once in FP32 (LU with
// partial pivoting) and solved by iterative refinement with FP64 residuals (the classical scheme
// analysed by Wilkinson and by Moler, 1967): x_0 = LU \ b, then r = b - K x_j in FP64,
// d = LU \ r in FP32, x_{j+1} = x_j + d, until the correction of the weight block is below 1e-12
// of the weights. Each step shrinks the error by about cond(K) eps_32 (~1e-3 for these stencils,
// cond(K) ~ 1e4 with scaled coordinates), so three or four steps reach the FP64 solution; what
// remains is FP64 rounding, of the same size as that of the elimination in phs_weights_k.
// The work moves from the FP64 pipe (2(m^3)/3 flops of elimination) to the FP32 pipes; FP64 keeps
// the matrix entries (m^2/2 square roots) and m n + n L multiply-adds per residual.
// A stencil that does not converge in IR_MAXIT steps, or meets an FP32 pivot below 2^-20 of its
// largest entry, is listed and solved again by phs_weights_k, which also decides singularity.
// Per warp in shared memory: the rows 0..n-1 of K = [A P] in FP64 (A is symmetric, so column i of
// these rows is row i of K restricted to its first n columns), the m x m FP32 copy that is
// factorised (multipliers below the diagonal), x, b, r in FP64, 1/u_kk and the row permutation.
// Strides are odd so that a warp reading a column touches distinct banks.
// ---------------------------------------------------------------------------------------------
constexpr int IR_MAXIT = 8;

struct IrLayout {
    size_t kd, xs, bd, rd, xh, yh, f, rinv, perm, bytes;
};
__host__ __device__ inline IrLayout ir_layout(int n, int m) {
    IrLayout o;
    const size_t ldd = (size_t)(m | 1), ldf = (size_t)(m | 1);
    size_t off = 0;
    o.kd = off; off += 8 * n * ldd;
    o.xs = off; off += 8 * (size_t)m;
    o.bd = off; off += 8 * (size_t)m;
    o.rd = off; off += 8 * (size_t)m;
    o.xh = off; off += 8 * (size_t)n;
    o.yh = off; off += 8 * (size_t)n;
    o.f = off; off += 4 * m * ldf;
    o.rinv = off; off += 4 * (size_t)m;
    o.perm = off; off += 4 * (size_t)m;
    o.bytes = (off + 15) & ~(size_t)15;
    return o;
}

__device__ __forceinline__ unsigned mag_bits_f(float v) {
    unsigned b = __float_as_uint(v) & 0x7fffffffu;
    return b > 0x7f800000u ? 0u : b;
}

template <int Q>
__device__ __forceinline__ float pick(const float (&z)[Q], int q) {
    float v = z[0];
#pragma unroll
    for (int p = 1; p < Q; ++p)
        if (q == p) v = z[p];
    return v;
}

// z = U^-1 L^-1 (P src) in FP32 with the factors in F (unit lower triangle below the diagonal);
// lane holds rows lane + 32 q in z[q]
template <int Q>
__device__ __forceinline__ void ir_solve(const float* F, int ldf, const float* rinv, const int* perm, const double* src,
                                         int m, int lane, float (&z)[Q]) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int r = lane + 32 * q;
        z[q] = r < m ? (float)src[perm[r]] : 0.0f;
    }
    for (int kk = 0; kk < m; ++kk) {
        const float zk = __shfl_sync(0xffffffffu, pick(z, kk >> 5), kk & 31);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = lane + 32 * q;
            if (r > kk && r < m) z[q] = fmaf(-F[r * ldf + kk], zk, z[q]);
        }
    }
    for (int kk = m - 1; kk >= 0; --kk) {
        const float xk = __shfl_sync(0xffffffffu, pick(z, kk >> 5), kk & 31) * rinv[kk];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int r = lane + 32 * q;
            if (r == kk) z[q] = xk;
            else if (r < kk) z[q] = fmaf(-F[r * ldf + kk], xk, z[q]);
        }
    }
}

template <int Q>
__global__ void __launch_bounds__(256) phs_weights_ir_k(PhsArgs a, int wpb, int32_t* retry, int* nretry) {
    extern __shared__ __align__(16) unsigned char sm_ir[];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int n = a.n, m = a.m, L = a.L, ldd = m | 1, ldf = m | 1;
    const IrLayout lay = ir_layout(n, m);
    unsigned char* base = sm_ir + lay.bytes * wi;
    double* Kd = (double*)(base + lay.kd);
    double* xs = (double*)(base + lay.xs);
    double* bd = (double*)(base + lay.bd);
    double* rd = (double*)(base + lay.rd);
    double* xh = (double*)(base + lay.xh);
    double* yh = (double*)(base + lay.yh);
    float* F = (float*)(base + lay.f);
    float* rinv = (float*)(base + lay.rinv);
    int* perm = (int*)(base + lay.perm);
    const int64_t i = (int64_t)blockIdx.x * wpb + wi;
    if (i >= a.N) return;
    const double s = stencil_coords(a, i, lane, xh, yh);
    if (!(s > 0.0)) {
        if (lane == 0) atomicMin(a.bad, (unsigned long long)i);
        return;
    }
    // K and b (eq. (rbf_fd_lap)), in FP64 and as the FP32 copy
    unsigned amaxb = 0;
    const int tri = n * (n + 1) / 2;
    for (int e = lane; e < tri; e += 32) {
        int r, c;
        tri_rc(e, n, &r, &c);
        double dx = xh[r] - xh[c], dy = yh[r] - yh[c];
        double v = phs(dx * dx + dy * dy, a.k);
        Kd[r * ldd + c] = v;
        Kd[c * ldd + r] = v;
        const float f = (float)v;
        F[r * ldf + c] = f;
        F[c * ldf + r] = f;
        amaxb = max(amaxb, mag_bits_f(f));
    }
    for (int e = lane; e < n * (L + 1); e += 32) {
        int r = e / (L + 1), t = e - r * (L + 1);
        if (t < L) {
            int pa, pb;
            mono_pow(t, &pa, &pb);
            double v = monomial(xh[r], yh[r], pa, pb);
            Kd[r * ldd + n + t] = v;
            const float f = (float)v;
            F[r * ldf + n + t] = f;
            F[(n + t) * ldf + r] = f;
            amaxb = max(amaxb, mag_bits_f(f));
        } else {
            bd[r] = phs_lap(xh[r] * xh[r] + yh[r] * yh[r], a.k);
        }
    }
    for (int e = lane; e < L * L; e += 32) {
        int t = e / L, c = e - t * L;
        F[(n + t) * ldf + n + c] = 0.0f;
    }
    for (int t = lane; t < L; t += 32) {
        int pa, pb;
        mono_pow(t, &pa, &pb);
        bd[n + t] = ((pa == 2 && pb == 0) || (pa == 0 && pb == 2)) ? 2.0 : 0.0;
    }
    for (int j = lane; j < m; j += 32) perm[j] = j;
    for (int o = 16; o; o >>= 1) amaxb = max(amaxb, __shfl_xor_sync(0xffffffffu, amaxb, o));
    const unsigned tolb = __float_as_uint(ldexpf(__uint_as_float(amaxb), -20));
    __syncwarp();
    // FP32 LU with partial pivoting (first row of maximal |f_rk|)
    bool ok = true;
    for (int kk = 0; kk < m; ++kk) {
        unsigned best = 0;
        int piv = m;
        for (int r = kk + lane; r < m; r += 32) {
            unsigned v = mag_bits_f(F[r * ldf + kk]);
            if (piv == m || v > best) { best = v; piv = r; }
        }
        for (int o = 16; o; o >>= 1) {
            unsigned ob = __shfl_xor_sync(0xffffffffu, best, o);
            int op = __shfl_xor_sync(0xffffffffu, piv, o);
            if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
        }
        if (!(best > tolb)) { ok = false; break; }  // warp-uniform after the reduction
        if (piv != kk) {
            for (int j = lane; j < m; j += 32) {
                float t = F[kk * ldf + j];
                F[kk * ldf + j] = F[piv * ldf + j];
                F[piv * ldf + j] = t;
            }
            if (lane == 0) {
                int t = perm[kk];
                perm[kk] = perm[piv];
                perm[piv] = t;
            }
        }
        __syncwarp();
        const float rk = 1.0f / F[kk * ldf + kk];
        if (lane == 0) rinv[kk] = rk;
        for (int r = kk + 1 + lane; r < m; r += 32) F[r * ldf + kk] = F[r * ldf + kk] * rk;
        __syncwarp();
        for (int cb = kk + 1; cb < m; cb += 32) {
            const int c = cb + lane;
            const bool act = c < m;
            const float pk = act ? F[kk * ldf + c] : 0.0f;
            int r = kk + 1;
            for (; r + 3 < m; r += 4) {
                const float l0 = F[r * ldf + kk], l1 = F[(r + 1) * ldf + kk], l2 = F[(r + 2) * ldf + kk],
                            l3 = F[(r + 3) * ldf + kk];
                if (act) {
                    float v0 = F[r * ldf + c], v1 = F[(r + 1) * ldf + c], v2 = F[(r + 2) * ldf + c],
                          v3 = F[(r + 3) * ldf + c];
                    F[r * ldf + c] = fmaf(-l0, pk, v0);
                    F[(r + 1) * ldf + c] = fmaf(-l1, pk, v1);
                    F[(r + 2) * ldf + c] = fmaf(-l2, pk, v2);
                    F[(r + 3) * ldf + c] = fmaf(-l3, pk, v3);
                }
            }
            for (; r < m; ++r) {
                const float l0 = F[r * ldf + kk];
                if (act) F[r * ldf + c] = fmaf(-l0, pk, F[r * ldf + c]);
            }
        }
        __syncwarp();
    }
    bool conv = false;
    if (ok) {
        float z[Q];
        ir_solve<Q>(F, ldf, rinv, perm, bd, m, lane, z);
#pragma unroll
        for (int q = 0; q < Q; ++q)
            if (lane + 32 * q < m) xs[lane + 32 * q] = (double)z[q];
        __syncwarp();
        for (int it = 0; it < IR_MAXIT; ++it) {
            // r = b - K x in FP64; row i reads column i of the stored rows (A symmetric)
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int r = lane + 32 * q;
                if (r < m) {
                    double acc = bd[r];
                    for (int j = 0; j < n; ++j) acc = fma(-Kd[j * ldd + r], xs[j], acc);
                    if (r < n)
                        for (int t = 0; t < L; ++t) acc = fma(-Kd[r * ldd + n + t], xs[n + t], acc);
                    rd[r] = acc;
                }
            }
            __syncwarp();
            ir_solve<Q>(F, ldf, rinv, perm, rd, m, lane, z);
            double dmax = 0.0, xmax = 0.0;
            bool fin = true;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int r = lane + 32 * q;
                if (r < m) {
                    const double d = (double)z[q];
                    const double xn = xs[r] + d;
                    xs[r] = xn;
                    fin = fin && isfinite(xn);
                    if (r < n) {
                        dmax = fmax(dmax, fabs(d));
                        xmax = fmax(xmax, fabs(xn));
                    }
                }
            }
            dmax = warp_max_d(dmax);
            xmax = warp_max_d(xmax);
            fin = __all_sync(0xffffffffu, fin);
            __syncwarp();
            if (!fin) break;
            if (dmax <= 1e-12 * xmax) {
                conv = true;
                break;
            }
        }
    }
    if (conv) {
        const double s2 = s * s;
        for (int j = lane; j < n; j += 32) a.w[i * n + j] = xs[j] / s2;
    } else if (lane == 0) {
        retry[atomicAdd(nretry, 1)] = (int32_t)i;
    }
}

// ---------------------------------------------------------------------------------------------
// The same refinement with the FP32 factorisation held in registers, for the two stencil shapes
// used most (m = 36: n = 30, ell = 2; m = 60: n = 50, ell = 3). Lane l holds rows l and l + 32 of
// the saddle matrix (all m columns, fully unrolled so every register index is static). Partial
// pivoting is implicit: rows stay in their lanes, a row chosen as pivot is marked done and keeps
// its U row, the others store their multipliers in place; the triangular solves follow the
// recorded pivot order. Shared memory keeps only the FP64 rows of [A P] for the residuals, so
// several times more warps fit on an SM than with the shared-memory factorisation.
// ---------------------------------------------------------------------------------------------
// FP32 value of an FP64 number rounded toward zero, by integer operations on its IEEE-754 fields
// (the FP64 pipe is the scarce one). Magnitudes below FP32's normal range give a signed zero, above
// it infinity; the factorisation only needs K to FP32 accuracy.
__device__ __forceinline__ float d2f_trunc(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)e << 23) | mant);
}

constexpr int RL_MAXD = 7;  // largest polynomial degree of the register kernel

struct RlLayout {
    size_t kd, xs, bd, xh, yh, rinv, piv, prow, bytes;
};
__host__ __device__ inline RlLayout rl_layout(int n, int m) {
    RlLayout o;
    const size_t ldd = (size_t)(m | 1);
    size_t off = 0;
    o.kd = off; off += 8 * n * ldd;
    o.xs = off; off += 8 * (size_t)m;
    o.bd = off; off += 8 * (size_t)m;
    o.xh = off; off += 8 * (size_t)n;
    o.yh = off; off += 8 * (size_t)n;
    o.rinv = off; off += 4 * (size_t)m;
    o.piv = off; off += 4 * (size_t)m;
    o.prow = (off + 15) & ~(size_t)15; off = o.prow + 4 * (size_t)m;  // the pivot row of one elimination step
    o.bytes = (off + 15) & ~(size_t)15;
    return o;
}

// column c of a row held as pairs of adjacent columns (c static after unrolling)
__device__ __forceinline__ float col_of(const float2* a, int c) { return (c & 1) ? a[c >> 1].y : a[c >> 1].x; }
__device__ __forceinline__ void set_col(float2* a, int c, float v) {
    if (c & 1) a[c >> 1].y = v;
    else a[c >> 1].x = v;
}

// z <- U^-1 L^-1 P z with the register factors; on return x0, x1 hold solution components lane and
// lane + 32. s0, s1: the step at which each row became the pivot (M: never).
template <int M>
__device__ __forceinline__ void rl_solve(const float2 (&a0)[M / 2], const float2 (&a1)[M / 2], int s0, int s1,
                                         const int* piv, const float* rinv, float z0, float z1, float& x0, float& x1,
                                         int lane) {
#pragma unroll
    for (int kk = 0; kk < M; ++kk) {
        const int p = piv[kk];
        const float y = __shfl_sync(0xffffffffu, p >= 32 ? z1 : z0, p & 31);
        if (s0 > kk) z0 = fmaf(-col_of(a0, kk), y, z0);
        if (s1 > kk) z1 = fmaf(-col_of(a1, kk), y, z1);
    }
#pragma unroll
    for (int kk = M - 1; kk >= 0; --kk) {
        const int p = piv[kk];
        const float xk = __shfl_sync(0xffffffffu, p >= 32 ? z1 : z0, p & 31) * rinv[kk];
        if (s0 < kk) z0 = fmaf(-col_of(a0, kk), xk, z0);
        if (s1 < kk) z1 = fmaf(-col_of(a1, kk), xk, z1);
        if (lane == (kk & 31)) {
            if (kk < 32) x0 = xk;
            else x1 = xk;
        }
    }
}

template <int M>
__global__ void __launch_bounds__(256) phs_weights_rl_k(PhsArgs a, int wpb, int32_t* retry, int* nretry) {
    static_assert(M <= 64, "two rows a lane");
    constexpr int LDD = M | 1;
    extern __shared__ __align__(16) unsigned char sm_rl[];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int n = a.n, L = M - n;
    const RlLayout lay = rl_layout(n, M);
    unsigned char* base = sm_rl + lay.bytes * wi;
    double* Kd = (double*)(base + lay.kd);
    double* xs = (double*)(base + lay.xs);
    double* bd = (double*)(base + lay.bd);
    double* xh = (double*)(base + lay.xh);
    double* yh = (double*)(base + lay.yh);
    float* rinv = (float*)(base + lay.rinv);
    int* piv = (int*)(base + lay.piv);
    float4* prow = (float4*)(base + lay.prow);
    const int64_t i = (int64_t)blockIdx.x * wpb + wi;
    if (i >= a.N) return;
    const double s = stencil_coords(a, i, lane, xh, yh);
    if (!(s > 0.0)) {
        if (lane == 0) atomicMin(a.bad, (unsigned long long)i);
        return;
    }
    // rows 0..n-1 of K = [A P] and b in FP64 (eq. (rbf_fd_lap))
    unsigned long long amaxb = 0;
    const int tri = n * (n + 1) / 2;
    for (int e = lane; e < tri; e += 32) {
        int r, c;
        tri_rc(e, n, &r, &c);
        double dx = xh[r] - xh[c], dy = yh[r] - yh[c];
        double v = phs(dx * dx + dy * dy, a.k);
        Kd[r * LDD + c] = v;
        Kd[c * LDD + r] = v;
        amaxb = max(amaxb, mag_bits(v));
    }
    // the monomials of one point a lane, in the order of mono_pow, with the powers of x and y
    // shared: x^a y^b is x^a (x multiplied in a - 1 times) times y, b times, exactly the
    // operations of monomial(), so the same numbers, at one multiplication a monomial or less
    // and with every lane of the warp on the same degree
    for (int r = lane; r < n; r += 32) {
        const double x = xh[r], y = yh[r];
        double px[RL_MAXD + 1], py[RL_MAXD + 1];
        px[0] = 1.0;
        py[0] = 1.0;
#pragma unroll
        for (int d = 1; d <= RL_MAXD; ++d) {
            px[d] = 0.0;
            py[d] = 0.0;
            if (d <= a.ell) {
                px[d] = d == 1 ? x : px[d - 1] * x;
                py[d] = d == 1 ? y : py[d - 1] * y;
            }
        }
        double* row = Kd + r * LDD + n;
#pragma unroll
        for (int d = 0; d <= RL_MAXD; ++d) {
            if (d <= a.ell) {
#pragma unroll
                for (int off = 0; off <= d; ++off) {
                    double v;
                    if (off == 0) {
                        v = px[d];
                    } else if (off == d) {
                        v = py[d];
                    } else {
                        v = px[d - off];
#pragma unroll
                        for (int q = 0; q < off; ++q) v = v * y;
                    }
                    row[d * (d + 1) / 2 + off] = v;
                    amaxb = max(amaxb, mag_bits(v));
                }
            }
        }
    }
    for (int r = lane; r < n; r += 32) bd[r] = phs_lap(xh[r] * xh[r] + yh[r] * yh[r], a.k);
    for (int t = lane; t < L; t += 32) {
        int pa, pb;
        mono_pow(t, &pa, &pb);
        bd[n + t] = ((pa == 2 && pb == 0) || (pa == 0 && pb == 2)) ? 2.0 : 0.0;
    }
    for (int o = 16; o; o >>= 1) amaxb = max(amaxb, __shfl_xor_sync(0xffffffffu, amaxb, o));
    const unsigned tolb = __float_as_uint(ldexpf((float)__longlong_as_double((long long)amaxb), -20));
    __syncwarp();
    // FP32 copy into registers, as pairs of adjacent columns: row r < n is row r of [A P]; row n + t
    // is column n + t of it (P^T, then the zero block); rows >= M are absent
    static_assert(M % 4 == 0, "rows are stored as pairs of columns, published four columns at a time");
    constexpr int MP = M / 2;
    const int r0 = lane, r1 = lane + 32;
    float2 a0[MP], a1[MP];
    {
        const double* p0 = r0 < n ? Kd + r0 * LDD : Kd + r0;
        const double* p1 = r1 < n ? Kd + r1 * LDD : Kd + r1;
        const int st0 = r0 < n ? 1 : LDD, st1 = r1 < n ? 1 : LDD;
        const int lim0 = r0 < n ? M : (r0 < M ? n : 0), lim1 = r1 < n ? M : (r1 < M ? n : 0);
#pragma unroll
        for (int q = 0; q < MP; ++q) {
            const int c = 2 * q;
            a0[q] = make_float2(c < lim0 ? d2f_trunc(p0[c * st0]) : 0.0f, c + 1 < lim0 ? d2f_trunc(p0[(c + 1) * st0]) : 0.0f);
            a1[q] = make_float2(c < lim1 ? d2f_trunc(p1[c * st1]) : 0.0f, c + 1 < lim1 ? d2f_trunc(p1[(c + 1) * st1]) : 0.0f);
        }
    }
    // FP32 LU with implicit partial pivoting (first row of maximal |a_rk| among rows not yet used).
    // The pivot row's lane publishes the row's remaining columns in shared memory (four a store),
    // every lane reads them back as a broadcast and updates both of its rows with paired FMAs.
    bool d0 = r0 >= M, d1 = r1 >= M;
    int s0 = M, s1 = M;
    bool ok = true;
    const float* prowf = reinterpret_cast<const float*>(prow);
#pragma unroll
    for (int kk = 0; kk < M; ++kk) {
        const float f0 = col_of(a0, kk), f1 = col_of(a1, kk);
        const unsigned b0 = d0 ? 0u : mag_bits_f(f0);
        const unsigned b1 = d1 ? 0u : mag_bits_f(f1);
        // warp maximum in one reduction; the first row holding it (rows lane, then lane + 32)
        const unsigned best = __reduce_max_sync(0xffffffffu, max(b0, b1));
        const unsigned m0 = __ballot_sync(0xffffffffu, !d0 && b0 == best);
        const unsigned m1 = __ballot_sync(0xffffffffu, !d1 && b1 == best);
        ok = ok && best > tolb;  // warp-uniform; a failed factorisation is discarded
        const int p = m0 ? __ffs(m0) - 1 : 32 + __ffs(m1) - 1, pl = p & 31;
        const bool hi = p >= 32;
        if (p == r0) { d0 = true; s0 = kk; }
        if (p == r1) { d1 = true; s1 = kk; }
        // columns kk.. of the pivot row, from the first group of four that holds column kk
        const int g0 = (kk / 4) * 2;  // first pair published
        if (lane == pl) {
            if (hi) {
#pragma unroll
                for (int q = g0; q < MP; q += 2) prow[q >> 1] = make_float4(a1[q].x, a1[q].y, a1[q + 1].x, a1[q + 1].y);
            } else {
#pragma unroll
                for (int q = g0; q < MP; q += 2) prow[q >> 1] = make_float4(a0[q].x, a0[q].y, a0[q + 1].x, a0[q + 1].y);
            }
        }
        __syncwarp();
        const float rk = 1.0f / prowf[kk];
        if (lane == 0) {
            piv[kk] = p;
            rinv[kk] = rk;
        }
        const float l0 = d0 ? 0.0f : f0 * rk;
        const float l1 = d1 ? 0.0f : f1 * rk;
        const float2 n0 = make_float2(-l0, -l0), n1 = make_float2(-l1, -l1);
        // columns > kk: the pairs from (kk + 1) / 2; for even kk the first pair also holds column kk,
        // which the multiplier overwrites below (done rows have l = 0 and keep their entries)
#pragma unroll
        for (int q = (kk + 1) / 2; q < MP; ++q) {
            const float4 v4 = prow[q >> 1];
            const float2 v = (q & 1) ? make_float2(v4.z, v4.w) : make_float2(v4.x, v4.y);
            a0[q] = __ffma2_rn(n0, v, a0[q]);
            a1[q] = __ffma2_rn(n1, v, a1[q]);
        }
        if (!d0) set_col(a0, kk, l0);
        if (!d1) set_col(a1, kk, l1);
        __syncwarp();  // the pivot row is read before the next step overwrites it
    }
    __syncwarp();
    bool conv = false;
    if (ok) {
        for (int it = 0; it <= IR_MAXIT; ++it) {
            // r = b - K x in FP64 (x = 0 at it = 0); row i reads column i of the stored rows
            double q0 = 0.0, q1 = 0.0;
            if (r0 < M) q0 = bd[r0];
            if (r1 < M) q1 = bd[r1];
            if (it > 0) {
                for (int j = 0; j < n; ++j) {
                    const double xj = xs[j];
                    if (r0 < M) q0 = fma(-Kd[j * LDD + r0], xj, q0);
                    if (r1 < M) q1 = fma(-Kd[j * LDD + r1], xj, q1);
                }
                for (int t = 0; t < L; ++t) {
                    const double xt = xs[n + t];
                    if (r0 < n) q0 = fma(-Kd[r0 * LDD + n + t], xt, q0);
                    if (r1 < n) q1 = fma(-Kd[r1 * LDD + n + t], xt, q1);
                }
            }
            float x0 = 0.0f, x1 = 0.0f;
            rl_solve<M>(a0, a1, s0, s1, piv, rinv, (float)q0, (float)q1, x0, x1, lane);
            __syncwarp();
            // magnitudes compared as bits (FP32 for the correction), keeping the FP64 pipe free
            unsigned dmb = 0;
            unsigned long long xmb = 0;
            bool fin = true;
            if (r0 < M) {
                const double xn = (it > 0 ? xs[r0] : 0.0) + (double)x0;
                xs[r0] = xn;
                const unsigned long long b = (unsigned long long)__double_as_longlong(xn) & 0x7fffffffffffffffull;
                fin = fin && b < 0x7ff0000000000000ull && mag_bits_f(x0) == (__float_as_uint(x0) & 0x7fffffffu);
                if (r0 < n) { dmb = max(dmb, mag_bits_f(x0)); xmb = max(xmb, b); }
            }
            if (r1 < M) {
                const double xn = (it > 0 ? xs[r1] : 0.0) + (double)x1;
                xs[r1] = xn;
                const unsigned long long b = (unsigned long long)__double_as_longlong(xn) & 0x7fffffffffffffffull;
                fin = fin && b < 0x7ff0000000000000ull && mag_bits_f(x1) == (__float_as_uint(x1) & 0x7fffffffu);
                if (r1 < n) { dmb = max(dmb, mag_bits_f(x1)); xmb = max(xmb, b); }
            }
            for (int o = 16; o; o >>= 1) {
                dmb = max(dmb, __shfl_xor_sync(0xffffffffu, dmb, o));
                xmb = max(xmb, __shfl_xor_sync(0xffffffffu, xmb, o));
            }
            fin = __all_sync(0xffffffffu, fin);
            __syncwarp();
            if (!fin) break;
            if (it > 0 && (double)__uint_as_float(dmb) <= 1e-12 * __longlong_as_double((long long)xmb)) {
                conv = true;
                break;
            }
        }
    }
    if (conv) {
        const double s2 = s * s;
        for (int j = lane; j < n; j += 32) a.w[i * n + j] = xs[j] / s2;
    } else if (lane == 0) {
        retry[atomicAdd(nretry, 1)] = (int32_t)i;
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
// assembly: one warp per row; the row's (column, position) keys are staged in shared memory and
// each entry is placed by rank, so columns come out ascending (stable for repeats, which are
// reported)
// ---------------------------------------------------------------------------------------------
constexpr int ASM_WARPS = 8, ASM_MAX = 256;
__global__ void __launch_bounds__(ASM_WARPS * 32) assemble_k(int64_t N, int n, const int32_t* idx, const double* w,
                                                             double mu, int poisson, int32_t* rp, int32_t* col,
                                                             double* val, int* dup) {
    __shared__ unsigned long long key[ASM_WARPS][ASM_MAX];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * ASM_WARPS + wi;
    if (i > N) return;
    if (lane == 0) rp[i] = (int32_t)(i * n);
    if (i == N) return;
    for (int j = lane; j < n; j += 32)
        key[wi][j] = ((unsigned long long)(uint32_t)idx[i * n + j] << 32) | (unsigned)j;
    __syncwarp();
    bool rep = false;
    for (int j = lane; j < n; j += 32) {
        const unsigned long long k = key[wi][j];
        const int32_t cj = (int32_t)(k >> 32);
        int rank = 0;
        for (int u = 0; u < n; ++u) {
            const unsigned long long ku = key[wi][u];
            rank += ku < k ? 1 : 0;
            rep = rep || (u != j && (int32_t)(ku >> 32) == cj);
        }
        const double wj = w[i * n + j];
        double vj;
        if (poisson) vj = wj;
        else {
            const double t = mu * wj;
            vj = (cj == i) ? 1.0 - t : -t;
        }
        col[i * n + rank] = cj;
        val[i * n + rank] = vj;
    }
    if (__any_sync(0xffffffffu, rep) && lane == 0) atomicOr(dup, 1);
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
                       double* w, double* wy, int grad, unsigned long long* bad, cudaStream_t s,
                       const int32_t* rows = nullptr, int64_t nrows = 0) {
    const int m = n + L, ld = m + (grad ? 2 : 1);
    if (m > MAX_M) fail(MGM_ERR_UNSUPPORTED, "n + (ell+1)(ell+2)/2 must be <= 128");
    const size_t per = sizeof(double) * ((size_t)m * ld + 2 * n + 2 * m);
    int wpb = (int)std::min<size_t>(8, (227 * 1024) / per);
    if (wpb < 1) wpb = 1;
    const size_t smem = per * wpb;
    CK(cudaFuncSetAttribute(phs_weights_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    PhsArgs a{xyz, nrm, idx, N, n, k, ell, L, m, w, wy, grad, bad, rows, nrows};
    phs_weights_k<<<grid_for(rows ? nrows : N, wpb), 32 * wpb, smem, s>>>(a, wpb);
    CK_LAUNCH();
}

// FP32 LU + FP64 refinement, then FP64 elimination for the stencils it lists; returns their count
static int64_t phs_mixed(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, int n, int k, int ell,
                         int L, double* w, unsigned long long* bad, cudaStream_t s) {
    const int m = n + L;
    if (m > MAX_M) fail(MGM_ERR_UNSUPPORTED, "n + (ell+1)(ell+2)/2 must be <= 128");
    const IrLayout lay = ir_layout(n, m);
    int wpb = (int)std::min<size_t>(8, (227 * 1024) / lay.bytes);
    if (wpb < 1) wpb = 1;
    const size_t smem = lay.bytes * wpb;
    Temp<int32_t> retry(N, s);
    Temp<int> nretry(1, s);
    CK(cudaMemsetAsync(nretry.get(), 0, sizeof(int), s));
    PhsArgs a{xyz, nrm, idx, N, n, k, ell, L, m, w, nullptr, 0, bad, nullptr, 0};
    if ((m == 36 || m == 60) && a.ell <= RL_MAXD) {  // (m = 60 allows ell <= 6 with L <= n)
        // four warps a block: m = 60 takes 255 registers a thread (two blocks an SM), m = 36 about
        // 160 (three blocks)
        const RlLayout rl = rl_layout(n, m);
        const int wr = (int)std::min<size_t>(4, (227 * 1024) / rl.bytes);
        const size_t sm = rl.bytes * wr;
        if (m == 36) {
            CK(cudaFuncSetAttribute(phs_weights_rl_k<36>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            phs_weights_rl_k<36><<<grid_for(N, wr), 32 * wr, sm, s>>>(a, wr, retry.get(), nretry.get());
        } else {
            CK(cudaFuncSetAttribute(phs_weights_rl_k<60>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            phs_weights_rl_k<60><<<grid_for(N, wr), 32 * wr, sm, s>>>(a, wr, retry.get(), nretry.get());
        }
    } else if (m <= 64) {
        CK(cudaFuncSetAttribute(phs_weights_ir_k<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        phs_weights_ir_k<2><<<grid_for(N, wpb), 32 * wpb, smem, s>>>(a, wpb, retry.get(), nretry.get());
    } else {
        CK(cudaFuncSetAttribute(phs_weights_ir_k<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        phs_weights_ir_k<4><<<grid_for(N, wpb), 32 * wpb, smem, s>>>(a, wpb, retry.get(), nretry.get());
    }
    CK_LAUNCH();
    const int cnt = read1(nretry.get(), s);
    if (cnt > 0) phs_launch(xyz, nrm, N, idx, n, k, ell, L, w, nullptr, 0, bad, s, retry.get(), cnt);
    return cnt;
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
    REQUIRE(sp->weights == MGM_WEIGHTS_F64 || sp->weights == MGM_WEIGHTS_MIXED, "unknown weights mode");
    set_bad_row(-1);
    set_fp64_rows(0);
    Temp<unsigned long long> bad(1, s);
    CK(cudaMemsetAsync(bad.get(), 0xff, sizeof(unsigned long long), s));
    if (sp->method == MGM_RBF_FD) {
        REQUIRE(sp->k >= 1 && sp->k <= 8, "PHS order k must be in [1, 8]");
        if (sp->weights == MGM_WEIGHTS_MIXED) set_fp64_rows(phs_mixed(xyz, nrm, N, idx, n, sp->k, ell, L, w, bad.get(), s));
        else phs_launch(xyz, nrm, N, idx, n, sp->k, ell, L, w, nullptr, 0, bad.get(), s);
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
    REQUIRE(n <= ASM_MAX, "stencil size above 256");
    assemble_k<<<grid_for(N + 1, ASM_WARPS), ASM_WARPS * 32, 0, s>>>(N, n, idx, w, mu, poisson, rp, col, val, dup.get());
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

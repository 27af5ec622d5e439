// Eigenpairs of a hierarchy's operator L of smallest magnitude by shift-invert (paper Sec. 6.1:
// Arnoldi on the shifted inverse, each application an MGM-preconditioned GMRES solve; with
// L = I - D the shift is sigma = -1 for the surface operator -D).
//
// Method: block Krylov subspace for A = L^-1 with thick restarts and explicit Rayleigh-Ritz.
// Each expansion step applies A to a block of b orthonormal vectors (one mgm_solve_multi call for
// the b right-hand sides), so V (basis) and W = A V are both kept; the Rayleigh quotient
// G = V^T W is formed in full, its eigenpairs (theta, y) give the Ritz pairs (theta, V y) with
// residual W y - theta V y. After a cycle of s steps the basis restarts from the wanted Ritz
// vectors (real basis: a complex pair contributes its real and imaginary parts) and continues
// from the images of the last ones. Eigenvalues of L are 1 / theta.
//
// Device work: the solves, tall-skinny products V^T W (two passes, fixed summation order) and
// V S (S small), orthogonalisation by two rounds of classical Gram-Schmidt against the basis and
// Cholesky QR (twice) within the block. Host work: the small dense eigenproblem of G (Householder
// reduction to Hessenberg form, complex single-shift QR with Givens rotations, eigenvectors of the
// triangular Schur factor by back substitution) and Cholesky factors of b x b Gram matrices.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "hier.cuh"

namespace mgm {

typedef std::complex<double> cd;

// ------------------------------ device kernels ------------------------------------------------
constexpr int TS_THREADS = 256;
constexpr int TS_CHUNK = 16;    // rows staged per pass
constexpr int TS_MAXC = 96;     // columns of either factor

// part[blk][i][j] = sum over the block's rows of A[row][i] B[row][j]  (A: N x ka, B: N x kb, column-major)
__global__ void __launch_bounds__(TS_THREADS) tsgemm_tn_part_k(const double* A, int ka, const double* B, int kb,
                                                               int64_t N, int64_t rows_per_block, double* part) {
    __shared__ double sa[TS_CHUNK][TS_MAXC + 1];
    __shared__ double sb[TS_CHUNK][TS_MAXC + 1];
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_block;
    const int64_t r1 = r0 + rows_per_block < N ? r0 + rows_per_block : N;
    const int pairs = ka * kb;
    double acc[(TS_MAXC * TS_MAXC + TS_THREADS - 1) / TS_THREADS];
    const int np = (pairs + TS_THREADS - 1) / TS_THREADS;
    for (int q = 0; q < np; ++q) acc[q] = 0.0;
    for (int64_t c0 = r0; c0 < r1; c0 += TS_CHUNK) {
        const int nr = r1 - c0 < TS_CHUNK ? (int)(r1 - c0) : TS_CHUNK;
        for (int t = threadIdx.x; t < TS_CHUNK * ka; t += TS_THREADS) {
            const int rr = t % TS_CHUNK, cc = t / TS_CHUNK;
            sa[rr][cc] = rr < nr ? A[(int64_t)cc * N + c0 + rr] : 0.0;
        }
        for (int t = threadIdx.x; t < TS_CHUNK * kb; t += TS_THREADS) {
            const int rr = t % TS_CHUNK, cc = t / TS_CHUNK;
            sb[rr][cc] = rr < nr ? B[(int64_t)cc * N + c0 + rr] : 0.0;
        }
        __syncthreads();
        for (int q = 0; q < np; ++q) {
            const int p = threadIdx.x + q * TS_THREADS;
            if (p < pairs) {
                const int i = p % ka, j = p / ka;
                double s = acc[q];
                for (int rr = 0; rr < TS_CHUNK; ++rr) s = fma(sa[rr][i], sb[rr][j], s);
                acc[q] = s;
            }
        }
        __syncthreads();
    }
    for (int q = 0; q < np; ++q) {
        const int p = threadIdx.x + q * TS_THREADS;
        if (p < pairs) part[(int64_t)blockIdx.x * pairs + p] = acc[q];
    }
}
// C[p] = sum over blocks in order (deterministic)
__global__ void tsgemm_tn_sum_k(const double* part, int nblocks, int pairs, double* C) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= pairs) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * pairs + p];
    C[p] = s;
}
// C (N x l) = A (N x ka) S (ka x l), or C -= A S (sub), S column-major on the device
__global__ void tsgemm_nn_k(const double* A, int ka, const double* S, int l, int64_t N, double* C, int sub) {
    __shared__ double ss[TS_MAXC * 16];
    for (int t = threadIdx.x; t < ka * l; t += blockDim.x) ss[t] = S[t];
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    double out[16];
    for (int j = 0; j < l; ++j) out[j] = sub ? C[(int64_t)j * N + r] : 0.0;
    for (int i = 0; i < ka; ++i) {
        const double a = A[(int64_t)i * N + r];
        for (int j = 0; j < l; ++j) out[j] = sub ? fma(-a, ss[j * ka + i], out[j]) : fma(a, ss[j * ka + i], out[j]);
    }
    for (int j = 0; j < l; ++j) C[(int64_t)j * N + r] = out[j];
}
// uniform(-1, 1) entries from a counter-based SplitMix64 stream
__global__ void fill_uniform_k(double* x, int64_t n, unsigned long long seed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = seed + ((unsigned long long)i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// ------------------------------ host helpers ---------------------------------------------------
struct Ts {
    Temp<double> part, c;
    int nblocks = 0;
};

// host C (ka x kb, column-major) = A^T B
static void tsgemm_tn(Ts& w, const double* A, int ka, const double* B, int kb, int64_t N, std::vector<double>& C,
                      cudaStream_t s) {
    REQUIRE(ka <= TS_MAXC && kb <= TS_MAXC, "block too wide");
    const int pairs = ka * kb;
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(152 * 4, (N + 4095) / 4096));
    const int64_t rpb = (N + nb - 1) / nb;
    if ((int64_t)w.part.n < (int64_t)nb * pairs) w.part.alloc((int64_t)nb * pairs, s);
    if ((int64_t)w.c.n < pairs) w.c.alloc(pairs, s);
    tsgemm_tn_part_k<<<nb, TS_THREADS, 0, s>>>(A, ka, B, kb, N, rpb, w.part.get());
    CK_LAUNCH();
    tsgemm_tn_sum_k<<<grid_for(pairs, 128), 128, 0, s>>>(w.part.get(), nb, pairs, w.c.get());
    CK_LAUNCH();
    C.resize(pairs);
    to_host(C.data(), w.c.get(), pairs, s);
}

// C = A S or C -= A S with S (ka x l) given on the host (l <= 16)
static void tsgemm_nn(Temp<double>& sdev, const double* A, int ka, const std::vector<double>& S, int l, int64_t N,
                      double* C, bool sub, cudaStream_t s) {
    REQUIRE(ka * l <= TS_MAXC * 16 && l <= 16, "block too wide");
    if ((int64_t)sdev.n < ka * l) sdev.alloc(ka * l, s);
    CK(cudaMemcpyAsync(sdev.get(), S.data(), sizeof(double) * ka * l, cudaMemcpyHostToDevice, s));
    tsgemm_nn_k<<<grid_for(N, 256), 256, 0, s>>>(A, ka, sdev.get(), l, N, C, sub ? 1 : 0);
    CK_LAUNCH();
    CK(cudaStreamSynchronize(s));  // S is a host vector that may change before the copy runs otherwise
}

// C = A S for S with up to TS_MAXC columns, in slices of 16
static void tsgemm_nn_wide(Temp<double>& sdev, const double* A, int ka, const std::vector<double>& S, int l, int64_t N,
                           double* C, cudaStream_t s) {
    for (int j0 = 0; j0 < l; j0 += 16) {
        const int lj = std::min(16, l - j0);
        std::vector<double> Sj(S.begin() + (size_t)j0 * ka, S.begin() + (size_t)(j0 + lj) * ka);
        tsgemm_nn(sdev, A, ka, Sj, lj, N, C + (int64_t)j0 * N, false, s);
    }
}

// Eigen-decomposition of a small symmetric matrix S (n x n, column-major) by cyclic Jacobi
// rotations: S = U diag(w) U^T, U column-major.
static void jacobi_eig(int n, std::vector<double> S, std::vector<double>& w, std::vector<double>& U) {
    U.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) U[i + (size_t)i * n] = 1.0;
    auto a = [&](int i, int j) -> double& { return S[i + (size_t)j * n]; };
    double fro = 0.0;
    for (double x : S) fro += x * x;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += 2.0 * a(i, j) * a(i, j);
        if (off <= 1e-30 * fro) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (a(p, q) == 0.0) continue;
                const double theta = (a(q, q) - a(p, p)) / (2.0 * a(p, q));
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    const double x = a(k, p), y = a(k, q);
                    a(k, p) = c * x - sn * y;
                    a(k, q) = sn * x + c * y;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    const double x = a(p, k), y = a(q, k);
                    a(p, k) = c * x - sn * y;
                    a(q, k) = sn * x + c * y;
                }
                for (int k = 0; k < n; ++k) {
                    const double x = U[k + (size_t)p * n], y = U[k + (size_t)q * n];
                    U[k + (size_t)p * n] = c * x - sn * y;
                    U[k + (size_t)q * n] = sn * x + c * y;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = a(i, i);
}

// SVQB (Stathopoulos and Wu): for the Gram matrix G of n columns, the transform T with X T
// orthonormal, T = D U diag(w)^-1/2 from D G D = U diag(w) U^T, D = diag(G)^-1/2; directions with
// w <= 1e-14 max(w) are numerically absent and flagged in `drop` (their columns of T are zero).
static void svqb_transform(int n, const std::vector<double>& G, std::vector<double>& T, std::vector<char>& drop) {
    std::vector<double> d(n), S((size_t)n * n), w, U;
    for (int i = 0; i < n; ++i) d[i] = G[i + (size_t)i * n] > 0.0 ? 1.0 / std::sqrt(G[i + (size_t)i * n]) : 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) S[i + (size_t)j * n] = d[i] * G[i + (size_t)j * n] * d[j];
    jacobi_eig(n, S, w, U);
    double wmax = 0.0;
    for (double x : w) wmax = std::max(wmax, x);
    T.assign((size_t)n * n, 0.0);
    drop.assign(n, 0);
    for (int j = 0; j < n; ++j) {
        if (!(w[j] > 1e-14 * wmax)) { drop[j] = 1; continue; }
        const double f = 1.0 / std::sqrt(w[j]);
        for (int i = 0; i < n; ++i) T[i + (size_t)j * n] = d[i] * U[i + (size_t)j * n] * f;
    }
}

// Eigenpairs of a small dense real matrix G (k x k, column-major): lam[k], Y (k x k complex,
// column-major, unit 2-norm columns).
static void small_eig(int k, const std::vector<double>& G, std::vector<cd>& lam, std::vector<cd>& Y) {
    std::vector<cd> T((size_t)k * k), Q((size_t)k * k, cd(0.0));  // row-major
    auto t = [&](int i, int j) -> cd& { return T[(size_t)i * k + j]; };
    auto q = [&](int i, int j) -> cd& { return Q[(size_t)i * k + j]; };
    double gnorm = 0.0;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            t(i, j) = G[i + (size_t)j * k];
            gnorm = std::max(gnorm, std::abs(G[i + (size_t)j * k]));
        }
    for (int i = 0; i < k; ++i) q(i, i) = 1.0;
    // Householder reduction to upper Hessenberg form: T <- H T H, Q <- Q H
    std::vector<cd> v(k);
    for (int c = 0; c + 2 < k; ++c) {
        double a2 = 0.0;
        for (int r = c + 1; r < k; ++r) a2 += std::norm(t(r, c));
        const double alpha = std::sqrt(a2);
        if (alpha == 0.0) continue;
        const cd x0 = t(c + 1, c);
        const cd ph = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cd(1.0);
        std::fill(v.begin(), v.end(), cd(0.0));
        v[c + 1] = x0 + ph * alpha;
        for (int r = c + 2; r < k; ++r) v[r] = t(r, c);
        double vn2 = 0.0;
        for (int r = c + 1; r < k; ++r) vn2 += std::norm(v[r]);
        if (vn2 == 0.0) continue;
        const double f = 2.0 / vn2;
        for (int j = 0; j < k; ++j) {
            cd sacc = 0.0;
            for (int r = c + 1; r < k; ++r) sacc += std::conj(v[r]) * t(r, j);
            sacc *= f;
            for (int r = c + 1; r < k; ++r) t(r, j) -= v[r] * sacc;
        }
        for (int i = 0; i < k; ++i) {
            cd sacc = 0.0;
            for (int r = c + 1; r < k; ++r) sacc += t(i, r) * v[r];
            sacc *= f;
            for (int r = c + 1; r < k; ++r) t(i, r) -= sacc * std::conj(v[r]);
        }
        for (int i = 0; i < k; ++i) {
            cd sacc = 0.0;
            for (int r = c + 1; r < k; ++r) sacc += q(i, r) * v[r];
            sacc *= f;
            for (int r = c + 1; r < k; ++r) q(i, r) -= sacc * std::conj(v[r]);
        }
        for (int r = c + 2; r < k; ++r) t(r, c) = 0.0;
    }
    // shifted QR iterations (implicit single shift, Givens rotations), deflating from the bottom
    int hi = k - 1, iter = 0, total = 0;
    const double eps = 1e-15;
    while (hi > 0 && total < 60 * k) {
        int l = hi;
        while (l > 0) {
            const double sc = std::abs(t(l, l)) + std::abs(t(l - 1, l - 1));
            if (std::abs(t(l, l - 1)) <= eps * (sc > 0.0 ? sc : gnorm)) {
                t(l, l - 1) = 0.0;
                break;
            }
            --l;
        }
        if (l == hi) {
            --hi;
            iter = 0;
            continue;
        }
        ++iter;
        ++total;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer its last entry
        const cd a = t(hi - 1, hi - 1), b = t(hi - 1, hi), c = t(hi, hi - 1), d = t(hi, hi);
        const cd tr = a + d, det = a * d - b * c;
        const cd disc = std::sqrt(tr * tr * 0.25 - det);
        const cd m1 = tr * 0.5 + disc, m2 = tr * 0.5 - disc;
        cd mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
        if (iter % 10 == 0) mu = d + cd(0.75 * std::abs(t(hi, hi - 1)), 0.25 * std::abs(t(hi, hi - 1)));  // exceptional shift
        cd x = t(l, l) - mu, y = t(l + 1, l);
        for (int j = l; j < hi; ++j) {
            const double r = std::sqrt(std::norm(x) + std::norm(y));
            double cs;
            cd sn;
            if (r == 0.0) { cs = 1.0; sn = 0.0; }
            else if (std::abs(x) == 0.0) { cs = 0.0; sn = std::conj(y) / r; }
            else { cs = std::abs(x) / r; sn = (x / std::abs(x)) * std::conj(y) / r; }
            for (int qq = (j > l ? j - 1 : l); qq < k; ++qq) {
                const cd t1 = t(j, qq), t2 = t(j + 1, qq);
                t(j, qq) = cs * t1 + sn * t2;
                t(j + 1, qq) = -std::conj(sn) * t1 + cs * t2;
            }
            for (int qq = 0; qq <= std::min(j + 2, hi); ++qq) {
                const cd t1 = t(qq, j), t2 = t(qq, j + 1);
                t(qq, j) = cs * t1 + std::conj(sn) * t2;
                t(qq, j + 1) = -sn * t1 + cs * t2;
            }
            for (int qq = 0; qq < k; ++qq) {
                const cd t1 = q(qq, j), t2 = q(qq, j + 1);
                q(qq, j) = cs * t1 + std::conj(sn) * t2;
                q(qq, j + 1) = -sn * t1 + cs * t2;
            }
            if (j + 1 < hi) {
                x = t(j + 1, j);
                y = t(j + 2, j);
            }
        }
    }
    // eigenvectors of the triangular factor, mapped back by Q
    lam.resize(k);
    Y.assign((size_t)k * k, cd(0.0));
    std::vector<cd> z(k);
    for (int e = 0; e < k; ++e) {
        lam[e] = t(e, e);
        std::fill(z.begin(), z.end(), cd(0.0));
        z[e] = 1.0;
        for (int i = e - 1; i >= 0; --i) {
            cd sacc = 0.0;
            for (int j = i + 1; j <= e; ++j) sacc += t(i, j) * z[j];
            cd den = t(i, i) - lam[e];
            if (std::abs(den) < 1e-14 * gnorm) den = 1e-14 * gnorm;
            z[i] = -sacc / den;
        }
        double nn = 0.0;
        for (int i = 0; i < k; ++i) {
            cd sacc = 0.0;
            for (int j = 0; j <= e; ++j) sacc += q(i, j) * z[j];
            Y[i + (size_t)e * k] = sacc;
            nn += std::norm(sacc);
        }
        nn = std::sqrt(nn);
        // phase: the largest component real and positive
        int p = 0;
        for (int i = 1; i < k; ++i)
            if (std::abs(Y[i + (size_t)e * k]) > std::abs(Y[p + (size_t)e * k])) p = i;
        const cd ph = std::abs(Y[p + (size_t)e * k]) > 0.0 ? std::conj(Y[p + (size_t)e * k]) / std::abs(Y[p + (size_t)e * k]) : cd(1.0);
        for (int i = 0; i < k; ++i) Y[i + (size_t)e * k] *= ph / nn;
    }
}

// orthonormalise the b columns of X (N x b) against Vb (N x k, orthonormal) and among themselves
// (two rounds of Gram-Schmidt against Vb, then SVQB twice); numerically absent directions are
// replaced by random columns (seeded) and the whole is repeated
static void orthonormalise(Ts& w, Temp<double>& sdev, const double* Vb, int k, double* X, int b, int64_t N,
                           unsigned long long& seed, cudaStream_t s) {
    std::vector<double> C, G, T;
    std::vector<char> drop;
    Temp<double> tmp((int64_t)N * b, s);
    for (int attempt = 0; attempt < 6; ++attempt) {
        for (int pass = 0; pass < 2; ++pass) {
            if (k > 0) {
                tsgemm_tn(w, Vb, k, X, b, N, C, s);
                tsgemm_nn(sdev, Vb, k, C, b, N, X, true, s);
            }
        }
        bool good = true;
        for (int pass = 0; pass < 2; ++pass) {
            tsgemm_tn(w, X, b, X, b, N, G, s);
            svqb_transform(b, G, T, drop);
            CK(cudaMemcpyAsync(tmp.get(), X, sizeof(double) * N * b, cudaMemcpyDeviceToDevice, s));
            tsgemm_nn(sdev, tmp.get(), b, T, b, N, X, false, s);
            bool any = false;
            for (int j = 0; j < b; ++j)
                if (drop[j]) {
                    any = true;
                    fill_uniform_k<<<grid_for(N, 256), 256, 0, s>>>(X + (int64_t)j * N, N, seed);
                    CK_LAUNCH();
                    seed += 0x9E3779B97F4A7C15ull;
                }
            if (any) { good = false; break; }
        }
        if (good) return;
    }
    fail(MGM_ERR_BREAKDOWN, "eigensolver: could not orthonormalise a block");
}

void eigs(mgm_hierarchy* H, int nev, int b, int s_steps, int max_cycles, double tol, const mgm_solve_params* sp,
          uint64_t seed0, double* lam_re, double* lam_im, double* evec, double* resid, int* nconv, int* nsolves,
          cudaStream_t s) {
    REQUIRE(H && sp && lam_re && lam_im && nconv && nsolves, "null argument");
    REQUIRE(!H->bordered, "eigenpairs: not for constrained (bordered) hierarchies");
    REQUIRE(b >= 1 && b <= 8, "block size must be in [1, 8]");
    REQUIRE(nev >= 1 && s_steps >= 1 && max_cycles >= 1 && tol > 0.0, "bad eigensolver parameters");
    const int keep = nev + b;
    const int cap = keep + s_steps * b;
    REQUIRE(cap <= TS_MAXC, "nev + (s + 1) b must be <= 96");
    const int64_t N = H->N;
    REQUIRE(N >= cap, "basis larger than the problem");
    Temp<double> V((int64_t)N * cap, s), W((int64_t)N * cap, s), V2((int64_t)N * keep, s), W2((int64_t)N * keep, s);
    Temp<double> B((int64_t)N * b, s), Rb((int64_t)N * keep, s);
    Ts ts;
    Temp<double> sdev;
    unsigned long long seed = seed0 * 0x2545F4914F6CDD1Dull + 12345ull;
    fill_uniform_k<<<grid_for(N * b, 256), 256, 0, s>>>(B.get(), N * b, seed);
    CK_LAUNCH();
    seed += 0x9E3779B97F4A7C15ull;
    int k = 0, solves = 0;
    std::vector<cd> lam, Y;
    std::vector<double> G;
    for (int cycle = 0;; ++cycle) {
        // expansion: s_steps blocks of the block Krylov sequence
        for (int j = 0; j < s_steps; ++j) {
            orthonormalise(ts, sdev, V.get(), k, B.get(), b, N, seed, s);
            CK(cudaMemcpyAsync(V.get() + (int64_t)k * N, B.get(), sizeof(double) * N * b, cudaMemcpyDeviceToDevice, s));
            CK(cudaMemsetAsync(W.get() + (int64_t)k * N, 0, sizeof(double) * N * b, s));
            std::vector<mgm_solve_info> info(b);
            for (auto& x : info) x = mgm_solve_info{};
            solve_multi(H, b, V.get() + (int64_t)k * N, W.get() + (int64_t)k * N, sp, info.data(), s);
            solves += b;
            k += b;
            CK(cudaMemcpyAsync(B.get(), W.get() + (int64_t)(k - b) * N, sizeof(double) * N * b, cudaMemcpyDeviceToDevice, s));
        }
        // Rayleigh-Ritz: G = V^T W, Ritz values theta in decreasing magnitude
        tsgemm_tn(ts, V.get(), k, W.get(), k, N, G, s);
        small_eig(k, G, lam, Y);
        std::vector<int> order(k);
        for (int i = 0; i < k; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return std::abs(lam[a]) > std::abs(lam[c]); });
        // real basis Yk of the wanted Ritz vectors with V^T A V Yk ~ Yk Th: a real theta gives
        // Re(y) and Th = theta; a complex pair gives (Re y, Im y) and the block
        // [[Re theta, Im theta], [-Im theta, Re theta]]
        std::vector<double> Yk;
        std::vector<cd> thc;         // eigenvalue of each column (conjugate for the second of a pair)
        std::vector<int> pair;      // 0 real, 1 first of a pair, 2 second
        std::vector<char> used(k, 0);
        for (int t = 0; t < k && (int)thc.size() < keep; ++t) {
            const int e = order[t];
            if (used[e]) continue;
            used[e] = 1;
            const bool cplx = std::abs(lam[e].imag()) > 1e-10 * std::abs(lam[e]);
            if (cplx) {
                for (int u = t + 1; u < k; ++u)
                    if (!used[order[u]] && std::abs(lam[order[u]] - std::conj(lam[e])) < 1e-8 * std::abs(lam[e])) {
                        used[order[u]] = 1;
                        break;
                    }
                if ((int)thc.size() + 2 > keep) break;
                for (int part = 0; part < 2; ++part) {
                    for (int i = 0; i < k; ++i)
                        Yk.push_back(part == 0 ? Y[i + (size_t)e * k].real() : Y[i + (size_t)e * k].imag());
                    thc.push_back(part == 0 ? lam[e] : std::conj(lam[e]));
                    pair.push_back(part + 1);
                }
            } else {
                for (int i = 0; i < k; ++i) Yk.push_back(Y[i + (size_t)e * k].real());
                thc.push_back(cd(lam[e].real(), 0.0));
                pair.push_back(0);
            }
        }
        const int q = (int)thc.size();
        // Yk Th (k x q)
        std::vector<double> YT((size_t)k * q);
        for (int c = 0; c < q; ++c) {
            const double tr = thc[c].real();
            for (int i = 0; i < k; ++i) {
                double v = Yk[i + (size_t)c * k] * tr;
                if (pair[c] == 1) v -= Yk[i + (size_t)(c + 1) * k] * thc[c].imag();      // A yr = tr yr - ti yi
                if (pair[c] == 2) v += Yk[i + (size_t)(c - 1) * k] * thc[c - 1].imag();  // A yi = ti yr + tr yi
                YT[i + (size_t)c * k] = v;
            }
        }
        // residual vectors R = W Yk - V Yk Th and relative norms (pairs: the norm of both columns)
        std::vector<double> rn(q, 0.0), r2(q, 0.0), y2(q, 0.0);
        for (int j0 = 0; j0 < q; j0 += 16) {
            const int lj = std::min(16, q - j0);
            double* Rj = Rb.get() + (int64_t)j0 * N;
            std::vector<double> Sj(Yk.begin() + (size_t)j0 * k, Yk.begin() + (size_t)(j0 + lj) * k);
            tsgemm_nn(sdev, W.get(), k, Sj, lj, N, Rj, false, s);
            std::vector<double> Tj(YT.begin() + (size_t)j0 * k, YT.begin() + (size_t)(j0 + lj) * k);
            tsgemm_nn(sdev, V.get(), k, Tj, lj, N, Rj, true, s);
            std::vector<double> RR;
            tsgemm_tn(ts, Rj, lj, Rj, lj, N, RR, s);
            for (int c = 0; c < lj; ++c) r2[j0 + c] = std::max(RR[c + (size_t)c * lj], 0.0);
        }
        for (int c = 0; c < q; ++c)
            for (int i = 0; i < k; ++i) y2[c] += Yk[i + (size_t)c * k] * Yk[i + (size_t)c * k];  // ||V y|| = ||y||
        for (int c = 0; c < q; ++c) {
            const int c0 = pair[c] == 2 ? c - 1 : c, c1 = pair[c] == 1 ? c + 1 : c;
            double rr = 0.0, yy = 0.0;
            for (int u = c0; u <= c1; ++u) { rr += r2[u]; yy += y2[u]; }
            rn[c] = std::sqrt(rr) / (std::abs(thc[c]) * std::sqrt(yy));
        }
        const int nchk = std::min(nev, q);
        int conv = 0;
        for (int i = 0; i < nchk; ++i) conv += rn[i] <= tol ? 1 : 0;
        if (conv >= nev || cycle + 1 >= max_cycles) {
            // outputs: eigenvalues of L = 1 / theta; eigenvectors V y (unit norm; a complex pair: the
            // real and imaginary parts of the first eigenvalue's eigenvector)
            for (int i = 0; i < nev; ++i) {
                const cd th = i < q ? thc[i] : cd(0.0);
                const cd ev = std::abs(th) > 0.0 ? 1.0 / th : cd(0.0);
                lam_re[i] = ev.real();
                lam_im[i] = ev.imag();
                if (resid) resid[i] = i < q ? rn[i] : -1.0;
            }
            if (evec) {
                const int ne = std::min(nev, q);
                std::vector<double> Sx(Yk.begin(), Yk.begin() + (size_t)ne * k);
                for (int c = 0; c < ne; ++c) {  // a pair shares one factor: (Re y, Im y) stays an eigenvector
                    const int c0 = pair[c] == 2 ? c - 1 : c, c1 = pair[c] == 1 ? c + 1 : c;
                    double yy = 0.0;
                    for (int u = c0; u <= c1 && u < q; ++u) yy += y2[u];
                    const double f = 1.0 / std::sqrt(std::max(yy, 1e-300));
                    for (int i = 0; i < k; ++i) Sx[i + (size_t)c * k] *= f;
                }
                tsgemm_nn_wide(sdev, V.get(), k, Sx, ne, N, evec, s);
            }
            *nconv = conv;
            break;
        }
        // the next block: residuals of the least converged wanted pairs (then of the other kept
        // ones; random columns if fewer than b remain)
        std::vector<int> pick;
        for (int i = 0; i < nchk; ++i)
            if (rn[i] > tol) pick.push_back(i);
        std::stable_sort(pick.begin(), pick.end(), [&](int a, int c) { return rn[a] > rn[c]; });
        for (int i = nchk; i < q && (int)pick.size() < b; ++i) pick.push_back(i);
        if ((int)pick.size() > b) pick.resize(b);
        for (int c = 0; c < b; ++c) {
            if (c < (int)pick.size()) {
                CK(cudaMemcpyAsync(B.get() + (int64_t)c * N, Rb.get() + (int64_t)pick[c] * N, sizeof(double) * N,
                                   cudaMemcpyDeviceToDevice, s));
            } else {
                fill_uniform_k<<<grid_for(N, 256), 256, 0, s>>>(B.get() + (int64_t)c * N, N, seed);
                CK_LAUNCH();
                seed += 0x9E3779B97F4A7C15ull;
            }
        }
        // thick restart: V <- V Yk T, W <- W Yk T with T from SVQB (twice); absent directions dropped
        tsgemm_nn_wide(sdev, V.get(), k, Yk, q, N, V2.get(), s);
        tsgemm_nn_wide(sdev, W.get(), k, Yk, q, N, W2.get(), s);
        int qk = q;
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<double> GG, T;
            std::vector<char> drop;
            tsgemm_tn(ts, V2.get(), qk, V2.get(), qk, N, GG, s);
            svqb_transform(qk, GG, T, drop);
            std::vector<double> Tc;  // kept columns only
            int nk = 0;
            for (int j = 0; j < qk; ++j)
                if (!drop[j]) {
                    Tc.insert(Tc.end(), T.begin() + (size_t)j * qk, T.begin() + (size_t)(j + 1) * qk);
                    ++nk;
                }
            tsgemm_nn_wide(sdev, V2.get(), qk, Tc, nk, N, V.get(), s);
            tsgemm_nn_wide(sdev, W2.get(), qk, Tc, nk, N, W.get(), s);
            qk = nk;
            if (pass == 0) {
                CK(cudaMemcpyAsync(V2.get(), V.get(), sizeof(double) * N * qk, cudaMemcpyDeviceToDevice, s));
                CK(cudaMemcpyAsync(W2.get(), W.get(), sizeof(double) * N * qk, cudaMemcpyDeviceToDevice, s));
            }
        }
        k = qk;
    }
    *nsolves = solves;
}

}  // namespace mgm

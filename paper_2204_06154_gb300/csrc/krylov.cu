// Outer solver (paper Sec. 4.6 and Sec. 5): right-preconditioned flexible GMRES(restart) in FP64
// with one MGM V-cycle per iteration, or MGM as a standalone iteration (Sec. 5.1).
//
// All vectors live on the device in the level-0 solve order (the caller's f and u are permuted
// once on entry and once on exit). Per iteration: z_k = M v_k (V-cycle, its precision; z_k is
// stored in that precision, FP32 in the mixed mode), w = L z_k in FP64, classical Gram-Schmidt
// with one reorthogonalisation (CGS2: two passes of "h = V^T w; w -= V h"), then |w|. The dot
// products use fixed per-block partial sums and a fixed reduction order, so results repeat
// exactly from run to run. The (k+1)-vector of coefficients goes to the host, where the Givens
// rotations and the convergence test run (one synchronisation per iteration). The solution is
// updated at restarts and at exit, and the true FP64 residual |f - L u| decides convergence.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "hier.cuh"

namespace mgm {

void add_output(mgm_hierarchy* H, double* dst, const int32_t* scatter, cudaStream_t s);

constexpr int KG = 4;            // lanes per row in the FP64 operator (4: 0.189 ms at 1M rows; 8: 0.279; 16: 0.389)
constexpr int KBLOCK = 256;
constexpr int DOT_BLOCKS = 304;  // 2 per SM on 152 SMs

// y = f - L x (RESID) or y = L x, L in solve order (lower and upper parts, diagonal apart). Lane gl
// of KG takes every KG-th quad of entries of the row's lower part, then of its upper part; the
// columns and values of up to two quads, then their gathered x, are loaded before the products,
// so a warp has all of its rows' loads in flight at once (rows of up to 32 entries a part take one round).
// The products are added quad by quad in that order.
template <bool RESID>
__global__ void __launch_bounds__(KBLOCK) spmv64_k(const int32_t* __restrict__ lo, const int32_t* __restrict__ up,
                                                   const int32_t* __restrict__ sc, const double* __restrict__ sv,
                                                   const double* __restrict__ diag, const double* __restrict__ x,
                                                   const double* __restrict__ f, double* y, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * KBLOCK + threadIdx.x;
    const int64_t row = t / KG;
    const int gl = (int)(t & (KG - 1));
    double acc = 0.0;
    if (row < n) {
        const int32_t l0 = lo[row], l1 = lo[row + 1], u0 = up[row], u1 = up[row + 1];
        const int32_t nql = l1 > l0 + 4 * gl ? (l1 - l0 - 4 * gl + 4 * KG - 1) / (4 * KG) : 0;
        const int32_t nqu = u1 > u0 + 4 * gl ? (u1 - u0 - 4 * gl + 4 * KG - 1) / (4 * KG) : 0;
        const int32_t nq = nql + nqu;
#pragma unroll 1
        for (int32_t t0 = 0; t0 < nq; t0 += 2) {
            int4 c[2];
            double2 va[2], vb[2];
            double xv[2][4];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int32_t k = t0 + q;
                if (k < nq) {
                    const int32_t p = k < nql ? l0 + 4 * (gl + KG * k) : u0 + 4 * (gl + KG * (k - nql));
                    c[q] = __ldcs(reinterpret_cast<const int4*>(sc + p));
                    va[q] = __ldcs(reinterpret_cast<const double2*>(sv + p));
                    vb[q] = __ldcs(reinterpret_cast<const double2*>(sv + p + 2));
                }
            }
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (t0 + q < nq) {
                    xv[q][0] = x[c[q].x];
                    xv[q][1] = x[c[q].y];
                    xv[q][2] = x[c[q].z];
                    xv[q][3] = x[c[q].w];
                }
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (t0 + q < nq) {
                    acc = fma(va[q].x, xv[q][0], acc);
                    acc = fma(va[q].y, xv[q][1], acc);
                    acc = fma(vb[q].x, xv[q][2], acc);
                    acc = fma(vb[q].y, xv[q][3], acc);
                }
        }
    }
    for (int o = KG / 2; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (row < n && gl == 0) {
        double lx = fma(diag[row], x[row], acc);
        y[row] = RESID ? f[row] - lx : lx;
    }
}

// xd = (double) x
__global__ void widen_k(const float* __restrict__ x, double* __restrict__ xd, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xd[i] = (double)x[i];
}

// partial[b * k1 + t] = sum over block b's chunk of V_t . w
__global__ void __launch_bounds__(256) multidot_k(const double* __restrict__ V, int64_t ldv, int k1,
                                                  const double* __restrict__ w, int64_t n, double* partial) {
    __shared__ double red[8];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    for (int t = 0; t < k1; ++t) {
        const double* v = V + (int64_t)t * ldv;
        double acc = 0.0;
        for (int64_t i = b0 + threadIdx.x; i < b1; i += 256) acc = fma(v[i], w[i], acc);
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < 8; ++q) s += red[q];
            partial[(int64_t)blockIdx.x * k1 + t] = s;
        }
        __syncthreads();
    }
}
// h[t] = sum_b partial[b * k1 + t] (one warp per t; fixed order)
__global__ void reduce_partials_k(const double* partial, int nb, int k1, double* h) {
    int t = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) acc += partial[(int64_t)b * k1 + t];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) h[t] = acc;
}
// w -= V h (k1 vectors)
__global__ void multiaxpy_k(const double* __restrict__ V, int64_t ldv, int k1, const double* __restrict__ h, double* w,
                            int64_t n) {
    __shared__ double sh[256];
    for (int t = threadIdx.x; t < k1; t += blockDim.x) sh[t] = h[t];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = w[i];
    for (int t = 0; t < k1; ++t) acc = fma(-sh[t], V[(int64_t)t * ldv + i], acc);
    w[i] = acc;
}
// x += Z y
template <class TZ>
__global__ void update_x_k(const TZ* __restrict__ Z, int64_t ldz, int k, const double* __restrict__ y, double* x, int64_t n) {
    __shared__ double sy[256];
    for (int t = threadIdx.x; t < k; t += blockDim.x) sy[t] = y[t];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = x[i];
    for (int t = 0; t < k; ++t) acc = fma(sy[t], (double)Z[(int64_t)t * ldz + i], acc);
    x[i] = acc;
}
__global__ void scale_k(const double* a, double s, double* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i] * s;
}
__global__ void gather64_k(const double* in, const int32_t* idx, double* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[idx[i]];
}
__global__ void scatter64_k(const double* in, const int32_t* idx, double* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[idx[i]] = in[i];
}

// Bordered operator of Sec. 4.4 on (n+1)-vectors [u; lambda]: [L u + lambda 1; 1 . u]. The border
// sum uses fixed block partials (deterministic); y_n = f_n - sum for the residual form.
template <class TX>
__global__ void __launch_bounds__(256) bsum_k(const TX* __restrict__ x, int64_t n, double* part) {
    __shared__ double red[8];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    double acc = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += 256) acc += (double)x[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q];
        part[blockIdx.x] = t;
    }
}
__global__ void bsum_final_k(const double* part, int nb, const double* f_last, double* y_last) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) acc += part[b];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) *y_last = f_last ? *f_last - acc : acc;
}
// y_i += sign * lambda, lambda = x[n]
template <class TX>
__global__ void badd_k(const TX* lam, double* y, int64_t n, double sign) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = y[i] + sign * (double)*lam;
}
template <class TA, class TB>
__global__ void copy1_k(const TA* a, TB* b) { *b = (TB)*a; }

// BiCGSTAB updates: p = r + beta (p - omega v); s = r - alpha v; x += alpha ph + omega sh, r = s - omega t
__global__ void bicg_p_k(const double* r, const double* v, double* p, double beta, double omega, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = r[i] + beta * (p[i] - omega * v[i]);
}
__global__ void bicg_s_k(const double* r, const double* v, double* sv, double alpha, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sv[i] = r[i] - alpha * v[i];
}
__global__ void bicg_x_k(double* x, const double* ph, const double* sh, double alpha, double omega, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = x[i] + alpha * ph[i] + omega * (sh ? sh[i] : 0.0);
}
__global__ void bicg_r_k(const double* sv, const double* t, double* r, double omega, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = sv[i] - omega * t[i];
}

// ------------------------------ host side -------------------------------------------------------
struct Ops {
    mgm_hierarchy* H;
    cudaStream_t s;
    int64_t n;   // rows of L
    int64_t nv;  // length of the outer vectors: n, or n + 1 (bordered: [u; lambda])
    Level& L0() { return H->lv[0]; }

    // An FP32 x is widened once into an FP64 copy first: the product then converts n values
    // instead of one per stored entry (each conversion is an FP64-pipe instruction, and the FP64
    // pipe, not HBM, would otherwise bound the product). The result is the same bit for bit.
    template <bool RESID, class TX>
    void spmv(const TX* x, const double* f, double* y) {
        Level& L = L0();
        const double* xd;
        if constexpr (std::is_same<TX, float>::value) {
            widen_k<<<grid_for(n, 256), 256, 0, s>>>(x, H->zd.get(), n);
            CK_LAUNCH();
            xd = H->zd.get();
        } else {
            xd = x;
        }
        spmv64_k<RESID><<<grid_for(n * KG, KBLOCK), KBLOCK, 0, s>>>(L.lo.get(), L.up.get(), L.sc.get(), L.sv64.get(), L.diag64.get(),
                                                                   xd, f, y, n);
        CK_LAUNCH();
    }
    // y = f - L~ x (RESID) or y = L~ x, with the border of Sec. 4.4 when the hierarchy has one
    template <bool RESID, class TX>
    void op_apply(const TX* x, const double* f, double* y) {
        spmv<RESID, TX>(x, f, y);
        if (!H->bordered) return;
        badd_k<TX><<<grid_for(n, 256), 256, 0, s>>>(x + n, y, n, RESID ? -1.0 : 1.0);
        CK_LAUNCH();
        bsum_k<TX><<<DOT_BLOCKS, 256, 0, s>>>(x, n, H->part.get());
        CK_LAUNCH();
        bsum_final_k<<<1, 32, 0, s>>>(H->part.get(), DOT_BLOCKS, RESID ? f + n : nullptr, y + n);
        CK_LAUNCH();
    }
    // z = M v: one V-cycle (bordered: v_n is the constraint component, z_n the multiplier)
    template <class TZ>
    void precondition(const double* v, TZ* z) {
        load_input(H, v, MGM_F64, nullptr, s);
        if (H->bordered) {
            copy1_k<double, double><<<1, 1, 0, s>>>(v + n, H->sres.get());
            CK_LAUNCH();
        }
        vcycle_core(H, s);
        store_output(H, z, std::is_same<TZ, float>::value ? MGM_F32 : MGM_F64, nullptr, s);
        if (H->bordered) {
            Level& C = H->lv[H->p - 1];
            if (H->precision == MGM_F32) copy1_k<float, TZ><<<1, 1, 0, s>>>(C.e32.get() + H->np, z + n);
            else copy1_k<double, TZ><<<1, 1, 0, s>>>(C.e64.get() + H->np, z + n);
            CK_LAUNCH();
        }
    }
    // h (device, k1 entries) = V[0..k1)^T w
    void dots(const double* V, int64_t ldv, int k1, const double* w, double* h) {
        multidot_k<<<DOT_BLOCKS, 256, 0, s>>>(V, ldv, k1, w, nv, H->part.get());
        CK_LAUNCH();
        reduce_partials_k<<<k1, 32, 0, s>>>(H->part.get(), DOT_BLOCKS, k1, h);
        CK_LAUNCH();
    }
    void axpys(const double* V, int64_t ldv, int k1, const double* h, double* w) {
        multiaxpy_k<<<grid_for(nv, 256), 256, 0, s>>>(V, ldv, k1, h, w, nv);
        CK_LAUNCH();
    }
    double norm(const double* w) {
        dots(w, nv, 1, w, H->hbuf.get());
        double v = read1(H->hbuf.get(), s);
        return std::sqrt(v);
    }
    double dot(const double* a, const double* b) {
        dots(a, nv, 1, b, H->hbuf.get());
        return read1(H->hbuf.get(), s);
    }
};

// Right-preconditioned BiCGSTAB (paper Sec. 4.6: MGM as the preconditioner of BiCGSTAB), FP64,
// two V-cycles per step; `it` counts V-cycles. Returns the status; u, rel, hist updated.
static mgm_status bicgstab(mgm_hierarchy* H, Ops& op, const mgm_solve_params* sp, double fn, std::vector<double>& hist,
                           int& it, double& rel) {
    const int64_t n = op.n;
    cudaStream_t s = op.s;
    double* W = H->V.get();  // 8 work vectors
    double *r = W, *rh = W + n, *p = W + 2 * n, *v = W + 3 * n, *ph = W + 4 * n, *sv = W + 5 * n, *sh = W + 6 * n,
           *t = W + 7 * n;
    double* u = H->u.get();
    const unsigned gb = grid_for(n, 256);
    op.spmv<true, double>(u, H->f.get(), r);
    CK(cudaMemcpyAsync(rh, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(p, 0, sizeof(double) * n, s));
    CK(cudaMemsetAsync(v, 0, sizeof(double) * n, s));
    rel = op.norm(r) / fn;
    hist.push_back(rel);
    if (!std::isfinite(rel)) return MGM_ERR_BREAKDOWN;
    if (rel <= sp->tol) return MGM_OK;
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    mgm_status st = MGM_ERR_NOT_CONVERGED;
    while (it + 1 <= sp->maxit) {
        const double rho = op.dot(rh, r);
        if (rho == 0.0 || !std::isfinite(rho)) { st = MGM_ERR_BREAKDOWN; break; }
        const double beta = (rho / rho_old) * (alpha / omega);
        bicg_p_k<<<gb, 256, 0, s>>>(r, v, p, beta, omega, n);
        CK_LAUNCH();
        op.precondition(p, ph);
        ++it;
        op.spmv<false, double>(ph, nullptr, v);
        alpha = rho / op.dot(rh, v);
        bicg_s_k<<<gb, 256, 0, s>>>(r, v, sv, alpha, n);
        CK_LAUNCH();
        rel = op.norm(sv) / fn;
        hist.push_back(rel);
        if (!std::isfinite(rel)) { st = MGM_ERR_BREAKDOWN; break; }
        if (rel <= sp->tol || it + 1 > sp->maxit) {
            bicg_x_k<<<gb, 256, 0, s>>>(u, ph, nullptr, alpha, 0.0, n);
            CK_LAUNCH();
            break;
        }
        op.precondition(sv, sh);
        ++it;
        op.spmv<false, double>(sh, nullptr, t);
        const double tt = op.dot(t, t);
        if (tt == 0.0 || !std::isfinite(tt)) {
            bicg_x_k<<<gb, 256, 0, s>>>(u, ph, nullptr, alpha, 0.0, n);
            CK_LAUNCH();
            st = MGM_ERR_BREAKDOWN;
            break;
        }
        omega = op.dot(t, sv) / tt;
        bicg_x_k<<<gb, 256, 0, s>>>(u, ph, sh, alpha, omega, n);
        CK_LAUNCH();
        bicg_r_k<<<gb, 256, 0, s>>>(sv, t, r, omega, n);
        CK_LAUNCH();
        rel = op.norm(r) / fn;
        hist.push_back(rel);
        if (!std::isfinite(rel)) { st = MGM_ERR_BREAKDOWN; break; }
        if (rel <= sp->tol) break;
        rho_old = rho;
    }
    // the true residual decides
    op.spmv<true, double>(u, H->f.get(), r);
    rel = op.norm(r) / fn;
    if (st != MGM_ERR_BREAKDOWN) st = rel <= sp->tol ? MGM_OK : MGM_ERR_NOT_CONVERGED;
    return st;
}

static void ensure_workspace(mgm_hierarchy* H, int m) {
    const int64_t n = H->N + (H->bordered ? 1 : 0);
    if (H->krylov_m >= m && H->V.get()) return;
    H->V.alloc((int64_t)(m + 1) * n);
    if (H->precision == MGM_F32) {
        H->Z32.alloc((int64_t)m * n);
        H->zd.alloc(n);
    } else {
        H->Z64.alloc((int64_t)m * n);
    }
    H->f.alloc(n); H->u.alloc(n); H->w.alloc(n); H->r.alloc(n);
    H->part.alloc((int64_t)DOT_BLOCKS * (2 * (m + 1) + 2));
    H->hbuf.alloc(2 * (m + 2) + 2);
    H->ydev.alloc(m + 1);
    if (H->hhost) cudaFreeHost(H->hhost);
    H->hhost = nullptr;
    CK(cudaMallocHost((void**)&H->hhost, sizeof(double) * (2 * (m + 2) + 2)));
    H->krylov_m = m;
}

// times the FP64 operator application w = L z of the outer iteration (z in the V-cycle precision)
void profile_spmv(mgm_hierarchy* H, int reps, mgm_profile_info* out, cudaStream_t s) {
    ensure_workspace(H, std::max(H->krylov_m, 1));
    const int64_t n = H->N;
    Ops op{H, s, n, n};
    Level& L = H->lv[0];
    const bool f32 = H->precision == MGM_F32;
    if (f32) CK(cudaMemsetAsync(H->Z32.get(), 0, sizeof(float) * n, s));
    else CK(cudaMemsetAsync(H->Z64.get(), 0, sizeof(double) * n, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int t = 0; t < reps + 2; ++t) {
        if (t == 2) CK(cudaEventRecord(e0, s));
        if (f32) op.spmv<false, float>(H->Z32.get(), nullptr, H->w.get());
        else op.spmv<false, double>(H->Z64.get(), nullptr, H->w.get());
    }
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out->spmv_ms = ms / reps;
    out->spmv_bytes = (L.nlow + L.nupp) * 12 + n * (4 + 8 + 8 + (f32 ? 4 : 8));
}

// ------------------------------ FGMRES driven on the device -------------------------------------
// The same right-preconditioned FGMRES(m) as the host-driven loop below, with no host
// synchronisation: the restart cycle and the Arnoldi step are the bodies of two nested WHILE
// conditional nodes of one CUDA graph; one-thread kernels apply the Givens rotations, test
// convergence and set the loop conditions (cudaGraphSetConditional); the Arnoldi index k lives in
// device memory and the kernels that depend on it read it there. Launched once per solve (or as a
// child of a larger graph, e.g. a time step), it leaves the iteration count, the last true relative
// residual and the estimates in device memory.
enum { GS_FN = 0, GS_TOL, GS_BETA, GS_REL, GS_EST, GS_INV, GS_G };  // doubles; then g (m+1), cs, sn (m), Hm ((m+1) m), y (m)
enum { GI_K = 0, GI_IT, GI_CONV, GI_MAXIT, GI_NH };                 // ints

__device__ __forceinline__ double* gs_g(double* d) { return d + GS_G; }
__device__ __forceinline__ double* gs_cs(double* d, int m) { return d + GS_G + (m + 1); }
__device__ __forceinline__ double* gs_sn(double* d, int m) { return d + GS_G + (m + 1) + m; }
__device__ __forceinline__ double* gs_hm(double* d, int m) { return d + GS_G + (m + 1) + 2 * m; }
__device__ __forceinline__ double* gs_y(double* d, int m) { return d + GS_G + (m + 1) + 2 * m + (m + 1) * m; }

__global__ void gs_start_k(const double* hb, double* d, int* iv, cudaGraphConditionalHandle ho) {
    double fn = sqrt(hb[0]);
    iv[GI_IT] = 0;
    iv[GI_K] = 0;
    iv[GI_NH] = 0;
    if (!isfinite(fn)) { iv[GI_CONV] = 2; cudaGraphSetConditional(ho, 0); return; }
    if (fn == 0.0) fn = 1.0;
    d[GS_FN] = fn;
    iv[GI_CONV] = 0;
    cudaGraphSetConditional(ho, 1);
}
// start of a restart cycle from r = f - L u (beta = |r|): converged, out of iterations, or g = beta e1
__global__ void gs_cycle_k(const double* hb, double* d, int* iv, double* hist, int m, cudaGraphConditionalHandle ho,
                           cudaGraphConditionalHandle hi) {
    const double beta = sqrt(hb[0]);
    const double rel = beta / d[GS_FN];
    d[GS_REL] = rel;
    iv[GI_K] = 0;
    if (iv[GI_NH] == 0) hist[iv[GI_NH]++] = rel;
    bool stop = false;
    if (!isfinite(rel)) { iv[GI_CONV] = 2; stop = true; }
    else if (rel <= d[GS_TOL]) { iv[GI_CONV] = 1; stop = true; }
    else if (iv[GI_IT] >= iv[GI_MAXIT]) stop = true;
    if (stop) {
        cudaGraphSetConditional(ho, 0);
        cudaGraphSetConditional(hi, 0);
        return;
    }
    double* g = gs_g(d);
    g[0] = beta;
    for (int i = 1; i <= m; ++i) g[i] = 0.0;
    d[GS_INV] = 1.0 / beta;
    cudaGraphSetConditional(hi, 1);
}
// Arnoldi column k from h = h1 + h2 (two Gram-Schmidt passes) and |w|: rotations, estimate, next k
__global__ void gs_arnoldi_k(const double* hb, double* d, int* iv, double* hist, int m, cudaGraphConditionalHandle hi) {
    const int k = iv[GI_K], k1 = k + 1;
    double* Hm = gs_hm(d, m);
    double* cs = gs_cs(d, m);
    double* sn = gs_sn(d, m);
    double* g = gs_g(d);
    const double* h1 = hb;
    const double* h2 = hb + (m + 1);
    for (int i = 0; i < k1; ++i) Hm[(size_t)i * m + k] = h1[i] + h2[i];
    const double hn = sqrt(hb[2 * (m + 1)]);
    Hm[(size_t)k1 * m + k] = hn;
    if (!isfinite(hn)) {
        iv[GI_CONV] = 2;
        cudaGraphSetConditional(hi, 0);
        return;
    }
    d[GS_INV] = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int i = 0; i < k; ++i) {
        const double a = Hm[(size_t)i * m + k], b = Hm[(size_t)(i + 1) * m + k];
        Hm[(size_t)i * m + k] = cs[i] * a + sn[i] * b;
        Hm[(size_t)(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
    }
    const double a = Hm[(size_t)k * m + k], b = Hm[(size_t)k1 * m + k];
    const double rr = sqrt(a * a + b * b);
    cs[k] = rr == 0.0 ? 1.0 : a / rr;
    sn[k] = rr == 0.0 ? 0.0 : b / rr;
    Hm[(size_t)k * m + k] = rr;
    Hm[(size_t)k1 * m + k] = 0.0;
    g[k1] = -sn[k] * g[k];
    g[k] = cs[k] * g[k];
    const int it = ++iv[GI_IT];
    const double est = fabs(g[k1]) / d[GS_FN];
    d[GS_EST] = est;
    hist[iv[GI_NH]++] = est;
    iv[GI_K] = k1;
    cudaGraphSetConditional(hi, (k1 < m && est > d[GS_TOL] && hn != 0.0 && it < iv[GI_MAXIT]) ? 1 : 0);
}
// y = H(0:k, 0:k)^-1 g(0:k) (back substitution); a breakdown ends the restart loop
__global__ void gs_solve_y_k(double* d, const int* iv, int m, cudaGraphConditionalHandle ho) {
    const int k = iv[GI_K];
    const double* Hm = gs_hm(d, m);
    const double* g = gs_g(d);
    double* y = gs_y(d, m);
    for (int i = k - 1; i >= 0; --i) {
        double acc = g[i];
        for (int j = i + 1; j < k; ++j) acc -= Hm[(size_t)i * m + j] * y[j];
        y[i] = acc / Hm[(size_t)i * m + i];
    }
    if (iv[GI_CONV] == 2) cudaGraphSetConditional(ho, 0);
}
// vector kernels indexed by the device-resident k
template <class T>
__global__ void gs_loadv_k(const double* V, int64_t nv, const int* kp, T* b0, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b0[i] = (T)V[(int64_t)*kp * nv + i];
}
template <class T>
__global__ void gs_storez_k(const T* e0, T* Z, int64_t nv, const int* kp, double* zd, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T v = e0[i];
    Z[(int64_t)*kp * nv + i] = v;
    zd[i] = (double)v;
}
__global__ void gs_scale0_k(double* V, const double* inv, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) V[i] = V[i] * *inv;
}
__global__ void gs_scalek_k(const double* w, double* V, int64_t nv, const int* kp, const double* inv, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) V[(int64_t)*kp * nv + i] = w[i] * *inv;
}
// partial[b * m1 + t] = block b's part of V_t . w, t < k + 1 (k from the device)
__global__ void __launch_bounds__(256) gs_multidot_k(const double* __restrict__ V, int64_t ldv, const int* kp, int m1,
                                                     const double* __restrict__ w, int64_t n, double* partial) {
    __shared__ double red[8];
    const int k1 = *kp + 1;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    for (int t = 0; t < k1; ++t) {
        const double* v = V + (int64_t)t * ldv;
        double acc = 0.0;
        for (int64_t i = b0 + threadIdx.x; i < b1; i += 256) acc = fma(v[i], w[i], acc);
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < 8; ++q) s += red[q];
            partial[(int64_t)blockIdx.x * m1 + t] = s;
        }
        __syncthreads();
    }
}
__global__ void gs_reduce_k(const double* partial, int nb, const int* kp, int m1, double* h) {
    const int t = blockIdx.x;
    if (t > *kp) return;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) acc += partial[(int64_t)b * m1 + t];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) h[t] = acc;
}
__global__ void gs_multiaxpy_k(const double* __restrict__ V, int64_t ldv, const int* kp, const double* __restrict__ h,
                               double* w, int64_t n) {
    __shared__ double sh[256];
    const int k1 = *kp + 1;
    for (int t = threadIdx.x; t < k1; t += blockDim.x) sh[t] = h[t];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = w[i];
    for (int t = 0; t < k1; ++t) acc = fma(-sh[t], V[(int64_t)t * ldv + i], acc);
    w[i] = acc;
}
template <class TZ>
__global__ void gs_update_x_k(const TZ* __restrict__ Z, int64_t ldz, const int* kp, const double* __restrict__ y,
                              double* x, int64_t n) {
    __shared__ double sy[256];
    const int k = *kp;
    for (int t = threadIdx.x; t < k; t += blockDim.x) sy[t] = y[t];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = x[i];
    for (int t = 0; t < k; ++t) acc = fma(sy[t], (double)Z[(int64_t)t * ldz + i], acc);
    x[i] = acc;
}

bool solve_graph_supported(const mgm_hierarchy* H, const mgm_solve_params* sp) {
    if (H->bordered || H->learned || H->cycle != MGM_CYCLE_V || H->sweep_mode == MGM_SWEEP_BARRIER ||
        H->sweep_mode == MGM_SWEEP_FLAGS || sp->krylov != MGM_KRYLOV_FGMRES_GRAPH || sp->restart > 255)
        return false;
    for (int j = 0; j + 1 < H->p; ++j)
        if (H->lv[j].stream) return false;  // cooperative launches have no place in conditional bodies
    return true;
}

// the graph a capture on cs is building
static cudaGraph_t captured_graph(cudaStream_t cs) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    CK(cudaStreamGetCaptureInfo(cs, &st, nullptr, &g, nullptr, nullptr, nullptr));
    REQUIRE(st == cudaStreamCaptureStatusActive && g, "no active capture");
    return g;
}
// During a capture on cs: a WHILE node on handle h after the capture's current dependencies; its
// body graph is returned, to be filled by a capture on another stream.
static cudaGraph_t add_while(cudaStream_t cs, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(cs, &st, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
    CK(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return p.conditional.phGraph_out[0];
}

// State of the device-driven solve (sized for any restart up to 255 and `maxit` iterations, so
// that graphs built on it stay valid)
static void ensure_graph_state(mgm_hierarchy* H, int maxit) {
    constexpr int MMAX = 255;
    if (!H->gsd.get()) {
        H->gsd.alloc(GS_G + (MMAX + 1) + 2 * MMAX + (size_t)(MMAX + 1) * MMAX + MMAX);
        H->gsi.alloc(8);
    }
    if (H->ghist.n < (size_t)maxit + 2) {
        if (H->sgraph) { cudaGraphExecDestroy(H->sgraph); H->sgraph = nullptr; }
        H->ghist.alloc((size_t)std::max(maxit + 2, 256));
    }
    if (!H->zd.get()) H->zd.alloc(H->N);
}

// Appends the device-driven FGMRES(m) of H to the capture running on c1 (f and u in H->f, H->u,
// solve order):
//   |f|, start; WHILE (restart loop) { r = f - L u, |r|, cycle start, v_0 = r/|r|,
//   WHILE (Arnoldi) { z_k = M v_k, w = L z_k, CGS2, |w|, rotations, v_{k+1} }, y, u += Z y }
// The loop bodies are captured on two auxiliary streams. The V-cycle keeps its programmatic
// dependent launches when `pdl` (the caller retries without them where a driver does not admit
// them inside conditional bodies); the solve's own kernels are plain launches.
static void enqueue_solve_graph(mgm_hierarchy* H, int m, cudaStream_t c1, bool pdl) {
    const int64_t n = H->N;
    const bool f32 = H->precision == MGM_F32;
    const int m1 = m + 1;
    if (H->part.n < (size_t)DOT_BLOCKS * m1) H->part.alloc((size_t)DOT_BLOCKS * m1);
    double* d = H->gsd.get();
    int* iv = H->gsi.get();
    double* hist = H->ghist.get();
    double* hb = H->hbuf.get();
    double* V = H->V.get();
    double* w = H->w.get();
    double* part = H->part.get();
    Level& L0 = H->lv[0];
    const unsigned gb = grid_for(n, 256);
    cudaStream_t c2 = nullptr, c3 = nullptr;
    CK(cudaStreamCreateWithFlags(&c2, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&c3, cudaStreamNonBlocking));
    auto dots1 = [&](const double* a, const double* b, double* out, cudaStream_t s) {  // out = a . b
        multidot_k<<<DOT_BLOCKS, 256, 0, s>>>(a, n, 1, b, n, part);
        CK_LAUNCH();
        reduce_partials_k<<<1, 32, 0, s>>>(part, DOT_BLOCKS, 1, out);
        CK_LAUNCH();
    };
    const bool pdl_was = pdl_off();
    pdl_off() = true;
    try {
        dots1(H->f.get(), H->f.get(), hb, c1);
        cudaGraphConditionalHandle ho, hi;
        CK(cudaGraphConditionalHandleCreate(&ho, captured_graph(c1), 0, cudaGraphCondAssignDefault));
        gs_start_k<<<1, 1, 0, c1>>>(hb, d, iv, ho);
        CK_LAUNCH();
        cudaGraph_t body_o = add_while(c1, ho);
        // ---- restart cycle: r = f - L u, beta, start of the cycle, Arnoldi loop, update of u
        CK(cudaStreamBeginCaptureToGraph(c2, body_o, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        spmv64_k<true><<<grid_for(n * KG, KBLOCK), KBLOCK, 0, c2>>>(L0.lo.get(), L0.up.get(), L0.sc.get(), L0.sv64.get(),
                                                                  L0.diag64.get(), H->u.get(), H->f.get(), V, n);
        CK_LAUNCH();
        dots1(V, V, hb, c2);
        CK(cudaGraphConditionalHandleCreate(&hi, captured_graph(c2), 0, cudaGraphCondAssignDefault));
        gs_cycle_k<<<1, 1, 0, c2>>>(hb, d, iv, hist, m, ho, hi);
        CK_LAUNCH();
        gs_scale0_k<<<gb, 256, 0, c2>>>(V, d + GS_INV, n);
        CK_LAUNCH();
        cudaGraph_t body_i = add_while(c2, hi);
        // ---- one Arnoldi step: z_k = M v_k, w = L z_k, two Gram-Schmidt passes, |w|, rotations
        CK(cudaStreamBeginCaptureToGraph(c3, body_i, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (f32) gs_loadv_k<float><<<gb, 256, 0, c3>>>(V, n, iv + GI_K, L0.b32.get(), n);
        else gs_loadv_k<double><<<gb, 256, 0, c3>>>(V, n, iv + GI_K, L0.b64.get(), n);
        CK_LAUNCH();
        pdl_off() = !pdl;
        vcycle_enqueue(H, c3);
        pdl_off() = true;
        if (f32) gs_storez_k<float><<<gb, 256, 0, c3>>>(L0.e32.get(), H->Z32.get(), n, iv + GI_K, H->zd.get(), n);
        else gs_storez_k<double><<<gb, 256, 0, c3>>>(L0.e64.get(), H->Z64.get(), n, iv + GI_K, H->zd.get(), n);
        CK_LAUNCH();
        spmv64_k<false><<<grid_for(n * KG, KBLOCK), KBLOCK, 0, c3>>>(L0.lo.get(), L0.up.get(), L0.sc.get(), L0.sv64.get(),
                                                                    L0.diag64.get(), H->zd.get(), nullptr, w, n);
        CK_LAUNCH();
        for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice: h1, then h2
            double* h = hb + pass * m1;
            gs_multidot_k<<<DOT_BLOCKS, 256, 0, c3>>>(V, n, iv + GI_K, m1, w, n, part);
            CK_LAUNCH();
            gs_reduce_k<<<m1, 32, 0, c3>>>(part, DOT_BLOCKS, iv + GI_K, m1, h);
            CK_LAUNCH();
            gs_multiaxpy_k<<<gb, 256, 0, c3>>>(V, n, iv + GI_K, h, w, n);
            CK_LAUNCH();
        }
        dots1(w, w, hb + 2 * m1, c3);
        gs_arnoldi_k<<<1, 1, 0, c3>>>(hb, d, iv, hist, m, hi);
        CK_LAUNCH();
        gs_scalek_k<<<gb, 256, 0, c3>>>(w, V, n, iv + GI_K, d + GS_INV, n);
        CK_LAUNCH();
        CK(cudaStreamEndCapture(c3, &body_i));
        // ---- after the Arnoldi loop: y, u += Z y
        gs_solve_y_k<<<1, 1, 0, c2>>>(d, iv, m, ho);
        CK_LAUNCH();
        double* y = d + GS_G + (m + 1) + 2 * m + (size_t)(m + 1) * m;
        if (f32) gs_update_x_k<float><<<gb, 256, 0, c2>>>(H->Z32.get(), n, iv + GI_K, y, H->u.get(), n);
        else gs_update_x_k<double><<<gb, 256, 0, c2>>>(H->Z64.get(), n, iv + GI_K, y, H->u.get(), n);
        CK_LAUNCH();
        CK(cudaStreamEndCapture(c2, &body_o));
    } catch (...) {
        pdl_off() = pdl_was;
        cudaStreamCaptureStatus st;
        for (cudaStream_t c : {c3, c2})
            if (cudaStreamIsCapturing(c, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(c, &g);
            }
        cudaStreamDestroy(c2);
        cudaStreamDestroy(c3);
        throw;
    }
    pdl_off() = pdl_was;
    cudaStreamDestroy(c2);
    cudaStreamDestroy(c3);
}

static void build_solve_graph_pdl(mgm_hierarchy* H, int m, int maxit, bool pdl) {
    ensure_graph_state(H, maxit);
    cudaStream_t c1 = nullptr;
    CK(cudaStreamCreateWithFlags(&c1, cudaStreamNonBlocking));
    cudaGraph_t top = nullptr;
    const int64_t before = thread_launches();
    try {
        CK(cudaStreamBeginCapture(c1, cudaStreamCaptureModeThreadLocal));
        enqueue_solve_graph(H, m, c1, pdl);
        CK(cudaStreamEndCapture(c1, &top));
    } catch (...) {
        cudaStreamCaptureStatus st;
        if (cudaStreamIsCapturing(c1, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaStreamEndCapture(c1, &top);
            if (top) cudaGraphDestroy(top);
        }
        cudaStreamDestroy(c1);
        throw;
    }
    note_launch(-(thread_launches() - before));
    if (H->sgraph) cudaGraphExecDestroy(H->sgraph);
    H->sgraph = nullptr;
    cudaError_t e = cudaGraphInstantiate(&H->sgraph, top, 0);
    cudaGraphDestroy(top);
    cudaStreamDestroy(c1);
    CK(e);
    H->sgraph_m = m;
    H->sgraph_maxit = maxit;
}

// with the V-cycle's programmatic launches first; without them if that graph is refused
static void build_solve_graph(mgm_hierarchy* H, int m, int maxit) {
    if (guarded([&] { build_solve_graph_pdl(H, m, maxit, true); }) == MGM_OK) return;
    (void)cudaGetLastError();
    build_solve_graph_pdl(H, m, maxit, false);
}

// one solve through the device-driven graph (f, u already in H->f, H->u)
static void run_solve_graph(mgm_hierarchy* H, const mgm_solve_params* sp, cudaStream_t s) {
    const int m = sp->restart;
    ensure_graph_state(H, std::max(sp->maxit, 1));
    if (!H->sgraph || H->sgraph_m != m) build_solve_graph(H, m, std::max(sp->maxit, 1));
    const double tol = sp->tol;
    const int maxit = sp->maxit;
    CK(cudaMemcpyAsync(H->gsd.get() + GS_TOL, &tol, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(H->gsi.get() + GI_MAXIT, &maxit, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaGraphLaunch(H->sgraph, s));
    note_launch(1);
}

// ------------------------------ reaction-diffusion steps as graphs ----------------------------
// iterations of both solves of step t, and whether both converged
__global__ void rd_record_k(const int* gu, const int* gv, int* rec, int* step, int* failed) {
    const int t = *step;
    rec[2 * t] = gu[GI_IT];
    rec[2 * t + 1] = gv[GI_IT];
    if (gu[GI_CONV] != 1 || gv[GI_CONV] != 1) *failed = 1;
    *step = t + 1;
}

// IMEX Euler steps of the reaction-diffusion system (Sec. 6.2's scheme class; the time-stepping of
// config 5): each step one launch of a graph holding the fused right-hand sides, the gathers into
// the two hierarchies' solve orders (warm start from the current state), both device-driven FGMRES
// solves and the scatters back. The host launches the graph `steps` times and synchronises once.
static cudaGraphExec_t reaction_step_graph(mgm_hierarchy* Hu, mgm_hierarchy* Hv, int model, const double* prm, double dt,
                                           double* u, double* v, double* ru, double* rv, int* rec, int* step, int* failed,
                                           int m, bool pdl);

void reaction_steps(mgm_hierarchy* Hu, mgm_hierarchy* Hv, int model, const double* prm, double dt, double* u, double* v,
                    int steps, const mgm_solve_params* sp, int* iters_out, cudaStream_t s) {
    REQUIRE(Hu && Hv && Hu != Hv && prm && u && v && sp && steps >= 0, "bad argument");
    REQUIRE(Hu->N == Hv->N, "the two hierarchies must have the same points");
    REQUIRE(sp->restart >= 1 && sp->restart <= 200 && sp->maxit >= 1 && sp->tol >= 0.0, "bad solve parameters");
    mgm_solve_params gp = *sp;
    gp.krylov = MGM_KRYLOV_FGMRES_GRAPH;
    REQUIRE(solve_graph_supported(Hu, &gp) && solve_graph_supported(Hv, &gp),
            "hierarchies must admit the device-driven solve (see MGM_KRYLOV_FGMRES_GRAPH)");
    if (steps == 0) return;
    const int64_t n = Hu->N;
    const int m = sp->restart;
    for (mgm_hierarchy* H : {Hu, Hv}) {
        ensure_workspace(H, m);
        vcycle_prepare(H);
        ensure_graph_state(H, sp->maxit);
        CK(cudaMemcpyAsync(H->gsd.get() + GS_TOL, &sp->tol, sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(H->gsi.get() + GI_MAXIT, &sp->maxit, sizeof(int), cudaMemcpyHostToDevice, s));
    }
    Temp<double> ru(n, s), rv(n, s);
    Temp<int> rec((size_t)2 * steps + 2, s);
    CK(cudaMemsetAsync(rec.get(), 0, sizeof(int) * (2 * (size_t)steps + 2), s));
    int* step = rec.get() + 2 * steps;
    int* failed = step + 1;
    cudaGraphExec_t ex = nullptr;
    if (guarded([&] { ex = reaction_step_graph(Hu, Hv, model, prm, dt, u, v, ru.get(), rv.get(), rec.get(), step, failed, m,
                                               true); }) != MGM_OK) {
        (void)cudaGetLastError();
        ex = reaction_step_graph(Hu, Hv, model, prm, dt, u, v, ru.get(), rv.get(), rec.get(), step, failed, m, false);
    }
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < steps; ++t) {
        e = cudaGraphLaunch(ex, s);
        if (e != cudaSuccess) break;
        note_launch(1);
    }
    std::vector<int> h((size_t)2 * steps + 2);
    cudaError_t e2 = cudaMemcpyAsync(h.data(), rec.get(), sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    cudaGraphExecDestroy(ex);
    CK(e);
    CK(e2);
    CK(e3);
    for (mgm_hierarchy* H : {Hu, Hv})
        if (H->persistent) check_device_error(H, s);
    if (iters_out)
        for (int t = 0; t < 2 * steps; ++t) iters_out[t] = h[t];
    if (h[2 * steps + 1]) fail(MGM_ERR_NOT_CONVERGED, "a reaction-diffusion solve did not reach tol (or broke down)");
}

static cudaGraphExec_t reaction_step_graph(mgm_hierarchy* Hu, mgm_hierarchy* Hv, int model, const double* prm, double dt,
                                           double* u, double* v, double* ru, double* rv, int* rec, int* step, int* failed,
                                           int m, bool pdl) {
    const int64_t n = Hu->N;
    const unsigned gb = grid_for(n, 256);
    cudaStream_t c1 = nullptr;
    CK(cudaStreamCreateWithFlags(&c1, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    const int64_t before = thread_launches();
    try {
        CK(cudaStreamBeginCapture(c1, cudaStreamCaptureModeThreadLocal));
        reaction_rhs(model, MGM_RD_EULER, n, u, v, nullptr, nullptr, prm, dt, ru, rv, c1);
        gather64_k<<<gb, 256, 0, c1>>>(ru, Hu->ord_caller.get(), Hu->f.get(), n);
        CK_LAUNCH();
        gather64_k<<<gb, 256, 0, c1>>>(u, Hu->ord_caller.get(), Hu->u.get(), n);
        CK_LAUNCH();
        gather64_k<<<gb, 256, 0, c1>>>(rv, Hv->ord_caller.get(), Hv->f.get(), n);
        CK_LAUNCH();
        gather64_k<<<gb, 256, 0, c1>>>(v, Hv->ord_caller.get(), Hv->u.get(), n);
        CK_LAUNCH();
        enqueue_solve_graph(Hu, m, c1, pdl);
        enqueue_solve_graph(Hv, m, c1, pdl);
        scatter64_k<<<gb, 256, 0, c1>>>(Hu->u.get(), Hu->ord_caller.get(), u, n);
        CK_LAUNCH();
        scatter64_k<<<gb, 256, 0, c1>>>(Hv->u.get(), Hv->ord_caller.get(), v, n);
        CK_LAUNCH();
        rd_record_k<<<1, 1, 0, c1>>>(Hu->gsi.get(), Hv->gsi.get(), rec, step, failed);
        CK_LAUNCH();
        CK(cudaStreamEndCapture(c1, &g));
    } catch (...) {
        cudaStreamCaptureStatus st;
        if (cudaStreamIsCapturing(c1, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
            cudaStreamEndCapture(c1, &g);
            if (g) cudaGraphDestroy(g);
        }
        cudaStreamDestroy(c1);
        throw;
    }
    note_launch(-(thread_launches() - before));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    cudaStreamDestroy(c1);
    CK(e);
    return ex;
}

void solve(mgm_hierarchy* H, const double* f_in, double* u_io, const mgm_solve_params* sp, mgm_solve_info* info,
           cudaStream_t s) {
    REQUIRE(H && f_in && u_io && sp, "null argument");
    REQUIRE(sp->krylov == MGM_KRYLOV_FGMRES || sp->krylov == MGM_KRYLOV_NONE || sp->krylov == MGM_KRYLOV_BICGSTAB ||
                sp->krylov == MGM_KRYLOV_FGMRES_GRAPH,
            "unknown krylov method");
    REQUIRE(sp->maxit >= 0 && sp->tol >= 0.0, "maxit and tol must be >= 0");
    const bool fgmres = sp->krylov == MGM_KRYLOV_FGMRES || sp->krylov == MGM_KRYLOV_FGMRES_GRAPH;
    REQUIRE(!fgmres || (sp->restart >= 1 && sp->restart <= 200), "restart must be in [1, 200]");
    REQUIRE(!H->bordered || fgmres, "a constrained hierarchy is solved with FGMRES");
    const bool on_graph = sp->krylov == MGM_KRYLOV_FGMRES_GRAPH && solve_graph_supported(H, sp);
    const int m = fgmres ? sp->restart : sp->krylov == MGM_KRYLOV_BICGSTAB ? 8 : 1;
    ensure_workspace(H, m);
    vcycle_prepare(H);
    const int64_t n = H->N;
    const int64_t nv = n + (H->bordered ? 1 : 0);  // bordered: [u; lambda], f = [f; 0], lambda_0 = 0
    Ops op{H, s, n, nv};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
    const int32_t* ordc = H->ord_caller.get();
    gather64_k<<<grid_for(n, 256), 256, 0, s>>>(f_in, ordc, H->f.get(), n);
    CK_LAUNCH();
    gather64_k<<<grid_for(n, 256), 256, 0, s>>>(u_io, ordc, H->u.get(), n);
    CK_LAUNCH();
    if (H->bordered) {
        CK(cudaMemsetAsync(H->f.get() + n, 0, sizeof(double), s));
        CK(cudaMemsetAsync(H->u.get() + n, 0, sizeof(double), s));
    }
    double fn = op.norm(H->f.get());
    if (!std::isfinite(fn)) fail(MGM_ERR_INVALID_ARG, "right-hand side is not finite");
    if (fn == 0.0) fn = 1.0;
    std::vector<double> hist;
    int it = 0;
    double rel = 0.0;
    mgm_status status = MGM_ERR_NOT_CONVERGED;
    const bool f32 = H->precision == MGM_F32;
    // a learned correction that stops reducing the residual is switched off for the rest of the
    // solve (the flexible outer iteration tolerates the change of preconditioner): FGMRES when
    // five iterations reduce the estimate by less than 20% (GMRES estimates never increase, and
    // the first iterations of a good preconditioner may reduce little), the standalone iteration
    // as soon as the residual grows
    H->learned_active = true;
    auto fallback_if = [&](bool stalled) {
        if (H->learned && H->learned_active && stalled) {
            H->learned_active = false;
            ++H->learned_fallbacks;
        }
    };
    if (on_graph) {
        run_solve_graph(H, sp, s);
        int ivh[8];
        double dh[GS_G];
        to_host(ivh, H->gsi.get(), 8, s);
        to_host(dh, H->gsd.get(), (size_t)GS_G, s);
        it = ivh[GI_IT];
        rel = dh[GS_REL];
        hist.resize(std::max(0, ivh[GI_NH]));
        to_host(hist.data(), H->ghist.get(), hist.size(), s);
        status = ivh[GI_CONV] == 1 ? MGM_OK : ivh[GI_CONV] == 2 ? MGM_ERR_BREAKDOWN : MGM_ERR_NOT_CONVERGED;
        if (ivh[GI_CONV] == 2 && !std::isfinite(fn)) fail(MGM_ERR_INVALID_ARG, "right-hand side is not finite");
    } else if (sp->krylov == MGM_KRYLOV_BICGSTAB) {
        H->learned_active = false;  // BiCGSTAB needs a linear preconditioner
        status = bicgstab(H, op, sp, fn, hist, it, rel);
    } else if (sp->krylov == MGM_KRYLOV_NONE) {
        for (;;) {
            op.spmv<true, double>(H->u.get(), H->f.get(), H->r.get());
            rel = op.norm(H->r.get()) / fn;
            if (!hist.empty()) fallback_if(!(rel < hist.back()));
            hist.push_back(rel);
            if (!std::isfinite(rel)) { status = MGM_ERR_BREAKDOWN; break; }
            if (rel <= sp->tol) { status = MGM_OK; break; }
            if (it >= sp->maxit) break;
            load_input(H, H->r.get(), MGM_F64, nullptr, s);
            vcycle_core(H, s);
            add_output(H, H->u.get(), nullptr, s);
            ++it;
        }
    } else {
        std::vector<double> Hm((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), y(m);
        double* V = H->V.get();
        for (;;) {
            op.op_apply<true, double>(H->u.get(), H->f.get(), V);
            double beta = op.norm(V);
            rel = beta / fn;
            if (hist.empty()) hist.push_back(rel);
            if (!std::isfinite(rel)) { status = MGM_ERR_BREAKDOWN; break; }
            if (rel <= sp->tol) { status = MGM_OK; break; }
            if (it >= sp->maxit) break;
            scale_k<<<grid_for(nv, 256), 256, 0, s>>>(V, 1.0 / beta, V, nv);
            CK_LAUNCH();
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            int k = 0;
            bool stop = false;
            for (; k < m && it < sp->maxit; ++k) {
                double* vk = V + (int64_t)k * nv;
                double* w = H->w.get();
                if (f32) {
                    float* zk = H->Z32.get() + (int64_t)k * nv;
                    op.precondition(vk, zk);
                    op.op_apply<false, float>(zk, nullptr, w);
                } else {
                    double* zk = H->Z64.get() + (int64_t)k * nv;
                    op.precondition(vk, zk);
                    op.op_apply<false, double>(zk, nullptr, w);
                }
                const int k1 = k + 1;
                double* h1 = H->hbuf.get();
                double* h2 = h1 + (m + 1);
                double* hn2 = h2 + (m + 1);
                op.dots(V, nv, k1, w, h1);
                op.axpys(V, nv, k1, h1, w);
                op.dots(V, nv, k1, w, h2);
                op.axpys(V, nv, k1, h2, w);
                op.dots(w, nv, 1, w, hn2);
                CK(cudaMemcpyAsync(H->hhost, H->hbuf.get(), sizeof(double) * (2 * (m + 1) + 1), cudaMemcpyDeviceToHost, s));
                CK(cudaStreamSynchronize(s));
                const double* hh = H->hhost;
                for (int i = 0; i < k1; ++i) Hm[(size_t)i * m + k] = hh[i] + hh[(m + 1) + i];
                double hn = std::sqrt(hh[2 * (m + 1)]);
                Hm[(size_t)k1 * m + k] = hn;
                if (!std::isfinite(hn)) { status = MGM_ERR_BREAKDOWN; stop = true; break; }
                if (hn > 0.0 && k1 < m + 1) {
                    scale_k<<<grid_for(nv, 256), 256, 0, s>>>(w, 1.0 / hn, V + (int64_t)k1 * nv, nv);
                    CK_LAUNCH();
                }
                for (int i = 0; i < k; ++i) {
                    double a = Hm[(size_t)i * m + k], b = Hm[(size_t)(i + 1) * m + k];
                    Hm[(size_t)i * m + k] = cs[i] * a + sn[i] * b;
                    Hm[(size_t)(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
                }
                double a = Hm[(size_t)k * m + k], b = Hm[(size_t)k1 * m + k];
                double rr = std::sqrt(a * a + b * b);
                cs[k] = rr == 0.0 ? 1.0 : a / rr;
                sn[k] = rr == 0.0 ? 0.0 : b / rr;
                Hm[(size_t)k * m + k] = rr;
                Hm[(size_t)k1 * m + k] = 0.0;
                g[k1] = -sn[k] * g[k];
                g[k] = cs[k] * g[k];
                ++it;
                double est = std::fabs(g[k1]) / fn;
                if (hist.size() >= 5) fallback_if(!(est < 0.8 * hist[hist.size() - 5]));
                hist.push_back(est);
                if (est <= sp->tol || hn == 0.0) { ++k; break; }
            }
            if (stop) break;
            for (int i = k - 1; i >= 0; --i) {
                double acc = g[i];
                for (int j = i + 1; j < k; ++j) acc -= Hm[(size_t)i * m + j] * y[j];
                y[i] = acc / Hm[(size_t)i * m + i];
            }
            if (k > 0) {
                CK(cudaMemcpyAsync(H->ydev.get(), y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
                if (f32) update_x_k<float><<<grid_for(nv, 256), 256, 0, s>>>(H->Z32.get(), nv, k, H->ydev.get(), H->u.get(), nv);
                else update_x_k<double><<<grid_for(nv, 256), 256, 0, s>>>(H->Z64.get(), nv, k, H->ydev.get(), H->u.get(), nv);
                CK_LAUNCH();
                CK(cudaStreamSynchronize(s));  // y is pageable host memory
            }
        }
    }
    scatter64_k<<<grid_for(n, 256), 256, 0, s>>>(H->u.get(), ordc, u_io, n);
    CK_LAUNCH();
    if (H->persistent) check_device_error(H, s);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
        info->iters = it;
        info->rel_res = rel;
        info->solve_ms = ms;
        info->multiplier = H->bordered ? read1(H->u.get() + n, s) : 0.0;
        if (info->history && info->history_len > 0)
            for (int i = 0; i < info->history_len; ++i) info->history[i] = i < (int)hist.size() ? hist[i] : 0.0;
    }
    if (status != MGM_OK) {
        if (status == MGM_ERR_NOT_CONVERGED)
            set_error("not converged: relative residual " + std::to_string(rel) + " after " + std::to_string(it) + " iterations");
        else
            set_error("breakdown: non-finite value in the iteration");
        throw Fail{status};
    }
}

}  // namespace mgm

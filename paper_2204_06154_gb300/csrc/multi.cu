// Many right-hand sides on one hierarchy, and batches of hierarchies (the batched solve).
//
// With R right-hand sides the V-cycle and the outer operator stream each stored matrix and
// transfer entry once for all R: vectors are interleaved [row][R] (R = 1, 2, 4 or 8), so a
// gathered neighbour brings R consecutive values (one 32-byte sector for R = 8 in FP32) and each
// lane keeps R accumulators. R independent right-preconditioned FGMRES processes (paper Sec. 4.6)
// advance in lockstep: shared kernels, per-column dot products, Givens rotations and convergence
// tests per right-hand side on the host. A column that has converged stops contributing to its
// solution; a zero right-hand side (padding up to R) is converged from the start.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "hier.cuh"

namespace mgm {

constexpr int MG = 8;          // lanes per row
constexpr int MBLOCK = 256;
constexpr int BATCH_THREADS = 8;  // host threads (and streams) of a batched solve

template <int R, class T>
struct VecR {
    T v[R];
};

template <class T, int R>
__device__ __forceinline__ void load_row(const T* x, int32_t c, T* out) {
#pragma unroll
    for (int r = 0; r < R; ++r) out[r] = x[(int64_t)c * R + r];
}

// acc[r] += this lane's products v_p x[c_p][r] over [beg, end) (multiples of 4), MG lanes per row
// (the caller sums the lanes)
template <class T, int R>
__device__ __forceinline__ void row_sum_R(const int32_t* __restrict__ sc, const T* __restrict__ sv, int32_t beg,
                                          int32_t end, const T* x, int gl, T* acc) {
    for (int32_t p = beg + 4 * gl; p < end; p += 4 * MG) {
        int4 c = __ldg(reinterpret_cast<const int4*>(sc + p));
        T v[4] = {__ldg(sv + p), __ldg(sv + p + 1), __ldg(sv + p + 2), __ldg(sv + p + 3)};
        int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T xr[R];
            load_row<T, R>(x, cc[q], xr);
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fma(v[q], xr[r], acc[r]);
        }
    }
}

// MODE 0: first sweep from zero (lower part); 1: full sweep; 2: s = -U e; 3: s = b - A e
template <int MODE, class T, int R>
__global__ void __launch_bounds__(MBLOCK) rowR_k(const int32_t* __restrict__ lo, const int32_t* __restrict__ up,
                                                 const int32_t* __restrict__ sc, const T* __restrict__ sv,
                                                 const T* __restrict__ dv, const T* __restrict__ b, T* e, T* s, int32_t r0,
                                                 int32_t r1) {
    const int t = blockIdx.x * MBLOCK + threadIdx.x;
    const int32_t row = r0 + t / MG;
    const int gl = t & (MG - 1);
    const bool act = row < r1;
    T acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = T(0);
    int32_t b0 = 0, e0 = 0, b1 = 0, e1 = 0;  // lower part, then upper part
    if (act) {
        if (MODE != 2) { b0 = lo[row]; e0 = lo[row + 1]; }
        if (MODE != 0) { b1 = up[row]; e1 = up[row + 1]; }
    }
    row_sum_R<T, R>(sc, sv, b0, e0, e, gl, acc);
    row_sum_R<T, R>(sc, sv, b1, e1, e, gl, acc);
#pragma unroll
    for (int r = 0; r < R; ++r)
        for (int o = MG / 2; o; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (act && gl < R) {
        const int64_t o = (int64_t)row * R + gl;
        T a = acc[0];
#pragma unroll
        for (int r = 1; r < R; ++r) if (gl == r) a = acc[r];
        if (MODE == 0 || MODE == 1) e[o] = (b[o] - a) * dv[row];
        else if (MODE == 2) s[o] = -a;
        else s[o] = b[o] - dv[row] * e[o] - a;
    }
}

template <class T, int R>
__global__ void restrictR_k(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const T* __restrict__ v,
                            const T* __restrict__ s, T* bn, int64_t nc) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc * R) return;
    int64_t c = t / R;
    int r = (int)(t - c * R);
    T acc = T(0);
    for (int32_t q = rp[c]; q < rp[c + 1]; ++q) acc += v[q] * s[(int64_t)ci[q] * R + r];
    bn[t] = acc;
}

template <class T, int R>
__global__ void interpR_k(const int32_t* __restrict__ pc, const T* __restrict__ pv, int pw, const T* __restrict__ en,
                          T* e, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * R) return;
    int64_t i = t / R;
    int r = (int)(t - i * R);
    T acc = e[t];
    for (int q = 0; q < pw; ++q) acc += pv[i * pw + q] * en[(int64_t)pc[i * pw + q] * R + r];
    e[t] = acc;
}

template <class T, int R>
__global__ void coarseR_k(const double* __restrict__ Ainv, const T* __restrict__ b, T* e, int64_t n) {
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
        double a = Ainv[row * n + j];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = fma(a, (double)b[j * R + r], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        double v = warp_sum(acc[r]);
        if (lane == 0) e[row * R + r] = (T)v;
    }
}

// caller layout (column r at src + r * n, caller order) <-> interleaved solve-order vectors
template <class TO, int R>
__global__ void gatherR_k(const double* src, int nrhs, const int32_t* ord, TO* dst, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * R) return;
    int64_t i = t / R;
    int r = (int)(t - i * R);
    dst[t] = r < nrhs ? (TO)src[(int64_t)r * n + (ord ? ord[i] : i)] : TO(0);
}
template <class TI, int R>
__global__ void scatterR_k(const TI* src, int nrhs, const int32_t* ord, double* dst, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * R) return;
    int64_t i = t / R;
    int r = (int)(t - i * R);
    if (r < nrhs) dst[(int64_t)r * n + (ord ? ord[i] : i)] = (double)src[t];
}
template <class TI, class TO>
__global__ void castR_k(const TI* a, TO* b, int64_t m) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) b[t] = (TO)a[t];
}

// ------------------------------ outer FP64 kernels --------------------------------------------
template <bool RESID, class TX, int R>
__global__ void __launch_bounds__(MBLOCK) spmvR_k(const int32_t* __restrict__ lo, const int32_t* __restrict__ up,
                                                  const int32_t* __restrict__ sc,
                                                  const double* __restrict__ sv, const double* __restrict__ diag,
                                                  const TX* __restrict__ x, const double* __restrict__ f, double* y,
                                                  int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * MBLOCK + threadIdx.x;
    const int64_t row = t / MG;
    const int gl = (int)(t & (MG - 1));
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    if (row < n) {
        for (int part = 0; part < 2; ++part) {  // lower part, then upper part
            const int32_t b = part ? up[row] : lo[row], e = part ? up[row + 1] : lo[row + 1];
            for (int32_t p = b + 4 * gl; p < e; p += 4 * MG) {
                int4 c = __ldg(reinterpret_cast<const int4*>(sc + p));
                double v[4] = {__ldg(sv + p), __ldg(sv + p + 1), __ldg(sv + p + 2), __ldg(sv + p + 3)};
                int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int r = 0; r < R; ++r) acc[r] = fma(v[q], (double)x[(int64_t)cc[q] * R + r], acc[r]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        for (int o = MG / 2; o; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (row < n && gl < R) {
        double a = acc[0];
#pragma unroll
        for (int r = 1; r < R; ++r) if (gl == r) a = acc[r];
        const int64_t o = row * R + gl;
        double lx = fma(diag[row], (double)x[o], a);
        y[o] = RESID ? f[o] - lx : lx;
    }
}

constexpr int RDOT_BLOCKS = 304;
// partial[(b * k1 + t) * R + r] = sum over block b's rows of V_t[i][r] w[i][r]
template <int R>
__global__ void __launch_bounds__(256) multidotR_k(const double* __restrict__ V, int64_t ldv, int k1,
                                                   const double* __restrict__ w, int64_t n, double* partial) {
    __shared__ double red[8][R];
    const int64_t m = n * R;
    const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x) * R;
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(m, b0 + chunk);
    const int lane = threadIdx.x & 31;
    // element e = i*R + r; b0 and the stride 256 are multiples of R, so each thread sees one r
    for (int t = 0; t < k1; ++t) {
        const double* v = V + (int64_t)t * ldv;
        double acc = 0.0;
        for (int64_t e = b0 + threadIdx.x; e < b1; e += 256) acc = fma(v[e], w[e], acc);
        for (int o = 16; o >= R; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);  // lanes of equal r
        if (lane < R) red[threadIdx.x >> 5][lane] = acc;
        __syncthreads();
        if (threadIdx.x < R) {
            double s = 0.0;
            for (int q = 0; q < 8; ++q) s += red[q][threadIdx.x];
            partial[((int64_t)blockIdx.x * k1 + t) * R + threadIdx.x] = s;
        }
        __syncthreads();
    }
}
template <int R>
__global__ void reduce_partialsR_k(const double* partial, int nb, int k1, double* h) {
    const int t = blockIdx.x / R, r = blockIdx.x % R;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) acc += partial[((int64_t)b * k1 + t) * R + r];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) h[t * R + r] = acc;
}
// w[i][r] -= sum_t h[t][r] V_t[i][r]
template <int R>
__global__ void multiaxpyR_k(const double* __restrict__ V, int64_t ldv, int k1, const double* __restrict__ h, double* w,
                             int64_t m) {
    __shared__ double sh[256 * 8];
    for (int q = threadIdx.x; q < k1 * R; q += blockDim.x) sh[q] = h[q];
    __syncthreads();
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int r = (int)(e % R);
    double acc = w[e];
    for (int t = 0; t < k1; ++t) acc = fma(-sh[t * R + r], V[(int64_t)t * ldv + e], acc);
    w[e] = acc;
}
template <int R>
__global__ void scaleR_k(const double* a, const double* inv, double* b, int64_t m) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) b[e] = a[e] * inv[e % R];
}
template <class TZ, int R>
__global__ void updateR_k(const TZ* __restrict__ Z, int64_t ldz, int k, const double* __restrict__ y, double* x, int64_t m) {
    __shared__ double sy[256 * 8];
    for (int q = threadIdx.x; q < k * R; q += blockDim.x) sy[q] = y[q];
    __syncthreads();
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int r = (int)(e % R);
    double acc = x[e];
    for (int t = 0; t < k; ++t) acc = fma(sy[t * R + r], (double)Z[(int64_t)t * ldz + e], acc);
    x[e] = acc;
}

// ------------------------------ host side -------------------------------------------------------
struct MultiWork {
    int R = 0, m = 0, p = 0;
    std::vector<Buf<float>> b32, e32, s32;
    std::vector<Buf<double>> b64, e64, s64;
    Buf<double> V, f, u, w, part, hbuf, inv, y;
    Buf<float> Z32;
    Buf<double> Z64;
    Buf<double> zd;  // FP64 copy of an FP32 z_k for the outer product
    // the R-column V-cycle (b_0 -> e_0 of this workspace), captured once into a graph
    cudaGraphExec_t vgraph = nullptr;
    int64_t vgraph_kernels = 0;
    cudaStream_t cap = nullptr;
    void drop_graph() {
        if (vgraph) cudaGraphExecDestroy(vgraph);
        vgraph = nullptr;
    }
    ~MultiWork() {
        drop_graph();
        if (cap) cudaStreamDestroy(cap);
    }
};

static MultiWork& multi_work(mgm_hierarchy* H, int R, int m) {
    if (!H->multi) H->multi = new MultiWork();
    MultiWork& W = *static_cast<MultiWork*>(H->multi);
    if (W.R == R && W.m >= m) return W;
    W.drop_graph();
    W.R = R;
    W.m = m;
    W.p = H->p;
    const bool f32 = H->precision == MGM_F32;
    W.b32.clear(); W.e32.clear(); W.s32.clear(); W.b64.clear(); W.e64.clear(); W.s64.clear();
    W.b32.resize(H->p); W.e32.resize(H->p); W.s32.resize(H->p);
    W.b64.resize(H->p); W.e64.resize(H->p); W.s64.resize(H->p);
    for (int j = 0; j < H->p; ++j) {
        const size_t len = (size_t)H->lv[j].n * R;
        if (f32) {
            W.b32[j].alloc(len); W.e32[j].alloc(len); W.s32[j].alloc(len);
            CK(cudaMemset(W.e32[j].get(), 0, len * sizeof(float)));
        } else {
            W.b64[j].alloc(len); W.e64[j].alloc(len); W.s64[j].alloc(len);
            CK(cudaMemset(W.e64[j].get(), 0, len * sizeof(double)));
        }
    }
    const int64_t nR = H->N * R;
    W.V.alloc((int64_t)(m + 1) * nR);
    if (f32) {
        W.Z32.alloc((int64_t)m * nR);
        W.zd.alloc(nR);
    } else {
        W.Z64.alloc((int64_t)m * nR);
    }
    W.f.alloc(nR); W.u.alloc(nR); W.w.alloc(nR);
    W.part.alloc((int64_t)RDOT_BLOCKS * (m + 2) * R);
    W.hbuf.alloc((int64_t)(2 * (m + 2) + 2) * R);
    W.inv.alloc(R);
    W.y.alloc((int64_t)(m + 1) * R);
    return W;
}

template <class T> struct WV;
template <> struct WV<float> {
    static float* b(MultiWork& W, int j) { return W.b32[j].get(); }
    static float* e(MultiWork& W, int j) { return W.e32[j].get(); }
    static float* s(MultiWork& W, int j) { return W.s32[j].get(); }
    static const float* sv(Level& L) { return L.sv32.get(); }
    static const float* diag(Level& L) { return L.diag32.get(); }
    static const float* dinv(Level& L) { return L.dinv32.get(); }
    static const float* pv(Level& L) { return L.pv32.get(); }
    static const float* rv(Level& L) { return L.r_v32.get(); }
};
template <> struct WV<double> {
    static double* b(MultiWork& W, int j) { return W.b64[j].get(); }
    static double* e(MultiWork& W, int j) { return W.e64[j].get(); }
    static double* s(MultiWork& W, int j) { return W.s64[j].get(); }
    static const double* sv(Level& L) { return L.sv64.get(); }
    static const double* diag(Level& L) { return L.diag64.get(); }
    static const double* dinv(Level& L) { return L.dinv64.get(); }
    static const double* pv(Level& L) { return L.pv64.get(); }
    static const double* rv(Level& L) { return L.r_v64.get(); }
};

template <int MODE, class T, int R>
static void rows_R(MultiWork& W, Level& L, int j, int32_t r0, int32_t r1, cudaStream_t s) {
    if (r1 <= r0) return;
    const T* dv = MODE == 3 ? WV<T>::diag(L) : WV<T>::dinv(L);
    rowR_k<MODE, T, R><<<grid_for((int64_t)(r1 - r0) * MG, MBLOCK), MBLOCK, 0, s>>>(
        L.lo.get(), L.up.get(), L.sc.get(), WV<T>::sv(L), dv, WV<T>::b(W, j), WV<T>::e(W, j), WV<T>::s(W, j), r0, r1);
    CK_LAUNCH();
}

template <class T, int R>
static void sweep_R(MultiWork& W, Level& L, int j, bool from_zero, cudaStream_t s) {
    for (size_t c = 0; c + 1 < L.cptr.size(); ++c) {
        if (from_zero) rows_R<0, T, R>(W, L, j, L.cptr[c], L.cptr[c + 1], s);
        else rows_R<1, T, R>(W, L, j, L.cptr[c], L.cptr[c + 1], s);
    }
}

// Alg. 3 from zero for R right-hand sides: b_0 (interleaved) -> e_0
template <class T, int R>
static void vcycle_R(mgm_hierarchy* H, MultiWork& W, cudaStream_t s) {
    const int p = H->p;
    for (int j = 0; j + 1 < p; ++j) {
        Level& L = H->lv[j];
        Level& C = H->lv[j + 1];
        const T* rsrc;
        if (H->nu1 >= 1) {
            sweep_R<T, R>(W, L, j, true, s);
            for (int t = 1; t < H->nu1; ++t) sweep_R<T, R>(W, L, j, false, s);
            if (H->nu1 == 1) rows_R<2, T, R>(W, L, j, 0, (int32_t)L.n, s);
            else rows_R<3, T, R>(W, L, j, 0, (int32_t)L.n, s);
            rsrc = WV<T>::s(W, j);
        } else {
            CK(cudaMemsetAsync(WV<T>::e(W, j), 0, sizeof(T) * L.n * R, s));
            rsrc = WV<T>::b(W, j);
        }
        restrictR_k<T, R><<<grid_for(C.n * R, 256), 256, 0, s>>>(L.r_rp.get(), L.r_ci.get(), WV<T>::rv(L), rsrc,
                                                                WV<T>::b(W, j + 1), C.n);
        CK_LAUNCH();
    }
    Level& Cp = H->lv[p - 1];
    coarseR_k<T, R><<<grid_for(Cp.n * 32, 256), 256, 0, s>>>(H->Ainv.get(), WV<T>::b(W, p - 1), WV<T>::e(W, p - 1), Cp.n);
    CK_LAUNCH();
    for (int j = p - 2; j >= 0; --j) {
        Level& L = H->lv[j];
        interpR_k<T, R><<<grid_for(L.n * R, 256), 256, 0, s>>>(L.pc.get(), WV<T>::pv(L), L.pw, WV<T>::e(W, j + 1),
                                                              WV<T>::e(W, j), L.n);
        CK_LAUNCH();
        for (int t = 0; t < H->nu2; ++t) sweep_R<T, R>(W, L, j, false, s);
    }
}

// the R-column V-cycle as one graph launch (captured on first use; the workspace's buffers are fixed
// until it is reallocated, which drops the graph)
template <class T, int R>
static void vcycle_R_graph(mgm_hierarchy* H, MultiWork& W, cudaStream_t s) {
    if (!W.vgraph) {
        if (!W.cap) CK(cudaStreamCreateWithFlags(&W.cap, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        const int64_t before = thread_launches();
        CK(cudaStreamBeginCapture(W.cap, cudaStreamCaptureModeThreadLocal));
        try {
            vcycle_R<T, R>(H, W, W.cap);
        } catch (...) {
            cudaStreamEndCapture(W.cap, &g);
            if (g) cudaGraphDestroy(g);
            throw;
        }
        CK(cudaStreamEndCapture(W.cap, &g));
        W.vgraph_kernels = thread_launches() - before;
        note_launch(-W.vgraph_kernels);
        cudaError_t e = cudaGraphInstantiate(&W.vgraph, g, 0);
        cudaGraphDestroy(g);
        CK(e);
    }
    CK(cudaGraphLaunch(W.vgraph, s));
    note_launch(W.vgraph_kernels);
}

template <class T, int R>
static void solve_multi_t(mgm_hierarchy* H, int nrhs, const double* F, double* U, const mgm_solve_params* sp,
                          mgm_solve_info* info, cudaStream_t s) {
    const int m = sp->krylov == MGM_KRYLOV_FGMRES ? sp->restart : 1;
    MultiWork& W = multi_work(H, R, m);
    const int64_t n = H->N, nR = n * R;
    Level& L0 = H->lv[0];
    const int32_t* ordc = H->ord_caller.get();
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, s));
    gatherR_k<double, R><<<grid_for(nR, 256), 256, 0, s>>>(F, nrhs, ordc, W.f.get(), n);
    CK_LAUNCH();
    gatherR_k<double, R><<<grid_for(nR, 256), 256, 0, s>>>(U, nrhs, ordc, W.u.get(), n);
    CK_LAUNCH();
    std::vector<double> hh((size_t)(2 * (m + 2) + 2) * R);
    auto dots = [&](const double* V, int64_t ldv, int k1, const double* w, double* h) {
        multidotR_k<R><<<RDOT_BLOCKS, 256, 0, s>>>(V, ldv, k1, w, n, W.part.get());
        CK_LAUNCH();
        reduce_partialsR_k<R><<<k1 * R, 32, 0, s>>>(W.part.get(), RDOT_BLOCKS, k1, h);
        CK_LAUNCH();
    };
    auto norms = [&](const double* w, std::vector<double>& out) {
        dots(w, nR, 1, w, W.hbuf.get());
        out.resize(R);
        to_host(out.data(), W.hbuf.get(), R, s);
        for (auto& v : out) v = std::sqrt(v);
    };
    auto spmv = [&](const auto* x, const double* f, double* y, bool resid) {
        using TX = std::remove_const_t<std::remove_pointer_t<decltype(x)>>;
        if (resid) spmvR_k<true, TX, R><<<grid_for(n * MG, MBLOCK), MBLOCK, 0, s>>>(L0.lo.get(), L0.up.get(), L0.sc.get(), L0.sv64.get(),
                                                                                  L0.diag64.get(), x, f, y, n);
        else spmvR_k<false, TX, R><<<grid_for(n * MG, MBLOCK), MBLOCK, 0, s>>>(L0.lo.get(), L0.up.get(), L0.sc.get(), L0.sv64.get(),
                                                                             L0.diag64.get(), x, f, y, n);
        CK_LAUNCH();
    };
    auto precond = [&](const double* v, T* z) {
        castR_k<double, T><<<grid_for(nR, 256), 256, 0, s>>>(v, WV<T>::b(W, 0), nR);
        CK_LAUNCH();
        vcycle_R_graph<T, R>(H, W, s);
        castR_k<T, T><<<grid_for(nR, 256), 256, 0, s>>>(WV<T>::e(W, 0), z, nR);
        CK_LAUNCH();
    };
    std::vector<double> fn;
    norms(W.f.get(), fn);
    for (auto& v : fn) if (v == 0.0) v = 1.0;
    std::vector<int> iters(R, 0), done(R, 0);
    std::vector<double> rel(R, 0.0);
    std::vector<std::vector<double>> hist(R);
    int it = 0;
    bool breakdown = false;
    T* Z = nullptr;
    if constexpr (sizeof(T) == 4) Z = W.Z32.get(); else Z = W.Z64.get();
    for (;;) {
        // true residuals r = f - L u
        spmv((const double*)W.u.get(), W.f.get(), W.V.get(), true);
        std::vector<double> beta;
        norms(W.V.get(), beta);
        bool all = true;
        for (int r = 0; r < R; ++r) {
            rel[r] = beta[r] / fn[r];
            if (hist[r].empty()) hist[r].push_back(rel[r]);
            if (!std::isfinite(rel[r])) breakdown = true;
            if (rel[r] <= sp->tol || r >= nrhs) done[r] = 1;
            all = all && done[r];
        }
        if (all || breakdown || it >= sp->maxit) break;
        std::vector<double> inv(R);
        for (int r = 0; r < R; ++r) inv[r] = done[r] ? 0.0 : 1.0 / beta[r];
        CK(cudaMemcpyAsync(W.inv.get(), inv.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s));
        scaleR_k<R><<<grid_for(nR, 256), 256, 0, s>>>(W.V.get(), W.inv.get(), W.V.get(), nR);
        CK_LAUNCH();
        if (sp->krylov == MGM_KRYLOV_NONE) {
            // standalone MGM: u += M r (columns already converged have r scaled to zero)
            precond(W.V.get(), Z);
            std::vector<double> yb(R);
            for (int r = 0; r < R; ++r) yb[r] = done[r] ? 0.0 : beta[r];
            CK(cudaMemcpyAsync(W.y.get(), yb.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s));
            updateR_k<T, R><<<grid_for(nR, 256), 256, 0, s>>>(Z, nR, 1, W.y.get(), W.u.get(), nR);
            CK_LAUNCH();
            CK(cudaStreamSynchronize(s));
            ++it;
            for (int r = 0; r < R; ++r) if (!done[r]) iters[r] = it;
            continue;
        }
        std::vector<std::vector<double>> Hm(R, std::vector<double>((size_t)(m + 1) * m, 0.0)), g(R, std::vector<double>(m + 1, 0.0));
        std::vector<std::vector<double>> cs(R, std::vector<double>(m)), sn(R, std::vector<double>(m));
        std::vector<int> kr(R, 0), frozen(R, 0);
        for (int r = 0; r < R; ++r) { g[r][0] = done[r] ? 0.0 : beta[r]; frozen[r] = done[r]; }
        int k = 0;
        for (; k < m && it < sp->maxit; ++k) {
            double* vk = W.V.get() + (int64_t)k * nR;
            T* zk = Z + (int64_t)k * nR;
            precond(vk, zk);
            if constexpr (std::is_same<T, float>::value) {
                // widened once, so that the product converts nR values instead of one per entry
                castR_k<float, double><<<grid_for(nR, 256), 256, 0, s>>>(zk, W.zd.get(), nR);
                CK_LAUNCH();
                spmv((const double*)W.zd.get(), nullptr, W.w.get(), false);
            } else {
                spmv((const T*)zk, nullptr, W.w.get(), false);
            }
            const int k1 = k + 1;
            double* h1 = W.hbuf.get();
            double* h2 = h1 + (size_t)(m + 1) * R;
            double* hn2 = h2 + (size_t)(m + 1) * R;
            dots(W.V.get(), nR, k1, W.w.get(), h1);
            multiaxpyR_k<R><<<grid_for(nR, 256), 256, 0, s>>>(W.V.get(), nR, k1, h1, W.w.get(), nR);
            CK_LAUNCH();
            dots(W.V.get(), nR, k1, W.w.get(), h2);
            multiaxpyR_k<R><<<grid_for(nR, 256), 256, 0, s>>>(W.V.get(), nR, k1, h2, W.w.get(), nR);
            CK_LAUNCH();
            dots(W.w.get(), nR, 1, W.w.get(), hn2);
            to_host(hh.data(), W.hbuf.get(), (size_t)(2 * (m + 1) + 1) * R, s);
            ++it;
            std::vector<double> inv2(R, 0.0);
            bool stop = true;
            for (int r = 0; r < R; ++r) {
                double hn = std::sqrt(hh[(size_t)2 * (m + 1) * R + r]);
                if (frozen[r]) continue;
                std::vector<double>& Hr = Hm[r];
                for (int i = 0; i < k1; ++i) Hr[(size_t)i * m + k] = hh[(size_t)i * R + r] + hh[(size_t)(m + 1) * R + i * R + r];
                Hr[(size_t)k1 * m + k] = hn;
                if (!std::isfinite(hn)) { breakdown = true; continue; }
                inv2[r] = hn > 0.0 ? 1.0 / hn : 0.0;
                for (int i = 0; i < k; ++i) {
                    double a = Hr[(size_t)i * m + k], b = Hr[(size_t)(i + 1) * m + k];
                    Hr[(size_t)i * m + k] = cs[r][i] * a + sn[r][i] * b;
                    Hr[(size_t)(i + 1) * m + k] = -sn[r][i] * a + cs[r][i] * b;
                }
                double a = Hr[(size_t)k * m + k], b = Hr[(size_t)k1 * m + k];
                double rr = std::sqrt(a * a + b * b);
                cs[r][k] = rr == 0.0 ? 1.0 : a / rr;
                sn[r][k] = rr == 0.0 ? 0.0 : b / rr;
                Hr[(size_t)k * m + k] = rr;
                Hr[(size_t)k1 * m + k] = 0.0;
                g[r][k1] = -sn[r][k] * g[r][k];
                g[r][k] = cs[r][k] * g[r][k];
                kr[r] = k1;
                iters[r] += 1;
                double est = std::fabs(g[r][k1]) / fn[r];
                hist[r].push_back(est);
                if (est <= sp->tol || hn == 0.0) frozen[r] = 1;
                else stop = false;
            }
            if (breakdown) break;
            CK(cudaMemcpyAsync(W.inv.get(), inv2.data(), sizeof(double) * R, cudaMemcpyHostToDevice, s));
            scaleR_k<R><<<grid_for(nR, 256), 256, 0, s>>>(W.w.get(), W.inv.get(), W.V.get() + (int64_t)k1 * nR, nR);
            CK_LAUNCH();
            if (stop) { ++k; break; }
        }
        if (breakdown) break;
        // u += Z y per column (y_r has kr[r] entries)
        std::vector<double> Y((size_t)(m + 1) * R, 0.0);
        int kmax = 0;
        for (int r = 0; r < R; ++r) {
            const int kk = kr[r];
            kmax = std::max(kmax, kk);
            std::vector<double> yr(kk);
            for (int i = kk - 1; i >= 0; --i) {
                double acc = g[r][i];
                for (int j2 = i + 1; j2 < kk; ++j2) acc -= Hm[r][(size_t)i * m + j2] * yr[j2];
                yr[i] = acc / Hm[r][(size_t)i * m + i];
            }
            for (int i = 0; i < kk; ++i) Y[(size_t)i * R + r] = yr[i];
        }
        if (kmax > 0) {
            CK(cudaMemcpyAsync(W.y.get(), Y.data(), sizeof(double) * kmax * R, cudaMemcpyHostToDevice, s));
            updateR_k<T, R><<<grid_for(nR, 256), 256, 0, s>>>(Z, nR, kmax, W.y.get(), W.u.get(), nR);
            CK_LAUNCH();
            CK(cudaStreamSynchronize(s));
        }
    }
    scatterR_k<double, R><<<grid_for(nR, 256), 256, 0, s>>>(W.u.get(), nrhs, ordc, U, n);
    CK_LAUNCH();
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bool all_ok = !breakdown;
    for (int r = 0; r < nrhs; ++r) {
        all_ok = all_ok && rel[r] <= sp->tol;
        if (info) {
            info[r].iters = iters[r];
            info[r].rel_res = rel[r];
            info[r].solve_ms = ms;
            if (info[r].history && info[r].history_len > 0)
                for (int i = 0; i < info[r].history_len; ++i) info[r].history[i] = i < (int)hist[r].size() ? hist[r][i] : 0.0;
        }
    }
    if (breakdown) fail(MGM_ERR_BREAKDOWN, "breakdown: non-finite value in the iteration");
    if (!all_ok) {
        set_error("not converged: at least one right-hand side above tol after maxit");
        throw Fail{MGM_ERR_NOT_CONVERGED};
    }
}

void solve_multi(mgm_hierarchy* H, int nrhs, const double* F, double* U, const mgm_solve_params* sp, mgm_solve_info* info,
                 cudaStream_t s) {
    REQUIRE(H && F && U && sp, "null argument");
    REQUIRE(nrhs >= 1 && nrhs <= 8, "nrhs must be in [1, 8]");
    REQUIRE(!H->bordered, "many right-hand sides: not for constrained (bordered) hierarchies");
    REQUIRE(H->cycle == MGM_CYCLE_V, "many right-hand sides: V-cycle hierarchies only");
    REQUIRE(sp->krylov == MGM_KRYLOV_FGMRES || sp->krylov == MGM_KRYLOV_NONE, "unknown krylov method");
    REQUIRE(sp->maxit >= 0 && sp->tol >= 0.0, "maxit and tol must be >= 0");
    REQUIRE(sp->krylov != MGM_KRYLOV_FGMRES || (sp->restart >= 1 && sp->restart <= 200), "restart must be in [1, 200]");
    const int R = nrhs <= 1 ? 1 : nrhs <= 2 ? 2 : nrhs <= 4 ? 4 : 8;
    const bool f32 = H->precision == MGM_F32;
#define MGM_CASE(RR)                                                               \
    case RR:                                                                       \
        if (f32) solve_multi_t<float, RR>(H, nrhs, F, U, sp, info, s);             \
        else solve_multi_t<double, RR>(H, nrhs, F, U, sp, info, s);                \
        break;
    switch (R) {
        MGM_CASE(1)
        MGM_CASE(2)
        MGM_CASE(4)
        MGM_CASE(8)
    }
#undef MGM_CASE
}

// Problems of a batch on a pool of host threads, each driving its problems' solves on a stream of
// its own: the problems' kernels run concurrently on the device (a small problem alone leaves most
// of the SMs idle between its dependent launches). The pool takes problems from a shared counter.
void solve_batched(mgm_hierarchy* const* H, int nprob, const double* const* F, double* const* U, int nrhs,
                   const mgm_solve_params* sp, mgm_solve_info* info, mgm_status* status, cudaStream_t s) {
    REQUIRE(H && F && U && sp && nprob >= 1, "bad argument");
    for (int q = 0; q < nprob; ++q) {
        REQUIRE(H[q] && F[q] && U[q], "null problem");
        for (int r = 0; r < q; ++r) REQUIRE(H[r] != H[q], "a hierarchy appears twice in the batch");
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    cudaEvent_t start;
    CK(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    CK(cudaEventRecord(start, s));  // work of the caller's stream before the batch (F, U) comes first
    const int nthreads = std::min(nprob, BATCH_THREADS);
    std::atomic<int> next{0};
    std::vector<mgm_status> st(nprob, MGM_OK);
    std::vector<std::string> msg(nprob);
    std::vector<cudaEvent_t> done(nthreads, nullptr);
    std::vector<std::thread> pool;
    std::vector<std::string> setup_err(nthreads);
    for (int t = 0; t < nthreads; ++t) {
        pool.emplace_back([&, t] {
            cudaStream_t ws = nullptr;
            const mgm_status ok = guarded([&] {
                CK(cudaSetDevice(dev));
                CK(cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking));
                CK(cudaStreamWaitEvent(ws, start, 0));
                CK(cudaEventCreateWithFlags(&done[t], cudaEventDisableTiming));
            });
            if (ok != MGM_OK) { setup_err[t] = error_message(); return; }
            for (int q = next++; q < nprob; q = next++) {
                st[q] = guarded([&] { solve_multi(H[q], nrhs, F[q], U[q], sp, info ? info + (size_t)q * nrhs : nullptr, ws); });
                if (st[q] != MGM_OK) msg[q] = error_message();
            }
            cudaEventRecord(done[t], ws);
            cudaStreamDestroy(ws);
        });
    }
    for (auto& th : pool) th.join();
    for (int t = 0; t < nthreads; ++t)
        if (done[t]) {
            cudaStreamWaitEvent(s, done[t], 0);
            cudaEventDestroy(done[t]);
        }
    cudaEventDestroy(start);
    for (int t = 0; t < nthreads; ++t)
        if (!setup_err[t].empty()) fail(MGM_ERR_CUDA, "batched solve: worker set-up failed: " + setup_err[t]);
    if (status)
        for (int q = 0; q < nprob; ++q) status[q] = st[q];
    // the most severe status of the batch (by code: breakdown, CUDA and OOM above non-convergence)
    int worst = -1;
    for (int q = 0; q < nprob; ++q)
        if (st[q] != MGM_OK && (worst < 0 || st[q] > st[worst])) worst = q;
    if (worst >= 0) {
        set_error("problem " + std::to_string(worst) + ": " + msg[worst]);
        throw Fail{st[worst]};
    }
}

void free_multi(mgm_hierarchy* H) {
    delete static_cast<MultiWork*>(H->multi);
    H->multi = nullptr;
}

}  // namespace mgm

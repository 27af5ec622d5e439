// The MGM V(nu1, nu2)-cycle (paper Alg. 3) on the device, as the linear preconditioner z = M r
// (zero initial guess on every level).
//
// Smoother: forward Gauss-Seidel (eq. (smoother), Table 1) in multicolour order: the rows of one
// colour are mutually independent, so a sweep is one kernel per colour over a contiguous row
// range. Rows are stored split into lower-colour and upper-colour parts (see hier.cuh). Starting
// from zero, the first sweep only needs the lower part (upper-colour unknowns are still zero),
// and its residual is then exactly -U e, because (D + L_lower) e = b row by row. So pre-smoothing
// plus the residual stream each level's matrix once, and post-smoothing streams it once more.
//
// Kernels assign G = 8 lanes to a row and read columns and values with 16-byte vector loads
// (rows start at multiples of 4 entries); gathered vector entries come from L1/L2 (RCM order
// keeps them local). The restriction (CSR of the transposed interpolation) and interpolation
// (ELL, width m) are one thread per row; the coarsest solve multiplies by the explicit FP64
// inverse, one warp per row. The whole cycle is captured once into a CUDA graph.
#include <algorithm>

#include "hier.cuh"

namespace mgm {

constexpr int G = 8;          // lanes per row
constexpr int VBLOCK = 256;   // threads per block -> 32 rows per block

template <class T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// same sums with L2-coherent loads of x (ld.global.cg): inside one persistent launch, x is written
// by other blocks between grid barriers, so it must not be served from a stale L1 line
__device__ __forceinline__ float row_sum_cg(const int32_t* __restrict__ sc, const float* __restrict__ sv, int32_t beg,
                                            int32_t end, const float* x, int gl, float acc) {
    for (int32_t p = beg + 4 * gl; p < end; p += 4 * G) {
        int4 c = __ldg(reinterpret_cast<const int4*>(sc + p));
        float4 v = __ldg(reinterpret_cast<const float4*>(sv + p));
        acc = fmaf(v.x, __ldcg(x + c.x), acc);
        acc = fmaf(v.y, __ldcg(x + c.y), acc);
        acc = fmaf(v.z, __ldcg(x + c.z), acc);
        acc = fmaf(v.w, __ldcg(x + c.w), acc);
    }
    return acc;
}
__device__ __forceinline__ double row_sum_cg(const int32_t* __restrict__ sc, const double* __restrict__ sv, int32_t beg,
                                             int32_t end, const double* x, int gl, double acc) {
    for (int32_t p = beg + 4 * gl; p < end; p += 4 * G) {
        int4 c = __ldg(reinterpret_cast<const int4*>(sc + p));
        double2 v0 = __ldg(reinterpret_cast<const double2*>(sv + p));
        double2 v1 = __ldg(reinterpret_cast<const double2*>(sv + p + 2));
        acc = fma(v0.x, __ldcg(x + c.x), acc);
        acc = fma(v0.y, __ldcg(x + c.y), acc);
        acc = fma(v1.x, __ldcg(x + c.z), acc);
        acc = fma(v1.y, __ldcg(x + c.w), acc);
    }
    return acc;
}

template <class T>
__device__ __forceinline__ T group_reduce(T v) {
    for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Programmatic dependent launch (pdl_trigger / pdl_wait / launch_pdl in common.cuh): every kernel
// of the cycle lets its successor be scheduled as soon as all of its own blocks are running, and
// waits for its predecessor's completion and memory before it reads anything the predecessor
// writes. Work that only reads the level's static operators (row structure, columns, values) is
// issued before the wait, so it overlaps the predecessor's tail.

// Streamed operator data (columns, values, row structure) is loaded with an L2 evict-first policy,
// so that it does not push the gathered vector out of L2 (the matrix of a level is far larger than
// L2; the vector is a few MB and is gathered ~50 times per pass).
__device__ __forceinline__ uint64_t stream_policy() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ int4 ld_stream(const int4* q, uint64_t pol) {
    int4 v;
    asm("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(q), "l"(pol));
    return v;
}
__device__ __forceinline__ float4 ld_stream(const float4* q, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(q), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_stream(const double2* q, uint64_t pol) {
    double2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(q), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_stream(const int32_t* q, uint64_t pol) {
    int32_t v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(q), "l"(pol));
    return v;
}

__device__ __forceinline__ float ld_stream_t(const float* q, uint64_t pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(q), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_stream_t(const double* q, uint64_t pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(q), "l"(pol));
    return v;
}

// a transfer weight: FP32 as stored, or a BF16 bit pattern widened to FP32 (exact)
__device__ __forceinline__ float ld_weight(const float* q, uint64_t pol) { return ld_stream_t(q, pol); }
__device__ __forceinline__ double ld_weight(const double* q, uint64_t pol) { return ld_stream_t(q, pol); }
__device__ __forceinline__ float ld_weight(const uint16_t* q, uint64_t pol) {
    unsigned short v;
    asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(q), "l"(pol));
    return __uint_as_float((unsigned)v << 16);
}

template <class T>
struct Quad;
template <>
struct Quad<float> {
    float x, y, z, w;
    __device__ __forceinline__ static Quad load(const float* p) {
        float4 v = __ldg(reinterpret_cast<const float4*>(p));
        return {v.x, v.y, v.z, v.w};
    }
    __device__ __forceinline__ static Quad load(const float* p, uint64_t pol) {
        float4 v = ld_stream(reinterpret_cast<const float4*>(p), pol);
        return {v.x, v.y, v.z, v.w};
    }
};
template <>
struct Quad<double> {
    double x, y, z, w;
    __device__ __forceinline__ static Quad load(const double* p) {
        double2 a = __ldg(reinterpret_cast<const double2*>(p));
        double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
        return {a.x, a.y, b.x, b.y};
    }
    __device__ __forceinline__ static Quad load(const double* p, uint64_t pol) {
        double2 a = ld_stream(reinterpret_cast<const double2*>(p), pol);
        double2 b = ld_stream(reinterpret_cast<const double2*>(p + 2), pol);
        return {a.x, a.y, b.x, b.y};
    }
};
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// MODE 0: e = (b - lower e) dinv   (first sweep from zero)
// MODE 1: e = (b - offdiag e) dinv (full sweep)
// MODE 2: s = -upper e             (residual after a first sweep from zero)
// MODE 3: s = b - diag e - offdiag e
// A row's products are summed lane-strided over its lower part, then over its upper part.
template <int MODE, class T>
__global__ void __launch_bounds__(VBLOCK) row_kernel(const int32_t* __restrict__ lo, const int32_t* __restrict__ up,
                                                     const int32_t* __restrict__ sc, const T* __restrict__ sv,
                                                     const T* __restrict__ dv, const T* __restrict__ b, T* e, T* s,
                                                     int32_t r0, int32_t r1) {
    pdl_trigger();
    const uint64_t pol = stream_policy();
    const int t = blockIdx.x * VBLOCK + threadIdx.x;
    const int32_t row = r0 + t / G;
    const int gl = t & (G - 1);
    const bool act = row < r1;
    // ranges [b0, e0) then [b1, e1)
    int32_t b0 = 0, e0 = 0, b1 = 0, e1 = 0;
    if (act) {
        if (MODE == 2) { b0 = ld_stream(up + row, pol); e0 = ld_stream(up + row + 1, pol); }
        else { b0 = ld_stream(lo + row, pol); e0 = ld_stream(lo + row + 1, pol); }
        if (MODE == 1 || MODE == 3) { b1 = ld_stream(up + row, pol); e1 = ld_stream(up + row + 1, pol); }
    }
    // the lane's first quad of columns and values of each range (static data) before the wait
    const int32_t p0 = b0 + 4 * gl, p1 = b1 + 4 * gl;
    const bool h0 = p0 < e0, h1 = p1 < e1;
    int4 c0 = make_int4(0, 0, 0, 0), c1 = make_int4(0, 0, 0, 0);
    Quad<T> v0{}, v1{};
    if (h0) { c0 = ld_stream(reinterpret_cast<const int4*>(sc + p0), pol); v0 = Quad<T>::load(sv + p0, pol); }
    if (h1) { c1 = ld_stream(reinterpret_cast<const int4*>(sc + p1), pol); v1 = Quad<T>::load(sv + p1, pol); }
    pdl_wait();
    T acc = T(0);
    if (h0) {
        acc = fma_t(v0.x, e[c0.x], acc);
        acc = fma_t(v0.y, e[c0.y], acc);
        acc = fma_t(v0.z, e[c0.z], acc);
        acc = fma_t(v0.w, e[c0.w], acc);
    }
    for (int32_t p = p0 + 4 * G; p < e0; p += 4 * G) {
        const int4 c = ld_stream(reinterpret_cast<const int4*>(sc + p), pol);
        const Quad<T> v = Quad<T>::load(sv + p, pol);
        acc = fma_t(v.x, e[c.x], acc);
        acc = fma_t(v.y, e[c.y], acc);
        acc = fma_t(v.z, e[c.z], acc);
        acc = fma_t(v.w, e[c.w], acc);
    }
    if (h1) {
        acc = fma_t(v1.x, e[c1.x], acc);
        acc = fma_t(v1.y, e[c1.y], acc);
        acc = fma_t(v1.z, e[c1.z], acc);
        acc = fma_t(v1.w, e[c1.w], acc);
    }
    for (int32_t p = p1 + 4 * G; p < e1; p += 4 * G) {
        const int4 c = ld_stream(reinterpret_cast<const int4*>(sc + p), pol);
        const Quad<T> v = Quad<T>::load(sv + p, pol);
        acc = fma_t(v.x, e[c.x], acc);
        acc = fma_t(v.y, e[c.y], acc);
        acc = fma_t(v.z, e[c.z], acc);
        acc = fma_t(v.w, e[c.w], acc);
    }
    acc = group_reduce(acc);
    if (act && gl == 0) {
        if (MODE == 0 || MODE == 1) e[row] = (b[row] - acc) * dv[row];
        else if (MODE == 2) s[row] = -acc;
        else s[row] = b[row] - dv[row] * e[row] - acc;
    }
}

// ------------------------------ persistent multicolour sweep ----------------------------------
// One cooperative launch runs every colour of a sweep; blocks meet at a grid barrier between
// colours. The barrier is a counter in global memory; each wait is bounded (spin limit), after
// which the block records MGM_ERR_TIMEOUT in the error word and every block leaves.
constexpr int PS_THREADS = 512;
constexpr int PS_ROWS = PS_THREADS / G;   // rows per block pass
constexpr unsigned long long PS_SPIN_LIMIT = 4000000ull;


template <int MODE, class T>
__global__ void __launch_bounds__(PS_THREADS) psweep_k(const int32_t* __restrict__ lo, const int32_t* __restrict__ up,
                                                       const int32_t* __restrict__ sc, const T* __restrict__ sv,
                                                       const T* __restrict__ dinv, const T* __restrict__ b, T* e,
                                                       const int32_t* __restrict__ cptr, int ncolors, unsigned* bar,
                                                       int* err, unsigned long long limit) {
    __shared__ int ok;
    const int gl = threadIdx.x & (G - 1);
    const int rloc = threadIdx.x / G;
    unsigned target = 0;
    for (int c = 0; c < ncolors; ++c) {
        const int32_t r0 = cptr[c], r1 = cptr[c + 1];
        for (int32_t base = r0 + (int32_t)blockIdx.x * PS_ROWS; base < r1; base += (int32_t)gridDim.x * PS_ROWS) {
            const int32_t row = base + rloc;
            const bool act = row < r1;
            T acc = T(0);
            if (act) {
                acc = row_sum_cg(sc, sv, lo[row], lo[row + 1], e, gl, acc);
                if (MODE != 0) acc = row_sum_cg(sc, sv, up[row], up[row + 1], e, gl, acc);
            }
            acc = group_reduce(acc);
            if (act && gl == 0) e[row] = (b[row] - acc) * dinv[row];
        }
        if (c + 1 < ncolors) {
            target += gridDim.x;
            if (gridDim.x == 1) __syncthreads();
            else if (!grid_barrier(bar, target, limit, err, &ok)) return;
        }
    }
}

// ------------------------------ dependency-driven multicolour sweep ---------------------------
// One launch per sweep. Rows are taken in groups of at most four consecutive rows of one colour,
// one warp per group (G lanes per row), the groups dealt round-robin to the resident warps; each
// warp takes its groups in increasing order, so the lowest unfinished group always finds its
// inputs ready and the sweep cannot deadlock. A group starts once every lower-part column of its
// rows carries its ready flag, which a row sets (release) right after storing its new value;
// upper-part columns are read from eold, a copy of e taken before the sweep. Every row therefore
// reads exactly the values it reads under per-colour launches, in the same order: the result is
// bit-identical. Waits are bounded: past the spin limit the warp records MGM_ERR_TIMEOUT in the
// error word and every warp leaves at its next wait.
constexpr int DS_THREADS = 256;
constexpr int DS_WARPS = DS_THREADS / 32;

__device__ __forceinline__ int ld_acquire_i32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_i32(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}



template <int MODE, class T>
__global__ void __launch_bounds__(DS_THREADS) dsweep_k(const int32_t* __restrict__ lo, const int32_t* __restrict__ up,
                                                       const int32_t* __restrict__ sc, const T* __restrict__ sv,
                                                       const T* __restrict__ dinv, const T* __restrict__ b, T* e,
                                                       const T* __restrict__ eold, const int32_t* __restrict__ gptr,
                                                       int32_t ngroups, int* flag, int* err, unsigned long long limit) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const int64_t W = (int64_t)gridDim.x * DS_WARPS;
    for (int64_t g = (int64_t)blockIdx.x * DS_WARPS + (threadIdx.x >> 5); g < ngroups; g += W) {
        const int32_t row = gptr[g] + lane / G;
        const bool act = row < gptr[g + 1];
        int32_t beg = 0, m = 0, ub = 0, ue = 0;
        if (act) {
            beg = lo[row];
            m = lo[row + 1];
            if (MODE != 0) { ub = up[row]; ue = up[row + 1]; }
        }
        unsigned long long it = 0;
        for (;;) {  // every lower-part column final? (padding entries point at the row itself)
            bool ready = true;
            for (int32_t p = beg + 4 * gl; p < m && ready; p += 4 * G) {
                const int4 c = __ldg(reinterpret_cast<const int4*>(sc + p));
                ready = (c.x == row || ld_acquire_i32(flag + c.x)) && (c.y == row || ld_acquire_i32(flag + c.y)) &&
                        (c.z == row || ld_acquire_i32(flag + c.z)) && (c.w == row || ld_acquire_i32(flag + c.w));
            }
            if (__all_sync(0xffffffffu, ready)) break;
            int quit = 0;
            if (lane == 0) {
                if (*(volatile int*)err) quit = 1;
                else if (++it > limit) { atomicOr(err, MGM_ERR_TIMEOUT); quit = 1; }
            }
            if (__shfl_sync(0xffffffffu, quit, 0)) return;
            __nanosleep(64);
        }
        T acc = T(0);
        for (int32_t p = beg + 4 * gl; p < m; p += 4 * G) {  // the order of row_kernel
            const int4 c = __ldg(reinterpret_cast<const int4*>(sc + p));
            const Quad<T> v = Quad<T>::load(sv + p);
            acc = fma_t(v.x, __ldcg(e + c.x), acc);
            acc = fma_t(v.y, __ldcg(e + c.y), acc);
            acc = fma_t(v.z, __ldcg(e + c.z), acc);
            acc = fma_t(v.w, __ldcg(e + c.w), acc);
        }
        for (int32_t p = ub + 4 * gl; p < ue; p += 4 * G) {
            const int4 c = __ldg(reinterpret_cast<const int4*>(sc + p));
            const Quad<T> v = Quad<T>::load(sv + p);
            acc = fma_t(v.x, __ldg(eold + c.x), acc);
            acc = fma_t(v.y, __ldg(eold + c.y), acc);
            acc = fma_t(v.z, __ldg(eold + c.z), acc);
            acc = fma_t(v.w, __ldg(eold + c.w), acc);
        }
        acc = group_reduce(acc);
        if (act && gl == 0) {
            e[row] = (b[row] - acc) * dinv[row];
            st_release_i32(flag + row, 1);
        }
    }
}

// a barrier that nobody completes: the wait must end at its limit with MGM_ERR_TIMEOUT
__global__ void barrier_timeout_probe_k(unsigned* bar, int* err, unsigned long long limit) {
    __shared__ int ok;
    grid_barrier(bar, gridDim.x + 1, limit, err, &ok);
}

// W: the stored weight type (T, or uint16_t BF16 bit patterns for the FP32 cycle)
template <class T, class W = T>
__global__ void restrict_k(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, const W* __restrict__ v,
                           const T* __restrict__ s, T* bn, int64_t nc) {
    pdl_trigger();
    pdl_wait();
    const uint64_t pol = stream_policy();
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    T acc = T(0);
    for (int32_t q = rp[c]; q < rp[c + 1]; ++q) acc += (T)ld_weight(v + q, pol) * s[ld_stream(ci + q, pol)];
    bn[c] = acc;
}

template <class T, class W = T>
__global__ void interp_k(const int32_t* __restrict__ pc, const W* __restrict__ pv, int pw, const T* __restrict__ en, T* e,
                         int64_t n) {
    pdl_trigger();
    pdl_wait();
    const uint64_t pol = stream_policy();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T acc = e[i];
    for (int t = 0; t < pw; ++t) acc += (T)ld_weight(pv + i * pw + t, pol) * en[ld_stream(pc + i * pw + t, pol)];
    e[i] = acc;
}

// restriction / interpolation launches of one level pair, with the level's stored weight type
template <class T>
static void launch_restrict(mgm_hierarchy* H, Level& L, Level& C, const T* rsrc, cudaStream_t s);
template <class T>
static void launch_interp(mgm_hierarchy* H, Level& L, Level& C, cudaStream_t s);

template <class T>
__global__ void coarse_k(const double* __restrict__ Ainv, const T* __restrict__ b, T* e, int64_t n) {
    pdl_trigger();
    pdl_wait();
    int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double acc = 0.0;
    for (int64_t j = lane; j < n; j += 32) acc = fma(Ainv[row * n + j], (double)b[j], acc);
    acc = warp_sum(acc);
    if (lane == 0) e[row] = (T)acc;
}

template <class T>
__global__ void copy_k(const T* a, T* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

template <class TI, class TO>
__global__ void load_k(const TI* src, const int32_t* gather, TO* dst, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (TO)src[gather ? gather[i] : i];
}
template <class TI, class TO>
__global__ void store_k(const TI* src, const int32_t* scatter, TO* dst, int64_t n, int add) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = scatter ? scatter[i] : i;
    dst[j] = add ? (TO)((double)dst[j] + (double)src[i]) : (TO)src[i];
}

// ------------------------------ level accessors ----------------------------------------------
template <class T> struct LV;
template <> struct LV<float> {
    static float* b(Level& L) { return L.b32.get(); }
    static float* e(Level& L) { return L.e32.get(); }
    static float* s(Level& L) { return L.s32.get(); }
    static const float* sv(Level& L) { return L.sv32.get(); }
    static const float* diag(Level& L) { return L.diag32.get(); }
    static const float* dinv(Level& L) { return L.dinv32.get(); }
    static const float* pv(Level& L) { return L.pv32.get(); }
    static const float* rv(Level& L) { return L.r_v32.get(); }
    static float* eold(Level& L) { return L.eold32.get(); }
    static const float* c(Level& L) { return L.c32.get(); }
};
template <> struct LV<double> {
    static double* b(Level& L) { return L.b64.get(); }
    static double* e(Level& L) { return L.e64.get(); }
    static double* s(Level& L) { return L.s64.get(); }
    static const double* sv(Level& L) { return L.sv64.get(); }
    static const double* diag(Level& L) { return L.diag64.get(); }
    static const double* dinv(Level& L) { return L.dinv64.get(); }
    static const double* pv(Level& L) { return L.pv64.get(); }
    static const double* rv(Level& L) { return L.r_v64.get(); }
    static double* eold(Level& L) { return L.eold64.get(); }
    static const double* c(Level& L) { return L.c64.get(); }
};

template <class T>
static void launch_restrict(mgm_hierarchy* H, Level& L, Level& C, const T* rsrc, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (H->transfer_bf16) {
            launch_pdl(restrict_k<float, uint16_t>, grid_for(C.n, 256), 256, s, (const int32_t*)L.r_rp.get(),
                       (const int32_t*)L.r_ci.get(), (const uint16_t*)L.r_v16.get(), rsrc, LV<T>::b(C), (int64_t)C.n);
            return;
        }
    }
    launch_pdl(restrict_k<T>, grid_for(C.n, 256), 256, s, (const int32_t*)L.r_rp.get(), (const int32_t*)L.r_ci.get(),
               LV<T>::rv(L), rsrc, LV<T>::b(C), (int64_t)C.n);
}

template <class T>
static void launch_interp(mgm_hierarchy* H, Level& L, Level& C, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (H->transfer_bf16) {
            launch_pdl(interp_k<float, uint16_t>, grid_for(L.n, 256), 256, s, (const int32_t*)L.pc.get(),
                       (const uint16_t*)L.pv16.get(), L.pw, (const T*)LV<T>::e(C), LV<T>::e(L), (int64_t)L.n);
            return;
        }
    }
    launch_pdl(interp_k<T>, grid_for(L.n, 256), 256, s, (const int32_t*)L.pc.get(), LV<T>::pv(L), L.pw,
               (const T*)LV<T>::e(C), LV<T>::e(L), (int64_t)L.n);
}

template <int MODE, class T>
static void launch_rows(Level& L, int32_t r0, int32_t r1, cudaStream_t s) {
    if (r1 <= r0) return;
    const int64_t threads = (int64_t)(r1 - r0) * G;
    const T* dv = (MODE == 3) ? LV<T>::diag(L) : LV<T>::dinv(L);
    launch_pdl(row_kernel<MODE, T>, grid_for(threads, VBLOCK), VBLOCK, s, (const int32_t*)L.lo.get(),
               (const int32_t*)L.up.get(), (const int32_t*)L.sc.get(), LV<T>::sv(L), dv, (const T*)LV<T>::b(L),
               LV<T>::e(L), LV<T>::s(L), r0, r1);
}

// blocks for a persistent sweep: enough to cover the largest colour in one pass, at most what can
// be co-resident (a cooperative launch requires all blocks resident)
template <int MODE, class T>
static void launch_psweep(mgm_hierarchy* H, Level& L, cudaStream_t s) {
    const int nc = (int)L.cptr.size() - 1;
    if (nc <= 0) return;
    int maxrows = 0;
    for (int c = 0; c < nc; ++c) maxrows = std::max(maxrows, L.cptr[c + 1] - L.cptr[c]);
    const int mb = coresident_blocks((const void*)psweep_k<MODE, T>, PS_THREADS, 0, 0);
    const int nblocks = std::max(1, std::min(mb, (maxrows + PS_ROWS - 1) / PS_ROWS));
    CK(cudaMemsetAsync(L.bar.get(), 0, sizeof(unsigned), s));
    const int32_t* lo = L.lo.get();
    const int32_t* up = L.up.get();
    const int32_t* sc = L.sc.get();
    const T* sv = LV<T>::sv(L);
    const T* dv = LV<T>::dinv(L);
    const T* b = LV<T>::b(L);
    T* e = LV<T>::e(L);
    const int32_t* cp = L.cptr_dev.get();
    unsigned* bar = L.bar.get();
    int* err = H->err.get();
    unsigned long long limit = PS_SPIN_LIMIT;
    void* args[] = {(void*)&lo, (void*)&up, (void*)&sc, (void*)&sv, (void*)&dv, (void*)&b, (void*)&e, (void*)&cp,
                    (void*)&nc, (void*)&bar, (void*)&err, (void*)&limit};
    CK(cudaLaunchCooperativeKernel((const void*)psweep_k<MODE, T>, dim3(nblocks), dim3(PS_THREADS), args, 0, s));
    CK_LAUNCH();
}

template <int MODE, class T>
static void launch_dsweep(mgm_hierarchy* H, Level& L, cudaStream_t s) {
    if (L.ngroups <= 0) return;
    const int mb = coresident_blocks((const void*)dsweep_k<MODE, T>, DS_THREADS, 0, 0);
    const int nblocks = std::max(1, std::min(mb, (L.ngroups + DS_WARPS - 1) / DS_WARPS));
    CK(cudaMemsetAsync(L.flag.get(), 0, sizeof(int) * L.n, s));
    T* e = LV<T>::e(L);
    T* eold = LV<T>::eold(L);
    if (MODE == 1) CK(cudaMemcpyAsync(eold, e, sizeof(T) * L.n, cudaMemcpyDeviceToDevice, s));
    const int32_t* lo = L.lo.get();
    const int32_t* up = L.up.get();
    const int32_t* sc = L.sc.get();
    const T* sv = LV<T>::sv(L);
    const T* dv = LV<T>::dinv(L);
    const T* b = LV<T>::b(L);
    const T* eo = eold;
    const int32_t* gp = L.gptr.get();
    int32_t ng = L.ngroups;
    int* flag = L.flag.get();
    int* err = H->err.get();
    unsigned long long limit = PS_SPIN_LIMIT;
    void* args[] = {(void*)&lo, (void*)&up, (void*)&sc, (void*)&sv, (void*)&dv, (void*)&b, (void*)&e, (void*)&eo,
                    (void*)&gp, (void*)&ng, (void*)&flag, (void*)&err, (void*)&limit};
    CK(cudaLaunchCooperativeKernel((const void*)dsweep_k<MODE, T>, dim3(nblocks), dim3(DS_THREADS), args, 0, s));
    CK_LAUNCH();
}

template <class T>
static void sweep(Level& L, bool from_zero, cudaStream_t s) {
    for (size_t c = 0; c + 1 < L.cptr.size(); ++c) {
        if (from_zero) launch_rows<0, T>(L, L.cptr[c], L.cptr[c + 1], s);
        else launch_rows<1, T>(L, L.cptr[c], L.cptr[c + 1], s);
    }
}

// one forward sweep of level L (from zero: lower parts only)
template <class T>
static void sweep_any(mgm_hierarchy* H, Level& L, bool from_zero, cudaStream_t s) {
    if (L.stream) {
        stream_sweep<T>(H, L, from_zero ? 0 : 1, false, s);
    } else if (L.csched) {
        colour_sweep<T>(H, L, from_zero ? 0 : 1, s);
    } else if (H->sweep_mode == 2) {
        if (from_zero) launch_dsweep<0, T>(H, L, s);
        else launch_dsweep<1, T>(H, L, s);
    } else if (H->sweep_mode == 1) {
        if (from_zero) launch_psweep<0, T>(H, L, s);
        else launch_psweep<1, T>(H, L, s);
    } else {
        sweep<T>(L, from_zero, s);
    }
}

// pre-smoothing of level L from a zero initial guess and its residual s = b - L e (Alg. 3's
// descent at one level): nu1 sweeps, the first from zero; with nu1 = 1 the residual is -U e
template <class T>
static const T* presmooth_residual(mgm_hierarchy* H, Level& L, cudaStream_t s) {
    if (H->nu1 == 1 && L.stream) {
        stream_sweep<T>(H, L, 0, true, s);  // sweep and residual in one launch
        return LV<T>::s(L);
    }
    sweep_any<T>(H, L, true, s);
    for (int t = 1; t < H->nu1; ++t) sweep_any<T>(H, L, false, s);
    if (H->nu1 == 1) launch_rows<2, T>(L, 0, (int32_t)L.n, s);
    else launch_rows<3, T>(L, 0, (int32_t)L.n, s);
    return LV<T>::s(L);
}

// ------------------------------ the bordered cycle (Sec. 4.4) -------------------------------------
// Constraint residual chain of the descent: s_{j+1} = s_j - c_j . e_j (the border row of level j
// is c_j^T), accumulated in FP64 with fixed block partials; the coarsest right-hand side carries
// s_p in its last entry. Before post-smoothing, b_j <- b_j - c_j mu with mu the coarsest
// multiplier (passed up unchanged by the interpolation), so the sweep smooths u only.
constexpr int BDOT_BLOCKS = 256;
template <class T>
__global__ void __launch_bounds__(256) bdot_k(const T* __restrict__ c, const T* __restrict__ e, int64_t n, double* part) {
    __shared__ double red[8];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t)blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    double acc = 0.0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += 256) acc = fma((double)c[i], (double)e[i], acc);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q];
        part[blockIdx.x] = t;
    }
}
template <class T>
__global__ void bdot_final_k(const double* part, int nb, double* sres, int j, T* bcoarse) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) acc += part[b];
    acc = warp_sum(acc);
    if (threadIdx.x == 0) {
        const double v = sres[j] - acc;
        sres[j + 1] = v;
        if (bcoarse) *bcoarse = (T)v;
    }
}
template <class T>
__global__ void bshift_k(T* b, const T* __restrict__ c, const T* mu, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = b[i] - c[i] * *mu;
}

template <class T>
static void cycle_rec(mgm_hierarchy* H, int j, int type, bool zero_start, cudaStream_t s);

template <class T>
static void vcycle_launches(mgm_hierarchy* H, cudaStream_t s) {
    if (H->cycle != MGM_CYCLE_V) {
        cycle_rec<T>(H, 0, H->cycle, true, s);
        return;
    }
    const int p = H->p;
    // levels tail_top..p-1 in one cluster launch (FP32 unconstrained V(1,1)-cycles; tail.cu)
    const int top = (sizeof(T) == 4 && !H->bordered) ? H->tail_top : 0;
    const int jd = top ? top : p - 1;  // levels smoothed by per-colour launches: 0..jd-1
    for (int j = 0; j < jd; ++j) {  // pre-smoothing and restricted residuals
        Level& L = H->lv[j];
        Level& C = H->lv[j + 1];
        const T* rsrc;
        if (H->nu1 >= 1) {
            rsrc = presmooth_residual<T>(H, L, s);
        } else {
            CK(cudaMemsetAsync(LV<T>::e(L), 0, sizeof(T) * L.n, s));
            rsrc = LV<T>::b(L);
        }
        if (H->bordered) {  // s_{j+1} = s_j - c_j . e_j
            bdot_k<T><<<BDOT_BLOCKS, 256, 0, s>>>(LV<T>::c(L), LV<T>::e(L), L.n, H->bpart.get());
            CK_LAUNCH();
            bdot_final_k<T><<<1, 32, 0, s>>>(H->bpart.get(), BDOT_BLOCKS, H->sres.get(), j,
                                             j + 2 == p ? LV<T>::b(C) + C.n : nullptr);
            CK_LAUNCH();
        }
        launch_restrict<T>(H, L, C, rsrc, s);
    }
    if (top) {
        tail_launch(H, s);
    } else {   // coarsest defect (bordered: with the multiplier in the last entry)
        Level& C = H->lv[p - 1];
        launch_pdl(coarse_k<T>, grid_for(H->nb * 32, 256), 256, s, (const double*)H->Ainv.get(), (const T*)LV<T>::b(C),
                   LV<T>::e(C), (int64_t)H->nb);
    }
    for (int j = jd - 1; j >= 0; --j) {  // interpolate / correct, post-smooth
        Level& L = H->lv[j];
        Level& C = H->lv[j + 1];
        launch_interp<T>(H, L, C, s);
        if (H->bordered) {  // smooth u only: b_j <- b_j - c_j mu
            const T* mu = LV<T>::e(H->lv[p - 1]) + H->np;
            bshift_k<T><<<grid_for(L.n, 256), 256, 0, s>>>(LV<T>::b(L), LV<T>::c(L), mu, L.n);
            CK_LAUNCH();
        }
        for (int t = 0; t < H->nu2; ++t) sweep_any<T>(H, L, false, s);
    }
}

// W- and F-cycles (Sec. 4.5), recursive: level j smooths (from zero on a first visit, with the
// lower-part sweep and the -U e residual identity, as the V-cycle; otherwise full sweeps from the
// current iterate and the full residual), restricts, visits level j+1 (V: once; W: twice, the second
// from the first's result; F: an F-cycle, then a V-cycle from its result), interpolates and
// post-smooths. The coarsest visit applies the inverse, which ignores the starting iterate.
template <class T>
static void cycle_rec(mgm_hierarchy* H, int j, int type, bool zero_start, cudaStream_t s) {
    const int p = H->p;
    if (j == p - 1) {
        Level& C = H->lv[p - 1];
        launch_pdl(coarse_k<T>, grid_for(H->nb * 32, 256), 256, s, (const double*)H->Ainv.get(), (const T*)LV<T>::b(C),
                   LV<T>::e(C), (int64_t)H->nb);
        return;
    }
    Level& L = H->lv[j];
    Level& C = H->lv[j + 1];
    const T* rsrc;
    if (zero_start && H->nu1 >= 1) {
        rsrc = presmooth_residual<T>(H, L, s);
    } else if (zero_start) {
        CK(cudaMemsetAsync(LV<T>::e(L), 0, sizeof(T) * L.n, s));
        rsrc = LV<T>::b(L);
    } else {
        for (int t = 0; t < H->nu1; ++t) sweep_any<T>(H, L, false, s);
        launch_rows<3, T>(L, 0, (int32_t)L.n, s);  // s = b - L e
        rsrc = LV<T>::s(L);
    }
    launch_restrict<T>(H, L, C, rsrc, s);
    if (type == MGM_CYCLE_V) {
        cycle_rec<T>(H, j + 1, MGM_CYCLE_V, true, s);
    } else if (type == MGM_CYCLE_W) {
        cycle_rec<T>(H, j + 1, MGM_CYCLE_W, true, s);
        cycle_rec<T>(H, j + 1, MGM_CYCLE_W, false, s);
    } else {
        cycle_rec<T>(H, j + 1, MGM_CYCLE_F, true, s);
        cycle_rec<T>(H, j + 1, MGM_CYCLE_V, false, s);
    }
    launch_interp<T>(H, L, C, s);
    for (int t = 0; t < H->nu2; ++t) sweep_any<T>(H, L, false, s);
}

void alloc_work(mgm_hierarchy* H) {
    H->err.alloc(1);
    CK(cudaMemset(H->err.get(), 0, sizeof(int)));
    for (int j = 0; j < H->p; ++j) {
        Level& L = H->lv[j];
        const bool smooth = j + 1 < H->p;
        if (smooth) {
            L.bar.alloc(1);
            L.cptr_dev.alloc(L.cptr.size());
            CK(cudaMemcpy(L.cptr_dev.get(), L.cptr.data(), sizeof(int32_t) * L.cptr.size(), cudaMemcpyHostToDevice));
        }
        if (smooth && H->sweep_mode == 2) {  // groups of <= 4 rows that never straddle a colour
            std::vector<int32_t> gp;
            for (size_t c = 0; c + 1 < L.cptr.size(); ++c)
                for (int32_t r = L.cptr[c]; r < L.cptr[c + 1]; r += 4) gp.push_back(r);
            gp.push_back((int32_t)L.n);
            L.ngroups = (int32_t)gp.size() - 1;
            L.gptr.alloc(gp.size());
            CK(cudaMemcpy(L.gptr.get(), gp.data(), sizeof(int32_t) * gp.size(), cudaMemcpyHostToDevice));
            L.flag.alloc(L.n);
            if (H->precision == MGM_F32) L.eold32.alloc(L.n);
            else L.eold64.alloc(L.n);
        }
        const int64_t nv = L.n + ((H->bordered && !smooth) ? 1 : 0);  // coarsest bordered: + multiplier
        if (H->precision == MGM_F32) {
            L.b32.alloc(nv); L.e32.alloc(nv);
            CK(cudaMemset(L.e32.get(), 0, sizeof(float) * nv));
            CK(cudaMemset(L.b32.get(), 0, sizeof(float) * nv));
            if (smooth) { L.s32.alloc(L.n); CK(cudaMemset(L.s32.get(), 0, sizeof(float) * L.n)); }
        } else {
            L.b64.alloc(nv); L.e64.alloc(nv);
            CK(cudaMemset(L.e64.get(), 0, sizeof(double) * nv));
            CK(cudaMemset(L.b64.get(), 0, sizeof(double) * nv));
            if (smooth) { L.s64.alloc(L.n); CK(cudaMemset(L.s64.get(), 0, sizeof(double) * L.n)); }
        }
    }
}

// the plain cycle's launches on s (into a capture the caller runs)
void vcycle_enqueue(mgm_hierarchy* H, cudaStream_t s) {
    if (H->precision == MGM_F32) vcycle_launches<float>(H, s);
    else vcycle_launches<double>(H, s);
}

bool& pdl_off() {
    static thread_local bool off = false;
    return off;
}

static cudaGraphExec_t capture(mgm_hierarchy* H, bool learned, int64_t* kernels) {
    cudaGraph_t g = nullptr;
    const int64_t before = thread_launches();
    CK(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal));
    try {
        if (H->precision == MGM_F32) {
            vcycle_launches<float>(H, H->cap_stream);
            if (learned) {  // s_0 = b_0 - L_0 e_0, then the learned correction of e_0
                Level& L0 = H->lv[0];
                launch_rows<3, float>(L0, 0, (int32_t)L0.n, H->cap_stream);
                learned_correct(H, H->cap_stream);
            }
        } else {
            vcycle_launches<double>(H, H->cap_stream);
        }
    } catch (...) {
        cudaStreamEndCapture(H->cap_stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    CK(cudaStreamEndCapture(H->cap_stream, &g));
    *kernels = thread_launches() - before;  // captured, not executed: counted per graph launch
    note_launch(-*kernels);
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return ex;
}

// drop the captured cycle graphs (after a level's sweep schedule changed); recaptured on next use
void invalidate_graphs(mgm_hierarchy* H) {
    if (H->vgraph) { CK(cudaGraphExecDestroy(H->vgraph)); H->vgraph = nullptr; }
    if (H->lgraph) { CK(cudaGraphExecDestroy(H->lgraph)); H->lgraph = nullptr; }
}

// Device time (ms) of level j's smoothing work in one V-cycle: pre-smoothing from zero with its
// residual, then the post-smoothing sweeps, captured in a graph as the cycle runs them and
// replayed `reps` times after two warm-ups. Overwrites the level's work vectors.
float time_level_smoothing(mgm_hierarchy* H, int j, int reps, cudaStream_t s) {
    REQUIRE(j >= 0 && j + 1 < H->p && reps >= 1, "bad level");
    if (!H->cap_stream) CK(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
    Level& L = H->lv[j];
    cudaGraph_t g = nullptr;
    const int64_t before = thread_launches();
    CK(cudaStreamBeginCapture(H->cap_stream, cudaStreamCaptureModeThreadLocal));
    try {
        if (H->precision == MGM_F32) {
            presmooth_residual<float>(H, L, H->cap_stream);
            for (int t = 0; t < H->nu2; ++t) sweep_any<float>(H, L, false, H->cap_stream);
        } else {
            presmooth_residual<double>(H, L, H->cap_stream);
            for (int t = 0; t < H->nu2; ++t) sweep_any<double>(H, L, false, H->cap_stream);
        }
    } catch (...) {
        cudaStreamEndCapture(H->cap_stream, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    CK(cudaStreamEndCapture(H->cap_stream, &g));
    note_launch(-(thread_launches() - before));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(e);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int t = 0; t < 2; ++t) CK(cudaGraphLaunch(ex, s));
    CK(cudaEventRecord(e0, s));
    for (int t = 0; t < reps; ++t) CK(cudaGraphLaunch(ex, s));
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(ex);
    check_device_error(H, s);
    return ms / reps;
}

void vcycle_prepare(mgm_hierarchy* H) {
    if (!H->cap_stream) CK(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
    if (!H->vgraph) H->vgraph = capture(H, false, &H->graph_kernels);
    if (H->learned && !H->lgraph) H->lgraph = capture(H, true, &H->lgraph_kernels);
}

void vcycle_plain(mgm_hierarchy* H, cudaStream_t s) {
    vcycle_prepare(H);
    CK(cudaGraphLaunch(H->vgraph, s));
    note_launch(H->graph_kernels);
}

void vcycle_core(mgm_hierarchy* H, cudaStream_t s) {
    vcycle_prepare(H);
    if (H->learned && H->learned_active) {
        CK(cudaGraphLaunch(H->lgraph, s));
        note_launch(H->lgraph_kernels);
    } else {
        CK(cudaGraphLaunch(H->vgraph, s));
        note_launch(H->graph_kernels);
    }
}

void load_input(mgm_hierarchy* H, const void* src, int dt, const int32_t* gather, cudaStream_t s) {
    Level& L = H->lv[0];
    const int64_t n = L.n;
    if (H->precision == MGM_F32) {
        if (dt == MGM_F64) load_k<double, float><<<grid_for(n, 256), 256, 0, s>>>((const double*)src, gather, L.b32.get(), n);
        else load_k<float, float><<<grid_for(n, 256), 256, 0, s>>>((const float*)src, gather, L.b32.get(), n);
    } else {
        if (dt == MGM_F64) load_k<double, double><<<grid_for(n, 256), 256, 0, s>>>((const double*)src, gather, L.b64.get(), n);
        else load_k<float, double><<<grid_for(n, 256), 256, 0, s>>>((const float*)src, gather, L.b64.get(), n);
    }
    CK_LAUNCH();
}

void store_output(mgm_hierarchy* H, void* dst, int dt, const int32_t* scatter, cudaStream_t s) {
    Level& L = H->lv[0];
    const int64_t n = L.n;
    if (H->precision == MGM_F32) {
        if (dt == MGM_F64) store_k<float, double><<<grid_for(n, 256), 256, 0, s>>>(L.e32.get(), scatter, (double*)dst, n, 0);
        else store_k<float, float><<<grid_for(n, 256), 256, 0, s>>>(L.e32.get(), scatter, (float*)dst, n, 0);
    } else {
        if (dt == MGM_F64) store_k<double, double><<<grid_for(n, 256), 256, 0, s>>>(L.e64.get(), scatter, (double*)dst, n, 0);
        else store_k<double, float><<<grid_for(n, 256), 256, 0, s>>>(L.e64.get(), scatter, (float*)dst, n, 0);
    }
    CK_LAUNCH();
}

// u[scatter[i]] += e_0[i] (FP64 accumulation), for the standalone MGM iteration
void add_output(mgm_hierarchy* H, double* dst, const int32_t* scatter, cudaStream_t s) {
    Level& L = H->lv[0];
    const int64_t n = L.n;
    if (H->precision == MGM_F32) store_k<float, double><<<grid_for(n, 256), 256, 0, s>>>(L.e32.get(), scatter, dst, n, 1);
    else store_k<double, double><<<grid_for(n, 256), 256, 0, s>>>(L.e64.get(), scatter, dst, n, 1);
    CK_LAUNCH();
}

// Algorithmic bytes of one V-cycle on level j (j + 1 < p): every stored off-diagonal entry (value +
// column) is read once per pass, per-row arrays (row starts, diagonal inverse, b, e, s) once per
// pass, transfer entries once; gathered vector entries are L2 hits and not counted.
static int64_t level_bytes(const mgm_hierarchy* H, int j) {
    const int64_t vs = H->precision == MGM_F32 ? 4 : 8, ent = vs + 4;
    const int64_t went = (H->transfer_bf16 ? 2 : vs) + 4;  // a transfer entry: weight + column
    const Level& L = H->lv[j];
    const Level& C = H->lv[j + 1];
    const int64_t n = L.n, nnzo = L.nlow + L.nupp;
    int64_t b = 0;
    if (H->nu1 >= 1) {
        b += L.nlow * ent + n * (8 + 3 * vs);                      // first sweep from zero (lower part)
        b += (int64_t)(H->nu1 - 1) * (nnzo * ent + n * (4 + 3 * vs));
        b += (H->nu1 == 1 ? L.nupp * ent + n * (4 + vs)           // residual -U e
                          : nnzo * ent + n * (4 + 4 * vs));        // residual b - A e
    }
    b += L.pnnz * went + (C.n + 1) * 4 + n * vs + C.n * vs;       // restriction
    b += L.pnnz * went + 2 * n * vs;                              // interpolation + correction
    b += (int64_t)H->nu2 * (nnzo * ent + n * (4 + 3 * vs));       // post-smoothing sweeps
    return b;
}

// the smoothing part of level_bytes: the pre-smoothing sweeps with their residual and the
// post-smoothing sweeps (what time_level_smoothing times)
int64_t level_smoothing_bytes(const mgm_hierarchy* H, int j) {
    const Level& L = H->lv[j];
    const Level& C = H->lv[j + 1];
    const int64_t vs = H->precision == MGM_F32 ? 4 : 8;
    const int64_t went = (H->transfer_bf16 ? 2 : vs) + 4;
    const int64_t transfers = L.pnnz * went + (C.n + 1) * 4 + L.n * vs + C.n * vs + L.pnnz * went + 2 * L.n * vs;
    return level_bytes(H, j) - transfers;
}

int64_t vcycle_bytes(const mgm_hierarchy* H) {
    int64_t b = 0;
    for (int j = 0; j + 1 < H->p; ++j) b += level_bytes(H, j);
    const int64_t vs = H->precision == MGM_F32 ? 4 : 8;
    b += H->np * H->np * 8 + 2 * H->np * vs;                          // coarsest solve
    return b;
}

// Lower bound of one V-cycle's time for schedules that separate a sweep's colours by kernel
// boundaries: level by level, the larger of its bytes at `gbs` GB/s and its chain of dependent
// launches (nu1 + nu2 sweeps of one launch per colour, residual, restriction, interpolation) at
// `chain_us` each, plus one launch for the coarsest solve. Bytes may overlap the latency of
// launches (a launch prefetches while its predecessor runs) but neither can shrink below itself.
double vcycle_floor_ms(const mgm_hierarchy* H, double chain_us, double gbs, double* bytes_ms, double* chain_ms) {
    double f = 0.0, bt = 0.0, ch = 0.0;
    for (int j = 0; j + 1 < H->p; ++j) {
        const Level& L = H->lv[j];
        const int64_t C = (int64_t)L.cptr.size() - 1;
        const double tb = (double)level_bytes(H, j) / (gbs * 1e6);
        const double tc = (double)((H->nu1 + H->nu2) * C + 3) * chain_us * 1e-3;
        f += std::max(tb, tc);
        bt += tb;
        ch += tc;
    }
    f += chain_us * 1e-3;
    ch += chain_us * 1e-3;
    if (bytes_ms) *bytes_ms = bt;
    if (chain_ms) *chain_ms = ch;
    return f;
}

void profile_vcycle(mgm_hierarchy* H, int reps, mgm_profile_info* out, cudaStream_t s) {
    REQUIRE(H && out && reps >= 1, "bad argument");
    vcycle_prepare(H);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float ms = 0.0f;
    out->learned_vcycle_ms = 0.0f;
    out->learned_ms = 0.0f;
    out->learned_bytes = 0;
    if (H->learned) {  // the cycle with the learned correction, and the correction kernel alone
        H->learned_active = true;
        for (int t = 0; t < 2; ++t) vcycle_core(H, s);
        CK(cudaEventRecord(e0, s));
        for (int t = 0; t < reps; ++t) vcycle_core(H, s);
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        out->learned_vcycle_ms = ms / reps;
        for (int t = 0; t < 2; ++t) learned_correct(H, s);
        CK(cudaEventRecord(e0, s));
        for (int t = 0; t < reps; ++t) learned_correct(H, s);
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        out->learned_ms = ms / reps;
        // per row: n stencil indices, 64 FP16 first-layer geometric terms, diagonal, e read and written
        out->learned_bytes = H->N * (4 * (int64_t)H->ln + 64 * 2 + 4 + 8);
    }
    for (int t = 0; t < 2; ++t) vcycle_plain(H, s);
    CK(cudaEventRecord(e0, s));
    for (int t = 0; t < reps; ++t) vcycle_plain(H, s);
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    out->vcycle_ms = ms / reps;
    out->vcycle_bytes = vcycle_bytes(H);
    out->vcycle_kernels = H->graph_kernels;
    out->sweep_ms = 0.0f;
    out->sweep_bytes = 0;
    out->sweep_launches = 0;
    if (H->p >= 2) {
        Level& L = H->lv[0];
        const int64_t vs = H->precision == MGM_F32 ? 4 : 8;
        for (int t = 0; t < 2; ++t) {
            if (H->precision == MGM_F32) sweep_any<float>(H, L, false, s);
            else sweep_any<double>(H, L, false, s);
        }
        CK(cudaEventRecord(e0, s));
        for (int t = 0; t < reps; ++t) {
            if (H->precision == MGM_F32) sweep_any<float>(H, L, false, s);
            else sweep_any<double>(H, L, false, s);
        }
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
        out->sweep_ms = ms / reps;
        out->sweep_bytes = (L.nlow + L.nupp) * (vs + 4) + L.n * (4 + 3 * vs);
        // kernels a sweep (copies not counted): one for the persistent and streamed schedules, one a
        // colour for the per-colour launches (plain or staged)
        const bool one = L.stream || (!L.csched && (H->sweep_mode == 1 || H->sweep_mode == 2));
        out->sweep_launches = one ? 1 : (int32_t)(L.cptr.size() - 1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

// reads and clears the device error word of the persistent kernels
void check_device_error(mgm_hierarchy* H, cudaStream_t s) {
    int e = read1(H->err.get(), s);
    if (e) {
        CK(cudaMemsetAsync(H->err.get(), 0, sizeof(int), s));
        stream_reset(H, s);
        fail(MGM_ERR_TIMEOUT, "a device-side barrier wait gave up (spin limit reached)");
    }
}

// Runs a grid barrier that can never complete (one arrival short) with the given spin limit and
// returns the error word: exercises the bounded-wait path without hanging anything.
int barrier_timeout_probe(int nblocks, unsigned long long limit, cudaStream_t s) {
    Temp<unsigned> bar(1, s);
    Temp<int> err(1, s);
    CK(cudaMemsetAsync(bar.get(), 0, sizeof(unsigned), s));
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    unsigned* b = bar.get();
    int* e = err.get();
    void* args[] = {(void*)&b, (void*)&e, (void*)&limit};
    CK(cudaLaunchCooperativeKernel((const void*)barrier_timeout_probe_k, dim3(nblocks), dim3(32), args, 0, s));
    CK_LAUNCH();
    return read1(err.get(), s);
}

template <class TA, class TB>
__global__ void cast1_k(const TA* a, TB* b) { *b = (TB)*a; }

void vcycle_api(mgm_hierarchy* H, const void* r, void* z, int dtype, cudaStream_t s) {
    REQUIRE(H && r && z, "null argument");
    REQUIRE(dtype == MGM_F32 || dtype == MGM_F64, "dtype must be MGM_F32 or MGM_F64");
    load_input(H, r, dtype, H->ord_caller.get(), s);
    if (H->bordered) {  // r_N: the constraint component
        if (dtype == MGM_F64) cast1_k<double, double><<<1, 1, 0, s>>>((const double*)r + H->N, H->sres.get());
        else cast1_k<float, double><<<1, 1, 0, s>>>((const float*)r + H->N, H->sres.get());
        CK_LAUNCH();
    }
    H->learned_active = true;
    vcycle_core(H, s);
    store_output(H, z, dtype, H->ord_caller.get(), s);
    if (H->bordered) {  // z_N: the multiplier correction
        Level& C = H->lv[H->p - 1];
        if (H->precision == MGM_F32) {
            if (dtype == MGM_F64) cast1_k<float, double><<<1, 1, 0, s>>>(C.e32.get() + H->np, (double*)z + H->N);
            else cast1_k<float, float><<<1, 1, 0, s>>>(C.e32.get() + H->np, (float*)z + H->N);
        } else {
            if (dtype == MGM_F64) cast1_k<double, double><<<1, 1, 0, s>>>(C.e64.get() + H->np, (double*)z + H->N);
            else cast1_k<double, float><<<1, 1, 0, s>>>(C.e64.get() + H->np, (float*)z + H->N);
        }
        CK_LAUNCH();
    }
    if (H->persistent) check_device_error(H, s);
}

}  // namespace mgm

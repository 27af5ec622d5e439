// Learned correction after the MGM V-cycle (an addition to the paper's method; plain multicolour
// Gauss-Seidel stays the fallback and the FP64 oracle judges every number).
//
// For the finest level, with stencil idx_i (centre first), tangent-plane offsets (xh, yh) and
// support s_i of Sec. 2.1, LBO weights c_ij and the residual r = b - L e left by the cycle:
//   features f[4j..4j+3] = (xh_j / s, yh_j / s, c_ij s^2, r_{idx_ij} / rho_i),
//   rho_i = sqrt(mean_j r_{idx_ij}^2),
//   out_i = w3 . relu(W2 relu(W1 f_i))        (4n -> 64 -> 64 -> 1, no biases),
//   e_i  += rho_i out_i / l_ii.
// Training minimises the relative residual left by the correction, J = |r - L delta|^2 / |r|^2,
// with dJ/d out_i = -2 (rho_i / l_ii) (L^T (r - L delta))_i / |r|^2 and Adam on FP32 master weights.
//
// Inference (once per V-cycle) splits W1 into its geometric columns, applied once per weight
// update (hg = W1_geo f_geo, 64 values per row), and its residual columns, so a cycle only gathers
// n residuals per row: h1 = relu(hg + W1_r r_stencil / rho). Weights are BF16 in memory and
// expanded exactly to FP32 in shared memory; all arithmetic accumulates in FP32. Per-row arrays
// are stored column-major ([j][N]) so one-thread-per-row loads coalesce.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "geom.cuh"
#include "hier.cuh"

struct mgm_mlp {
    int n = 0, din = 0;
    mgm::Buf<float> W, m, v;  // [W1 64 x din | W2 64 x 64 | w3 64], Adam moments
    int step = 0;
};

namespace mgm {

constexpr int HID = 64;
constexpr int LMAX_N = 48;
constexpr int LMAX_DIN = 4 * LMAX_N;
constexpr int OP_THREADS = 256;
constexpr int OP_TILE = 32;                                   // rows staged per outer-product step
constexpr int OP_MAXQ = (HID * LMAX_DIN + OP_THREADS - 1) / OP_THREADS;
constexpr int OP_CHUNKS = 304;                                // 2 x 152 SMs

inline int64_t mlp_count(int din) { return (int64_t)HID * din + HID * HID + HID; }

// ------------------------------ geometry and features ----------------------------------------
__global__ void attach_k(const double* xyz, const double* nrm, const int32_t* idx, const double* w, int n, int64_t N,
                         const int32_t* ordc, const int32_t* invc, int32_t* nbr, float* geo) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int64_t i = ordc[s];
    const int32_t* id = idx + i * n;
    double xh[LMAX_N], yh[LMAX_N];
    const double sup = project_support(xyz, nrm, i, id, n, xh, yh);
    for (int j = 0; j < n; ++j) {
        nbr[(int64_t)j * N + s] = invc[id[j]];
        geo[(int64_t)(3 * j + 0) * N + s] = sup > 0.0 ? (float)(xh[j] / sup) : 0.0f;
        geo[(int64_t)(3 * j + 1) * N + s] = sup > 0.0 ? (float)(yh[j] / sup) : 0.0f;
        geo[(int64_t)(3 * j + 2) * N + s] = (float)(w[i * n + j] * (sup * sup));
    }
}

__global__ void gather_cast_k(const double* src, const int32_t* ordc, float* dst, int64_t N) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < N) dst[s] = (float)src[ordc[s]];
}

// rows of features (row-major [row][4n]) in solve order, or at the caller's row when ordc is set
__global__ void features_k(const int32_t* nbr, const float* geo, const float* r, const float* diag, int n, int64_t N,
                           const int32_t* ordc, float* feat, float* rho_out, float* scale_out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    float ss = 0.0f;
    for (int j = 0; j < n; ++j) {
        const float v = r[nbr[(int64_t)j * N + s]];
        ss = fmaf(v, v, ss);
    }
    const float rho = sqrtf(ss / (float)n);
    const float ir = rho > 0.0f ? 1.0f / rho : 0.0f;
    const int64_t o = ordc ? (int64_t)ordc[s] : s;
    float* f = feat + o * 4 * n;
    for (int j = 0; j < n; ++j) {
        f[4 * j + 0] = geo[(int64_t)(3 * j + 0) * N + s];
        f[4 * j + 1] = geo[(int64_t)(3 * j + 1) * N + s];
        f[4 * j + 2] = geo[(int64_t)(3 * j + 2) * N + s];
        f[4 * j + 3] = r[nbr[(int64_t)j * N + s]] * ir;
    }
    if (rho_out) rho_out[o] = rho;
    if (scale_out) scale_out[o] = rho / diag[s];
}

// ------------------------------ FP32 network (training) ----------------------------------------
// W in shared memory as W1^T [din][64], W2 [64][64], w3 [64]
__device__ __forceinline__ void load_weights_t(const float* W, int din, float* sm) {
    const int n1 = HID * din;
    for (int q = threadIdx.x; q < n1; q += blockDim.x) {
        const int a = q / din, k = q - a * din;
        sm[k * HID + a] = W[q];
    }
    for (int q = threadIdx.x; q < HID * HID + HID; q += blockDim.x) sm[n1 + q] = W[n1 + q];
    __syncthreads();
}

// out = w3 . relu(W2 relu(W1 f)); activations stored column-major [64][B] when requested
__global__ void __launch_bounds__(128) fwd_k(const float* __restrict__ feat, int din, int64_t B, const float* __restrict__ W,
                                             float* out, float* h1s, float* h2s) {
    extern __shared__ __align__(16) float wsm[];
    load_weights_t(W, din, wsm);
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float* W1t = wsm;
    const float* W2 = wsm + HID * din;
    const float* w3 = W2 + HID * HID;
    const float* f = feat + b * din;
    float h[HID];
#pragma unroll
    for (int a = 0; a < HID; ++a) h[a] = 0.0f;
    for (int k = 0; k < din; ++k) {
        const float fk = f[k];
        const float4* wk = reinterpret_cast<const float4*>(W1t + k * HID);
#pragma unroll
        for (int q = 0; q < HID / 4; ++q) {
            const float4 c = wk[q];
            h[4 * q + 0] = fmaf(c.x, fk, h[4 * q + 0]);
            h[4 * q + 1] = fmaf(c.y, fk, h[4 * q + 1]);
            h[4 * q + 2] = fmaf(c.z, fk, h[4 * q + 2]);
            h[4 * q + 3] = fmaf(c.w, fk, h[4 * q + 3]);
        }
    }
#pragma unroll
    for (int a = 0; a < HID; ++a) h[a] = fmaxf(h[a], 0.0f);
    if (h1s) {
#pragma unroll
        for (int a = 0; a < HID; ++a) h1s[(int64_t)a * B + b] = h[a];
    }
    float o = 0.0f;
    for (int a = 0; a < HID; ++a) {
        const float4* wa = reinterpret_cast<const float4*>(W2 + a * HID);
        float z = 0.0f;
#pragma unroll
        for (int q = 0; q < HID / 4; ++q) {
            const float4 c = wa[q];
            z = fmaf(c.x, h[4 * q + 0], z);
            z = fmaf(c.y, h[4 * q + 1], z);
            z = fmaf(c.z, h[4 * q + 2], z);
            z = fmaf(c.w, h[4 * q + 3], z);
        }
        z = fmaxf(z, 0.0f);
        if (h2s) h2s[(int64_t)a * B + b] = z;
        o = fmaf(w3[a], z, o);
    }
    out[b] = o;
}

// d2 = g w3 [h2 > 0], d1 = (W2^T d2) [h1 > 0]   (relu(z) > 0 exactly when z > 0)
__global__ void __launch_bounds__(128) bwd_k(const float* __restrict__ gout, const float* __restrict__ W, int din, int64_t B,
                                             const float* __restrict__ h1s, const float* __restrict__ h2s, float* d1s,
                                             float* d2s) {
    __shared__ __align__(16) float sm[HID * HID + HID];
    for (int q = threadIdx.x; q < HID * HID + HID; q += blockDim.x) sm[q] = W[(int64_t)HID * din + q];
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float g = gout[b];
    float acc[HID];
#pragma unroll
    for (int k = 0; k < HID; ++k) acc[k] = 0.0f;
    for (int a = 0; a < HID; ++a) {
        const float d2 = h2s[(int64_t)a * B + b] > 0.0f ? g * sm[HID * HID + a] : 0.0f;
        d2s[(int64_t)a * B + b] = d2;
        const float4* wa = reinterpret_cast<const float4*>(sm + a * HID);
#pragma unroll
        for (int q = 0; q < HID / 4; ++q) {
            const float4 c = wa[q];
            acc[4 * q + 0] = fmaf(c.x, d2, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(c.y, d2, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(c.z, d2, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(c.w, d2, acc[4 * q + 3]);
        }
    }
#pragma unroll
    for (int k = 0; k < HID; ++k) d1s[(int64_t)k * B + b] = h1s[(int64_t)k * B + b] > 0.0f ? acc[k] : 0.0f;
}

// partial[c][a][k] = sum over the rows of chunk c of U[a][row] V[row][k]; U column-major [du][B]
// (du = 1 allowed), V row-major [B][dv] (vrow) or column-major [dv][B]. Fixed chunks, fixed order.
__global__ void __launch_bounds__(OP_THREADS) outer_partial_k(const float* __restrict__ U, int du, const float* __restrict__ V,
                                                              int dv, bool vrow, int64_t B, int64_t chunk, float* partial) {
    __shared__ float us[OP_TILE][HID];
    __shared__ float vs[OP_TILE][LMAX_DIN];
    const int total = du * dv;
    const int64_t r0 = (int64_t)blockIdx.x * chunk;
    const int64_t r1 = min(B, r0 + chunk);
    float acc[OP_MAXQ];
#pragma unroll
    for (int q = 0; q < OP_MAXQ; ++q) acc[q] = 0.0f;
    for (int64_t t0 = r0; t0 < r1; t0 += OP_TILE) {
        const int rows = (int)min((int64_t)OP_TILE, r1 - t0);
        __syncthreads();
        for (int q = threadIdx.x; q < OP_TILE * du; q += OP_THREADS) {
            const int a = q / OP_TILE, rr = q - a * OP_TILE;
            us[rr][a] = rr < rows ? U[(int64_t)a * B + t0 + rr] : 0.0f;
        }
        for (int q = threadIdx.x; q < OP_TILE * dv; q += OP_THREADS) {
            int rr, k;
            if (vrow) { rr = q / dv; k = q - rr * dv; }
            else { k = q / OP_TILE; rr = q - k * OP_TILE; }
            float val = 0.0f;
            if (rr < rows) val = vrow ? V[(t0 + rr) * dv + k] : V[(int64_t)k * B + t0 + rr];
            vs[rr][k] = val;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < OP_MAXQ; ++q) {
            const int o = threadIdx.x + q * OP_THREADS;
            if (o < total) {
                const int a = o / dv, k = o - a * dv;
                float s = acc[q];
                for (int rr = 0; rr < OP_TILE; ++rr) s = fmaf(us[rr][a], vs[rr][k], s);
                acc[q] = s;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < OP_MAXQ; ++q) {
        const int o = threadIdx.x + q * OP_THREADS;
        if (o < total) partial[(int64_t)blockIdx.x * total + o] = acc[q];
    }
}

__global__ void reduce_partials_k(const float* partial, int nchunks, int total, float* G) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    float s = 0.0f;
    for (int c = 0; c < nchunks; ++c) s += partial[(int64_t)c * total + t];
    G[t] = s;
}

__global__ void nonfinite_k(const float* G, int64_t cnt, int* bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt && !isfinite(G[t])) atomicOr(bad, 1);
}

__global__ void adam_k(float* W, const float* G, float* m, float* v, int64_t cnt, float lr, float b1, float b2, float eps,
                       float bc1, float bc2) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const float g = G[t];
    const float mt = b1 * m[t] + (1.0f - b1) * g;
    const float vt = b2 * v[t] + (1.0f - b2) * g * g;
    m[t] = mt;
    v[t] = vt;
    W[t] -= lr * (mt / bc1) / (sqrtf(vt / bc2) + eps);
}

// ------------------------------ residual objective ---------------------------------------------
// s = r - L (scale * out); per-block FP64 partial sums of s^2 and r^2
constexpr int RB = 256;
__global__ void __launch_bounds__(RB) loss_res_k(const int32_t* rp, const int32_t* ci, const float* val, const float* out,
                                                 const float* scale, const float* r, int64_t N, float* sres, double* part) {
    __shared__ double red[2][RB / 32];
    const int64_t i = (int64_t)blockIdx.x * RB + threadIdx.x;
    double a = 0.0, b = 0.0;
    if (i < N) {
        float acc = 0.0f;
        for (int32_t q = rp[i]; q < rp[i + 1]; ++q) {
            const int32_t c = ci[q];
            acc = fmaf(val[q], scale[c] * out[c], acc);
        }
        const float s = r[i] - acc;
        sres[i] = s;
        a = (double)s * s;
        b = (double)r[i] * r[i];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a; red[1][threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < RB / 32; ++w) { x += red[0][w]; y += red[1][w]; }
        part[2 * blockIdx.x] = x;
        part[2 * blockIdx.x + 1] = y;
    }
}

__global__ void sum_pairs_k(const double* part, int nb, double* sums) {
    double x = 0.0, y = 0.0;
    for (int b = threadIdx.x; b < nb; b += 32) { x += part[2 * b]; y += part[2 * b + 1]; }
    x = warp_sum(x);
    y = warp_sum(y);
    if (threadIdx.x == 0) { sums[0] = x; sums[1] = y; }
}

// gout = -2 scale (L^T s) / |r|^2
__global__ void gout_k(const int32_t* trp, const int32_t* tci, const float* tval, const float* sres, const float* scale,
                       const double* sums, int64_t N, float* gout) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float acc = 0.0f;
    for (int32_t q = trp[i]; q < trp[i + 1]; ++q) acc = fmaf(tval[q], sres[tci[q]], acc);
    const double rr = sums[1];
    gout[i] = rr > 0.0 ? (float)(-2.0 * (double)scale[i] * (double)acc / rr) : 0.0f;
}

// r_out[caller] = r_in[caller] - (L e)[s]
__global__ void cycle_res_k(const int32_t* rp, const int32_t* ci, const float* val, const float* e, const double* rin,
                            const int32_t* ordc, int64_t N, double* rout) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = 0.0;
    for (int32_t q = rp[i]; q < rp[i + 1]; ++q) acc += (double)val[q] * (double)e[ci[q]];
    const int64_t o = ordc[i];
    rout[o] = rin[o] - acc;
}

__global__ void f64_to_f32_k(const double* a, float* b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

// ------------------------------ inference (BF16 weights, FP32 arithmetic) ----------------------
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// packed inference weights: [W1 residual columns as [j][64] | W2 [64][64] | w3 [64]]
__global__ void pack_k(const float* W, int n, uint16_t* lw) {
    const int din = 4 * n;
    const int tot = n * HID + HID * HID + HID;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tot) return;
    float v;
    if (t < n * HID) {
        const int j = t / HID, a = t - j * HID;
        v = W[a * din + 4 * j + 3];
    } else {
        v = W[HID * din + (t - n * HID)];
    }
    lw[t] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// hg[s][a] = sum_j sum_{q<3} bf16(W1[a][4j+q]) geo[3j+q][s], accumulated in FP32 and stored as FP16
// (row-major: 128 contiguous bytes a row; |hg| stays far below the FP16 range, relative rounding
// 2^-11)
__global__ void __launch_bounds__(128) hg_k(const float* __restrict__ geo, int n, int64_t N, const float* __restrict__ W,
                                            __half* hg) {
    extern __shared__ __align__(16) float gsm[];  // [3n][64]
    const int din = 4 * n;
    for (int q = threadIdx.x; q < 3 * n * HID; q += blockDim.x) {
        const int jq = q / HID, a = q - jq * HID;
        const int j = jq / 3, c = jq - 3 * j;
        gsm[q] = bf16r(W[a * din + 4 * j + c]);
    }
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    float h[HID];
#pragma unroll
    for (int a = 0; a < HID; ++a) h[a] = 0.0f;
    for (int jq = 0; jq < 3 * n; ++jq) {
        const float g = geo[(int64_t)jq * N + s];
        const float4* w4 = reinterpret_cast<const float4*>(gsm + jq * HID);
#pragma unroll
        for (int q = 0; q < HID / 4; ++q) {
            const float4 c = w4[q];
            h[4 * q + 0] = fmaf(c.x, g, h[4 * q + 0]);
            h[4 * q + 1] = fmaf(c.y, g, h[4 * q + 1]);
            h[4 * q + 2] = fmaf(c.z, g, h[4 * q + 2]);
            h[4 * q + 3] = fmaf(c.w, g, h[4 * q + 3]);
        }
    }
    __half2* out = reinterpret_cast<__half2*>(hg + s * HID);
#pragma unroll
    for (int q = 0; q < HID / 2; ++q) out[q] = __floats2half2_rn(h[2 * q], h[2 * q + 1]);
}

// e[s] += rho out / l_ss from the residual r (solve order); rows with a zero stencil residual are
// left unchanged. Tensor cores (mma.sync m16n8k16, BF16 in, FP32 accumulate), one warp per tile of
// 16 rows:
//   GEMM1  D1 = X W1_r^T   X = r_stencil / rho (16 x K1, K1 = n rounded up to 16), W1_r 64 x K1
//   h1 = relu(D1 + hg)     (hg: the geometric part, FP16, row-major [N][64])
//   GEMM2  D2 = h1 W2^T,   out = w3 . relu(D2)
// Activations are split into BF16 hi + lo parts (x = hi + lo to ~2^-16 relative), each multiplied
// by the exact BF16 weights, so the products carry FP32-like accuracy. GEMM2's A fragments are
// GEMM1's accumulators, re-packed in registers (the m16n8 accumulator layout of two adjacent
// n-tiles is the m16k16 operand layout).
constexpr int CW = 4;                 // warps per block
constexpr int W2S = HID + 8;          // shared-memory row strides (bf16 units), padded against
__host__ __device__ constexpr int k1_of(int n) { return (n + 15) / 16 * 16; }   // bank conflicts

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {  // element k in the low half
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo_k)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi_k)) << 16);
}
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const float ha = __bfloat162float(__float2bfloat16_rn(a)), hb = __bfloat162float(__float2bfloat16_rn(b));
    hi = pack_bf16(ha, hb);
    lo = pack_bf16(a - ha, b - hb);
}
// four 8x8 b16 matrices from shared memory; lane l gives the address of row l % 8 of matrix l / 8
// (16 contiguous bytes, 16-byte aligned) and receives row l / 4, elements 2 (l % 4), +1 of each
__device__ __forceinline__ void ldsm_x4(uint32_t* r, const uint16_t* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(CW * 32) correct_k(const int32_t* __restrict__ nbr, const float* __restrict__ r,
                                                    const __half* __restrict__ hg, const float* __restrict__ diag,
                                                    const uint16_t* __restrict__ lw, int n, int64_t N, float* e) {
    extern __shared__ __align__(16) uint16_t lsm[];
    const int K1 = k1_of(n), S1 = K1 + 8;
    uint16_t* w1 = lsm;                       // [64][S1]: W1_r as [unit][stencil member]
    uint16_t* w2 = w1 + HID * S1;             // [64][W2S]
    float* w3 = reinterpret_cast<float*>(w2 + HID * W2S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint16_t* xs = reinterpret_cast<uint16_t*>(w3 + HID) + warp * 2 * 16 * S1;  // [hi|lo][16][S1]
    for (int q = threadIdx.x; q < HID * S1; q += blockDim.x) {
        const int a = q / S1, k = q - a * S1;
        w1[q] = k < n ? lw[k * HID + a] : (uint16_t)0;
    }
    for (int q = threadIdx.x; q < HID * W2S; q += blockDim.x) {
        const int a = q / W2S, k = q - a * W2S;
        w2[q] = k < HID ? lw[n * HID + a * HID + k] : (uint16_t)0;
    }
    for (int q = threadIdx.x; q < HID; q += blockDim.x) w3[q] = __uint_as_float((uint32_t)lw[n * HID + HID * HID + q] << 16);
    __syncthreads();
    const int g = lane >> 2, tg = lane & 3;
    const int64_t ntiles = (N + 15) / 16;
    for (int64_t tile = (int64_t)blockIdx.x * CW + warp; tile < ntiles; tile += (int64_t)gridDim.x * CW) {
        const int64_t r0 = tile * 16;
        // gather the stencil residuals: lane -> row (lane & 15), members j = (lane >> 4) + 2t
        const int64_t grow = r0 + (lane & 15);
        const bool gact = grow < N;
        float vals[(LMAX_N + 1) / 2];
        float ss = 0.0f;
#pragma unroll
        for (int t = 0; t < (LMAX_N + 1) / 2; ++t) {
            const int j = (lane >> 4) + 2 * t;
            float v = 0.0f;
            if (gact && j < n) v = r[nbr[(int64_t)j * N + grow]];
            vals[t] = v;
            ss = fmaf(v, v, ss);
        }
        ss += __shfl_xor_sync(0xffffffffu, ss, 16);
        const float rho = sqrtf(ss / (float)n);
        const float ir = rho > 0.0f ? 1.0f / rho : 0.0f;
        __syncwarp();
#pragma unroll
        for (int t = 0; t < (LMAX_N + 1) / 2; ++t) {
            const int j = (lane >> 4) + 2 * t;
            if (j < K1) {
                const float x = vals[t] * ir;
                const __nv_bfloat16 h = __float2bfloat16_rn(x);
                xs[(lane & 15) * S1 + j] = __bfloat16_as_ushort(h);
                xs[16 * S1 + (lane & 15) * S1 + j] = __bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h)));
            }
        }
        __syncwarp();
        // GEMM1: D1 (16 x 64) = X (16 x K1) W1_r^T, hi and lo parts of X
        float d1[8][4];
#pragma unroll
        for (int t = 0; t < 8; ++t) d1[t][0] = d1[t][1] = d1[t][2] = d1[t][3] = 0.0f;
        // fragments by ldmatrix: lane l addresses row (l % 8) + 8 ((l / 8) & 1) at column 8 (l / 16) of
        // the A tile (a0..a3), and for B rows n = 8 (l / 16) + l % 8 of a pair of n-tiles at
        // k + 8 ((l / 8) & 1) (b0, b1 of tile t, then of tile t + 1)
        const int lr = (lane & 7) + 8 * ((lane >> 3) & 1), lc = 8 * (lane >> 4);
        const int bn = 8 * (lane >> 4) + (lane & 7), bk = 8 * ((lane >> 3) & 1);
        for (int kk = 0; kk < K1; kk += 16) {
            uint32_t b[8][2];
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                uint32_t q[4];
                ldsm_x4(q, w1 + (8 * t + bn) * S1 + kk + bk);
                b[t][0] = q[0]; b[t][1] = q[1]; b[t + 1][0] = q[2]; b[t + 1][1] = q[3];
            }
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                uint32_t a[4];
                ldsm_x4(a, xs + part * 16 * S1 + lr * S1 + kk + lc);
#pragma unroll
                for (int t = 0; t < 8; ++t) mma16816(d1[t], a, b[t][0], b[t][1]);
            }
        }
        // h1 = relu(D1 + hg), re-packed as GEMM2's A operand (hi and lo)
        const int64_t ra = r0 + g, rb = r0 + g + 8;
        uint32_t ah[4][4], al[4][4];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int c = 8 * t + 2 * tg;
            float2 ga = make_float2(0.0f, 0.0f), gb = make_float2(0.0f, 0.0f);
            if (ra < N) ga = __half22float2(__ldg(reinterpret_cast<const __half2*>(hg + ra * HID + c)));
            if (rb < N) gb = __half22float2(__ldg(reinterpret_cast<const __half2*>(hg + rb * HID + c)));
            const float h0 = fmaxf(d1[t][0] + ga.x, 0.0f), h1v = fmaxf(d1[t][1] + ga.y, 0.0f);
            const float h2 = fmaxf(d1[t][2] + gb.x, 0.0f), h3 = fmaxf(d1[t][3] + gb.y, 0.0f);
            const int kb = t >> 1, half = (t & 1) * 2;   // k-step and register pair of the A fragment
            split2(h0, h1v, ah[kb][half + 0], al[kb][half + 0]);
            split2(h2, h3, ah[kb][half + 1], al[kb][half + 1]);
        }
        // GEMM2 per pair of output n-tiles, then relu, times w3, summed over the thread's columns
        float oa = 0.0f, ob = 0.0f;
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            float d2[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
                uint32_t q[4];
                ldsm_x4(q, w2 + (8 * t + bn) * W2S + 16 * kb + bk);
                mma16816(d2[0], ah[kb], q[0], q[1]);
                mma16816(d2[0], al[kb], q[0], q[1]);
                mma16816(d2[1], ah[kb], q[2], q[3]);
                mma16816(d2[1], al[kb], q[2], q[3]);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int c = 8 * (t + u) + 2 * tg;
                oa = fmaf(w3[c], fmaxf(d2[u][0], 0.0f), fmaf(w3[c + 1], fmaxf(d2[u][1], 0.0f), oa));
                ob = fmaf(w3[c], fmaxf(d2[u][2], 0.0f), fmaf(w3[c + 1], fmaxf(d2[u][3], 0.0f), ob));
            }
        }
        oa += __shfl_xor_sync(0xffffffffu, oa, 1);
        oa += __shfl_xor_sync(0xffffffffu, oa, 2);
        ob += __shfl_xor_sync(0xffffffffu, ob, 1);
        ob += __shfl_xor_sync(0xffffffffu, ob, 2);
        const float rho_a = __shfl_sync(0xffffffffu, rho, g);       // lane g holds row g's rho
        const float rho_b = __shfl_sync(0xffffffffu, rho, g + 8);
        if (tg == 0) {
            if (ra < N && rho_a > 0.0f) e[ra] += rho_a * oa / diag[ra];
            if (rb < N && rho_b > 0.0f) e[rb] += rho_b * ob / diag[rb];
        }
        __syncwarp();
    }
}

// ------------------------------ host side ------------------------------------------------------
static size_t fwd_smem(int din) { return sizeof(float) * (size_t)mlp_count(din); }
static size_t correct_smem(int n) {
    return sizeof(uint16_t) * (size_t)(HID * (k1_of(n) + 8) + HID * W2S) + sizeof(float) * HID +
           sizeof(uint16_t) * (size_t)CW * 2 * 16 * (k1_of(n) + 8);
}

static void set_smem_limits() {
    static bool done = false;
    if (done) return;
    CK(cudaFuncSetAttribute(fwd_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(LMAX_DIN)));
    CK(cudaFuncSetAttribute(hg_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float) * 3 * LMAX_N * HID)));
    CK(cudaFuncSetAttribute(correct_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)correct_smem(LMAX_N)));
    done = true;
}

static void forward(const float* feat, int din, int64_t B, const float* W, float* out, float* h1s, float* h2s,
                    cudaStream_t s) {
    set_smem_limits();
    fwd_k<<<grid_for(B, 128), 128, fwd_smem(din), s>>>(feat, din, B, W, out, h1s, h2s);
    CK_LAUNCH();
}

// G (device, mlp_count(din) floats) = gradients of sum_b gout_b out_b, from stored activations
static void gradients(const float* feat, const float* gout, int din, int64_t B, const float* W, const float* h1s,
                      const float* h2s, float* G, cudaStream_t s) {
    Temp<float> d1(B * HID, s), d2(B * HID, s);
    bwd_k<<<grid_for(B, 128), 128, 0, s>>>(gout, W, din, B, h1s, h2s, d1.get(), d2.get());
    CK_LAUNCH();
    const int64_t per = (B + OP_CHUNKS - 1) / OP_CHUNKS;
    const int64_t chunk = std::max<int64_t>(OP_TILE, (per + OP_TILE - 1) / OP_TILE * OP_TILE);
    const int nch = (int)((B + chunk - 1) / chunk);
    Temp<float> part((size_t)nch * HID * std::max(din, HID), s);
    struct Job {
        const float* U;
        int du;
        const float* V;
        int dv;
        bool vrow;
        float* G;
    };
    const Job jobs[3] = {{d1.get(), HID, feat, din, true, G},
                         {d2.get(), HID, h1s, HID, false, G + (int64_t)HID * din},
                         {gout, 1, h2s, HID, false, G + (int64_t)HID * din + HID * HID}};
    for (const Job& jb : jobs) {
        outer_partial_k<<<nch, OP_THREADS, 0, s>>>(jb.U, jb.du, jb.V, jb.dv, jb.vrow, B, chunk, part.get());
        CK_LAUNCH();
        reduce_partials_k<<<grid_for(jb.du * jb.dv, 256), 256, 0, s>>>(part.get(), nch, jb.du * jb.dv, jb.G);
        CK_LAUNCH();
    }
}

static void check_mlp(const mgm_mlp* M) { REQUIRE(M && M->din == 4 * M->n && M->W.get(), "invalid network handle"); }

static void check_attached(const mgm_hierarchy* H) {
    REQUIRE(H, "null hierarchy");
    REQUIRE(H->ln > 0, "learned correction: call mgm_learned_attach first");
}

void learned_attach(mgm_hierarchy* H, const double* xyz, const double* nrm, const int32_t* idx, const double* w, int n,
                    cudaStream_t s) {
    REQUIRE(H && xyz && nrm && idx && w, "null argument");
    REQUIRE(n >= 1 && n <= LMAX_N, "learned correction: stencil size must be in [1, 48]");
    REQUIRE(H->p >= 2, "learned correction needs a hierarchy with at least two levels");
    REQUIRE(H->precision == MGM_F32, "learned correction runs in FP32 V-cycles (precision MGM_F32)");
    REQUIRE(!H->bordered, "learned correction: not for constrained (bordered) hierarchies");
    const int64_t N = H->N;
    validate_index(idx, N * n, N, "stencil indices", s);
    Level& L0 = H->lv[0];
    Temp<int32_t> invc(N, s);
    invert_perm(H->ord_caller.get(), invc.get(), N, s);
    H->ln = 0;
    H->learned = false;
    if (H->lgraph) {  // captured with the previous buffers
        CK(cudaGraphExecDestroy(H->lgraph));
        H->lgraph = nullptr;
    }
    H->lnbr.alloc(N * n);
    H->lgeo.alloc(N * n * 3);
    H->lhg.alloc(N * HID);
    H->lw.alloc(n * HID + HID * HID + HID);
    attach_k<<<grid_for(N, 128), 128, 0, s>>>(xyz, nrm, idx, w, n, N, H->ord_caller.get(), invc.get(), H->lnbr.get(),
                                              H->lgeo.get());
    CK_LAUNCH();
    // L_0 in solve order as plain CSR (diagonal included) and its transpose, FP32
    const int64_t nnz = L0.nnz;
    Temp<int32_t> rp(N + 1, s), ci(nnz, s), trp(N + 1, s), tci(nnz, s);
    Temp<double> v(nnz, s), tv(nnz, s);
    csr_permute(N, L0.rp.get(), L0.ci.get(), L0.v.get(), L0.ord.get(), rp.get(), ci.get(), v.get(), s);
    csr_transpose(N, N, rp.get(), ci.get(), v.get(), trp.get(), tci.get(), tv.get(), s);
    H->lrp.alloc(N + 1); H->lci.alloc(nnz); H->lval.alloc(nnz);
    H->ltrp.alloc(N + 1); H->ltci.alloc(nnz); H->ltval.alloc(nnz);
    CK(cudaMemcpyAsync(H->lrp.get(), rp.get(), sizeof(int32_t) * (N + 1), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(H->lci.get(), ci.get(), sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(H->ltrp.get(), trp.get(), sizeof(int32_t) * (N + 1), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(H->ltci.get(), tci.get(), sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s));
    f64_to_f32_k<<<grid_for(nnz, 256), 256, 0, s>>>(v.get(), H->lval.get(), nnz);
    CK_LAUNCH();
    f64_to_f32_k<<<grid_for(nnz, 256), 256, 0, s>>>(tv.get(), H->ltval.get(), nnz);
    CK_LAUNCH();
    CK(cudaStreamSynchronize(s));
    H->ln = n;
    H->device_bytes += (int64_t)(H->lnbr.bytes() + H->lgeo.bytes() + H->lhg.bytes() + H->lw.bytes() + H->lrp.bytes() +
                                 H->lci.bytes() + H->lval.bytes() + H->ltrp.bytes() + H->ltci.bytes() + H->ltval.bytes());
}

void learned_features(mgm_hierarchy* H, const double* r, float* feat, float* rho, cudaStream_t s) {
    check_attached(H);
    REQUIRE(r && feat, "null argument");
    const int64_t N = H->N;
    Temp<float> r32(N, s);
    gather_cast_k<<<grid_for(N, 256), 256, 0, s>>>(r, H->ord_caller.get(), r32.get(), N);
    CK_LAUNCH();
    features_k<<<grid_for(N, 128), 128, 0, s>>>(H->lnbr.get(), H->lgeo.get(), r32.get(), H->lv[0].diag32.get(), H->ln, N,
                                                H->ord_caller.get(), feat, rho, nullptr);
    CK_LAUNCH();
    CK(cudaStreamSynchronize(s));
}

void learned_cycle_residual(mgm_hierarchy* H, const double* r, double* rout, cudaStream_t s) {
    check_attached(H);
    REQUIRE(r && rout, "null argument");
    const int64_t N = H->N;
    load_input(H, r, MGM_F64, H->ord_caller.get(), s);
    vcycle_plain(H, s);
    cycle_res_k<<<grid_for(N, 256), 256, 0, s>>>(H->lrp.get(), H->lci.get(), H->lval.get(), H->lv[0].e32.get(), r,
                                                 H->ord_caller.get(), N, rout);
    CK_LAUNCH();
    if (H->persistent) check_device_error(H, s);
    CK(cudaStreamSynchronize(s));
}

// J and dJ/dW on the sample r (caller order); optionally one Adam step of size lr
static double learned_objective(mgm_hierarchy* H, mgm_mlp* M, const double* r, float* grad_out, bool update, float lr,
                                cudaStream_t s) {
    check_attached(H);
    check_mlp(M);
    REQUIRE(r, "null argument");
    REQUIRE(M->n == H->ln, "network and attached stencil sizes differ");
    const int64_t N = H->N;
    const int n = H->ln, din = 4 * n;
    const int64_t cnt = mlp_count(din);
    Temp<float> r32(N, s), feat(N * din, s), scale(N, s), out(N, s), h1(N * HID, s), h2(N * HID, s), sres(N, s),
        gout(N, s), G(cnt, s);
    const unsigned nb = grid_for(N, RB);
    Temp<double> part(2 * (size_t)nb, s), sums(2, s);
    gather_cast_k<<<grid_for(N, 256), 256, 0, s>>>(r, H->ord_caller.get(), r32.get(), N);
    CK_LAUNCH();
    features_k<<<grid_for(N, 128), 128, 0, s>>>(H->lnbr.get(), H->lgeo.get(), r32.get(), H->lv[0].diag32.get(), n, N,
                                                nullptr, feat.get(), nullptr, scale.get());
    CK_LAUNCH();
    forward(feat.get(), din, N, M->W.get(), out.get(), h1.get(), h2.get(), s);
    loss_res_k<<<nb, RB, 0, s>>>(H->lrp.get(), H->lci.get(), H->lval.get(), out.get(), scale.get(), r32.get(), N, sres.get(),
                                 part.get());
    CK_LAUNCH();
    sum_pairs_k<<<1, 32, 0, s>>>(part.get(), (int)nb, sums.get());
    CK_LAUNCH();
    gout_k<<<grid_for(N, 256), 256, 0, s>>>(H->ltrp.get(), H->ltci.get(), H->ltval.get(), sres.get(), scale.get(),
                                            sums.get(), N, gout.get());
    CK_LAUNCH();
    gradients(feat.get(), gout.get(), din, N, M->W.get(), h1.get(), h2.get(), G.get(), s);
    if (grad_out) CK(cudaMemcpyAsync(grad_out, G.get(), sizeof(float) * cnt, cudaMemcpyDeviceToDevice, s));
    Temp<int> bad(1, s);
    CK(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    nonfinite_k<<<grid_for(cnt, 256), 256, 0, s>>>(G.get(), cnt, bad.get());
    CK_LAUNCH();
    double hs[2];
    to_host(hs, sums.get(), 2, s);
    const int nonfinite = read1(bad.get(), s);
    const double J = hs[1] > 0.0 ? hs[0] / hs[1] : 0.0;
    if (update && std::isfinite(J) && hs[1] > 0.0 && !nonfinite) {  // a sample that overflowed FP32 is skipped
        M->step += 1;
        const float bc1 = (float)(1.0 - std::pow(0.9, M->step)), bc2 = (float)(1.0 - std::pow(0.999, M->step));
        adam_k<<<grid_for(cnt, 256), 256, 0, s>>>(M->W.get(), G.get(), M->m.get(), M->v.get(), cnt, lr, 0.9f, 0.999f, 1e-8f,
                                                  bc1, bc2);
        CK_LAUNCH();
    }
    return J;
}

double learned_loss(mgm_hierarchy* H, const mgm_mlp* M, const double* r, float* grad, cudaStream_t s) {
    return learned_objective(H, const_cast<mgm_mlp*>(M), r, grad, false, 0.0f, s);
}

double learned_train_step(mgm_hierarchy* H, mgm_mlp* M, const double* r, float lr, cudaStream_t s) {
    REQUIRE(lr > 0.0f && std::isfinite(lr), "learning rate must be positive and finite");
    return learned_objective(H, M, r, nullptr, true, lr, s);
}

void learned_enable(mgm_hierarchy* H, const mgm_mlp* M, cudaStream_t s) {
    REQUIRE(H, "null hierarchy");
    if (!M) {
        H->learned = false;
        return;
    }
    check_attached(H);
    check_mlp(M);
    REQUIRE(M->n == H->ln, "network and attached stencil sizes differ");
    set_smem_limits();
    const int n = H->ln;
    const int64_t N = H->N;
    const int tot = n * HID + HID * HID + HID;
    pack_k<<<grid_for(tot, 256), 256, 0, s>>>(M->W.get(), n, H->lw.get());
    CK_LAUNCH();
    hg_k<<<grid_for(N, 128), 128, sizeof(float) * 3 * n * HID, s>>>(H->lgeo.get(), n, N, M->W.get(),
                                                                     reinterpret_cast<__half*>(H->lhg.get()));
    CK_LAUNCH();
    CK(cudaStreamSynchronize(s));
    H->learned = true;
    H->learned_active = true;
}

void learned_correct(mgm_hierarchy* H, cudaStream_t s) {
    set_smem_limits();
    Level& L0 = H->lv[0];
    static int blocks = 0;
    if (!blocks) {
        int per_sm = 0, dev = 0, sms = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, correct_k, CW * 32, correct_smem(LMAX_N)));
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        blocks = std::max(1, per_sm * sms);
    }
    const int64_t tiles = (H->N + 15) / 16;
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, (tiles + CW - 1) / CW));
    correct_k<<<nb, CW * 32, correct_smem(H->ln), s>>>(H->lnbr.get(), L0.s32.get(), reinterpret_cast<const __half*>(H->lhg.get()),
                                                     L0.diag32.get(),
                                                     H->lw.get(), H->ln, H->N, L0.e32.get());
    CK_LAUNCH();
}

// delta = correction for the residual r (caller order), through the inference kernel
void learned_correction(mgm_hierarchy* H, const double* r, double* delta, cudaStream_t s) {
    check_attached(H);
    REQUIRE(H->learned, "learned correction: no network enabled (mgm_learned_enable)");
    REQUIRE(r && delta, "null argument");
    const int64_t N = H->N;
    Level& L0 = H->lv[0];
    gather_cast_k<<<grid_for(N, 256), 256, 0, s>>>(r, H->ord_caller.get(), L0.s32.get(), N);
    CK_LAUNCH();
    CK(cudaMemsetAsync(L0.e32.get(), 0, sizeof(float) * N, s));
    learned_correct(H, s);
    store_output(H, delta, MGM_F64, H->ord_caller.get(), s);
    CK(cudaStreamSynchronize(s));
}

// ---- network handle
static uint64_t splitmix(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

mgm_mlp* mlp_create(int n, uint64_t seed) {
    REQUIRE(n >= 1 && n <= LMAX_N, "network stencil size must be in [1, 48]");
    const int din = 4 * n;
    const int64_t cnt = mlp_count(din), n1 = (int64_t)HID * din;
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) per layer from one SplitMix64 stream
    std::vector<float> w(cnt);
    uint64_t st = seed;
    for (int64_t q = 0; q < cnt; ++q) {
        const double fan = q < n1 ? (double)din : (double)HID;
        const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
        w[q] = (float)((2.0 * u - 1.0) / std::sqrt(fan));
    }
    auto* M = new mgm_mlp;
    M->n = n;
    M->din = din;
    try {
        M->W.alloc(cnt); M->m.alloc(cnt); M->v.alloc(cnt);
        CK(cudaMemcpy(M->W.get(), w.data(), sizeof(float) * cnt, cudaMemcpyHostToDevice));
        CK(cudaMemset(M->m.get(), 0, sizeof(float) * cnt));
        CK(cudaMemset(M->v.get(), 0, sizeof(float) * cnt));
    } catch (...) {
        delete M;
        throw;
    }
    return M;
}

void mlp_destroy(mgm_mlp* M) { delete M; }

void mlp_get(const mgm_mlp* M, float* W) {
    check_mlp(M);
    REQUIRE(W, "null argument");
    CK(cudaMemcpy(W, M->W.get(), sizeof(float) * mlp_count(M->din), cudaMemcpyDeviceToHost));
}

void mlp_set(mgm_mlp* M, const float* W) {
    check_mlp(M);
    REQUIRE(W, "null argument");
    const int64_t cnt = mlp_count(M->din);
    CK(cudaMemcpy(M->W.get(), W, sizeof(float) * cnt, cudaMemcpyHostToDevice));
    CK(cudaMemset(M->m.get(), 0, sizeof(float) * cnt));
    CK(cudaMemset(M->v.get(), 0, sizeof(float) * cnt));
    M->step = 0;
}

int64_t mlp_size(int n) { return n >= 1 && n <= LMAX_N ? mlp_count(4 * n) : -1; }

void mlp_forward_api(const mgm_mlp* M, const float* feat, int64_t B, float* out, cudaStream_t s) {
    check_mlp(M);
    REQUIRE(B >= 0 && (B == 0 || (feat && out)), "bad argument");
    if (B == 0) return;
    forward(feat, M->din, B, M->W.get(), out, nullptr, nullptr, s);
    CK(cudaStreamSynchronize(s));
}

void mlp_vjp_api(const mgm_mlp* M, const float* feat, const float* gout, int64_t B, float* grad, cudaStream_t s) {
    check_mlp(M);
    REQUIRE(B >= 1 && feat && gout && grad, "bad argument");
    Temp<float> out(B, s), h1(B * HID, s), h2(B * HID, s);
    forward(feat, M->din, B, M->W.get(), out.get(), h1.get(), h2.get(), s);
    gradients(feat, gout, M->din, B, M->W.get(), h1.get(), h2.get(), grad, s);
    CK(cudaStreamSynchronize(s));
}

}  // namespace mgm

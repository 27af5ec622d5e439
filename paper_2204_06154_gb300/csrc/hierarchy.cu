// MGM preprocessing on the device (paper Alg. 2) and the solve-order layouts the V-cycle runs on.
//
// Order of operations follows Alg. 2: RCM of L_1 and reordering of X_1; number of levels; per
// level: weighted sample elimination to floor(N_1/4^j) points, PHS interpolation, restriction =
// transpose, Galerkin product L_{j+1} = R (L_j P) (operand order of eq. (galerkin)), RCM of
// L_{j+1} with the matching renumbering of the coarse index of the transfers; and the coarsest
// factorisation (an
// explicit FP64 inverse by Gauss-Jordan elimination, so the coarsest solve is one matrix-vector
// product per cycle). Then, for the multicolour smoother: colourings of the RCM-ordered level
// operators, the colour-grouped solve orders, and FP32/FP64 copies of operators and transfers.
// Built with --fmad=false (the integer decisions and FP64 setup values are bit-reproducible).
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <string>
#include <vector>

#include "hier.cuh"

namespace mgm {

void rcm(int64_t N, const int32_t* rp, const int32_t* ci, int32_t* perm, cudaStream_t s);
void rcm(int64_t N, const int32_t* rp, const int32_t* ci, int32_t* perm, cudaStream_t s, Temp<int32_t>* keep_rp,
         Temp<int32_t>* keep_ci);
void permute_pattern(int64_t N, const int32_t* srp, const int32_t* sci, const int32_t* perm, Temp<int32_t>& nrp,
                     Temp<int32_t>& nci, cudaStream_t s);
void color(int64_t N, const int32_t* rp, const int32_t* ci, uint64_t seed, int32_t* colour, int32_t* ncolors,
           cudaStream_t s);
void color(int64_t N, const int32_t* rp, const int32_t* ci, uint64_t seed, int32_t* colour, int32_t* ncolors,
           cudaStream_t s, const int32_t* sym_rp, const int32_t* sym_ci);
void coarsen(const double* x, int64_t N, int64_t NH, int32_t* keep, cudaStream_t s, double* rmax_out);
int64_t interp(const double* xf, int64_t nf, const double* xc, int64_t nc, int m, int32_t* rp, int32_t* col, double* val,
               cudaStream_t s);
int64_t spgemm_symbolic(int64_t nA, const int32_t* arp, const int32_t* aci, const int32_t* brp, const int32_t* bci,
                        int32_t* crp, cudaStream_t s);
void spgemm_numeric(int64_t nA, const int32_t* arp, const int32_t* aci, const double* av, const int32_t* brp,
                    const int32_t* bci, const double* bv, const int32_t* crp, int32_t* cci, double* cv, cudaStream_t s);

int num_levels(int64_t N1, int64_t nmin) {
    if (N1 < nmin) return 1;
    int t = 0;
    __int128 pw = nmin;
    while (pw * 4 <= N1) { pw *= 4; ++t; }
    return t + 1;
}

// ------------------------------ helpers --------------------------------------------------------
__global__ void remap_cols_k(const int32_t* rp, const int32_t* ci, const double* v, const int32_t* inv, int64_t n,
                             int32_t* oci, double* ov) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t b = rp[i], e = rp[i + 1];
    for (int32_t p = b; p < e; ++p) { oci[p] = inv[ci[p]]; ov[p] = v[p]; }
    for (int32_t p = b + 1; p < e; ++p) {  // insertion sort by column
        int32_t c = oci[p];
        double x = ov[p];
        int32_t q = p;
        while (q > b && oci[q - 1] > c) { oci[q] = oci[q - 1]; ov[q] = ov[q - 1]; --q; }
        oci[q] = c;
        ov[q] = x;
    }
}

// rows of L into the left half of the augmented [A | I] (dimension nt >= n), identity on the right
__global__ void csr_to_dense_k(const int32_t* rp, const int32_t* ci, const double* v, int64_t n, double* A, int64_t ld,
                               int64_t nt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) A[i * ld + ci[p]] = v[p];
    A[i * ld + nt + i] = 1.0;  // augmented identity
}

// y = R x for the restriction stored with the level (rows: next level's vector order)
__global__ void restrict_vec_k(const int32_t* rp, const int32_t* ci, const double* v, const double* x, int64_t n,
                               double* y) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) acc = fma(v[p], x[ci[p]], acc);
    y[i] = acc;
}
__global__ void fill_ones_k(double* x, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 1.0;
}


// Gauss-Jordan with partial pivoting on [A | I] (n x 2n), every step in one cooperative launch.
// Step k reads buffer `cur` and writes `nxt` (so no block overwrites a row another block still
// reads), then all blocks meet at a grid barrier. Every block finds the pivot itself (first row
// of largest |a_ik|, i >= k: the same result everywhere), and updates its rows i = block, block +
// grid, ...: row k becomes the pivot row divided by a_pk; row p (p != k) takes the old row k, and
// every row r != k subtracts a_rk times that divided pivot row with a fused multiply-add (rows
// with a_rk = 0 are copied). These are the operations, in order, of a row swap, a division of
// the pivot row and one elimination step. Columns left of k are not written: no later step reads
// them. The waits are bounded (grid_barrier); a singular step leaves err = 1 in every block.
constexpr int GJ_THREADS = 256;
__global__ void __launch_bounds__(GJ_THREADS) gj_coop_k(double* A0, double* A1, int64_t n, unsigned* bar, int* err,
                                                       unsigned long long limit) {
    __shared__ double sv[GJ_THREADS / 32];
    __shared__ int si[GJ_THREADS / 32];
    __shared__ int ok;
    const int64_t ld = 2 * n;
    double* cur = A0;
    double* nxt = A1;
    unsigned target = 0;
    for (int64_t k = 0; k < n; ++k) {
        double best = -1.0;
        int64_t piv = k;
        for (int64_t i = k + threadIdx.x; i < n; i += blockDim.x) {
            const double v = fabs(cur[i * ld + k]);
            if (v > best) { best = v; piv = i; }
        }
        for (int o = 16; o; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int64_t op = __shfl_xor_sync(0xffffffffu, piv, o);
            if (ob > best || (ob == best && op < piv)) { best = ob; piv = op; }
        }
        if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = best; si[threadIdx.x >> 5] = (int)piv; }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int nw = blockDim.x >> 5;
            double b = threadIdx.x < nw ? sv[threadIdx.x] : -1.0;
            int p = threadIdx.x < nw ? si[threadIdx.x] : 0x7fffffff;
            for (int o = 16; o; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, b, o);
                const int op = __shfl_xor_sync(0xffffffffu, p, o);
                if (ob > b || (ob == b && op < p)) { b = ob; p = op; }
            }
            if (threadIdx.x == 0) { sv[0] = b; si[0] = p; }
        }
        __syncthreads();
        best = sv[0];
        piv = si[0];
        __syncthreads();  // everyone has read sv[0], si[0] before the next step overwrites them
        if (!(best > 0.0)) {
            if (threadIdx.x == 0) *err = 1;
            return;
        }
        const double rk = 1.0 / cur[piv * ld + k];  // the pivot row scaled by the reciprocal (dgetf2's form)
        for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
            const double* src = cur + (i == piv ? k : i) * ld;
            const double m = i == k ? 0.0 : src[k];
            for (int64_t j = k + threadIdx.x; j < ld; j += blockDim.x) {
                const double pr = cur[piv * ld + j] * rk;
                nxt[i * ld + j] = i == k ? pr : (m == 0.0 ? src[j] : fma(-m, pr, src[j]));
            }
        }
        target += gridDim.x;
        if (!grid_barrier(bar, target, limit, err, &ok)) return;
        double* t = cur;
        cur = nxt;
        nxt = t;
    }
}

__global__ void extract_inv_k(const double* A, int64_t n, double* inv) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    int64_t i = e / n, j = e - i * n;
    inv[e] = A[i * 2 * n + n + j];
}

// border of the coarsest constrained operator: [L c; c^T 0] in an (n+1) x 2(n+1) augmented matrix
__global__ void border_dense_k(const double* c, int64_t n, double* A) {
    const int64_t ld = 2 * (n + 1);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (i < n) {
        A[i * ld + n] = c[i];
        A[n * ld + i] = c[i];
    } else {
        A[n * ld + n] = 0.0;
        A[n * ld + (n + 1) + n] = 1.0;
    }
}

// inverse of L (border == nullptr) or of the bordered [L c; c^T 0]
static void dense_inverse(const Level& L, const double* border, Buf<double>& inv, cudaStream_t s) {
    const int64_t nl = L.n;
    const int64_t n = nl + (border ? 1 : 0);
    if (n > 8192) fail(MGM_ERR_UNSUPPORTED, "coarsest level larger than 8192 rows");
    Temp<double> A(2 * n * n, s), B(2 * n * n, s);
    Temp<int> err(1, s);
    Temp<unsigned> bar(1, s);
    CK(cudaMemsetAsync(A.get(), 0, sizeof(double) * 2 * n * n, s));
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    CK(cudaMemsetAsync(bar.get(), 0, sizeof(unsigned), s));
    csr_to_dense_k<<<grid_for(nl, 128), 128, 0, s>>>(L.rp.get(), L.ci.get(), L.v.get(), nl, A.get(), 2 * n, n);
    CK_LAUNCH();
    if (border) {
        border_dense_k<<<grid_for(n, 128), 128, 0, s>>>(border, nl, A.get());
        CK_LAUNCH();
    }
    const int mb = coresident_blocks((const void*)gj_coop_k, GJ_THREADS, 0, 1);
    const int nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(mb, n));
    double* a0 = A.get();
    double* a1 = B.get();
    unsigned* barp = bar.get();
    int* errp = err.get();
    int64_t nn = n;
    unsigned long long limit = 4000000ull;
    void* args[] = {(void*)&a0, (void*)&a1, (void*)&nn, (void*)&barp, (void*)&errp, (void*)&limit};
    CK(cudaLaunchCooperativeKernel((const void*)gj_coop_k, dim3(nblocks), dim3(GJ_THREADS), args, 0, s));
    CK_LAUNCH();
    const int e = read1(err.get(), s);
    if (e == 1) fail(MGM_ERR_BREAKDOWN, "coarsest operator is singular");
    if (e) fail(MGM_ERR_TIMEOUT, "coarsest factorisation: a grid barrier timed out");
    inv.alloc(n * n);
    extract_inv_k<<<grid_for(n * n, 256), 256, 0, s>>>((n % 2 == 0) ? A.get() : B.get(), n, inv.get());
    CK_LAUNCH();
}

// ------------------------------ solve-order layout ---------------------------------------------
// Stable grouping of rows by colour in one pass: blocks of 256 rows rank each row among the
// earlier rows of its colour in the block and count colours per block; a scan of the
// (colour, block) counts in colour-major order gives each block's base for each colour.
__global__ void __launch_bounds__(256) colour_rank_k(const int32_t* col, int64_t n, int nc, int nblocks, int32_t* lrank,
                                                      int32_t* hist) {
    extern __shared__ int32_t crk_sh[];
    int32_t* scol = crk_sh;
    int32_t* cnt = crk_sh + 256;
    const int t = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * 256 + t;
    const int c = i < n ? col[i] : -1;
    scol[t] = c;
    for (int q = t; q < nc; q += 256) cnt[q] = 0;
    __syncthreads();
    if (i < n) {
        int r = 0;
        for (int u = 0; u < t; ++u) r += scol[u] == c ? 1 : 0;
        lrank[i] = r;
        atomicAdd(&cnt[c], 1);
    }
    __syncthreads();
    for (int q = t; q < nc; q += 256) hist[(int64_t)q * nblocks + blockIdx.x] = cnt[q];
}
__global__ void colour_place_k(const int32_t* col, const int32_t* lrank, const int32_t* off, int64_t n, int nblocks,
                               int32_t* ord) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i < n) ord[off[(int64_t)col[i] * nblocks + blockIdx.x] + lrank[i]] = (int32_t)i;
}
__global__ void colour_bounds_k(const int32_t* off, int nc, int nblocks, int64_t n, int32_t* cp) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc) cp[c] = off[(int64_t)c * nblocks];
    if (c == nc) cp[c] = (int32_t)n;
}

__device__ __forceinline__ int32_t pad4(int32_t x) { return (x + 3) & ~3; }

__global__ void add_i32_k(int32_t* a, int32_t v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += v;
}

// lengths of the split rows; err bit 1: same colour off-diagonal, bit 2: missing/zero diagonal.
// One warp per row (lanes over its entries); the block sums its rows' counts before one atomic.
__global__ void __launch_bounds__(256) split_len_k(const int32_t* rp, const int32_t* ci, const double* v,
                                                   const int32_t* col, const int32_t* ord, int64_t n, int single,
                                                   int32_t* lenl, int32_t* lenu, int* err, unsigned long long* tot) {
    __shared__ unsigned long long bt[2];
    const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 2) bt[threadIdx.x] = 0;
    __syncthreads();
    if (s < n) {
        const int32_t r = ord[s];
        const int32_t cr = single ? 0 : col[r];
        int nl = 0, nu = 0;
        bool diag = false, same = false;
        for (int32_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
            const int32_t j = ci[p];
            if (j == r) { diag = v[p] != 0.0; continue; }
            const int32_t cj = single ? 1 : col[j];
            same = same || cj == cr;
            if (cj < cr) ++nl; else ++nu;
        }
        nl = warp_sum_i(nl);
        nu = warp_sum_i(nu);
        diag = __any_sync(0xffffffffu, diag);
        same = __any_sync(0xffffffffu, same);
        if (lane == 0) {
            if (same) atomicOr(err, 1);
            if (!diag) atomicOr(err, 2);
            lenl[s] = pad4(nl);
            lenu[s] = pad4(nu);
            atomicAdd(&bt[0], (unsigned long long)nl);
            atomicAdd(&bt[1], (unsigned long long)nu);
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 && bt[threadIdx.x]) atomicAdd(&tot[threadIdx.x], bt[threadIdx.x]);
}

// Rows in solve order, split in two regions of the same arrays: the lower parts (columns of earlier
// colours) of all rows, then the upper parts of all rows; each part sorted by solve-order column and
// padded to a multiple of 4 with (own row, 0). Row s: lower [lo[s], lo[s+1]), upper [up[s],
// up[s+1]). One warp per row; the entries are staged in shared memory and placed by rank (rows of up
// to SPLIT_MAX entries; longer rows take the thread path below).
constexpr int SPLIT_WARPS = 4, SPLIT_MAX = 256;
__global__ void __launch_bounds__(SPLIT_WARPS * 32) split_fill_k(
    const int32_t* rp, const int32_t* ci, const double* v, const int32_t* col, const int32_t* ord, const int32_t* inv,
    int64_t n, int single, const int32_t* lo, const int32_t* up, int32_t* sc, double* sv64, float* sv32, double* diag64,
    double* dinv64, float* diag32, float* dinv32, int* longrows) {
    __shared__ unsigned long long key[SPLIT_WARPS][SPLIT_MAX];  // (upper?, solve column) of each entry
    __shared__ double val[SPLIT_WARPS][SPLIT_MAX];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * SPLIT_WARPS + w;
    if (s >= n) return;
    const int32_t r = ord[s];
    const int32_t b = rp[r], e = rp[r + 1];
    if (e - b > SPLIT_MAX) {
        if (lane == 0) atomicAdd(longrows, 1);
        return;
    }
    const int32_t cr = single ? 0 : col[r];
    double d = 0.0;
    int nl = 0;
    for (int32_t p = b + lane; p < e; p += 32) {
        const int32_t j = ci[p];
        unsigned long long k = ~0ull;  // the diagonal sorts last and is not placed
        if (j == r) d = v[p];
        else {
            const int32_t cj = single ? 1 : col[j];
            const unsigned long long up = cj < cr ? 0ull : 1ull;
            if (!up) ++nl;
            k = (up << 32) | (unsigned)inv[j];
        }
        key[w][p - b] = k;
        val[w][p - b] = v[p];
    }
    nl = warp_sum_i(nl);
    for (int o = 16; o; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);  // one lane holds it, the others 0
    __syncwarp();
    const int32_t len = e - b, q0 = lo[s], qm = up[s];
    for (int32_t t = lane; t < len; t += 32) {
        const unsigned long long k = key[w][t];
        if (k == ~0ull) continue;
        int rank = 0;
        for (int32_t u = 0; u < len; ++u) rank += key[w][u] < k ? 1 : 0;
        const bool up = (k >> 32) != 0;
        const int32_t pos = up ? qm + (rank - nl) : q0 + rank;
        sc[pos] = (int32_t)(k & 0xffffffffull);
        sv64[pos] = val[w][t];
        sv32[pos] = (float)val[w][t];
    }
    const int32_t nu = len - nl - 1 >= 0 ? len - nl - 1 : 0;
    const int32_t ql = q0 + pad4(nl), qe = qm + pad4(nu);
    for (int32_t t = q0 + nl + lane; t < ql; t += 32) { sc[t] = (int32_t)s; sv64[t] = 0.0; sv32[t] = 0.0f; }
    for (int32_t t = qm + nu + lane; t < qe; t += 32) { sc[t] = (int32_t)s; sv64[t] = 0.0; sv32[t] = 0.0f; }
    if (lane == 0) {
        diag64[s] = d;
        dinv64[s] = 1.0 / d;
        diag32[s] = (float)d;
        dinv32[s] = (float)(1.0 / d);
    }
}

// rows longer than SPLIT_MAX: one thread per row, insertion into place
__global__ void split_fill_long_k(const int32_t* rp, const int32_t* ci, const double* v, const int32_t* col,
                                  const int32_t* ord, const int32_t* inv, int64_t n, int single, const int32_t* lo,
                                  const int32_t* up, int32_t* sc, double* sv64, float* sv32, double* diag64,
                                  double* dinv64, float* diag32, float* dinv32) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int32_t r = ord[s];
    if (rp[r + 1] - rp[r] <= SPLIT_MAX) return;
    int32_t cr = single ? 0 : col[r];
    double d = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        const int32_t start = pass == 0 ? lo[s] : up[s];
        int32_t q = start;
        for (int32_t p = rp[r]; p < rp[r + 1]; ++p) {
            int32_t j = ci[p];
            if (j == r) { d = v[p]; continue; }
            int32_t cj = single ? 1 : col[j];
            if ((pass == 0) != (cj < cr)) continue;
            int32_t js = inv[j];
            double x = v[p];
            int32_t t = q++;
            while (t > start && sc[t - 1] > js) { sc[t] = sc[t - 1]; sv64[t] = sv64[t - 1]; --t; }
            sc[t] = js;
            sv64[t] = x;
        }
        while ((q - start) & 3) { sc[q] = (int32_t)s; sv64[q] = 0.0; ++q; }
        for (int32_t t = start; t < q; ++t) sv32[t] = (float)sv64[t];
    }
    diag64[s] = d;
    dinv64[s] = 1.0 / d;
    diag32[s] = (float)d;
    dinv32[s] = (float)(1.0 / d);
}

static void build_solve_layout(Level& L, bool single, cudaStream_t s, bool lex = false) {
    const int64_t n = L.n;
    L.ord.alloc(n);
    L.inv.alloc(n);
    if (single) {
        iota_i32(L.ord.get(), n, s);
        L.cptr = {0, (int32_t)n};
    } else if (lex) {  // the rows in their own order, one class each
        iota_i32(L.ord.get(), n, s);
        L.cptr.resize(n + 1);
        for (int64_t i = 0; i <= n; ++i) L.cptr[i] = (int32_t)i;
    } else {
        const int nc = L.ncolors;
        const int nblocks = (int)grid_for(n, 256);
        Temp<int32_t> lrank(n, s), hist((int64_t)nc * nblocks + 1, s), off((int64_t)nc * nblocks + 1, s), cp(nc + 1, s);
        colour_rank_k<<<nblocks, 256, sizeof(int32_t) * (256 + nc), s>>>(L.colour.get(), n, nc, nblocks, lrank.get(),
                                                                         hist.get());
        CK_LAUNCH();
        exclusive_scan_i32(hist.get(), off.get(), (int64_t)nc * nblocks, s);
        colour_place_k<<<nblocks, 256, 0, s>>>(L.colour.get(), lrank.get(), off.get(), n, nblocks, L.ord.get());
        CK_LAUNCH();
        colour_bounds_k<<<grid_for(nc + 1, 128), 128, 0, s>>>(off.get(), nc, nblocks, n, cp.get());
        CK_LAUNCH();
        L.cptr.assign(nc + 1, 0);
        to_host(L.cptr.data(), cp.get(), nc + 1, s);
    }
    invert_perm(L.ord.get(), L.inv.get(), n, s);
    Temp<int32_t> lenl(n + 1, s), lenu(n + 1, s);
    Temp<int> err(1, s);
    Temp<unsigned long long> tot(2, s);
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    CK(cudaMemsetAsync(tot.get(), 0, 2 * sizeof(unsigned long long), s));
    split_len_k<<<grid_for(n, 8), 256, 0, s>>>(L.rp.get(), L.ci.get(), L.v.get(), L.colour.get(), L.ord.get(), n,
                                               single ? 1 : 0, lenl.get(), lenu.get(), err.get(), tot.get());
    CK_LAUNCH();
    unsigned long long th[2];
    to_host(th, tot.get(), 2, s);
    L.nlow = (int64_t)th[0];
    L.nupp = (int64_t)th[1];
    int e = read1(err.get(), s);
    if (e & 1) fail(MGM_ERR_INVALID_ARG, "colouring is not valid for the operator pattern");
    if (e & 2) fail(MGM_ERR_BREAKDOWN, "a level operator has a zero or missing diagonal entry");
    L.lo.alloc(n + 1);
    L.up.alloc(n + 1);
    exclusive_scan_i32(lenl.get(), L.lo.get(), n, s);
    exclusive_scan_i32(lenu.get(), L.up.get(), n, s);
    L.nl_pad = csr_nnz(L.lo.get(), n, s);
    L.snnz = L.nl_pad + csr_nnz(L.up.get(), n, s);
    REQUIRE(L.snnz <= INT32_MAX, "level operator too large for 32-bit entry offsets");
    add_i32_k<<<grid_for(n + 1, 256), 256, 0, s>>>(L.up.get(), (int32_t)L.nl_pad, n + 1);
    CK_LAUNCH();
    L.sc.alloc(std::max<int64_t>(L.snnz, 4));
    L.sv64.alloc(std::max<int64_t>(L.snnz, 4));
    L.sv32.alloc(std::max<int64_t>(L.snnz, 4));
    L.diag64.alloc(n); L.dinv64.alloc(n); L.diag32.alloc(n); L.dinv32.alloc(n);
    Temp<int> longrows(1, s);
    CK(cudaMemsetAsync(longrows.get(), 0, sizeof(int), s));
    split_fill_k<<<grid_for(n, SPLIT_WARPS), SPLIT_WARPS * 32, 0, s>>>(
        L.rp.get(), L.ci.get(), L.v.get(), L.colour.get(), L.ord.get(), L.inv.get(), n, single ? 1 : 0, L.lo.get(),
        L.up.get(), L.sc.get(), L.sv64.get(), L.sv32.get(), L.diag64.get(), L.dinv64.get(), L.diag32.get(),
        L.dinv32.get(), longrows.get());
    CK_LAUNCH();
    if (read1(longrows.get(), s) > 0) {
        split_fill_long_k<<<grid_for(n, 128), 128, 0, s>>>(L.rp.get(), L.ci.get(), L.v.get(), L.colour.get(), L.ord.get(),
                                                           L.inv.get(), n, single ? 1 : 0, L.lo.get(), L.up.get(),
                                                           L.sc.get(), L.sv64.get(), L.sv32.get(), L.diag64.get(),
                                                           L.dinv64.get(), L.diag32.get(), L.dinv32.get());
        CK_LAUNCH();
    }
}

// interpolation rows re-indexed to solve orders: compact CSR (for the transpose) and ELL
__global__ void p_solve_len_k(const int32_t* prp, const int32_t* ord, int64_t n, int32_t* len) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) { int32_t r = ord[s]; len[s] = prp[r + 1] - prp[r]; }
}
__global__ void p_solve_fill_k(const int32_t* prp, const int32_t* pci, const double* pv, const int32_t* ord,
                               const int32_t* next_inv, int64_t n, int pw, const int32_t* crp, int32_t* cci, double* cv,
                               int32_t* ec, double* ev64, float* ev32) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int32_t r = ord[s];
    int32_t b = prp[r], len = prp[r + 1] - b;
    int32_t q0 = crp[s];
    for (int t = 0; t < len; ++t) {
        int32_t c = next_inv ? next_inv[pci[b + t]] : pci[b + t];
        cci[q0 + t] = c;
        cv[q0 + t] = pv[b + t];
    }
    for (int t = 1; t < len; ++t) {  // sort by column
        int32_t c = cci[q0 + t];
        double x = cv[q0 + t];
        int u = t;
        while (u > 0 && cci[q0 + u - 1] > c) { cci[q0 + u] = cci[q0 + u - 1]; cv[q0 + u] = cv[q0 + u - 1]; --u; }
        cci[q0 + u] = c;
        cv[q0 + u] = x;
    }
    for (int t = 0; t < pw; ++t) {
        bool has = t < len;
        ec[s * pw + t] = has ? cci[q0 + t] : 0;
        ev64[s * pw + t] = has ? cv[q0 + t] : 0.0;
        ev32[s * pw + t] = has ? (float)cv[q0 + t] : 0.0f;
    }
}
__global__ void to_f32_k(const double* a, float* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

static void build_transfers(Level& F, const Level* C, int64_t nc, int m, cudaStream_t s) {
    const int64_t n = F.n;
    Temp<int32_t> len(n + 1, s), crp(n + 1, s);
    p_solve_len_k<<<grid_for(n, 256), 256, 0, s>>>(F.P_rp.get(), F.ord.get(), n, len.get());
    CK_LAUNCH();
    exclusive_scan_i32(len.get(), crp.get(), n, s);
    Temp<int32_t> cci(std::max<int64_t>(F.pnnz, 1), s);
    Temp<double> cv(std::max<int64_t>(F.pnnz, 1), s);
    F.pw = m;
    F.pc.alloc(n * m);
    F.pv64.alloc(n * m);
    F.pv32.alloc(n * m);
    p_solve_fill_k<<<grid_for(n, 128), 128, 0, s>>>(F.P_rp.get(), F.P_ci.get(), F.P_v.get(), F.ord.get(),
                                                    C ? C->inv.get() : nullptr, n, m, crp.get(), cci.get(), cv.get(),
                                                    F.pc.get(), F.pv64.get(), F.pv32.get());
    CK_LAUNCH();
    F.r_rp.alloc(nc + 1);
    F.r_ci.alloc(std::max<int64_t>(F.pnnz, 1));
    F.r_v64.alloc(std::max<int64_t>(F.pnnz, 1));
    F.r_v32.alloc(std::max<int64_t>(F.pnnz, 1));
    csr_transpose(n, nc, crp.get(), cci.get(), cv.get(), F.r_rp.get(), F.r_ci.get(), F.r_v64.get(), s);
    if (F.pnnz > 0) {
        to_f32_k<<<grid_for(F.pnnz, 256), 256, 0, s>>>(F.r_v64.get(), F.r_v32.get(), F.pnnz);
        CK_LAUNCH();
    }
}

// BF16 bit patterns of FP32 weights: the top 16 bits rounded to nearest, ties to even (finite inputs)
__global__ void to_bf16_bits_k(const float* in, int64_t n, uint16_t* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned u = __float_as_uint(in[i]);
    out[i] = (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

__global__ void compose_k(const int32_t* a, const int32_t* b, int64_t n, int32_t* out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[b[i]];
}

// ------------------------------ setup driver ---------------------------------------------------
// With MGM_TRACE set in the environment, setup synchronises at each phase boundary and prints the
// phase's wall time to stderr (tracing only; off by default, no effect on results).
struct Trace {
    cudaStream_t s;
    explicit Trace(cudaStream_t st) : s(st) { trace_mark(s, "start"); }
    void mark(const char* what, int level) { trace_mark(s, what, level); }
};

mgm_hierarchy* setup(const double* xyz, int64_t N, const int32_t* rp, const int32_t* ci, const double* v,
                     const mgm_params* prm, cudaStream_t s) {
    REQUIRE(prm != nullptr, "null params");
    REQUIRE(xyz && rp && ci && v, "null array");
    REQUIRE(N >= 1 && N < 0x7fffffff, "N out of range");
    REQUIRE(prm->n_min >= 1, "n_min must be >= 1");
    REQUIRE(prm->m >= 1 && prm->m <= 8, "m must be in [1, 8]");
    REQUIRE(prm->nu1 >= 0 && prm->nu1 <= 8 && prm->nu2 >= 0 && prm->nu2 <= 8, "nu1, nu2 must be in [0, 8]");
    REQUIRE(prm->precision == MGM_F32 || prm->precision == MGM_F64, "precision must be MGM_F32 or MGM_F64");
    std::unique_ptr<mgm_hierarchy> H(new mgm_hierarchy());
    H->precision = prm->precision;
    H->nu1 = prm->nu1;
    H->nu2 = prm->nu2;
    H->m = prm->m;
    H->seed = prm->seed;
    REQUIRE(prm->persistent_sweeps >= 0 && prm->persistent_sweeps <= 5, "persistent_sweeps must be 0 to 5");
    REQUIRE(prm->smoother == MGM_SMOOTHER_MC || prm->smoother == MGM_SMOOTHER_LEX, "unknown smoother");
    const bool lex = prm->smoother == MGM_SMOOTHER_LEX;
    H->sweep_mode = lex ? 2 : prm->persistent_sweeps;  // lexicographic: one row per group, flag-driven
    H->persistent = H->sweep_mode != 0;  // error word checked after each solve
    REQUIRE(prm->constraint == 0 || prm->constraint == 1, "constraint must be 0 or 1");
    H->bordered = prm->constraint == 1;
    REQUIRE(prm->cycle >= MGM_CYCLE_V && prm->cycle <= MGM_CYCLE_F, "unknown cycle type");
    REQUIRE(prm->cycle == MGM_CYCLE_V || !H->bordered, "W and F cycles: not for constrained hierarchies");
    H->cycle = prm->cycle;
    REQUIRE(prm->transfer_bf16 == 0 || prm->transfer_bf16 == 1, "transfer_bf16 must be 0 or 1");
    H->transfer_bf16 = prm->transfer_bf16 == 1 && prm->precision == MGM_F32;
    H->N = N;
    int p = num_levels(N, prm->n_min);
    if (p > 16) fail(MGM_ERR_UNSUPPORTED, "more than 16 levels");
    // coarse levels must keep at least m points for the interpolation
    while (p > 1 && N / ((int64_t)1 << (2 * (p - 1))) < prm->m) --p;
    H->p = p;
    H->lv.resize(p);
    const int64_t nnz = csr_nnz(rp, N, s);
    Trace tr(s);
    // The symmetric pattern RCM builds for a level's operator, renumbered by the RCM permutation,
    // is the pattern of the level's final (permuted) operator: the multicolour colouring takes it
    // from there instead of building it again (smoothed levels; the colours are a function of the
    // pattern as a set).
    Temp<int32_t> sym_rp, sym_ci;
    auto colour_level = [&](int j) {
        Level& L = H->lv[j];
        if (lex || j + 1 >= p) return;
        Temp<int32_t> nrp, nci;
        permute_pattern(L.n, sym_rp.get(), sym_ci.get(), L.perm.get(), nrp, nci, s);
        sym_rp.release();
        sym_ci.release();
        L.colour.alloc(L.n);
        int32_t nc = 0;
        color(L.n, L.rp.get(), L.ci.get(), prm->seed, L.colour.get(), &nc, s, nrp.get(), nci.get());
        L.ncolors = nc;
        tr.mark("colour", j);
    };
    {   // level 1: RCM of L_1 and X_1 (Alg. 2)
        Level& L = H->lv[0];
        L.n = N;
        L.nnz = nnz;
        L.perm.alloc(N);
        rcm(N, rp, ci, L.perm.get(), s, &sym_rp, &sym_ci);
        tr.mark("  rcm", 0);
        L.X.alloc(3 * N);
        gather_xyz(xyz, L.perm.get(), L.X.get(), N, s);
        L.rp.alloc(N + 1);
        L.ci.alloc(nnz);
        L.v.alloc(nnz);
        csr_permute(N, rp, ci, v, L.perm.get(), L.rp.get(), L.ci.get(), L.v.get(), s);
        tr.mark("rcm+permute", 0);
        colour_level(0);
    }
    for (int j = 1; j < p; ++j) {
        Level& F = H->lv[j - 1];
        Level& C = H->lv[j];
        const int64_t NH = N / ((int64_t)1 << (2 * j));
        C.n = NH;
        C.keep.alloc(NH);
        coarsen(F.X.get(), F.n, NH, C.keep.get(), s, nullptr);              // coarse point cloud
        tr.mark("coarsen", j);
        Temp<double> Xc(3 * NH, s);
        gather_xyz(F.X.get(), C.keep.get(), Xc.get(), NH, s);
        Temp<int32_t> P_rp(F.n + 1, s), P_ci(F.n * prm->m, s);
        Temp<double> P_v(F.n * prm->m, s);
        int64_t pnnz = interp(F.X.get(), F.n, Xc.get(), NH, prm->m, P_rp.get(), P_ci.get(), P_v.get(), s);  // interpolation
        tr.mark("interp", j);
        Temp<int32_t> R_rp(NH + 1, s), R_ci(std::max<int64_t>(pnnz, 1), s);
        Temp<double> R_v(std::max<int64_t>(pnnz, 1), s);
        csr_transpose(F.n, NH, P_rp.get(), P_ci.get(), P_v.get(), R_rp.get(), R_ci.get(), R_v.get(), s);  // restriction
        tr.mark("  transpose", j);
        // Galerkin operator L_{j+1} = R (L_j P)
        Temp<int32_t> T_rp(F.n + 1, s);
        int64_t tnnz = spgemm_symbolic(F.n, F.rp.get(), F.ci.get(), P_rp.get(), P_ci.get(), T_rp.get(), s);
        Temp<int32_t> T_ci(std::max<int64_t>(tnnz, 1), s);
        Temp<double> T_v(std::max<int64_t>(tnnz, 1), s);
        spgemm_numeric(F.n, F.rp.get(), F.ci.get(), F.v.get(), P_rp.get(), P_ci.get(), P_v.get(), T_rp.get(), T_ci.get(),
                       T_v.get(), s);
        tr.mark("  galerkin:LP", j);
        Temp<int32_t> G_rp(NH + 1, s);
        int64_t gnnz = spgemm_symbolic(NH, R_rp.get(), R_ci.get(), T_rp.get(), T_ci.get(), G_rp.get(), s);
        Temp<int32_t> G_ci(std::max<int64_t>(gnnz, 1), s);
        Temp<double> G_v(std::max<int64_t>(gnnz, 1), s);
        spgemm_numeric(NH, R_rp.get(), R_ci.get(), R_v.get(), T_rp.get(), T_ci.get(), T_v.get(), G_rp.get(), G_ci.get(),
                       G_v.get(), s);
        tr.mark("galerkin", j);
        // RCM of L_{j+1}; renumber coarse points and the interpolation's columns
        C.perm.alloc(NH);
        rcm(NH, G_rp.get(), G_ci.get(), C.perm.get(), s, &sym_rp, &sym_ci);
        tr.mark("  rcm", j);
        C.X.alloc(3 * NH);
        gather_xyz(Xc.get(), C.perm.get(), C.X.get(), NH, s);
        C.nnz = gnnz;
        C.rp.alloc(NH + 1);
        C.ci.alloc(std::max<int64_t>(gnnz, 1));
        C.v.alloc(std::max<int64_t>(gnnz, 1));
        csr_permute(NH, G_rp.get(), G_ci.get(), G_v.get(), C.perm.get(), C.rp.get(), C.ci.get(), C.v.get(), s);
        Temp<int32_t> cinv(NH, s);
        invert_perm(C.perm.get(), cinv.get(), NH, s);
        F.pnnz = pnnz;
        F.P_rp.alloc(F.n + 1);
        F.P_ci.alloc(std::max<int64_t>(pnnz, 1));
        F.P_v.alloc(std::max<int64_t>(pnnz, 1));
        CK(cudaMemcpyAsync(F.P_rp.get(), P_rp.get(), sizeof(int32_t) * (F.n + 1), cudaMemcpyDeviceToDevice, s));
        remap_cols_k<<<grid_for(F.n, 256), 256, 0, s>>>(P_rp.get(), P_ci.get(), P_v.get(), cinv.get(), F.n, F.P_ci.get(),
                                                      F.P_v.get());
        CK_LAUNCH();
        tr.mark("rcm+permute", j);
        colour_level(j);
    }
    // colourings (multicolour: done above, level by level) and solve orders
    for (int j = 0; j + 1 < p; ++j) {
        Level& L = H->lv[j];
        if (lex) {  // every row its own class, in the level's (RCM) order
            L.colour.alloc(L.n);
            iota_i32(L.colour.get(), L.n, s);
            L.ncolors = (int32_t)L.n;
            tr.mark("colour", j);
        }
        build_solve_layout(L, false, s, lex);
        tr.mark("layout", j);
    }
    // transfers
    if (p == 1) build_solve_layout(H->lv[0], true, s);  // one group: serves the outer operator only
    for (int j = 0; j + 1 < p; ++j)
        build_transfers(H->lv[j], (j + 2 < p) ? &H->lv[j + 1] : nullptr, H->lv[j + 1].n, prm->m, s);
    if (H->transfer_bf16) {  // BF16 copies of the FP32 transfer weights
        for (int j = 0; j + 1 < p; ++j) {
            Level& L = H->lv[j];
            L.pv16.alloc(L.n * L.pw);
            to_bf16_bits_k<<<grid_for(L.n * L.pw, 256), 256, 0, s>>>(L.pv32.get(), L.n * L.pw, L.pv16.get());
            CK_LAUNCH();
            L.r_v16.alloc(std::max<int64_t>(L.pnnz, 1));
            if (L.pnnz > 0) {
                to_bf16_bits_k<<<grid_for(L.pnnz, 256), 256, 0, s>>>(L.r_v32.get(), L.pnnz, L.r_v16.get());
                CK_LAUNCH();
            }
        }
    }
    tr.mark("transfers", -1);
    // constrained Poisson (Sec. 4.4): border vectors c_0 = 1, c_{j+1} = R_j c_j (eq. (gco_saddle_point))
    if (H->bordered) {
        REQUIRE(p >= 2, "a constrained hierarchy needs at least two levels");
        for (int j = 0; j < p; ++j) {
            Level& L = H->lv[j];
            L.c64.alloc(L.n);
            if (j == 0) {
                fill_ones_k<<<grid_for(L.n, 256), 256, 0, s>>>(L.c64.get(), L.n);
            } else {
                Level& F = H->lv[j - 1];
                restrict_vec_k<<<grid_for(L.n, 256), 256, 0, s>>>(F.r_rp.get(), F.r_ci.get(), F.r_v64.get(), F.c64.get(),
                                                                L.n, L.c64.get());
            }
            CK_LAUNCH();
            if (H->precision == MGM_F32) {
                L.c32.alloc(L.n);
                to_f32_k<<<grid_for(L.n, 256), 256, 0, s>>>(L.c64.get(), L.c32.get(), L.n);
                CK_LAUNCH();
            }
        }
        H->sres.alloc(p + 1);
        CK(cudaMemsetAsync(H->sres.get(), 0, sizeof(double) * (p + 1), s));
        H->bpart.alloc(1024);
    }
    // coarsest factorisation
    H->np = H->lv[p - 1].n;
    H->nb = H->np + (H->bordered ? 1 : 0);
    dense_inverse(H->lv[p - 1], H->bordered ? H->lv[p - 1].c64.get() : nullptr, H->Ainv, s);
    tr.mark("coarse-inv", p - 1);
    // caller index of each level-0 solve row
    H->ord_caller.alloc(N);
    compose_k<<<grid_for(N, 256), 256, 0, s>>>(H->lv[0].perm.get(), H->lv[0].ord.get(), N, H->ord_caller.get());
    CK_LAUNCH();
    alloc_work(H.get());
    if (H->sweep_mode == MGM_SWEEP_STREAM) {  // streamed sweeps on every level they fit
        const int maxb = stream_blocks_limit(H.get());
        for (int j = 0; j + 1 < p; ++j) {
            Level& L = H->lv[j];
            const int B = (int)std::max<int64_t>(1, std::min<int64_t>(maxb, (L.n + 2047) / 2048));
            stream_prepare(H.get(), L, B, 2, 2, s);
        }
        tr.mark("stream-tables", p - 1);
    } else if (H->sweep_mode == MGM_SWEEP_AUTO) {  // the faster schedule per level, timed
        autotune(H.get(), 5, true, s);
        tr.mark("autotune", p - 1);
    } else if (H->sweep_mode == MGM_SWEEP_STAGED) {  // staged per-colour launches on every level
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        for (int j = 0; j + 1 < p; ++j) {
            Level& L = H->lv[j];
            // measured on the 1M-point sphere (n = 50): four bands an SM and 2 lanes a row on levels
            // of 500k rows and more, three bands an SM and 4 lanes from 100k, one band an SM below,
            // with 4 lanes (>= 30k rows) or 8 (the levels there are bound by launch latency alone)
            const int B = L.n >= 500000 ? 4 * sms : (L.n >= 100000 ? 3 * sms : sms);
            const int G = L.n >= 500000 ? 2 : (L.n >= 30000 ? 4 : 8);
            colour_prepare(H.get(), L, B, G, s);  // (a level that does not fit keeps plain launches)
        }
        tail_prepare(H.get(), s);  // the coarse levels in one cluster launch, where they fit
        tr.mark("staged-tables", p - 1);
    }
    CK(cudaStreamSynchronize(s));
    int64_t bytes = H->Ainv.bytes() + H->ord_caller.bytes();
    for (auto& L : H->lv)
        bytes += L.X.bytes() + L.rp.bytes() + L.ci.bytes() + L.v.bytes() + L.perm.bytes() + L.keep.bytes() + L.P_rp.bytes() +
                 L.P_ci.bytes() + L.P_v.bytes() + L.colour.bytes() + L.ord.bytes() + L.inv.bytes() + L.lo.bytes() +
                 L.up.bytes() + L.sc.bytes() + L.sv32.bytes() + L.sv64.bytes() + 3 * L.diag64.bytes() + 3 * L.diag32.bytes() +
                 L.pc.bytes() + L.pv32.bytes() + L.pv16.bytes() + L.r_v16.bytes() + L.pv64.bytes() + L.r_rp.bytes() + L.r_ci.bytes() + L.r_v32.bytes() +
                 L.r_v64.bytes() + L.b32.bytes() * 3 + L.b64.bytes() * 3;
    H->device_bytes = bytes;
    return H.release();
}

void hierarchy_level(const mgm_hierarchy* H, int j, int32_t* perm, int32_t* keep, double* xyz, int32_t* lrp, int32_t* lci,
                     double* lv, int32_t* prp, int32_t* pci, double* pv, int32_t* colour, cudaStream_t s) {
    REQUIRE(H && j >= 0 && j < H->p, "level index out of range");
    const Level& L = H->lv[j];
    auto cp = [&](void* dst, const void* src, size_t bytes) {
        if (dst && src && bytes) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
    };
    cp(perm, L.perm.get(), L.perm.bytes());
    if (j >= 1) cp(keep, L.keep.get(), L.keep.bytes());
    cp(xyz, L.X.get(), sizeof(double) * 3 * L.n);
    cp(lrp, L.rp.get(), sizeof(int32_t) * (L.n + 1));
    cp(lci, L.ci.get(), sizeof(int32_t) * L.nnz);
    cp(lv, L.v.get(), sizeof(double) * L.nnz);
    if (j + 1 < H->p) {
        cp(prp, L.P_rp.get(), sizeof(int32_t) * (L.n + 1));
        cp(pci, L.P_ci.get(), sizeof(int32_t) * L.pnnz);
        cp(pv, L.P_v.get(), sizeof(double) * L.pnnz);
        cp(colour, L.colour.get(), sizeof(int32_t) * L.n);
    }
}

}  // namespace mgm

mgm_hierarchy::~mgm_hierarchy() {
    mgm::free_multi(this);
    if (vgraph) cudaGraphExecDestroy(vgraph);
    if (lgraph) cudaGraphExecDestroy(lgraph);
    if (sgraph) cudaGraphExecDestroy(sgraph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (hhost) cudaFreeHost(hhost);
}

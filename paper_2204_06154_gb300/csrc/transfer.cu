// Transfer operators and the Galerkin product (paper Sec. 3 and Sec. 4.2).
//
// Interpolation I_H^h (eq. (rbf_fd_interp)): per fine node the m nearest coarse nodes, a
// (m+1) x (m+1) PHS system with phi(r) = r plus a constant, solved in R^3 by Gaussian elimination
// with partial pivoting (one thread per row; same operation sequence as a sequential solve).
//
// SpGEMM C = A B (used as T = L P, then L_H = R T, eq. (galerkin)): one warp per row of C. The
// pattern is the union of the B rows selected by the A row, collected in a per-warp open-addressing
// hash set in shared memory, compacted and sorted by rank. Each lane then owns a few output
// columns j and accumulates sum_p a_ip b_{l_p j} over A's row in ascending order with fused
// multiply-adds (binary search of j in the sorted B row), which is exactly the order of a
// row-by-row sequential product: results are bit-reproducible. Built with --fmad=false.
#include <climits>

#include "common.cuh"

namespace mgm {

// ------------------------------ interpolation ------------------------------------------------
constexpr int MAX_INTERP_M = 8;

__device__ int gepp_small(double* a, int m, double tol, double* x) {
    const int ld = m + 1;
    double rinvs[MAX_INTERP_M + 1];
    for (int k = 0; k < m; ++k) {
        int piv = k;
        double best = fabs(a[k * ld + k]);
        for (int i = k + 1; i < m; ++i) {
            double v = fabs(a[i * ld + k]);
            if (v > best) { best = v; piv = i; }
        }
        if (!(best > tol)) return 1;
        if (piv != k)
            for (int j = 0; j < ld; ++j) { double t = a[k * ld + j]; a[k * ld + j] = a[piv * ld + j]; a[piv * ld + j] = t; }
        const double rinv = 1.0 / a[k * ld + k];
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
    for (int k = 0; k < m; ++k)
        if (!isfinite(x[k])) return 1;
    return 0;
}

__global__ void interp_len_k(const double* d2, int64_t nf, int m, int32_t* len) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) len[i] = d2[i * m] == 0.0 ? 1 : m;
}

__global__ void interp_fill_k(const double* xc, const int32_t* nb, const double* d2, int64_t nf, int m, const int32_t* rp,
                              int32_t* col, double* val, unsigned long long* bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const int32_t* id = nb + i * m;
    int32_t p = rp[i];
    if (d2[i * m] == 0.0) {
        col[p] = id[0];
        val[p] = 1.0;
        return;
    }
    double a[(MAX_INTERP_M + 1) * (MAX_INTERP_M + 2)], x[MAX_INTERP_M + 1];
    const int M = m + 1, ld = M + 1;
    double amax = 0.0;
    for (int r = 0; r < m; ++r) {
        const double* yr = xc + 3 * (int64_t)id[r];
        for (int c = 0; c < m; ++c) {
            const double* yc = xc + 3 * (int64_t)id[c];
            double dx = yr[0] - yc[0], dy = yr[1] - yc[1], dz = yr[2] - yc[2];
            a[r * ld + c] = sqrt((dx * dx + dy * dy) + dz * dz);
        }
        a[r * ld + m] = 1.0;
        a[r * ld + M] = sqrt(d2[i * m + r]);
    }
    for (int c = 0; c < m; ++c) a[m * ld + c] = 1.0;
    a[m * ld + m] = 0.0;
    a[m * ld + M] = 1.0;
    for (int r = 0; r < M; ++r)
        for (int c = 0; c < M; ++c) amax = fmax(amax, fabs(a[r * ld + c]));
    if (gepp_small(a, M, 1e-13 * amax, x)) {
        atomicMin(bad, (unsigned long long)i);
        return;
    }
    int32_t b = p;
    for (int r = 0; r < m; ++r) {
        int32_t c = id[r];
        double v = x[r];
        int32_t q = p;
        while (q > b && col[q - 1] > c) { col[q] = col[q - 1]; val[q] = val[q - 1]; --q; }
        col[q] = c;
        val[q] = v;
        ++p;
    }
}

// builds I_H^h as CSR; rp (nf+1) and col/val with capacity nf*m. Returns nnz.
int64_t interp(const double* xf, int64_t nf, const double* xc, int64_t nc, int m, int32_t* rp, int32_t* col, double* val,
               cudaStream_t s) {
    REQUIRE(xf && xc && rp && col && val, "null array");
    REQUIRE(m >= 1 && m <= MAX_INTERP_M && m <= nc, "interpolation stencil m must be in [1, min(8, N_c)]");
    REQUIRE(nf >= 1 && nf < 0x7fffffff && nf * (int64_t)m < 0x7fffffff, "N_f out of range");
    Temp<int32_t> nb(nf * m, s), len(nf + 1, s);
    Temp<double> d2(nf * m, s);
    knn_device(xc, nc, xf, nf, m, 0, nb.get(), d2.get(), s);
    interp_len_k<<<grid_for(nf, 256), 256, 0, s>>>(d2.get(), nf, m, len.get());
    CK_LAUNCH();
    exclusive_scan_i32(len.get(), rp, nf, s);
    set_bad_row(-1);
    Temp<unsigned long long> bad(1, s);
    CK(cudaMemsetAsync(bad.get(), 0xff, sizeof(unsigned long long), s));
    interp_fill_k<<<grid_for(nf, 128), 128, 0, s>>>(xc, nb.get(), d2.get(), nf, m, rp, col, val, bad.get());
    CK_LAUNCH();
    unsigned long long b = read1(bad.get(), s);
    if (b != ULLONG_MAX) {
        set_bad_row((int64_t)b);
        fail(MGM_ERR_SINGULAR_STENCIL, "interpolation: singular local system at fine row " + std::to_string(b));
    }
    return csr_nnz(rp, nf, s);
}

// ------------------------------ SpGEMM ---------------------------------------------------------
// Hash-set size per warp: the next power of two >= 2x the largest product count of any row
// (64..4096 slots); at most half the slots may be filled (distinct columns of one row).
constexpr int SG_WARPS = 4;
constexpr int SG_MAX_HASH = 4096;

__device__ __forceinline__ int sg_insert(int* slots, int hs, int col) {
    const int shift = 32 - (31 - __clz(hs));
    unsigned h = ((unsigned)col * 2654435761u) >> shift;
    for (int probe = 0; probe < hs; ++probe) {
        int old = atomicCAS(&slots[h], -1, col);
        if (old == -1) return 1;
        if (old == col) return 0;
        h = (h + 1) & (hs - 1);
    }
    return -1;
}

// per-warp: build the hash set of row i's columns; returns the unique count (warp-uniform)
__device__ int sg_collect(int* slots, int hs, const int32_t* arp, const int32_t* aci, const int32_t* brp,
                          const int32_t* bci, int64_t i, int lane, bool* overflow) {
    for (int t = lane; t < hs; t += 32) slots[t] = -1;
    __syncwarp();
    int added = 0;
    bool ovf = false;
    for (int32_t p = arp[i]; p < arp[i + 1]; ++p) {
        int32_t l = aci[p];
        for (int32_t q = brp[l] + lane; q < brp[l + 1]; q += 32) {
            int r = sg_insert(slots, hs, bci[q]);
            if (r < 0) ovf = true;
            else added += r;
        }
    }
    __syncwarp();
    added = warp_sum_i(added);
    *overflow = __any_sync(0xffffffffu, ovf) || added > hs / 2;
    return added;
}

__global__ void sg_maxprod_k(int64_t nA, const int32_t* arp, const int32_t* aci, const int32_t* brp, int* mx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nA) return;
    int c = 0;
    for (int32_t p = arp[i]; p < arp[i + 1]; ++p) c += brp[aci[p] + 1] - brp[aci[p]];
    atomicMax(mx, c);
}

__global__ void __launch_bounds__(SG_WARPS * 32) spgemm_symbolic_k(int64_t nA, const int32_t* arp, const int32_t* aci,
                                                                   const int32_t* brp, const int32_t* bci, int32_t* cnt,
                                                                   int hs, int* err) {
    extern __shared__ int sg_smem[];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t i = (int64_t)blockIdx.x * SG_WARPS + w;
    if (i >= nA) return;
    bool ovf;
    int u = sg_collect(sg_smem + w * hs, hs, arp, aci, brp, bci, i, lane, &ovf);
    if (lane == 0) {
        cnt[i] = u;
        if (ovf) atomicOr(err, 1);
    }
}

__global__ void __launch_bounds__(SG_WARPS * 32) spgemm_numeric_k(int64_t nA, const int32_t* arp, const int32_t* aci,
                                                                  const double* av, const int32_t* brp, const int32_t* bci,
                                                                  const double* bv, const int32_t* crp, int32_t* cci,
                                                                  double* cv, int hs, int* err) {
    extern __shared__ int sg_smem[];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int* slots = sg_smem + w * hs;
    int* lst = sg_smem + SG_WARPS * hs + w * (hs / 2);
    int64_t i = (int64_t)blockIdx.x * SG_WARPS + w;
    if (i >= nA) return;
    bool ovf;
    int u = sg_collect(slots, hs, arp, aci, brp, bci, i, lane, &ovf);
    if (ovf || u != crp[i + 1] - crp[i]) {
        if (lane == 0) atomicOr(err, 2);
        return;
    }
    // compact the set into lst
    int base = 0;
    for (int t = lane; t - lane < hs; t += 32) {
        int c = t < hs ? slots[t] : -1;
        unsigned m = __ballot_sync(0xffffffffu, c >= 0);
        if (c >= 0) lst[base + __popc(m & ((1u << lane) - 1u))] = c;
        base += __popc(m);
    }
    __syncwarp();
    // rank sort into the slot array (reused as the sorted column list)
    int* sorted = slots;
    for (int t = lane; t < u; t += 32) {
        int c = lst[t];
        int r = 0;
        for (int q = 0; q < u; ++q) r += lst[q] < c ? 1 : 0;
        sorted[r] = c;
    }
    __syncwarp();
    const int32_t c0 = crp[i];
    const int32_t ab = arp[i], ae = arp[i + 1];
    for (int t = lane; t < u; t += 32) {
        int j = sorted[t];
        double acc = 0.0;
        for (int32_t p = ab; p < ae; ++p) {
            int32_t l = aci[p];
            int32_t lo = brp[l], hi = brp[l + 1] - 1;
            while (lo <= hi) {
                int32_t mid = (lo + hi) >> 1;
                int32_t bc = bci[mid];
                if (bc == j) { acc = fma(av[p], bv[mid], acc); break; }
                if (bc < j) lo = mid + 1; else hi = mid - 1;
            }
        }
        cci[c0 + t] = j;
        cv[c0 + t] = acc;
    }
}

static int sg_hash_size(int64_t nA, const int32_t* arp, const int32_t* aci, const int32_t* brp, cudaStream_t s) {
    Temp<int> mx(1, s);
    CK(cudaMemsetAsync(mx.get(), 0, sizeof(int), s));
    if (nA > 0) {
        sg_maxprod_k<<<grid_for(nA, 256), 256, 0, s>>>(nA, arp, aci, brp, mx.get());
        CK_LAUNCH();
    }
    int m = read1(mx.get(), s);
    int hs = 64;
    while (hs < 2 * m && hs < SG_MAX_HASH) hs *= 2;
    return hs;
}

// symbolic phase: fills crp (nA+1), returns nnz
int64_t spgemm_symbolic(int64_t nA, const int32_t* arp, const int32_t* aci, const int32_t* brp, const int32_t* bci,
                        int32_t* crp, cudaStream_t s) {
    Temp<int32_t> cnt(nA + 1, s);
    Temp<int> err(1, s);
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    if (nA > 0) {
        const int hs = sg_hash_size(nA, arp, aci, brp, s);
        const size_t smem = sizeof(int) * SG_WARPS * hs;
        CK(cudaFuncSetAttribute(spgemm_symbolic_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        spgemm_symbolic_k<<<grid_for(nA, SG_WARPS), SG_WARPS * 32, smem, s>>>(nA, arp, aci, brp, bci, cnt.get(), hs,
                                                                             err.get());
        CK_LAUNCH();
    }
    if (read1(err.get(), s)) fail(MGM_ERR_UNSUPPORTED, "SpGEMM row exceeds 2048 distinct columns");
    exclusive_scan_i32(cnt.get(), crp, nA, s);
    return csr_nnz(crp, nA, s);
}

void spgemm_numeric(int64_t nA, const int32_t* arp, const int32_t* aci, const double* av, const int32_t* brp,
                    const int32_t* bci, const double* bv, const int32_t* crp, int32_t* cci, double* cv, cudaStream_t s) {
    if (nA <= 0) return;
    Temp<int> err(1, s);
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    const int hs = sg_hash_size(nA, arp, aci, brp, s);
    const size_t smem = sizeof(int) * SG_WARPS * (hs + hs / 2);
    CK(cudaFuncSetAttribute(spgemm_numeric_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    spgemm_numeric_k<<<grid_for(nA, SG_WARPS), SG_WARPS * 32, smem, s>>>(nA, arp, aci, av, brp, bci, bv, crp, cci, cv, hs,
                                                                        err.get());
    CK_LAUNCH();
    if (read1(err.get(), s)) fail(MGM_ERR_INVALID_ARG, "SpGEMM: row pointer does not match the product pattern");
}

}  // namespace mgm

// Transfer operators and the Galerkin product (paper Sec. 3 and Sec. 4.2).
//
// Interpolation I_H^h (eq. (rbf_fd_interp)): per fine node the m nearest coarse nodes, a
// (m+1) x (m+1) PHS system with phi(r) = r plus a constant, solved in R^3 by Gaussian elimination
// with partial pivoting (one thread per row; same operation sequence as a sequential solve).
//
// SpGEMM C = A B (used as T = L P, then L_H = R T, eq. (galerkin)): one warp per row of C. The
// warp first gathers the row's products into shared memory with all loads in flight at once
// (lanes over the A entries for the B row extents, then lanes over the flattened products for
// their columns and values). The pattern is the union of those columns, collected in a per-warp
// open-addressing hash set, compacted and sorted by rank. The values are then accumulated from
// shared memory with A's entries taken one at a time in ascending order and lanes over the B row
// of each (a B row holds each column once, so no two lanes meet), with fused multiply-adds: every
// c_ij is the sum over A's row in ascending order, exactly the order of a row-by-row sequential
// product, so results are bit-reproducible. Built with --fmad=false.
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
constexpr int SG_MAX_HASH = 4096;

__device__ __forceinline__ unsigned sg_hash(int col, int hs) {
    const int shift = 32 - (31 - __clz(hs));
    return ((unsigned)col * 2654435761u) >> shift;
}
__device__ __forceinline__ int sg_insert(int* slots, int hs, int col) {
    unsigned h = sg_hash(col, hs);
    for (int probe = 0; probe < hs; ++probe) {
        int old = atomicCAS(&slots[h], -1, col);
        if (old == -1) return 1;
        if (old == col) return 0;
        h = (h + 1) & (hs - 1);
    }
    return -1;
}
// slot of a column known to be in the set
__device__ __forceinline__ int sg_find(const int* slots, int hs, int col) {
    unsigned h = sg_hash(col, hs);
    for (int probe = 0; probe < hs && slots[h] != col; ++probe) h = (h + 1) & (hs - 1);
    return (int)h;
}

// Per-warp shared memory: hash slots[hs]; (numeric) rank[hs], reused after the ranking as the
// per-column counts and segment ends; the products' columns pj[mp] (in the numeric phase replaced
// by their columns' ranks), (numeric) their B values pv[mp] and A values pa[mp] (double), and the
// products sorted by column srt[mp] (first the compacted columns); per A entry its first product
// aoff[ma + 1]. mp: the largest product count of a row, ma: the largest A row.
struct SgLayout {
    size_t slots, rank, pj, pv, pa, srt, aoff, bytes;
};
__host__ __device__ inline SgLayout sg_layout(int hs, int mp, int ma, bool numeric) {
    SgLayout o;
    size_t off = 0;
    o.pv = off; off += numeric ? 8 * (size_t)mp : 0;
    o.pa = off; off += numeric ? 8 * (size_t)mp : 0;
    o.slots = off; off += 4 * (size_t)hs;
    o.rank = off; off += numeric ? 4 * (size_t)hs : 0;
    o.pj = off; off += 4 * (size_t)mp;
    o.srt = off; off += numeric ? 4 * (size_t)mp : 0;
    o.aoff = off; off += 4 * (size_t)(ma + 1);
    o.bytes = (off + 15) & ~(size_t)15;
    return o;
}

// Gathers row i's products into pj (and their B and A values into pv, pa when av is given) in
// A-row order, aoff[t] = first product of A entry t; then inserts the columns into the hash set.
// Returns the number of distinct columns (warp-uniform); *overflow when the set or the product
// buffer is too small.
__device__ int sg_gather(int* slots, int hs, int* pj, double* pv, int* aoff, double* pa, int mp, const int32_t* arp,
                         const int32_t* aci, const double* av, const int32_t* brp, const int32_t* bci, const double* bv,
                         int64_t i, int lane, bool* overflow) {
    for (int t = lane; t < hs; t += 32) slots[t] = -1;
    const int32_t ab = arp[i], ae = arp[i + 1];
    int base = 0;
    for (int32_t c0 = ab; c0 < ae; c0 += 32) {
        const int32_t p = c0 + lane;
        const bool has = p < ae;
        const int32_t l = has ? aci[p] : 0;
        const int32_t b0 = has ? brp[l] : 0;
        const int len = has ? brp[l + 1] - b0 : 0;
        const double al = has && av ? av[p] : 0.0;
        int incl = len;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - len, tot = __shfl_sync(0xffffffffu, incl, 31);
        if (has) aoff[p - ab] = base + excl;
        // lanes over the flattened products of these (up to) 32 A entries
        for (int e0 = 0; e0 < tot; e0 += 32) {
            const int e = e0 + lane;
            // the A entry whose products hold e: the last lane with excl <= e
            int lo = 0;
            for (int step = 16; step; step >>= 1) {
                const int x = __shfl_sync(0xffffffffu, excl, lo + step);
                if (lo + step < 32 && x <= e) lo += step;
            }
            const int32_t sb = __shfl_sync(0xffffffffu, b0, lo), se = __shfl_sync(0xffffffffu, excl, lo);
            const double ae = __shfl_sync(0xffffffffu, al, lo);
            if (e < tot && base + e < mp) {
                const int32_t q = sb + (e - se);
                pj[base + e] = bci[q];
                if (bv) pv[base + e] = bv[q];
                if (pa) pa[base + e] = ae;
            }
        }
        base += tot;
    }
    if (lane == 0 && ae > ab) aoff[ae - ab] = base;
    __syncwarp();
    bool ovf = base > mp;
    int added = 0;
    for (int e = lane; e < base && !ovf; e += 32) {
        const int r = sg_insert(slots, hs, pj[e]);
        if (r < 0) ovf = true;
        else added += r;
    }
    __syncwarp();
    added = warp_sum_i(added);
    *overflow = __any_sync(0xffffffffu, ovf) || added > hs / 2;
    return added;
}

// largest product count and largest A row over the rows: mx[0], mx[1]
__global__ void sg_maxprod_k(int64_t nA, const int32_t* arp, const int32_t* aci, const int32_t* brp, int* mx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nA) return;
    int c = 0;
    for (int32_t p = arp[i]; p < arp[i + 1]; ++p) c += brp[aci[p] + 1] - brp[aci[p]];
    atomicMax(mx, c);
    atomicMax(mx + 1, arp[i + 1] - arp[i]);
}

__global__ void spgemm_symbolic_k(int64_t nA, const int32_t* arp, const int32_t* aci, const int32_t* brp,
                                  const int32_t* bci, int32_t* cnt, int hs, int mp, int ma, int* err) {
    extern __shared__ __align__(16) unsigned char sg_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const SgLayout lay = sg_layout(hs, mp, ma, false);
    unsigned char* base = sg_smem + lay.bytes * w;
    const int64_t i = (int64_t)blockIdx.x * wpb + w;
    if (i >= nA) return;
    bool ovf;
    const int u = sg_gather((int*)(base + lay.slots), hs, (int*)(base + lay.pj), nullptr, (int*)(base + lay.aoff), nullptr,
                            mp, arp, aci, nullptr, brp, bci, nullptr, i, lane, &ovf);
    if (lane == 0) {
        cnt[i] = u;
        if (ovf) atomicOr(err, 1);
    }
}

// Row i of C = A B, a warp per row. Each column's sum takes its products in A-row order,
// c = fma(a_p, b, c) from c = 0, the order of the oracle's product: the products are ranked by
// column, stably sorted by rank (a chunk of 32 products at a time, equal ranks within a chunk
// placed by lane), and a lane a column then adds its segment in that order.
__global__ void spgemm_numeric_k(int64_t nA, const int32_t* arp, const int32_t* aci, const double* av,
                                 const int32_t* brp, const int32_t* bci, const double* bv, const int32_t* crp,
                                 int32_t* cci, double* cv, int hs, int mp, int ma, int* err) {
    extern __shared__ __align__(16) unsigned char sg_smem[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const SgLayout lay = sg_layout(hs, mp, ma, true);
    unsigned char* base = sg_smem + lay.bytes * w;
    int* slots = (int*)(base + lay.slots);
    int* rank = (int*)(base + lay.rank);
    int* pj = (int*)(base + lay.pj);
    double* pv = (double*)(base + lay.pv);
    double* pa = (double*)(base + lay.pa);
    int* srt = (int*)(base + lay.srt);
    int* aoff = (int*)(base + lay.aoff);
    const int64_t i = (int64_t)blockIdx.x * wpb + w;
    if (i >= nA) return;
    bool ovf;
    const int u = sg_gather(slots, hs, pj, pv, aoff, pa, mp, arp, aci, av, brp, bci, bv, i, lane, &ovf);
    if (ovf || u != crp[i + 1] - crp[i]) {
        if (lane == 0) atomicOr(err, 2);
        return;
    }
    const int na = arp[i + 1] - arp[i];
    const int tot = na > 0 ? aoff[na] : 0;  // products of the row
    // compact the set (into srt, free until the sort)
    int* lst = srt;
    int nb = 0;
    for (int t = lane; t - lane < hs; t += 32) {
        const int c = t < hs ? slots[t] : -1;
        const unsigned m = __ballot_sync(0xffffffffu, c >= 0);
        if (c >= 0) lst[nb + __popc(m & ((1u << lane) - 1u))] = c;
        nb += __popc(m);
    }
    __syncwarp();
    // rank of each column among the row's columns, kept at its hash slot; the sorted columns out
    const int32_t c0 = crp[i];
    for (int t = lane; t < u; t += 32) {
        const int c = lst[t];
        int r = 0;
        for (int q = 0; q < u; ++q) r += lst[q] < c ? 1 : 0;
        rank[sg_find(slots, hs, c)] = r;
        cci[c0 + r] = c;
    }
    __syncwarp();
    // each product's column rank, over its column
    for (int e = lane; e < tot; e += 32) pj[e] = rank[sg_find(slots, hs, pj[e])];
    __syncwarp();
    int* cnt = rank;            // products a column
    int* seg = rank + hs / 2;   // start, then end, of each column's segment in srt
    for (int t = lane; t < u; t += 32) cnt[t] = 0;
    __syncwarp();
    for (int e = lane; e < tot; e += 32) atomicAdd(&cnt[pj[e]], 1);
    __syncwarp();
    int carry = 0;
    for (int t0 = 0; t0 < u; t0 += 32) {
        const int t = t0 + lane;
        const int c = t < u ? cnt[t] : 0;
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (t < u) seg[t] = carry + incl - c;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    for (int e0 = 0; e0 < tot; e0 += 32) {
        const int e = e0 + lane;
        const int r = e < tot ? pj[e] : -1 - lane;  // idle lanes: keys of their own
        const unsigned grp = __match_any_sync(0xffffffffu, r);
        const int before = __popc(grp & ((1u << lane) - 1u));
        int at = 0;
        if (e < tot) at = seg[r] + before;
        __syncwarp();
        if (e < tot) {
            srt[at] = e;
            if (before == __popc(grp) - 1) seg[r] = at + 1;  // the group's last lane moves the cursor
        }
        __syncwarp();
    }
    for (int t = lane; t < u; t += 32) {
        const int e1 = seg[t], e0 = e1 - cnt[t];
        double acc = 0.0;
        for (int j = e0; j < e1; ++j) {
            const int e = srt[j];
            acc = fma(pa[e], pv[e], acc);
        }
        cv[c0 + t] = acc;
    }
}

struct SgShape {
    int hs, mp, ma;
};
static SgShape sg_shape(int64_t nA, const int32_t* arp, const int32_t* aci, const int32_t* brp, cudaStream_t s) {
    Temp<int> mx(2, s);
    CK(cudaMemsetAsync(mx.get(), 0, 2 * sizeof(int), s));
    if (nA > 0) {
        sg_maxprod_k<<<grid_for(nA, 256), 256, 0, s>>>(nA, arp, aci, brp, mx.get());
        CK_LAUNCH();
    }
    int h[2];
    to_host(h, mx.get(), 2, s);
    int hs = 64;
    while (hs < 2 * h[0] && hs < SG_MAX_HASH) hs *= 2;
    return {hs, std::max(h[0], 1), std::max(h[1], 1)};
}
// warps per block: up to 4, within 200 KB of shared memory
static int sg_warps(size_t per_warp) {
    int w = 4;
    while (w > 1 && per_warp * w > 200 * 1024) --w;
    return w;
}

// symbolic phase: fills crp (nA+1), returns nnz
int64_t spgemm_symbolic(int64_t nA, const int32_t* arp, const int32_t* aci, const int32_t* brp, const int32_t* bci,
                        int32_t* crp, cudaStream_t s) {
    Temp<int32_t> cnt(nA + 1, s);
    Temp<int> err(1, s);
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    if (nA > 0) {
        const SgShape sh = sg_shape(nA, arp, aci, brp, s);
        const size_t per = sg_layout(sh.hs, sh.mp, sh.ma, false).bytes;
        if (per > 200 * 1024) fail(MGM_ERR_UNSUPPORTED, "SpGEMM row has too many products");
        const int wpb = sg_warps(per);
        CK(cudaFuncSetAttribute(spgemm_symbolic_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(per * wpb)));
        spgemm_symbolic_k<<<grid_for(nA, wpb), wpb * 32, per * wpb, s>>>(nA, arp, aci, brp, bci, cnt.get(), sh.hs, sh.mp,
                                                                       sh.ma, err.get());
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
    const SgShape sh = sg_shape(nA, arp, aci, brp, s);
    const size_t per = sg_layout(sh.hs, sh.mp, sh.ma, true).bytes;
    if (per > 200 * 1024) fail(MGM_ERR_UNSUPPORTED, "SpGEMM row has too many products");
    const int wpb = sg_warps(per);
    CK(cudaFuncSetAttribute(spgemm_numeric_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(per * wpb)));
    spgemm_numeric_k<<<grid_for(nA, wpb), wpb * 32, per * wpb, s>>>(nA, arp, aci, av, brp, bci, bv, crp, cci, cv, sh.hs,
                                                                  sh.mp, sh.ma, err.get());
    CK_LAUNCH();
    if (read1(err.get(), s)) fail(MGM_ERR_INVALID_ARG, "SpGEMM: row pointer does not match the product pattern");
}

}  // namespace mgm

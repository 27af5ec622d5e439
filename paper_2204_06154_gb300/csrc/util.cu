// Device-wide building blocks for the setup phase: scans, permutations, CSR transpose and
// permutation, the symmetrised pattern used by RCM and colouring. Every output is deterministic
// (independent of thread scheduling): where atomics place entries, the rows are sorted afterwards.
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstdio>

#include <map>
#include <unordered_map>
#include <mutex>
#include <tuple>

#include "common.cuh"

namespace mgm {

// ---------------------------------------------------------------------------------------------
// error state
// ---------------------------------------------------------------------------------------------
static std::atomic<int64_t> g_launches{0};
static thread_local int64_t t_launches = 0;
void note_launch(int64_t n) {
    g_launches.fetch_add(n, std::memory_order_relaxed);
    t_launches += n;
}
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }
int64_t thread_launches() { return t_launches; }
static thread_local std::string g_msg;
static thread_local int64_t g_row = -1;
void set_error(const std::string& msg) { g_msg = msg; }
void set_bad_row(int64_t row) { g_row = row; }
const char* error_message() { return g_msg.c_str(); }
int64_t bad_row() { return g_row; }
static thread_local int64_t g_fp64_rows = 0;
void set_fp64_rows(int64_t n) { g_fp64_rows = n; }
int64_t fp64_rows() { return g_fp64_rows; }
void fail(mgm_status st, const std::string& msg) {
    set_error(msg);
    throw Fail{st};
}
void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
    if (e == cudaSuccess) return;
    (void)cudaGetLastError();
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) fail(MGM_ERR_OOM, buf);
    fail(MGM_ERR_CUDA, buf);
}

// ---------------------------------------------------------------------------------------------
// scans: block-level scan of 1024 items per block, then a scan of block totals (recursive)
// ---------------------------------------------------------------------------------------------
constexpr int SCAN_BLOCK = 512;
constexpr int SCAN_ITEMS = 2;  // per thread
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

template <class T>
__device__ T block_exclusive_scan(T v, T* smem, T* total) {
    // smem: SCAN_BLOCK/32 entries
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = lane < SCAN_BLOCK / 32 ? smem[lane] : T(0);
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SCAN_BLOCK / 32) smem[lane] = t;
    }
    __syncthreads();
    T before = (w > 0 ? smem[w - 1] : T(0)) + x - v;
    if (total) *total = smem[SCAN_BLOCK / 32 - 1];
    __syncthreads();
    return before;
}

template <class T>
__global__ void scan_tiles(const T* in, T* out, int64_t n, T* tile_sums) {
    __shared__ T sm[SCAN_BLOCK / 32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    T v[SCAN_ITEMS];
    T local = 0;
    for (int t = 0; t < SCAN_ITEMS; ++t) {
        int64_t i = base + t;
        v[t] = i < n ? in[i] : T(0);
        local += v[t];
    }
    T total;
    T pre = block_exclusive_scan<T>(local, sm, &total);
    for (int t = 0; t < SCAN_ITEMS; ++t) {
        int64_t i = base + t;
        if (i < n) out[i] = pre;
        pre += v[t];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

template <class T>
__global__ void scan_add(T* out, int64_t n, const T* tile_prefix, T* total_out) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    T add = tile_prefix[blockIdx.x];
    for (int t = threadIdx.x; t < SCAN_TILE; t += blockDim.x) {
        int64_t i = base + t;
        if (i < n) out[i] += add;
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = tile_prefix[gridDim.x];
}

template <class T>
static void exclusive_scan_impl(const T* in, T* out, int64_t n, cudaStream_t s) {
    // out has n+1 entries; out[n] = total
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles < 1) tiles = 1;
    Temp<T> sums(tiles + 1, s);
    scan_tiles<T><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(in, out, n, sums.get());
    CK_LAUNCH();
    // exclusive scan of tile sums (recursive), written in place, with total at [tiles]
    if (tiles == 1) {
        Temp<T> tmp(2, s);
        scan_tiles<T><<<1, SCAN_BLOCK, 0, s>>>(sums.get(), sums.get(), 1, tmp.get());
        CK_LAUNCH();
        CK(cudaMemcpyAsync(sums.get() + 1, tmp.get(), sizeof(T), cudaMemcpyDeviceToDevice, s));
    } else {
        exclusive_scan_impl<T>(sums.get(), sums.get(), tiles, s);
    }
    scan_add<T><<<(unsigned)tiles, SCAN_BLOCK, 0, s>>>(out, n, sums.get(), out + n);
    CK_LAUNCH();
}

__global__ void check_i32_total(const int64_t* t64, int32_t* out, int* overflow) {
    int64_t t = *t64;
    if (t > 0x7fffffffLL) *overflow = 1;
    *out = (int32_t)t;
}
__global__ void widen_i32(const int32_t* in, int64_t* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}
__global__ void narrow_i64(const int64_t* in, int32_t* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) out[i] = (int32_t)in[i];
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    exclusive_scan_impl<int64_t>(in, out, n, s);
}

void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
    // scan in int64 so the total cannot wrap, then check and narrow
    Temp<int64_t> w(n + 1, s);
    widen_i32<<<grid_for(n, 256), 256, 0, s>>>(in, w.get(), n);
    CK_LAUNCH();
    exclusive_scan_impl<int64_t>(w.get(), w.get(), n, s);
    int64_t total = read1(w.get() + n, s);
    if (total > 0x7fffffffLL) fail(MGM_ERR_UNSUPPORTED, "index total exceeds int32 range");
    narrow_i64<<<grid_for(n + 1, 256), 256, 0, s>>>(w.get(), out, n);
    CK_LAUNCH();
}

// ---------------------------------------------------------------------------------------------
// small element-wise helpers
// ---------------------------------------------------------------------------------------------
__global__ void fill_k(int32_t* p, int32_t v, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void iota_k(int32_t* p, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = (int32_t)i;
}
__global__ void invert_k(const int32_t* perm, int32_t* inv, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) inv[perm[i]] = (int32_t)i;
}
__global__ void gather_xyz_k(const double* in, const int32_t* idx, double* out, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int64_t j = idx[i];
        out[3 * i] = in[3 * j];
        out[3 * i + 1] = in[3 * j + 1];
        out[3 * i + 2] = in[3 * j + 2];
    }
}
void fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    fill_k<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
    CK_LAUNCH();
}
void iota_i32(int32_t* p, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    iota_k<<<grid_for(n, 256), 256, 0, s>>>(p, n);
    CK_LAUNCH();
}
void invert_perm(const int32_t* perm, int32_t* inv, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    invert_k<<<grid_for(n, 256), 256, 0, s>>>(perm, inv, n);
    CK_LAUNCH();
}
void gather_xyz(const double* in, const int32_t* idx, double* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    gather_xyz_k<<<grid_for(n, 256), 256, 0, s>>>(in, idx, out, n);
    CK_LAUNCH();
}

int64_t csr_nnz(const int32_t* rp, int64_t nrows, cudaStream_t s) { return (int64_t)read1(rp + nrows, s); }

// ---------------------------------------------------------------------------------------------
// validation of caller-supplied index data (so that bad input is an error, not a bad access)
// ---------------------------------------------------------------------------------------------
__global__ void check_rowptr_k(const int32_t* rp, int64_t n, int* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && rp[0] != 0) atomicOr(err, 1);
    if (i < n && rp[i + 1] < rp[i]) atomicOr(err, 1);
}
__global__ void check_range_k(const int32_t* a, int64_t cnt, int64_t hi, int* err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt && (a[i] < 0 || (int64_t)a[i] >= hi)) atomicOr(err, 2);
}
void validate_index(const int32_t* a, int64_t cnt, int64_t hi, const char* what, cudaStream_t s) {
    if (cnt <= 0) return;
    Temp<int> err(1, s);
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    check_range_k<<<grid_for(cnt, 256), 256, 0, s>>>(a, cnt, hi, err.get());
    CK_LAUNCH();
    if (read1(err.get(), s)) fail(MGM_ERR_INVALID_ARG, std::string(what) + ": index out of range");
}
void validate_csr(int64_t nrows, int64_t ncols, const int32_t* rp, const int32_t* ci, const char* what, cudaStream_t s) {
    Temp<int> err(1, s);
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    check_rowptr_k<<<grid_for(nrows + 1, 256), 256, 0, s>>>(rp, nrows, err.get());
    CK_LAUNCH();
    if (read1(err.get(), s)) fail(MGM_ERR_INVALID_ARG, std::string(what) + ": row pointers must start at 0 and not decrease");
    validate_index(ci, csr_nnz(rp, nrows, s), ncols, what, s);
}

// ---------------------------------------------------------------------------------------------
// CSR transpose: count per column, scan, place with atomics, then sort each row by source row
// ---------------------------------------------------------------------------------------------
__global__ void count_cols_k(const int32_t* rp, const int32_t* ci, int64_t nrows, int32_t* cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) atomicAdd(&cnt[ci[p]], 1);
}
__global__ void place_t_k(const int32_t* rp, const int32_t* ci, const double* v, int64_t nrows, const int32_t* trp,
                          int32_t* fill, int32_t* tci, double* tv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p) {
        int32_t c = ci[p];
        int32_t q = trp[c] + atomicAdd(&fill[c], 1);
        tci[q] = (int32_t)i;
        if (v) tv[q] = v[p];
    }
}
// sort each row's (col, val) by col: warp per row, rank placement through shared memory for
// rows of up to 256 entries (columns within a row are distinct), insertion sort beyond
constexpr int SR_WARPS = 8, SR_MAX = 256;
__global__ void __launch_bounds__(SR_WARPS * 32) sort_rows_k(const int32_t* rp, int32_t* ci, double* v, int64_t nrows) {
    __shared__ int32_t sc[SR_WARPS][SR_MAX];
    __shared__ double sv[SR_WARPS][SR_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * SR_WARPS + w;
    if (i >= nrows) return;
    const int32_t b = rp[i], e = rp[i + 1], len = e - b;
    if (len <= SR_MAX) {
        for (int32_t t = lane; t < len; t += 32) {
            sc[w][t] = ci[b + t];
            if (v) sv[w][t] = v[b + t];
        }
        __syncwarp();
        for (int32_t t = lane; t < len; t += 32) {
            const int32_t c = sc[w][t];
            int rank = 0;
            for (int32_t q = 0; q < len; ++q) rank += sc[w][q] < c ? 1 : 0;
            ci[b + rank] = c;
            if (v) v[b + rank] = sv[w][t];
        }
    } else if (lane == 0) {
        for (int32_t p = b + 1; p < e; ++p) {
            int32_t c = ci[p];
            double x = v ? v[p] : 0.0;
            int32_t q = p;
            while (q > b && ci[q - 1] > c) {
                ci[q] = ci[q - 1];
                if (v) v[q] = v[q - 1];
                --q;
            }
            ci[q] = c;
            if (v) v[q] = x;
        }
    }
}

void csr_transpose(int64_t nrows, int64_t ncols, const int32_t* rp, const int32_t* ci, const double* v,
                   int32_t* trp, int32_t* tci, double* tv, cudaStream_t s) {
    Temp<int32_t> cnt(ncols + 1, s);
    CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * (ncols + 1), s));
    if (nrows > 0) {
        count_cols_k<<<grid_for(nrows, 256), 256, 0, s>>>(rp, ci, nrows, cnt.get());
        CK_LAUNCH();
    }
    exclusive_scan_i32(cnt.get(), trp, ncols, s);
    CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * (ncols + 1), s));
    if (nrows > 0) {
        place_t_k<<<grid_for(nrows, 256), 256, 0, s>>>(rp, ci, v, nrows, trp, cnt.get(), tci, tv);
        CK_LAUNCH();
    }
    if (ncols > 0) {
        sort_rows_k<<<grid_for(ncols, SR_WARPS), SR_WARPS * 32, 0, s>>>(trp, tci, tv, ncols);
        CK_LAUNCH();
    }
}

// ---------------------------------------------------------------------------------------------
// B = A[perm][:, perm]
// ---------------------------------------------------------------------------------------------
__global__ void perm_rowlen_k(const int32_t* rp, const int32_t* perm, int64_t N, int32_t* len) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        int32_t o = perm[i];
        len[i] = rp[o + 1] - rp[o];
    }
}
// one warp per row: lanes over the source row's entries, so loads and stores coalesce and the
// renumbering gathers of a row are in flight together
constexpr int PF_WARPS = 8;
__global__ void __launch_bounds__(PF_WARPS * 32) perm_fill_k(const int32_t* rp, const int32_t* ci, const double* v,
                                                             const int32_t* perm, const int32_t* inv, int64_t N,
                                                             const int32_t* brp, int32_t* bci, double* bv) {
    const int64_t i = (int64_t)blockIdx.x * PF_WARPS + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    const int32_t o = perm[i];
    const int32_t b = rp[o], e = rp[o + 1], q = brp[i] - b;
    for (int32_t p = b + lane; p < e; p += 32) {
        bci[q + p] = inv[ci[p]];
        if (bv) bv[q + p] = v[p];
    }
}
void csr_permute(int64_t N, const int32_t* rp, const int32_t* ci, const double* v, const int32_t* perm,
                 int32_t* brp, int32_t* bci, double* bv, cudaStream_t s) {
    if (N <= 0) return;
    Temp<int32_t> len(N + 1, s), inv(N, s);
    perm_rowlen_k<<<grid_for(N, 256), 256, 0, s>>>(rp, perm, N, len.get());
    CK_LAUNCH();
    exclusive_scan_i32(len.get(), brp, N, s);
    invert_perm(perm, inv.get(), N, s);
    perm_fill_k<<<grid_for(N, PF_WARPS), PF_WARPS * 32, 0, s>>>(rp, ci, v, perm, inv.get(), N, brp, bci, bv);
    CK_LAUNCH();
    sort_rows_k<<<grid_for(N, SR_WARPS), SR_WARPS * 32, 0, s>>>(brp, bci, bv, N);
    CK_LAUNCH();
}

// ---------------------------------------------------------------------------------------------
// symmetrised pattern: union of row i of A and row i of A^T, diagonal dropped
// ---------------------------------------------------------------------------------------------
// One warp per row. Both sorted rows (of A and of A^T) are staged in shared memory; each entry
// finds its place in the merged sequence by a binary search in the other row (an entry of A
// before an equal entry of A^T), and a ballot scan compacts, in order, the entries that are
// neither the diagonal nor equal to the entry before them. Rows longer than UR_MAX are merged by
// one lane.
constexpr int UR_WARPS = 8, UR_MAX = 256;
__device__ __forceinline__ int lower_bound_i32(const int32_t* a, int n, int32_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}
template <bool WRITE>
__global__ void __launch_bounds__(UR_WARPS * 32) union_rows_k(const int32_t* rp, const int32_t* ci, const int32_t* trp,
                                                              const int32_t* tci, int64_t N, int32_t* cnt,
                                                              const int32_t* orp, int32_t* oci) {
    __shared__ int32_t sa[UR_WARPS][UR_MAX], st[UR_WARPS][UR_MAX], sm[UR_WARPS][2 * UR_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * UR_WARPS + w;
    if (i >= N) return;
    const int32_t a = rp[i], ae = rp[i + 1], b = trp[i], be = trp[i + 1];
    const int la = ae - a, lt = be - b;
    const int32_t q = WRITE ? orp[i] : 0;
    if (la > UR_MAX || lt > UR_MAX) {
        if (lane == 0) {
            int32_t c = 0, last = -1, x;
            for (int32_t p = a, r = b; p < ae || r < be;) {
                if (r >= be || (p < ae && ci[p] <= tci[r])) x = ci[p++];
                else x = tci[r++];
                if (x == i || x == last) continue;
                last = x;
                if (WRITE) oci[q + c] = x;
                ++c;
            }
            if (!WRITE) cnt[i] = c;
        }
        return;
    }
    for (int t = lane; t < la; t += 32) sa[w][t] = ci[a + t];
    for (int t = lane; t < lt; t += 32) st[w][t] = tci[b + t];
    __syncwarp();
    // the merged sequence, duplicates included (equal values end up next to each other)
    for (int t = lane; t < la; t += 32) {
        const int32_t x = sa[w][t];
        sm[w][t + lower_bound_i32(st[w], lt, x)] = x;
    }
    for (int t = lane; t < lt; t += 32) {
        const int32_t y = st[w][t];
        sm[w][t + lower_bound_i32(sa[w], la, y + 1)] = y;  // after the entries of A <= y
    }
    __syncwarp();
    // kept: not the diagonal, and not equal to the entry before it
    int32_t c = 0;
    for (int t0 = 0; t0 < la + lt; t0 += 32) {
        const int t = t0 + lane;
        const int32_t x = t < la + lt ? sm[w][t] : -1;
        const bool keep = t < la + lt && x != (int32_t)i && (t == 0 || sm[w][t - 1] != x);
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (WRITE && keep) oci[q + c + __popc(m & ((1u << lane) - 1u))] = x;
        c += __popc(m);
    }
    if (!WRITE && lane == 0) cnt[i] = c;
}
void sym_pattern(int64_t N, const int32_t* rp, const int32_t* ci, Temp<int32_t>& srp, Temp<int32_t>& sci,
                 cudaStream_t s) {
    int64_t nnz = csr_nnz(rp, N, s);
    Temp<int32_t> trp(N + 1, s), tci(nnz > 0 ? nnz : 1, s);
    csr_transpose(N, N, rp, ci, nullptr, trp.get(), tci.get(), nullptr, s);
    Temp<int32_t> cnt(N + 1, s);
    srp.alloc(N + 1, s);
    if (N > 0) {
        union_rows_k<false><<<grid_for(N, UR_WARPS), UR_WARPS * 32, 0, s>>>(rp, ci, trp.get(), tci.get(), N, cnt.get(),
                                                                           nullptr, nullptr);
        CK_LAUNCH();
    }
    exclusive_scan_i32(cnt.get(), srp.get(), N, s);
    int64_t snnz = csr_nnz(srp.get(), N, s);
    sci.alloc(snnz > 0 ? snnz : 1, s);
    if (N > 0) {
        union_rows_k<true><<<grid_for(N, UR_WARPS), UR_WARPS * 32, 0, s>>>(rp, ci, trp.get(), tci.get(), N, nullptr,
                                                                          srp.get(), sci.get());
        CK_LAUNCH();
    }
}

// Set-up tracing: with MGM_TRACE set in the environment, synchronise `s` and print the wall time
// since the calling thread's previous mark (off by default; no effect on results).
bool trace_on() {
    static const bool on = std::getenv("MGM_TRACE") != nullptr;
    return on;
}
void trace_mark(cudaStream_t s, const char* what, int level) {
    if (!trace_on()) return;
    static thread_local std::chrono::steady_clock::time_point last = std::chrono::steady_clock::now();
    cudaStreamSynchronize(s);
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[mgm setup] level %d %-16s %9.3f ms\n", level, what,
                 std::chrono::duration<double, std::milli>(now - last).count());
    last = now;
}

// The library's scratch pool on each device: stream-ordered allocations that are kept for reuse
// across synchronisations (the release threshold is unlimited) instead of being unmapped at every
// one, as the default pool does; heavy entry points hand the cached memory back with scratch_trim.
cudaMemPool_t scratch_pool() {
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto it = pools.find(dev);
    if (it != pools.end()) return it->second;
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.handleTypes = cudaMemHandleTypeNone;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = dev;
    cudaMemPool_t pool = nullptr;
    CK(cudaMemPoolCreate(&pool, &pp));
    uint64_t keep = ~0ull;
    CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    pools[dev] = pool;
    return pool;
}

void scratch_trim(size_t keep_bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPoolTrimTo(scratch_pool(), keep_bytes);
}

namespace {
struct BufCache {
    std::mutex mu;
    std::unordered_map<void*, std::pair<int, size_t>> live;      // block -> (device, bytes)
    std::map<int, std::multimap<size_t, void*>> free_blocks;      // device -> (bytes, block)
};
BufCache& buf_cache() {
    static BufCache* c = new BufCache();  // (never destroyed: buffers may be released at exit)
    return *c;
}
thread_local int g_cache_scope = 0;
}  // namespace

BufCacheScope::BufCacheScope() { ++g_cache_scope; }
BufCacheScope::~BufCacheScope() { --g_cache_scope; }

void* buf_alloc(size_t bytes) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    BufCache& c = buf_cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto& fb = c.free_blocks[dev];
        auto it = fb.lower_bound(bytes);
        if (it != fb.end() && it->first <= 2 * bytes) {
            void* p = it->second;
            c.live[p] = {dev, it->first};
            fb.erase(it);
            return p;
        }
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        release_cached_memory();
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            fail(MGM_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        }
    }
    std::lock_guard<std::mutex> lk(c.mu);
    c.live[p] = {dev, bytes};
    return p;
}

void buf_free(void* p) {
    BufCache& c = buf_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.live.find(p);
    if (it == c.live.end()) return;
    const int dev = it->second.first;
    const size_t bytes = it->second.second;
    c.live.erase(it);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) cur = -1;
    if (g_cache_scope > 0 && dev == cur) {  // (the scope's synchronisation covered this device only)
        c.free_blocks[dev].emplace(bytes, p);
    } else {
        cudaFree(p);
    }
}

void* host_stage() {
    thread_local void* p = nullptr;
    thread_local bool tried = false;
    if (!tried) {
        tried = true;
        if (cudaMallocHost(&p, HOST_STAGE_BYTES) != cudaSuccess) {
            (void)cudaGetLastError();
            p = nullptr;
        }
    }
    return p;
}

// Memory the caches may keep on a device between calls: 1/32 of its memory (8.9 GB on a GB300).
size_t cache_budget() {
    static std::mutex mu;
    static std::map<int, size_t> budget;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(mu);
    auto it = budget.find(dev);
    if (it != budget.end()) return it->second;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        (void)cudaGetLastError();
        tot = 0;
    }
    return budget[dev] = tot / 32;
}

void buf_cache_trim(size_t keep_bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    BufCache& c = buf_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto& fb = c.free_blocks[dev];
    size_t total = 0;
    for (auto& b : fb) total += b.first;
    while (total > keep_bytes && !fb.empty()) {  // largest blocks first
        auto it = std::prev(fb.end());
        total -= it->first;
        cudaFree(it->second);
        fb.erase(it);
    }
}

void release_cached_memory() {
    cudaDeviceSynchronize();
    scratch_trim(0);
    buf_cache_flush();
}

void buf_cache_flush() {
    BufCache& c = buf_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.free_blocks.empty()) return;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) cur = 0;
    for (auto& d : c.free_blocks) {
        if (d.second.empty()) continue;
        cudaSetDevice(d.first);
        cudaDeviceSynchronize();
        for (auto& b : d.second) cudaFree(b.second);
        d.second.clear();
    }
    cudaSetDevice(cur);
}

int coresident_blocks(const void* kernel, int threads, size_t smem, int per_sm_cap) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, size_t, int>, int> cache;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const auto key = std::make_tuple(kernel, dev, threads, smem, per_sm_cap);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int per_sm = 0, sms = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) fail(MGM_ERR_UNSUPPORTED, "a cooperative kernel cannot be resident on this device");
    if (per_sm_cap > 0) per_sm = std::min(per_sm, per_sm_cap);
    const int nb = per_sm * sms;
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = nb;
    return nb;
}

}  // namespace mgm

// Orderings of a level operator: reverse Cuthill-McKee (paper Sec. 4.2; Alg. 2)
// and the multicolouring used by the multicolour Gauss-Seidel smoother.
//
// RCM on the GPU: a level-synchronous breadth-first search that reproduces the sequential
// Cuthill-McKee order exactly. Within a level, a frontier node v (in CM order) appends its
// unvisited neighbours in increasing (degree, index); a node adjacent to several frontier nodes
// is appended by the first of them. So each unvisited neighbour takes the minimum CM position
// of its frontier neighbours (atomicMin), the children are counted by owner, a scan gives
// offsets, and each frontier node writes its children in its (degree, index) order.
//
// Colouring: Jones-Plassmann rounds. An uncoloured vertex whose (SplitMix64(seed, i), i) priority
// exceeds that of all uncoloured neighbours takes the smallest colour absent from its coloured
// neighbours. Such vertices are never adjacent, and the result equals sequential first-fit
// colouring in decreasing priority. That equality lets one launch compute it directly along the
// sorted priority order (jp_ordered_k, below); the rounds remain as its fallback.
#include <algorithm>
#include <climits>
#include <cstdlib>

#include "common.cuh"

namespace mgm {

// sort each row of the symmetrised adjacency by (degree, index): warp per row; the (degree,
// index) keys of a row (up to 256) are staged in shared memory and placed by rank
constexpr int SBD_WARPS = 8, SBD_MAX = 256;
__global__ void __launch_bounds__(SBD_WARPS * 32) sort_by_degree_k(const int32_t* rp, const int32_t* ci, int64_t N,
                                                                    int32_t* out) {
    __shared__ unsigned long long keys[SBD_WARPS][SBD_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * SBD_WARPS + w;
    if (row >= N) return;
    const int32_t b = rp[row], e = rp[row + 1], len = e - b;
    auto key = [&](int32_t u) { return ((unsigned long long)(uint32_t)(rp[u + 1] - rp[u]) << 32) | (uint32_t)u; };
    if (len <= SBD_MAX) {
        for (int32_t t = lane; t < len; t += 32) keys[w][t] = key(ci[b + t]);
        __syncwarp();
        for (int32_t t = lane; t < len; t += 32) {
            const unsigned long long k = keys[w][t];
            int rank = 0;
            for (int32_t q = 0; q < len; ++q) rank += keys[w][q] < k ? 1 : 0;
            out[b + rank] = (int32_t)(k & 0xffffffffull);
        }
    } else {
        for (int32_t p = b + lane; p < e; p += 32) {
            const unsigned long long k = key(ci[p]);
            int rank = 0;
            for (int32_t q = b; q < e; ++q) rank += key(ci[q]) < k ? 1 : 0;
            out[b + rank] = (int32_t)(k & 0xffffffffull);
        }
    }
}

// Device-resident BFS state: the host enqueues levels without reading anything back and checks
// for completion only every RCM_BATCH levels; kernels of an exhausted search return at once.
// A level is three launches: claim (frontier nodes claim their unvisited neighbours; a node's first
// claim lists it as touched), scan (one block: children counted from the touched list, offsets,
// the next frontier; when that is empty and nodes remain, the next component's start), write.
struct RcmState {
    int32_t fs, fe, tail;     // current frontier [fs, fe) in `order`, next free slot
    int32_t wfs, wfe, wtail;  // the frontier and first slot of the level being written
    int32_t ntouched;         // nodes first claimed at this level (listed in `touched`)
};
constexpr int RCM_BATCH = 16;
constexpr int RCM_SCAN_SMEM = 11264;  // frontier counts kept in the scan block's shared memory (44 KB)
constexpr int RCM_GRID = 152 * 8;  // blocks of 128 threads: 4 frontier nodes a block at a time

// claim: one warp per frontier node, lanes over its (degree, index)-sorted neighbours, so the
// dependent loads of a node's neighbours overlap instead of forming one long chain per thread
__global__ void rcm_claim_k(const int32_t* rp, const int32_t* adj, const int32_t* order, const int32_t* pos,
                            RcmState* st, int32_t* claim, int32_t* touched) {
    pdl_trigger();
    pdl_wait();
    const int32_t fs = st->fs, fe = st->fe;
    const int lane = threadIdx.x & 31;
    const int32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (int32_t t = fs + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < fe; t += nw) {
        const int32_t v = order[t];
        for (int32_t p0 = rp[v]; p0 < rp[v + 1]; p0 += 32) {
            const int32_t p = p0 + lane;
            int32_t u = -1;
            bool first = false;
            if (p < rp[v + 1]) {
                u = adj[p];
                if (pos[u] < 0) first = atomicMin(&claim[u], t) == INT_MAX;
            }
            const unsigned m = __ballot_sync(0xffffffffu, first);
            if (m) {
                int32_t at = 0;
                if (lane == __ffs(m) - 1) at = atomicAdd(&st->ntouched, __popc(m));
                at = __shfl_sync(0xffffffffu, at, __ffs(m) - 1);
                if (first) touched[at + __popc(m & ((1u << lane) - 1u))] = u;
            }
        }
    }
}

// one block: each touched node counts for the frontier node that claimed it; exclusive scan of
// the counts (chunk sums, then a two-level shuffle scan of the 1024 chunk sums); the next
// frontier; if it is empty and nodes remain, the unvisited node of least (degree, index) starts
// the next component (the first level of the search only does this)
__global__ void __launch_bounds__(1024) rcm_scan_k(const int32_t* rp, const int32_t* claim, const int32_t* touched,
                                                   int32_t* cnt, int32_t* off, int32_t* order, int32_t* pos, int64_t N,
                                                   RcmState* st) {
    pdl_trigger();
    pdl_wait();
    __shared__ int32_t wsum[32];
    __shared__ unsigned long long wbest[32];
    __shared__ int32_t scnt[RCM_SCAN_SMEM];
    const int32_t fs = st->fs, fe = st->fe, tail = st->tail, nt = st->ntouched;
    const int32_t n = fe - fs;
    if (n <= RCM_SCAN_SMEM) cnt = scnt;  // (block-uniform) the counts of a frontier that fits stay on chip
    for (int32_t i = threadIdx.x; i < n; i += 1024) cnt[i] = 0;
    __syncthreads();
    for (int32_t i = threadIdx.x; i < nt; i += 1024) atomicAdd(&cnt[claim[touched[i]] - fs], 1);
    __syncthreads();
    const int32_t per = (n + 1023) / 1024;
    const int32_t b = threadIdx.x * per, e = min(n, b + per);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t sum = 0;
    for (int32_t i = b; i < e; ++i) sum += cnt[i];
    int32_t x = sum;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t t = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const int32_t total = wsum[31];
    int32_t acc = (w > 0 ? wsum[w - 1] : 0) + x - sum;
    for (int32_t i = b; i < e; ++i) { off[i] = acc; acc += cnt[i]; }
    if (threadIdx.x == 0) {
        st->wfs = fs;
        st->wfe = fe;
        st->wtail = tail;
        st->fs = tail;
        st->fe = tail + total;
        st->tail = tail + total;
        st->ntouched = 0;
    }
    if (total > 0 || tail >= N) return;  // (block-uniform)
    unsigned long long best = ~0ull;
    for (int64_t i = threadIdx.x; i < N; i += 1024)
        if (pos[i] < 0) best = min(best, ((unsigned long long)(uint32_t)(rp[i + 1] - rp[i]) << 32) | (uint32_t)i);
    for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) wbest[w] = best;
    __syncthreads();
    if (w == 0) {
        best = wbest[lane];
        for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) {
            const int32_t s0 = (int32_t)(best & 0xffffffffull);
            order[tail] = s0;
            pos[s0] = tail;
            st->fs = tail;
            st->fe = tail + 1;
            st->tail = tail + 1;
        }
    }
}

__global__ void rcm_write_k(const int32_t* rp, const int32_t* adj, int32_t* order, int32_t* pos, const int32_t* claim,
                            const int32_t* off, const RcmState* st) {
    pdl_trigger();
    pdl_wait();
    const int32_t fs = st->wfs, fe = st->wfe, tail = st->wtail;
    const int lane = threadIdx.x & 31;
    const int32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (int32_t t = fs + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < fe; t += nw) {
        const int32_t v = order[t];
        int32_t q = tail + off[t - fs];
        for (int32_t p0 = rp[v]; p0 < rp[v + 1]; p0 += 32) {
            const int32_t p = p0 + lane;
            int32_t u = -1;
            bool mine = false;
            if (p < rp[v + 1]) {
                u = adj[p];
                mine = pos[u] < 0 && claim[u] == t;
            }
            const unsigned m = __ballot_sync(0xffffffffu, mine);
            if (mine) {
                const int32_t qq = q + __popc(m & ((1u << lane) - 1u));
                order[qq] = u;
                pos[u] = qq;
            }
            q += __popc(m);
        }
    }
}

__global__ void reverse_k(const int32_t* order, int64_t N, int32_t* perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) perm[i] = order[N - 1 - i];
}

void rcm(int64_t N, const int32_t* rp, const int32_t* ci, int32_t* perm, cudaStream_t s, Temp<int32_t>* keep_rp,
         Temp<int32_t>* keep_ci) {
    REQUIRE(N >= 1 && N < 0x7fffffff, "N out of range");
    REQUIRE(rp && ci && perm, "null array");
    Temp<int32_t> srp, sci;
    sym_pattern(N, rp, ci, srp, sci, s);
    int64_t snnz = csr_nnz(srp.get(), N, s);
    Temp<int32_t> adj(snnz > 0 ? snnz : 1, s);
    sort_by_degree_k<<<grid_for(N, SBD_WARPS), SBD_WARPS * 32, 0, s>>>(srp.get(), sci.get(), N, adj.get());
    CK_LAUNCH();
    trace_mark(s, "  rcm:pattern");
    Temp<int32_t> order(N, s), pos(N, s), claim(N, s), cnt(N + 1, s), off(N + 1, s), touched(N, s);
    fill_i32(pos.get(), -1, N, s);
    fill_i32(claim.get(), INT_MAX, N, s);
    Temp<RcmState> st(1, s);
    RcmState init{0, 0, 0, 0, 0, 0, 0};  // empty frontier: the first level's scan seeds the search
    CK(cudaMemcpyAsync(st.get(), &init, sizeof(RcmState), cudaMemcpyHostToDevice, s));
    const unsigned grid = (unsigned)std::min<int64_t>(grid_for(N, 4), RCM_GRID);
    // one BFS level: three kernels chained by programmatic dependent launch
    auto level = [&](cudaStream_t q) {
        launch_pdl(rcm_claim_k, grid, 128, q, (const int32_t*)srp.get(), (const int32_t*)adj.get(),
                   (const int32_t*)order.get(), (const int32_t*)pos.get(), st.get(), claim.get(), touched.get());
        launch_pdl(rcm_scan_k, 1, 1024, q, (const int32_t*)srp.get(), (const int32_t*)claim.get(),
                   (const int32_t*)touched.get(), cnt.get(), off.get(), order.get(), pos.get(), N, st.get());
        launch_pdl(rcm_write_k, grid, 128, q, (const int32_t*)srp.get(), (const int32_t*)adj.get(), order.get(),
                   pos.get(), (const int32_t*)claim.get(), (const int32_t*)off.get(), (const RcmState*)st.get());
    };
    // Large graphs: RCM_BATCH levels captured once as a CUDA graph and replayed (levels after the
    // last are no-ops); the host reads the state between replays.
    GraphBatch gb;
    if (N >= 32768) gb.capture([&](cudaStream_t q) { for (int l = 0; l < RCM_BATCH; ++l) level(q); });
    for (int64_t lv = 0;; lv += RCM_BATCH) {
        RcmState h;
        to_host(&h, st.get(), 1, s);
        if (h.tail >= N && h.fs == h.fe) break;
        if (lv > 4 * N + 64) fail(MGM_ERR_UNSUPPORTED, "RCM did not terminate");
        if (gb.exec) gb.launch(s);
        else
            for (int l = 0; l < RCM_BATCH; ++l) level(s);
    }
    trace_mark(s, "  rcm:bfs");
    reverse_k<<<grid_for(N, 256), 256, 0, s>>>(order.get(), N, perm);
    CK_LAUNCH();
    if (keep_rp && keep_ci) {  // the symmetric pattern, for the colouring of the permuted operator
        *keep_rp = std::move(srp);
        *keep_ci = std::move(sci);
    }
}

void rcm(int64_t N, const int32_t* rp, const int32_t* ci, int32_t* perm, cudaStream_t s) {
    rcm(N, rp, ci, perm, s, nullptr, nullptr);
}

// the symmetric pattern (srp, sci) of an operator, renumbered by perm (perm[new] = old, inv its
// inverse): row r of the result is row perm[r] with its columns mapped by inv (order within a row
// kept; the colouring treats a row as a set)
__global__ void perm_len_k(const int32_t* srp, const int32_t* perm, int64_t N, int32_t* len) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < N) len[r] = srp[perm[r] + 1] - srp[perm[r]];
}
__global__ void perm_fill_pattern_k(const int32_t* srp, const int32_t* sci, const int32_t* perm, const int32_t* inv,
                                    const int32_t* nrp, int64_t N, int32_t* nci) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = t >> 5;
    if (r >= N) return;
    const int32_t b = srp[perm[r]], e = srp[perm[r] + 1], o = nrp[r];
    for (int32_t q = b + (int32_t)(t & 31); q < e; q += 32) nci[o + (q - b)] = inv[sci[q]];
}
void permute_pattern(int64_t N, const int32_t* srp, const int32_t* sci, const int32_t* perm, Temp<int32_t>& nrp,
                     Temp<int32_t>& nci, cudaStream_t s) {
    Temp<int32_t> inv(N, s), len(N + 1, s);
    invert_perm(perm, inv.get(), N, s);
    perm_len_k<<<grid_for(N, 256), 256, 0, s>>>(srp, perm, N, len.get());
    CK_LAUNCH();
    nrp.alloc(N + 1, s);
    exclusive_scan_i32(len.get(), nrp.get(), N, s);
    const int64_t nnz = csr_nnz(nrp.get(), N, s);
    nci.alloc(nnz > 0 ? nnz : 1, s);
    perm_fill_pattern_k<<<grid_for(N * 32, 256), 256, 0, s>>>(srp, sci, perm, inv.get(), nrp.get(), N, nci.get());
    CK_LAUNCH();
}

// ---------------------------------------------------------------------------------------------
// colouring
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// One thread per vertex; coloured vertices return at once. Neighbours are examined eight at a
// time (indices, then their colours, then priorities) so that the dependent loads of a vertex
// overlap. `left` is set (not counted) while uncoloured vertices remain.
constexpr int JP_BATCH = 8;
__global__ void jp_select_k(const int32_t* rp, const int32_t* adj, const int32_t* col, int64_t N, unsigned long long seed,
                            char* sel, int* left) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    if (col[v] >= 0) {
        sel[v] = 0;
        return;
    }
    const unsigned am = __activemask();  // the uncoloured vertices of this warp
    if ((threadIdx.x & 31) == __ffs(am) - 1) *left = 1;
    const unsigned long long pv = splitmix64(seed, (unsigned long long)v);
    const int32_t e = rp[v + 1];
    bool top = true;
    for (int32_t p = rp[v]; p < e && top; p += JP_BATCH) {
        int32_t u[JP_BATCH];
        int32_t cu[JP_BATCH];
#pragma unroll
        for (int q = 0; q < JP_BATCH; ++q) u[q] = p + q < e ? adj[p + q] : -1;
#pragma unroll
        for (int q = 0; q < JP_BATCH; ++q) cu[q] = u[q] >= 0 ? col[u[q]] : 0;
#pragma unroll
        for (int q = 0; q < JP_BATCH; ++q) {
            if (u[q] >= 0 && cu[q] < 0) {
                const unsigned long long pu = splitmix64(seed, (unsigned long long)u[q]);
                if (!(pv > pu || (pv == pu && v > u[q]))) top = false;
            }
        }
    }
    sel[v] = top ? 1 : 0;
}

// smallest colour absent from the coloured neighbours, 64 candidate colours at a time
__global__ void jp_assign_k(const int32_t* rp, const int32_t* adj, int32_t* col, const char* sel, int64_t N) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N || !sel[v]) return;
    const int32_t b = rp[v], e = rp[v + 1];
    for (int base = 0;; base += 64) {
        unsigned long long used = 0;
        for (int32_t p = b; p < e; p += JP_BATCH) {
            int32_t c[JP_BATCH];
#pragma unroll
            for (int q = 0; q < JP_BATCH; ++q) c[q] = p + q < e ? adj[p + q] : -1;
#pragma unroll
            for (int q = 0; q < JP_BATCH; ++q) c[q] = c[q] >= 0 ? col[c[q]] : -1;
#pragma unroll
            for (int q = 0; q < JP_BATCH; ++q)
                if (c[q] >= base && c[q] < base + 64) used |= 1ull << (c[q] - base);
        }
        if (~used) {
            col[v] = base + __ffsll((long long)~used) - 1;
            return;
        }
    }
}

// ---- greedy colouring in one launch --------------------------------------------------------
// A JP round gives a selected vertex the smallest colour absent from its coloured neighbours, and
// those are exactly its neighbours of higher (priority, index): it is selected only once all of
// them are coloured, and none of its lower neighbours can be coloured before it. The colouring is
// therefore the evaluation of "smallest colour absent from the higher neighbours" in decreasing
// priority, and every schedule that respects that order gives the same colours. Vertices are
// sorted by decreasing (priority, index); blocks take consecutive slices of that order in the
// order they start (a ticket counter), so a vertex waits only for vertices of blocks that have
// started or of its own block, and every wait ends. Each wait is bounded all the same: past the
// limit the kernel records MGM_ERR_TIMEOUT, the other threads stop waiting, and the host colours
// by JP rounds instead.
__device__ __forceinline__ bool prio_gt(unsigned long long pu, int32_t u, unsigned long long pv, int32_t v) {
    return pu > pv || (pu == pv && u > v);
}
__device__ __forceinline__ int ld_relaxed_i32(const int32_t* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_i32(int32_t* p, int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// bucket of a vertex: the top B bits of its priority, reversed so that ascending buckets hold
// decreasing priorities
__device__ __forceinline__ int prio_bucket(unsigned long long pv, int B) {
    return (int)(((1ull << B) - 1ull) - (pv >> (64 - B)));
}
__global__ void prio_count_k(int64_t N, unsigned long long seed, int B, int32_t* cnt) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < N) atomicAdd(&cnt[prio_bucket(splitmix64(seed, (unsigned long long)v), B)], 1);
}
__global__ void prio_fill_k(int64_t N, unsigned long long seed, int B, const int32_t* start, int32_t* fill,
                            int32_t* ord) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    const int b = prio_bucket(splitmix64(seed, (unsigned long long)v), B);
    ord[start[b] + atomicAdd(&fill[b], 1)] = (int32_t)v;
}
// each bucket in decreasing (priority, index): insertion sort, one thread per bucket
__global__ void prio_sort_k(int64_t nb, unsigned long long seed, const int32_t* start, int32_t* ord) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int32_t* o = ord + start[b];
    const int n = start[b + 1] - start[b];
    for (int i = 1; i < n; ++i) {
        const int32_t x = o[i];
        const unsigned long long px = splitmix64(seed, (unsigned long long)x);
        int j = i;
        while (j > 0 && prio_gt(px, x, splitmix64(seed, (unsigned long long)o[j - 1]), o[j - 1])) {
            o[j] = o[j - 1];
            --j;
        }
        o[j] = x;
    }
}

__global__ void __launch_bounds__(256) jp_ordered_k(const int32_t* rp, const int32_t* adj, const int32_t* ord, int64_t N,
                                                    unsigned long long seed, unsigned* ticket, int32_t* col, int* err,
                                                    unsigned long long limit) {
    __shared__ unsigned slice;
    if (threadIdx.x == 0) slice = atomicAdd(ticket, 1u);
    __syncthreads();
    const int64_t t = (int64_t)slice * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int32_t v = ord[t];
    const unsigned long long pv = splitmix64(seed, (unsigned long long)v);
    const int32_t b = rp[v], e = rp[v + 1];
    unsigned long long used = 0;
    bool more = false;  // a higher neighbour has a colour >= 64
    for (int32_t p = b; p < e; p += JP_BATCH) {
        int32_t u[JP_BATCH];
        int c[JP_BATCH];
#pragma unroll
        for (int q = 0; q < JP_BATCH; ++q) u[q] = p + q < e ? adj[p + q] : -1;
#pragma unroll
        for (int q = 0; q < JP_BATCH; ++q)
            if (u[q] >= 0 && !prio_gt(splitmix64(seed, (unsigned long long)u[q]), u[q], pv, v)) u[q] = -1;
#pragma unroll
        for (int q = 0; q < JP_BATCH; ++q) c[q] = u[q] >= 0 ? ld_relaxed_i32(col + u[q]) : 0;
#pragma unroll
        for (int q = 0; q < JP_BATCH; ++q) {
            if (u[q] < 0) continue;
            for (unsigned long long it = 0; c[q] < 0; ++it) {
                if (*(volatile int*)err) return;
                if (it >= limit) {
                    atomicOr(err, MGM_ERR_TIMEOUT);
                    return;
                }
                __nanosleep(64);
                c[q] = ld_relaxed_i32(col + u[q]);
            }
            if (c[q] < 64) used |= 1ull << c[q];
            else more = true;
        }
    }
    int colour = ~used ? __ffsll((long long)~used) - 1 : -1;
    // all 64 lowest colours taken: the next windows (every higher neighbour is coloured by now)
    for (int base = 64; colour < 0 && more; base += 64) {
        unsigned long long w = 0;
        for (int32_t p = b; p < e; ++p) {
            const int32_t u = adj[p];
            if (!prio_gt(splitmix64(seed, (unsigned long long)u), u, pv, v)) continue;
            const int c = ld_relaxed_i32(col + u);
            if (c >= base && c < base + 64) w |= 1ull << (c - base);
        }
        if (~w) colour = base + __ffsll((long long)~w) - 1;
    }
    if (colour < 0) colour = 64;  // (only when no higher neighbour has a colour >= 64)
    st_relaxed_i32(col + v, colour);
}

// Greedy colouring along the priority order in one launch; false when a wait ran out (the
// colours are then incomplete and the caller colours by rounds).
static bool color_ordered(int64_t N, const int32_t* rp, const int32_t* adj, uint64_t seed, int32_t* colour,
                          cudaStream_t s) {
    int B = 1;
    while (B < 24 && ((int64_t)1 << B) < N) ++B;
    const int64_t nb = (int64_t)1 << B;
    Temp<int32_t> cnt(nb, s), start(nb + 1, s), fill(nb, s), ord(N, s);
    Temp<unsigned> ticket(1, s);
    Temp<int> err(1, s);
    CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * nb, s));
    CK(cudaMemsetAsync(fill.get(), 0, sizeof(int32_t) * nb, s));
    CK(cudaMemsetAsync(ticket.get(), 0, sizeof(unsigned), s));
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    prio_count_k<<<grid_for(N, 256), 256, 0, s>>>(N, seed, B, cnt.get());
    CK_LAUNCH();
    exclusive_scan_i32(cnt.get(), start.get(), nb, s);
    prio_fill_k<<<grid_for(N, 256), 256, 0, s>>>(N, seed, B, start.get(), fill.get(), ord.get());
    CK_LAUNCH();
    prio_sort_k<<<grid_for(nb, 256), 256, 0, s>>>(nb, seed, start.get(), ord.get());
    CK_LAUNCH();
    fill_i32(colour, -1, N, s);
    jp_ordered_k<<<grid_for(N, 256), 256, 0, s>>>(rp, adj, ord.get(), N, seed, ticket.get(), colour, err.get(),
                                                  1ull << 22);
    CK_LAUNCH();
    return read1(err.get(), s) == 0;
}

__global__ void max_i32_k(const int32_t* a, int64_t n, int* out) {
    int m = -1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, a[i]);
    for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

void color(int64_t N, const int32_t* rp, const int32_t* ci, uint64_t seed, int32_t* colour, int32_t* ncolors,
           cudaStream_t s, const int32_t* sym_rp, const int32_t* sym_ci) {
    REQUIRE(N >= 1 && N < 0x7fffffff, "N out of range");
    REQUIRE(rp && ci && colour, "null array");
    Temp<int32_t> srp_t, sci_t;
    const int32_t* srp_p = sym_rp;  // the symmetric pattern, given or built here
    const int32_t* sci_p = sym_ci;
    if (!srp_p || !sci_p) {
        sym_pattern(N, rp, ci, srp_t, sci_t, s);
        srp_p = srp_t.get();
        sci_p = sci_t.get();
    }
    trace_mark(s, "  colour:pattern");
    Temp<int> ctr(2, s);  // [0] uncoloured vertices remain, [1] max colour
    // MGM_COLOR_ROUNDS in the environment selects the JP rounds directly (they are otherwise the
    // fallback only; the tests use it to check that both give the same colours)
    const bool ordered = !std::getenv("MGM_COLOR_ROUNDS") && color_ordered(N, srp_p, sci_p, seed, colour, s);
    Temp<char> sel(ordered ? 1 : N, s);
    if (!ordered) fill_i32(colour, -1, N, s);
    const unsigned wgrid = grid_for(N, 256);
    for (int64_t round = 0; !ordered; ++round) {
        if (round > N) fail(MGM_ERR_UNSUPPORTED, "colouring did not terminate");
        CK(cudaMemsetAsync(ctr.get(), 0, sizeof(int), s));
        jp_select_k<<<wgrid, 256, 0, s>>>(srp_p, sci_p, colour, N, seed, sel.get(), ctr.get());
        CK_LAUNCH();
        if (round % 4 == 3 || round < 2) {
            if (read1(ctr.get(), s) == 0) break;
        }
        jp_assign_k<<<wgrid, 256, 0, s>>>(srp_p, sci_p, colour, sel.get(), N);
        CK_LAUNCH();
    }
    CK(cudaMemsetAsync(ctr.get() + 1, 0xff, sizeof(int), s));
    max_i32_k<<<(unsigned)std::min<int64_t>(grid_for(N, 256), 152 * 4), 256, 0, s>>>(colour, N, ctr.get() + 1);
    CK_LAUNCH();
    *ncolors = read1(ctr.get() + 1, s) + 1;
}

void color(int64_t N, const int32_t* rp, const int32_t* ci, uint64_t seed, int32_t* colour, int32_t* ncolors,
           cudaStream_t s) {
    color(N, rp, ci, seed, colour, ncolors, s, nullptr, nullptr);
}

}  // namespace mgm

// Orderings of a level operator: reverse Cuthill-McKee (paper Sec. 4.2; Alg. 2)
// and the multicolouring used by the multicolour Gauss-Seidel smoother.
//
// RCM on the GPU: a level-synchronous breadth-first search that reproduces the sequential
// Cuthill-McKee order exactly. Within a level, a frontier node v (in CM order) appends its
// unvisited neighbours in increasing (degree, index); a node adjacent to several frontier nodes
// is appended by the first of them. So each unvisited neighbour takes the minimum CM position
// of its frontier neighbours (atomicMin), frontier nodes count the children they own, a scan
// gives offsets, and each frontier node writes its children in its (degree, index) order.
//
// Colouring: Jones-Plassmann rounds. An uncoloured vertex whose (SplitMix64(seed, i), i) priority
// exceeds that of all uncoloured neighbours takes the smallest colour absent from its coloured
// neighbours. Such vertices are never adjacent, and the result equals sequential first-fit
// colouring in decreasing priority.
#include <algorithm>
#include <climits>

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
struct RcmState {
    int32_t fs, fe, tail, total;   // current frontier [fs, fe) in `order`, next free slot, children found
    unsigned long long best;       // (degree, index) key of the next component's start
};
constexpr int RCM_BATCH = 16;
constexpr int RCM_GRID = 152 * 8;

__global__ void rcm_start_k(const int32_t* rp, const int32_t* pos, int64_t N, RcmState* st) {
    if (st->fs != st->fe || st->tail >= N) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        if (pos[i] >= 0) continue;
        unsigned long long key = ((unsigned long long)(uint32_t)(rp[i + 1] - rp[i]) << 32) | (uint32_t)i;
        atomicMin(&st->best, key);
    }
}

__global__ void rcm_seed_k(int32_t* order, int32_t* pos, int64_t N, RcmState* st) {
    if (st->fs != st->fe || st->tail >= N) return;
    int32_t s = (int32_t)(st->best & 0xffffffffull);
    order[st->tail] = s;
    pos[s] = st->tail;
    st->fs = st->tail;
    st->fe = st->tail + 1;
    st->tail += 1;
    st->best = ~0ull;
}

__global__ void rcm_claim_k(const int32_t* rp, const int32_t* adj, const int32_t* order, const int32_t* pos,
                            const RcmState* st, int32_t* claim) {
    const int32_t fs = st->fs, fe = st->fe;
    for (int32_t t = fs + blockIdx.x * blockDim.x + threadIdx.x; t < fe; t += gridDim.x * blockDim.x) {
        int32_t v = order[t];
        for (int32_t p = rp[v]; p < rp[v + 1]; ++p) {
            int32_t u = adj[p];
            if (pos[u] < 0) atomicMin(&claim[u], t);
        }
    }
}

__global__ void rcm_count_k(const int32_t* rp, const int32_t* adj, const int32_t* order, const int32_t* pos,
                            const int32_t* claim, const RcmState* st, int32_t* cnt) {
    const int32_t fs = st->fs, fe = st->fe;
    for (int32_t t = fs + blockIdx.x * blockDim.x + threadIdx.x; t < fe; t += gridDim.x * blockDim.x) {
        int32_t v = order[t];
        int32_t c = 0;
        for (int32_t p = rp[v]; p < rp[v + 1]; ++p) {
            int32_t u = adj[p];
            if (pos[u] < 0 && claim[u] == t) ++c;
        }
        cnt[t - fs] = c;
    }
}

// exclusive scan of the frontier's child counts by one block; total into the state
__global__ void __launch_bounds__(1024) rcm_scan_k(const int32_t* cnt, int32_t* off, RcmState* st) {
    __shared__ int32_t part[1024];
    const int32_t n = st->fe - st->fs;
    const int32_t per = (n + 1023) / 1024;
    const int32_t b = threadIdx.x * per, e = min(n, b + per);
    int32_t sum = 0;
    for (int32_t i = b; i < e; ++i) sum += cnt[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int t = 0; t < 1024; ++t) { int32_t v = part[t]; part[t] = acc; acc += v; }
        st->total = acc;
    }
    __syncthreads();
    int32_t acc = part[threadIdx.x];
    for (int32_t i = b; i < e; ++i) { off[i] = acc; acc += cnt[i]; }
}

__global__ void rcm_write_k(const int32_t* rp, const int32_t* adj, int32_t* order, int32_t* pos, const int32_t* claim,
                            const int32_t* off, const RcmState* st) {
    const int32_t fs = st->fs, fe = st->fe, tail = st->tail;
    for (int32_t t = fs + blockIdx.x * blockDim.x + threadIdx.x; t < fe; t += gridDim.x * blockDim.x) {
        int32_t v = order[t];
        int32_t q = tail + off[t - fs];
        for (int32_t p = rp[v]; p < rp[v + 1]; ++p) {
            int32_t u = adj[p];
            if (pos[u] < 0 && claim[u] == t) {
                order[q] = u;
                pos[u] = q;
                ++q;
            }
        }
    }
}

__global__ void rcm_advance_k(RcmState* st) {
    if (st->fs == st->fe) return;
    st->fs = st->tail;
    st->fe = st->tail + st->total;
    st->tail += st->total;
    st->total = 0;
}

__global__ void reverse_k(const int32_t* order, int64_t N, int32_t* perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) perm[i] = order[N - 1 - i];
}

void rcm(int64_t N, const int32_t* rp, const int32_t* ci, int32_t* perm, cudaStream_t s) {
    REQUIRE(N >= 1 && N < 0x7fffffff, "N out of range");
    REQUIRE(rp && ci && perm, "null array");
    Temp<int32_t> srp, sci;
    sym_pattern(N, rp, ci, srp, sci, s);
    int64_t snnz = csr_nnz(srp.get(), N, s);
    Temp<int32_t> adj(snnz > 0 ? snnz : 1, s);
    sort_by_degree_k<<<grid_for(N, SBD_WARPS), SBD_WARPS * 32, 0, s>>>(srp.get(), sci.get(), N, adj.get());
    CK_LAUNCH();
    Temp<int32_t> order(N, s), pos(N, s), claim(N, s), cnt(N + 1, s), off(N + 1, s);
    fill_i32(pos.get(), -1, N, s);
    fill_i32(claim.get(), INT_MAX, N, s);
    Temp<RcmState> st(1, s);
    RcmState init{0, 0, 0, 0, ~0ull};
    CK(cudaMemcpyAsync(st.get(), &init, sizeof(RcmState), cudaMemcpyHostToDevice, s));
    const unsigned grid = (unsigned)std::min<int64_t>(grid_for(N, 128), RCM_GRID);
    for (int64_t level = 0;; ++level) {
        if (level % RCM_BATCH == 0) {
            RcmState h;
            to_host(&h, st.get(), 1, s);
            if (h.tail >= N && h.fs == h.fe) break;
            if (level > 4 * N + 64) fail(MGM_ERR_UNSUPPORTED, "RCM did not terminate");
        }
        rcm_start_k<<<grid, 128, 0, s>>>(srp.get(), pos.get(), N, st.get());
        CK_LAUNCH();
        rcm_seed_k<<<1, 1, 0, s>>>(order.get(), pos.get(), N, st.get());
        CK_LAUNCH();
        rcm_claim_k<<<grid, 128, 0, s>>>(srp.get(), adj.get(), order.get(), pos.get(), st.get(), claim.get());
        CK_LAUNCH();
        rcm_count_k<<<grid, 128, 0, s>>>(srp.get(), adj.get(), order.get(), pos.get(), claim.get(), st.get(), cnt.get());
        CK_LAUNCH();
        rcm_scan_k<<<1, 1024, 0, s>>>(cnt.get(), off.get(), st.get());
        CK_LAUNCH();
        rcm_write_k<<<grid, 128, 0, s>>>(srp.get(), adj.get(), order.get(), pos.get(), claim.get(), off.get(), st.get());
        CK_LAUNCH();
        rcm_advance_k<<<1, 1, 0, s>>>(st.get());
        CK_LAUNCH();
    }
    reverse_k<<<grid_for(N, 256), 256, 0, s>>>(order.get(), N, perm);
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

__global__ void jp_select_k(const int32_t* rp, const int32_t* adj, const int32_t* col, int64_t N, unsigned long long seed,
                            char* sel, int* nleft) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int left = 0;
    if (v < N) {
        sel[v] = 0;
        if (col[v] < 0) {
            left = 1;
            unsigned long long pv = splitmix64(seed, (unsigned long long)v);
            bool top = true;
            for (int32_t p = rp[v]; p < rp[v + 1] && top; ++p) {
                int32_t u = adj[p];
                if (col[u] >= 0) continue;
                unsigned long long pu = splitmix64(seed, (unsigned long long)u);
                if (!(pv > pu || (pv == pu && v > u))) top = false;
            }
            sel[v] = top ? 1 : 0;
        }
    }
    left = warp_sum_i(left);
    if ((threadIdx.x & 31) == 0 && left) atomicAdd(nleft, left);
}

__global__ void jp_assign_k(const int32_t* rp, const int32_t* adj, int32_t* col, const char* sel, int64_t N, int* maxc) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N || !sel[v]) return;
    for (int base = 0;; base += 64) {
        unsigned long long used = 0;
        for (int32_t p = rp[v]; p < rp[v + 1]; ++p) {
            int32_t c = col[adj[p]];
            if (c >= base && c < base + 64) used |= 1ull << (c - base);
        }
        if (~used) {
            int c = base + __ffsll((long long)~used) - 1;
            col[v] = c;
            atomicMax(maxc, c);
            return;
        }
    }
}

void color(int64_t N, const int32_t* rp, const int32_t* ci, uint64_t seed, int32_t* colour, int32_t* ncolors,
           cudaStream_t s) {
    REQUIRE(N >= 1 && N < 0x7fffffff, "N out of range");
    REQUIRE(rp && ci && colour, "null array");
    Temp<int32_t> srp, sci;
    sym_pattern(N, rp, ci, srp, sci, s);
    Temp<char> sel(N, s);
    Temp<int> ctr(2, s);  // [0] uncoloured count, [1] max colour
    fill_i32(colour, -1, N, s);
    CK(cudaMemsetAsync(ctr.get() + 1, 0, sizeof(int), s));
    for (int64_t round = 0;; ++round) {
        if (round > N) fail(MGM_ERR_UNSUPPORTED, "colouring did not terminate");
        CK(cudaMemsetAsync(ctr.get(), 0, sizeof(int), s));
        jp_select_k<<<grid_for(N, 256), 256, 0, s>>>(srp.get(), sci.get(), colour, N, seed, sel.get(), ctr.get());
        CK_LAUNCH();
        if (round % 4 == 3 || round < 2) {
            if (read1(ctr.get(), s) == 0) break;
        }
        jp_assign_k<<<grid_for(N, 256), 256, 0, s>>>(srp.get(), sci.get(), colour, sel.get(), N, ctr.get() + 1);
        CK_LAUNCH();
    }
    *ncolors = read1(ctr.get() + 1, s) + 1;
}

}  // namespace mgm

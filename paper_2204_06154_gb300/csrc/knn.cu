// Exact k-nearest-neighbour and fixed-radius searches on a uniform grid (paper Sec. 2: stencils
// are the n nearest nodes in Euclidean R^3; Sec. 3: the m nearest coarse nodes; Sec. 4.1: the
// elimination weights use all neighbours within 2 r_max).
//
// Design: points are binned into a dense 3-D grid of about 2 N cells (counting sort by cell,
// coordinates copied into cell order so a warp reads a cell with coalesced 24-byte loads). One
// warp answers one query: it scans Chebyshev shells of cells around the query's cell, appending
// (d^2, index) candidates to a per-warp shared-memory buffer (compacted to its k smallest keys
// whenever it fills), until at least k candidates lie strictly inside the radius r*h that the
// scanned block is guaranteed to cover. The k smallest
// keys are then placed by rank counting. The result is therefore exactly the (d^2, index) order
// the definition asks for, independent of the grid and of scheduling. Distances are computed as
// (dx*dx + dy*dy) + dz*dz without contraction (this file is built with --fmad=false).
#include <algorithm>
#include <cmath>
#include <cfloat>
#include <climits>

#include "common.cuh"
#include "knn_grid.cuh"

namespace mgm {


__device__ __forceinline__ double d2_pts(double ax, double ay, double az, double bx, double by, double bz) {
    double dx = ax - bx, dy = ay - by, dz = az - bz;
    return (dx * dx + dy * dy) + dz * dz;
}

// ------------------------------ grid construction --------------------------------------------
__global__ void bbox_partial_k(const double* x, int64_t n, double* part) {
    double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) {
            double v = x[3 * i + c];
            mn[c] = fmin(mn[c], v);
            mx[c] = fmax(mx[c], v);
        }
    __shared__ double s[6][32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = 0; c < 3; ++c) {
        double a = mn[c], b = mx[c];
        for (int o = 16; o; o >>= 1) {
            a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) { s[c][w] = a; s[3 + c][w] = b; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = blockDim.x / 32;
        for (int c = 0; c < 3; ++c) {
            double a = s[c][0], b = s[3 + c][0];
            for (int t = 1; t < nw; ++t) { a = fmin(a, s[c][t]); b = fmax(b, s[3 + c][t]); }
            part[6 * blockIdx.x + c] = a;
            part[6 * blockIdx.x + 3 + c] = b;
        }
    }
}

// one block of GRID_PARAMS_THREADS: reduce the partial boxes; then one thread chooses h so that the
// dense grid has at most `cells` cells
__global__ void __launch_bounds__(GRID_PARAMS_THREADS) grid_params_k(const double* part, int nparts, int64_t cells,
                                                                     double h_min, Grid* g) {
    __shared__ double red[6][GRID_PARAMS_THREADS / 32];
    double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x)
        for (int c = 0; c < 3; ++c) { mn[c] = fmin(mn[c], part[6 * b + c]); mx[c] = fmax(mx[c], part[6 * b + 3 + c]); }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = 0; c < 3; ++c)
        for (int o = 16; o; o >>= 1) {
            mn[c] = fmin(mn[c], __shfl_xor_sync(0xffffffffu, mn[c], o));
            mx[c] = fmax(mx[c], __shfl_xor_sync(0xffffffffu, mx[c], o));
        }
    if (lane == 0)
        for (int c = 0; c < 3; ++c) { red[c][w] = mn[c]; red[3 + c][w] = mx[c]; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int c = 0; c < 3; ++c)
        for (int t = 1; t < (int)(blockDim.x / 32); ++t) { mn[c] = fmin(mn[c], red[c][t]); mx[c] = fmax(mx[c], red[3 + c][t]); }
    double e[3], emax = 0.0;
    for (int c = 0; c < 3; ++c) {
        e[c] = mx[c] - mn[c];
        if (!(e[c] >= 0.0 && e[c] < 1e300)) e[c] = 0.0;  // non-finite coordinates: one cell along this axis
        emax = fmax(emax, e[c]);
    }
    if (!(emax > 0.0)) emax = 1.0;
    // bisection on h: count(h) = prod(floor(e/h) + 1) <= cells
    // (64 halvings take the bracket below one part in 1e9 of emax; one reciprocal per step, as a
    // single thread's FP64 divisions are slow)
    double lo = emax * 1e-9, hi = emax * 2.0 + 1.0;
    for (int it = 0; it < 64; ++it) {
        double mid = 0.5 * (lo + hi);
        const double inv = 1.0 / mid;
        double cnt = 1.0;
        for (int c = 0; c < 3; ++c) cnt *= floor(e[c] * inv) + 1.0;
        if (cnt <= (double)cells) hi = mid; else lo = mid;
    }
    // The dimensions use the same expression as the test above (floor(e * (1/h)) + 1, monotone in
    // h), so nx ny nz <= cells, the size of the arrays indexed by cell; the loop only guards that.
    double h = fmax(hi, h_min);
    int n3[3];
    for (int it = 0;; ++it) {
        const double inv = 1.0 / h;
        double cnt = 1.0;
        for (int c = 0; c < 3; ++c) {
            const double f = floor(e[c] * inv) + 1.0;
            n3[c] = (int)f;
            cnt *= f;
        }
        if (cnt <= (double)cells) break;
        h = it < 200 ? h * 1.0001 : emax * 2.0 + 1.0;  // the last: one cell
    }
    double amax = 0.0;
    for (int c = 0; c < 3; ++c) amax = fmax(amax, fmax(fabs(mn[c]), fabs(mx[c])));
    g->amax = (amax < 1e300) ? amax : INFINITY;
    g->x0 = mn[0]; g->y0 = mn[1]; g->z0 = mn[2]; g->h = h;
    g->nx = n3[0]; g->ny = n3[1]; g->nz = n3[2];
    g->ncells = (int64_t)g->nx * g->ny * g->nz;
}

__device__ __forceinline__ int cell_coord(double v, double o, double h, int nd) {
    double t = floor((v - o) / h);
    int c = (int)fmax(0.0, fmin(t, (double)(nd - 1)));
    return c;
}

__global__ void cell_count_k(const double* x, int64_t n, const Grid* gp, int32_t* cnt, int32_t* cell_of) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    Grid g = *gp;
    int cx = cell_coord(x[3 * i], g.x0, g.h, g.nx), cy = cell_coord(x[3 * i + 1], g.y0, g.h, g.ny),
        cz = cell_coord(x[3 * i + 2], g.z0, g.h, g.nz);
    int64_t c = ((int64_t)cz * g.ny + cy) * g.nx + cx;
    cell_of[i] = (int32_t)c;
    atomicAdd(&cnt[c], 1);
}
__global__ void cell_place_k(const double* x, int64_t n, const int32_t* cell_of, const int32_t* start, int32_t* fill,
                             int32_t* sidx, double* sxyz, float4* s32) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t c = cell_of[i];
    int32_t q = start[c] + atomicAdd(&fill[c], 1);
    sidx[q] = (int32_t)i;
    const double a = x[3 * i], b = x[3 * i + 1], d = x[3 * i + 2];
    sxyz[3 * (int64_t)q] = a;
    sxyz[3 * (int64_t)q + 1] = b;
    sxyz[3 * (int64_t)q + 2] = d;
    if (s32) s32[q] = make_float4((float)a, (float)b, (float)d, 0.0f);
}

struct DevGrid {
    Temp<Grid> g;
    Temp<int32_t> start, sidx;
    Temp<double> sxyz;
    Temp<float4> s32;  // the sorted coordinates rounded to FP32, for culling
    int64_t cells;
};

static void build_grid(const double* x, int64_t n, int64_t cells, double h_min, DevGrid& G, cudaStream_t s) {
    if (cells < 1) cells = 1;
    if (cells > (int64_t)1 << 27) cells = (int64_t)1 << 27;
    G.cells = cells;
    int nparts = (int)std::min<int64_t>(grid_for(n, 256), 1024);
    Temp<double> part(6 * nparts, s);
    bbox_partial_k<<<nparts, 256, 0, s>>>(x, n, part.get());
    CK_LAUNCH();
    G.g.alloc(1, s);
    grid_params_k<<<1, GRID_PARAMS_THREADS, 0, s>>>(part.get(), nparts, cells, h_min, G.g.get());
    CK_LAUNCH();
    Temp<int32_t> cnt(cells + 1, s), cell_of(n, s);
    CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * (cells + 1), s));
    cell_count_k<<<grid_for(n, 256), 256, 0, s>>>(x, n, G.g.get(), cnt.get(), cell_of.get());
    CK_LAUNCH();
    G.start.alloc(cells + 1, s);
    exclusive_scan_i32(cnt.get(), G.start.get(), cells, s);
    CK(cudaMemsetAsync(cnt.get(), 0, sizeof(int32_t) * (cells + 1), s));
    G.sidx.alloc(n, s);
    G.sxyz.alloc(3 * n, s);
    G.s32.alloc(n, s);
    cell_place_k<<<grid_for(n, 256), 256, 0, s>>>(x, n, cell_of.get(), G.start.get(), cnt.get(), G.sidx.get(),
                                                    G.sxyz.get(), G.s32.get());
    CK_LAUNCH();
}

// ------------------------------ kNN -----------------------------------------------------------
// Candidate keys are integers: the bit pattern of a non-negative double orders like its value, so
// key = bits(d^2) + 1 (0 for the query itself when it is the stencil centre) ranks exactly as
// (d^2, index) with integer compares, which GB300 executes far faster than FP64 compares.
typedef unsigned long long ukey;
__device__ __forceinline__ bool key_lt(ukey a, int ia, ukey b, int ib) { return a < b || (a == b && ia < ib); }
__device__ __forceinline__ ukey d2_key(double d2) { return (ukey)__double_as_longlong(d2) + 1ull; }

// Cells around (cx, cy, cz), 32 at a time: the cube of side W = 2R+1 (`shell` false; dz slowest,
// dx fastest), or only its surface, the cells with max(|dx|,|dy|,|dz|) = R (`shell` true: the two
// z faces, then the square rings of the layers between). Lane l takes cell c0 + l, loads its point
// range, and a warp scan flattens the ranges, so that the warp then walks all their points 32 at
// a time instead of one cell after another; chunk_slot maps a flattened position to the point's
// slot in the cell-sorted arrays.
struct CellChunk {
    int b, excl, total;
};
__host__ __device__ __forceinline__ int block_cells(int R, bool shell) {
    const int W = 2 * R + 1;
    return (!shell || R == 0) ? W * W * W : W * W * W - (W - 2) * (W - 2) * (W - 2);
}
__device__ __forceinline__ CellChunk cell_chunk(const Grid& g, const int32_t* start, int cx, int cy, int cz, int R,
                                                bool shell, int c0, int lane) {
    const int W = 2 * R + 1, cl = c0 + lane;
    int b = 0, len = 0;
    if (cl < block_cells(R, shell)) {
        int dz, dy, dx;
        if (!shell || R == 0) {
            dz = cl / (W * W) - R; dy = (cl / W) % W - R; dx = cl % W - R;
        } else if (cl < 2 * W * W) {
            const int q = cl % (W * W);
            dz = cl < W * W ? -R : R; dy = q / W - R; dx = q % W - R;
        } else {
            const int ring = 4 * (W - 1), q0 = cl - 2 * W * W, q = q0 % ring;
            dz = -R + 1 + q0 / ring;
            if (q < W) { dy = -R; dx = q - R; }
            else if (q < 2 * W) { dy = R; dx = q - W - R; }
            else { dy = -R + 1 + (q - 2 * W) / 2; dx = ((q - 2 * W) & 1) ? R : -R; }
        }
        const int z = cz + dz, y = cy + dy, x = cx + dx;
        if (z >= 0 && z < g.nz && y >= 0 && y < g.ny && x >= 0 && x < g.nx) {
            const int64_t c = ((int64_t)z * g.ny + y) * g.nx + x;
            b = start[c];
            len = start[c + 1] - b;
        }
    }
    int incl = len;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    return CellChunk{b, incl - len, __shfl_sync(0xffffffffu, incl, 31)};
}
// slot of flattened position t (all lanes take part; t is clamped by the caller)
__device__ __forceinline__ int chunk_slot(const CellChunk& ch, int t) {
    int lo = 0;
    for (int step = 16; step; step >>= 1) {
        const int probe = lo + step;
        const int ex = __shfl_sync(0xffffffffu, ch.excl, probe & 31);
        if (probe < 32 && ex <= t) lo = probe;
    }
    return __shfl_sync(0xffffffffu, ch.b, lo) + (t - __shfl_sync(0xffffffffu, ch.excl, lo));
}

// Keep only the k smallest keys of the buffer (stable, in place). A candidate outside the k
// smallest of a subset can never enter the k smallest of the full set, so this loses nothing.
__device__ int knn_compact(ukey* bd, int* bi, int count, int k, int lane) {
    ukey td = 0;
    int tj = 0;
    bool found = false;
    for (int t = lane; t < count; t += 32) {
        int rank = 0;
        for (int u = 0; u < count; ++u) rank += key_lt(bd[u], bi[u], bd[t], bi[t]) ? 1 : 0;
        if (rank == k - 1) { td = bd[t]; tj = bi[t]; found = true; }
    }
    unsigned fm = __ballot_sync(0xffffffffu, found);
    int src = __ffs(fm) - 1;
    td = __shfl_sync(0xffffffffu, td, src);
    tj = __shfl_sync(0xffffffffu, tj, src);
    int w = 0;
    for (int base = 0; base < count; base += 32) {
        int t = base + lane;
        bool has = t < count;
        ukey d = has ? bd[t] : 0;
        int j = has ? bi[t] : 0;
        bool keep = has && !key_lt(td, tj, d, j);
        __syncwarp();
        unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            int pos = w + __popc(km & ((1u << lane) - 1u));
            bd[pos] = d;
            bi[pos] = j;
        }
        w += __popc(km);
        __syncwarp();
    }
    return w;
}

__global__ void __launch_bounds__(KNN_WARPS * 32) knn_k(const Grid* gp, const int32_t* start, const int32_t* sidx,
                                                        const double* sxyz, const double* q, int64_t nq, int k,
                                                        int self_first, int32_t* idx_out, double* d2_out, int* err) {
    extern __shared__ __align__(16) unsigned char knn_smem[];
    ukey (*sd)[KNN_CAP] = reinterpret_cast<ukey (*)[KNN_CAP]>(knn_smem);
    int (*si)[KNN_CAP] = reinterpret_cast<int (*)[KNN_CAP]>(knn_smem + sizeof(ukey) * KNN_WARPS * KNN_CAP);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t qi = (int64_t)blockIdx.x * KNN_WARPS + w;
    if (qi >= nq) return;
    const Grid g = *gp;
    const double px = q[3 * qi], py = q[3 * qi + 1], pz = q[3 * qi + 2];
    const int cx = cell_coord(px, g.x0, g.h, g.nx), cy = cell_coord(py, g.y0, g.h, g.ny), cz = cell_coord(pz, g.z0, g.h, g.nz);
    const int rfull = max(max(max(cx, g.nx - 1 - cx), max(cy, g.ny - 1 - cy)), max(cz, g.nz - 1 - cz));
    ukey* bd = sd[w];
    int* bi = si[w];
    int count = 0;
    ukey lim2 = 0;
    bool all = false;
    for (int r = 0;; ++r) {
        const int ncell = block_cells(r, true);
        for (int c0 = 0; c0 < ncell; c0 += 32) {
            const CellChunk ch = cell_chunk(g, start, cx, cy, cz, r, true, c0, lane);
            for (int t0 = 0; t0 < ch.total; t0 += 32) {
                if (count + 32 > KNN_CAP) {
                    __syncwarp();
                    count = knn_compact(bd, bi, count, k, lane);
                }
                const int t = t0 + lane;
                const bool has = t < ch.total;
                const int slot = chunk_slot(ch, has ? t : ch.total - 1);
                ukey d = 0;
                int j = 0;
                if (has) {
                    j = sidx[slot];
                    d = (self_first && j == (int)qi)
                            ? 0ull
                            : d2_key(d2_pts(px, py, pz, sxyz[3 * (int64_t)slot], sxyz[3 * (int64_t)slot + 1],
                                            sxyz[3 * (int64_t)slot + 2]));
                }
                unsigned m = __ballot_sync(0xffffffffu, has);
                int pos = count + __popc(m & ((1u << lane) - 1u));
                if (has) { bd[pos] = d; bi[pos] = j; }
                count += __popc(m);
            }
        }
        if (r >= rfull) { all = true; break; }
        if (r >= 1) {
            double R = (double)r * g.h;
            lim2 = d2_key(R * R * (1.0 - 1e-9));
            __syncwarp();
            int nin = 0;
            for (int t = lane; t < count; t += 32) nin += bd[t] < lim2 ? 1 : 0;
            nin = warp_sum_i(nin);
            if (nin >= k) break;
        }
    }
    __syncwarp();
    if (all && count < k) {
        if (lane == 0) atomicOr(err, 2);
        return;
    }
    if (!all) {  // keep only candidates strictly inside the covered radius (stable, in place)
        int wpos = 0;
        for (int base = 0; base < count; base += 32) {
            int t = base + lane;
            bool has = t < count;
            ukey d = has ? bd[t] : 0;
            int j = has ? bi[t] : 0;
            bool keep = has && d < lim2;
            __syncwarp();
            unsigned km = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                int pos = wpos + __popc(km & ((1u << lane) - 1u));
                bd[pos] = d;
                bi[pos] = j;
            }
            wpos += __popc(km);
            __syncwarp();
        }
        count = wpos;
    }
    // rank the remaining candidates; the k smallest keys take their places
    for (int t = lane; t < count; t += 32) {
        ukey d = bd[t];
        int j = bi[t];
        int rank = 0;
        for (int u = 0; u < count; ++u) rank += key_lt(bd[u], bi[u], d, j) ? 1 : 0;
        if (rank < k) {
            idx_out[qi * k + rank] = j;
            if (d2_out) d2_out[qi * k + rank] = d == 0ull ? 0.0 : __longlong_as_double((long long)(d - 1ull));
        }
    }
}

// k <= 4: one thread per query, its k best (key, index) pairs kept sorted in registers. Same
// search and stopping rule as knn_k (the k best lie strictly inside the covered radius), so the
// same result.
template <int K>
__global__ void __launch_bounds__(128) knn_small_k(const Grid* gp, const int32_t* start, const int32_t* sidx,
                                                   const double* sxyz, const float4* s32, const double* q, int64_t nq,
                                                   int self_first, int32_t* idx_out, double* d2_out, int* err) {
    const int64_t qi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= nq) return;
    const Grid g = *gp;
    const double px = q[3 * qi], py = q[3 * qi + 1], pz = q[3 * qi + 2];
    const float pxf = (float)px, pyf = (float)py, pzf = (float)pz;
    const double A = g.amax + fmax(fabs(px), fmax(fabs(py), fabs(pz)));
    float far = INFINITY;  // candidates beyond it are farther than the current K-th
    const int cx = cell_coord(px, g.x0, g.h, g.nx), cy = cell_coord(py, g.y0, g.h, g.ny), cz = cell_coord(pz, g.z0, g.h, g.nz);
    const int rfull = max(max(max(cx, g.nx - 1 - cx), max(cy, g.ny - 1 - cy)), max(cz, g.nz - 1 - cz));
    ukey bk[K];
    int bj[K];
#pragma unroll
    for (int t = 0; t < K; ++t) { bk[t] = ~0ull; bj[t] = INT_MAX; }
    int found = 0;
    for (int r = 0;; ++r) {
        for (int dz = -r; dz <= r; ++dz) {
            const int z = cz + dz;
            if (z < 0 || z >= g.nz) continue;
            for (int dy = -r; dy <= r; ++dy) {
                const int y = cy + dy;
                if (y < 0 || y >= g.ny) continue;
                const bool face = (dz == -r || dz == r || dy == -r || dy == r);
                for (int dx = -r; dx <= r; dx += (face ? 1 : 2 * r)) {
                    const int x = cx + dx;
                    if (x >= 0 && x < g.nx) {
                        const int64_t c = ((int64_t)z * g.ny + y) * g.nx + x;
                        const int b = start[c], e = start[c + 1];
                        for (int t = b; t < e; ++t) {
                            ++found;
                            if (d2_f32(pxf, pyf, pzf, s32[t]) > far) continue;  // cannot enter the K best
                            const int j = sidx[t];
                            const ukey d = (self_first && j == (int)qi)
                                               ? 0ull
                                               : d2_key(d2_pts(px, py, pz, sxyz[3 * (int64_t)t], sxyz[3 * (int64_t)t + 1],
                                                               sxyz[3 * (int64_t)t + 2]));
                            if (key_lt(d, j, bk[K - 1], bj[K - 1])) {
                                bk[K - 1] = d;
                                bj[K - 1] = j;
#pragma unroll
                                for (int u = K - 1; u > 0; --u)
                                    if (key_lt(bk[u], bj[u], bk[u - 1], bj[u - 1])) {
                                        const ukey tk = bk[u]; bk[u] = bk[u - 1]; bk[u - 1] = tk;
                                        const int tj = bj[u]; bj[u] = bj[u - 1]; bj[u - 1] = tj;
                                    }
                                if (bk[K - 1] != ~0ull)
                                    far = far_sq_f32(bk[K - 1] ? sqrt(__longlong_as_double((long long)(bk[K - 1] - 1ull))) : 0.0, A);
                            }
                        }
                    }
                    if (r == 0) break;
                }
            }
        }
        if (r >= rfull) break;
        if (r >= 1 && found >= K) {
            const double R = (double)r * g.h;
            if (bk[K - 1] < d2_key(R * R * (1.0 - 1e-9))) break;
        }
    }
    if (found < K) {
        atomicOr(err, 2);
        return;
    }
#pragma unroll
    for (int t = 0; t < K; ++t) {
        idx_out[qi * K + t] = bj[t];
        if (d2_out) d2_out[qi * K + t] = bk[t] == 0ull ? 0.0 : __longlong_as_double((long long)(bk[t] - 1ull));
    }
}

__global__ void nonempty_cells_k(const int32_t* start, int64_t cells, int* out) {
    int c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x)
        c += start[i + 1] > start[i] ? 1 : 0;
    c = warp_sum_i(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

void knn_device(const double* data, int64_t nd, const double* query, int64_t nq, int k, int self_first,
                int32_t* idx_out, double* d2_out, cudaStream_t s) {
    REQUIRE(k >= 1 && k <= 256, "k must be in [1, 256]");
    REQUIRE(nd >= k, "k exceeds the number of data points");
    REQUIRE(nd < 0x7fffffff && nq < 0x7fffffff, "point counts must be < 2^31");
    REQUIRE(!self_first || (data == query && nd == nq), "self_first requires query == data");
    if (nq == 0) return;
    DevGrid G;
    // about 2 N cells for small k; fewer, larger cells for large k so that one ring of cells
    // usually covers the k-th neighbour
    const int64_t cells = std::max<int64_t>(1, (int64_t)((2.0 * nd) * std::min(1.0, 12.0 / k)));
    build_grid(data, nd, cells, 0.0, G, s);
    Temp<int> err(1, s);
    CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
    // Resize for the occupancy that suits the search. A surface crosses a cell over about h^2/1.5
    // of its area on average, so a non-empty cell holds occ ~ rho h^2 / 1.5 points (rho: points per
    // unit area), the disc of radius h about 4.7 occ and the 27-cell block about 16 occ. With
    // occ ~ 0.35 k the first ring covers the k-th neighbour (~1.6 k points within h) while the
    // candidates stay near 6 k. Occupancy scales with h^2 on surfaces, hence the exponent 3/2 on
    // the cell count. The result does not depend on the grid; only the work does.
    if (nd >= 4096) {
        nonempty_cells_k<<<(unsigned)std::min<int64_t>(grid_for(G.cells, 256), 152 * 8), 256, 0, s>>>(G.start.get(), G.cells,
                                                                                                     err.get());
        CK_LAUNCH();
        const int64_t ne = std::max(1, read1(err.get(), s));
        CK(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
        const double occ = (double)nd / (double)ne, target = std::max(1.0, 0.35 * k);
        if (occ > 1.5 * target || occ < target / 1.5) {
            const double want = (double)G.cells * std::pow(occ / target, 1.5);
            const int64_t c2 = std::max<int64_t>(1, std::min<int64_t>((int64_t)want, std::min<int64_t>(8 * nd, (int64_t)1 << 27)));
            if (c2 > G.cells * 5 / 4 || c2 < G.cells * 4 / 5) {
                DevGrid G2;
                build_grid(data, nd, c2, 0.0, G2, s);
                G.g = std::move(G2.g);
                G.start = std::move(G2.start);
                G.sidx = std::move(G2.sidx);
                G.sxyz = std::move(G2.sxyz);
                G.s32 = std::move(G2.s32);
                G.cells = G2.cells;
            }
        }
    }
    if (k <= 4) {
        auto kern = k == 1 ? knn_small_k<1> : k == 2 ? knn_small_k<2> : k == 3 ? knn_small_k<3> : knn_small_k<4>;
        kern<<<grid_for(nq, 128), 128, 0, s>>>(G.g.get(), G.start.get(), G.sidx.get(), G.sxyz.get(), G.s32.get(), query,
                                               nq, self_first, idx_out, d2_out, err.get());
        CK_LAUNCH();
    } else {
        const size_t smem = (sizeof(ukey) + sizeof(int)) * KNN_WARPS * KNN_CAP;
        CK(cudaFuncSetAttribute(knn_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        knn_k<<<grid_for(nq, KNN_WARPS), KNN_WARPS * 32, smem, s>>>(G.g.get(), G.start.get(), G.sidx.get(), G.sxyz.get(),
                                                                query, nq, k, self_first, idx_out, d2_out, err.get());
        CK_LAUNCH();
    }
    int e = read1(err.get(), s);
    if (e & 1) fail(MGM_ERR_UNSUPPORTED, "kNN candidate buffer overflow (points too clustered for the grid)");
    if (e & 2) fail(MGM_ERR_INVALID_ARG, "fewer than k data points");
}

// ------------------------------ fixed-radius neighbour lists (for elimination weights) --------
// For each point i: all j != i with sqrt(d2) < two_rmax, ascending j, with the elimination weight
// contribution f = (1 - max(d, rmin)/two_rmax)^8 (three squarings). Two passes: count, then fill.
constexpr int RAD_WARPS = 4;
constexpr int RAD_CAP = 1024;

template <bool FILL>
__global__ void __launch_bounds__(RAD_WARPS * 32) radius_k(const Grid* gp, const int32_t* start, const int32_t* sidx,
                                                           const double* sxyz, const double* x, int64_t n,
                                                           const double* prm /* two_rmax, rmin */, int32_t* cnt,
                                                           const int32_t* rowptr, int32_t* nbr, double* f, int* err,
                                                           const int32_t* rows, int64_t nrows) {
    __shared__ int si[RAD_WARPS][RAD_CAP];
    __shared__ double sdist[RAD_WARPS][RAD_CAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t t_ = (int64_t)blockIdx.x * RAD_WARPS + w;
    if (t_ >= (rows ? nrows : n)) return;
    const int64_t i = rows ? (int64_t)rows[t_] : t_;
    const Grid g = *gp;
    const double two_rmax = prm[0], rmin = prm[1];
    const double lim_sq = two_rmax * two_rmax * (1.0 + 1e-9);
    const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    const int cx = cell_coord(px, g.x0, g.h, g.nx), cy = cell_coord(py, g.y0, g.h, g.ny), cz = cell_coord(pz, g.z0, g.h, g.nz);
    // rings so that the scanned block covers the radius: with cells wider than 2 r_max (by far
    // more than rounding), neighbours differ by at most one cell per axis; otherwise one extra
    // ring absorbs rounding at the bin boundaries
    const int R = (g.h >= two_rmax * (1.0 + 1e-6)) ? 1 : (int)ceil(two_rmax / g.h) + 1;
    int count = 0;
    const int ncell = block_cells(R, false);
    for (int c0 = 0; c0 < ncell; c0 += 32) {
        const CellChunk ch = cell_chunk(g, start, cx, cy, cz, R, false, c0, lane);
        for (int t0 = 0; t0 < ch.total; t0 += 32) {
            const int t = t0 + lane;
            const int slot = chunk_slot(ch, t < ch.total ? t : ch.total - 1);
            bool has = false;
            int j = 0;
            double d = 0.0;
            if (t < ch.total) {
                j = sidx[slot];
                if (j != (int)i) {
                    double dd = d2_pts(px, py, pz, sxyz[3 * (int64_t)slot], sxyz[3 * (int64_t)slot + 1],
                                       sxyz[3 * (int64_t)slot + 2]);
                    // sqrt(dd) < two_rmax is decided exactly below; skip the sqrt where dd is
                    // clearly beyond (the factor leaves a margin far above rounding)
                    if (dd <= lim_sq) {
                        d = sqrt(dd);
                        has = d < two_rmax;
                    }
                }
            }
            unsigned m = __ballot_sync(0xffffffffu, has);
            int pos = count + __popc(m & ((1u << lane) - 1u));
            if (has && pos < RAD_CAP) { si[w][pos] = j; sdist[w][pos] = d; }
            count += __popc(m);
        }
    }
    if (count > RAD_CAP) {
        if (lane == 0) atomicOr(err, 1);
        return;
    }
    if (!FILL) {
        if (lane == 0) cnt[i] = count;
        return;
    }
    __syncwarp();
    const int64_t base = rowptr[i];
    for (int t = lane; t < count; t += 32) {
        int j = si[w][t];
        int rank = 0;
        for (int u = 0; u < count; ++u) rank += si[w][u] < j ? 1 : 0;
        double d = sdist[w][t];
        double dh = d > rmin ? d : rmin;
        double tt = 1.0 - dh / two_rmax;
        double t2 = tt * tt, t4 = t2 * t2;
        nbr[base + rank] = j;
        f[base + rank] = t4 * t4;
    }
}

// The same lists with one thread per point (the lists are short: ~15 entries on the surfaces here):
// the count pass counts every point and lists those above RT_CAP; the fill pass keeps each list
// sorted by index in local memory as it is found and writes rows of at most RT_CAP entries (the
// warp kernel above fills the listed longer ones). Same candidates and tests, so the same lists.
constexpr int RT_CAP = 48;
// STAGE (with FILL): one pass that also counts, writing each row of at most RT_CAP entries to its
// fixed slot i * RT_CAP of nbr / f (compacted after the scan of the counts)
template <bool FILL, bool STAGE = false>
__global__ void __launch_bounds__(128) radius_thread_k(const Grid* gp, const int32_t* start, const int32_t* sidx,
                                                       const double* sxyz, const float4* s32, const double* x, int64_t n,
                                                       const double* prm, int32_t* cnt, const int32_t* rowptr,
                                                       int32_t* nbr, double* f, int32_t* longrows, int* nlong) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Grid g = *gp;
    const double two_rmax = prm[0], rmin = prm[1];
    const double lim_sq = two_rmax * two_rmax * (1.0 + 1e-9);
    // below in_sq the square root is certainly below 2 r_max (the count pass needs no root there)
    const double in_sq = two_rmax * two_rmax * (1.0 - 1e-9);
    const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    const float pxf = (float)px, pyf = (float)py, pzf = (float)pz;
    const float far = far_sq_f32(two_rmax, g.amax + fmax(fabs(px), fmax(fabs(py), fabs(pz))));
    const int cx = cell_coord(px, g.x0, g.h, g.nx), cy = cell_coord(py, g.y0, g.h, g.ny), cz = cell_coord(pz, g.z0, g.h, g.nz);
    const int R = (g.h >= two_rmax * (1.0 + 1e-6)) ? 1 : (int)ceil(two_rmax / g.h) + 1;
    int count = 0;
    int jl[RT_CAP];
    double dl[RT_CAP];
    for (int z = max(cz - R, 0); z <= min(cz + R, g.nz - 1); ++z)
        for (int y = max(cy - R, 0); y <= min(cy + R, g.ny - 1); ++y)
            for (int xx = max(cx - R, 0); xx <= min(cx + R, g.nx - 1); ++xx) {
                const int64_t c = ((int64_t)z * g.ny + y) * g.nx + xx;
                const int b = start[c], e = start[c + 1];
                for (int t = b; t < e; ++t) {
                    if (d2_f32(pxf, pyf, pzf, s32[t]) > far) continue;  // certainly beyond 2 r_max
                    const int j = sidx[t];
                    if (j == (int)i) continue;
                    const double dd = d2_pts(px, py, pz, sxyz[3 * (int64_t)t], sxyz[3 * (int64_t)t + 1],
                                             sxyz[3 * (int64_t)t + 2]);
                    if (!(dd <= lim_sq)) continue;
                    double d = 0.0;
                    if (FILL || !(dd < in_sq)) {
                        d = sqrt(dd);
                        if (!(d < two_rmax)) continue;
                    }
                    if (FILL && count < RT_CAP) {  // insert by index
                        int q = count;
                        while (q > 0 && jl[q - 1] > j) { jl[q] = jl[q - 1]; dl[q] = dl[q - 1]; --q; }
                        jl[q] = j;
                        dl[q] = d;
                    }
                    ++count;
                }
            }
    if (!FILL || STAGE) {
        cnt[i] = count;
        if (count > RT_CAP) longrows[atomicAdd(nlong, 1)] = (int32_t)i;
        if (!FILL) return;
    }
    if (count > RT_CAP) return;
    const int64_t base = STAGE ? i * RT_CAP : (int64_t)rowptr[i];
    for (int q = 0; q < count; ++q) {
        const double dh = dl[q] > rmin ? dl[q] : rmin;
        const double tt = 1.0 - dh / two_rmax;
        const double t2 = tt * tt, t4 = t2 * t2;
        nbr[base + q] = jl[q];
        f[base + q] = t4 * t4;
    }
}

// rows of at most RT_CAP entries from their fixed slots to their CSR positions
__global__ void radius_compact_k(const int32_t* cnt, const int32_t* rowptr, const int32_t* snbr, const double* sf, int64_t n,
                                 int32_t* nbr, double* f) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = t / RT_CAP;
    const int q = (int)(t % RT_CAP);
    if (i >= n || q >= cnt[i] || cnt[i] > RT_CAP) return;
    nbr[rowptr[i] + q] = snbr[t];
    f[rowptr[i] + q] = sf[t];
}

// Builds the neighbour graph for the elimination. prm: device {two_rmax, rmin}; h_hint: a host
// estimate of two_rmax used to size the grid cells. One search pass writes the lists of at most
// RT_CAP entries to fixed slots and counts every row; after the scan they are compacted, and the
// longer lists are searched again by a warp each.
void radius_graph(const double* x, int64_t n, const double* prm, double h_hint, Temp<int32_t>& rowptr,
                  Temp<int32_t>& nbr, Temp<double>& f, cudaStream_t s) {
    DevGrid G;
    build_grid(x, n, 8 * n, h_hint * (1.0 + 1e-5), G, s);  // cells no narrower than 2 r_max: one ring
    Temp<int32_t> cnt(n + 1, s), longrows(n, s);
    Temp<int> err(2, s);  // [0] warp-kernel overflow, [1] rows above RT_CAP
    CK(cudaMemsetAsync(err.get(), 0, 2 * sizeof(int), s));
    Temp<int32_t> snbr(n * RT_CAP, s);
    Temp<double> sf(n * RT_CAP, s);
    radius_thread_k<true, true><<<grid_for(n, 128), 128, 0, s>>>(G.g.get(), G.start.get(), G.sidx.get(), G.sxyz.get(),
                                                                 G.s32.get(), x, n, prm, cnt.get(), nullptr, snbr.get(),
                                                                 sf.get(), longrows.get(), err.get() + 1);
    CK_LAUNCH();
    int ecnt[2];
    to_host(ecnt, err.get(), 2, s);
    rowptr.alloc(n + 1, s);
    exclusive_scan_i32(cnt.get(), rowptr.get(), n, s);
    int64_t nnz = csr_nnz(rowptr.get(), n, s);
    nbr.alloc(nnz > 0 ? nnz : 1, s);
    f.alloc(nnz > 0 ? nnz : 1, s);
    radius_compact_k<<<grid_for(n * RT_CAP, 256), 256, 0, s>>>(cnt.get(), rowptr.get(), snbr.get(), sf.get(), n, nbr.get(),
                                                             f.get());
    CK_LAUNCH();
    if (ecnt[1] > 0) {  // the longer lists, one warp each
        radius_k<true><<<grid_for(ecnt[1], RAD_WARPS), RAD_WARPS * 32, 0, s>>>(
            G.g.get(), G.start.get(), G.sidx.get(), G.sxyz.get(), x, n, prm, nullptr, rowptr.get(), nbr.get(), f.get(),
            err.get(), longrows.get(), (int64_t)ecnt[1]);
        CK_LAUNCH();
        if (read1(err.get(), s)) fail(MGM_ERR_UNSUPPORTED, "elimination neighbour list exceeds 1024 entries");
    }
}

}  // namespace mgm

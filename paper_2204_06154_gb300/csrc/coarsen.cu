// Poisson-disk coarsening by weighted sample elimination (paper Sec. 4.1; the elimination weights
// follow the cited WSE method of Yuksel: w_ij = (1 - max(d_ij, r_min)/(2 r_max))^8 for neighbours
// closer than 2 r_max).
//
// GPU formulation (rounds): the sequential method removes the point of largest weight one at a
// time. A point whose (weight, index) exceeds that of every live neighbour is removed before any
// of its neighbours by that rule (neighbour weights only fall), so all such local maxima can go in
// one round. Each round: count live points with positive weight, mark candidates, and if more
// candidates than remaining removals exist keep only the largest by (weight, index) (a 96-bit
// MSB-first threshold search in one block). Survivors adjacent to a removed point recompute their
// weight from scratch in ascending neighbour order, so every weight is the same IEEE sum as a
// sequential recomputation and the kept set is bit-reproducible. Built with --fmad=false.
#include <algorithm>
#include <cstdio>

#include "common.cuh"

namespace mgm {

void radius_graph(const double* x, int64_t n, const double* prm, double h_hint, Temp<int32_t>& rowptr,
                  Temp<int32_t>& nbr, Temp<double>& f, cudaStream_t s);

__global__ void nn_fixed_sum_k(const double* x, const int32_t* idx2, int64_t n, unsigned long long* S) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    long long v = 0;
    if (i < n) {
        int64_t j = idx2[2 * i + 1];
        double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1], dz = x[3 * i + 2] - x[3 * j + 2];
        double d = sqrt((dx * dx + dy * dy) + dz * dz);
        v = __double2ll_rn(d * 4294967296.0);
    }
    v = warp_sum<long long>(v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(S, (unsigned long long)v);
}

// r_max from the hexagonal-packing area estimate, r_min from weight limiting (beta 0.65, gamma 1.5)
__global__ void wse_params_k(const unsigned long long* S, int64_t N, int64_t NH, double* prm) {
    double dbar = ((double)(long long)*S / 4294967296.0) / (double)N;
    double area = (double)N * ((sqrt(3.0) * 0.5) * (dbar * dbar));
    double rmax = sqrt(area / ((2.0 * sqrt(3.0)) * (double)NH));
    double ratio = (double)NH / (double)N;
    double rmin = (rmax * (1.0 - ratio * sqrt(ratio))) * 0.65;
    prm[0] = 2.0 * rmax;
    prm[1] = rmin;
    prm[2] = rmax;
}

// w_i = sum over live neighbours in ascending order; with `only_dirty`, only rows flagged dirty
__global__ void weights_k(const int32_t* rp, const int32_t* nbr, const double* f, const char* live, char* dirty,
                          int64_t n, int only_dirty, double* w) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !live[i]) return;
    if (only_dirty) {
        if (!dirty[i]) return;
        dirty[i] = 0;
    }
    double acc = 0.0;
    for (int32_t p = rp[i]; p < rp[i + 1]; ++p)
        if (live[nbr[p]]) acc = acc + f[p];
    w[i] = acc;
}

// Device-resident round state: the host enqueues rounds without reading anything back and
// checks the live count every WSE_BATCH rounds; a round with nothing left to remove is a no-op.
struct WseState {
    long long nlive, need;
    int npos, ncand, selective;
};
constexpr int WSE_BATCH = 8;

__global__ void wse_round_begin_k(WseState* st, long long NH) {
    st->need = st->nlive - NH;
    st->npos = 0;
    st->ncand = 0;
    st->selective = 0;
}

__global__ void count_pos_k(const char* live, const double* w, int64_t n, WseState* st) {
    if (st->need <= 0) return;
    int c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += (live[i] && w[i] > 0.0) ? 1 : 0;
    c = warp_sum_i(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&st->npos, c);
}

__device__ __forceinline__ bool wgt_gt(double wa, int64_t a, double wb, int64_t b) { return wa > wb || (wa == wb && a > b); }

__global__ void candidates_k(const int32_t* rp, const int32_t* nbr, const char* live, const double* w, int64_t n,
                             WseState* st, int32_t* cand) {
    if (st->need <= 0) return;
    const bool anypos = st->npos > 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!live[i]) continue;
        if (anypos) {
            double wi = w[i];
            if (!(wi > 0.0)) continue;
            bool top = true;
            for (int32_t p = rp[i]; p < rp[i + 1] && top; ++p) {
                int32_t j = nbr[p];
                if (live[j] && !wgt_gt(wi, i, w[j], j)) top = false;
            }
            if (!top) continue;
        }
        int q = atomicAdd(&st->ncand, 1);
        cand[q] = (int32_t)i;
    }
}

// When more candidates than remaining removals exist, keep only the `need` largest by
// (weight, index): the need-th largest 96-bit key (weight bits, index) is found digit by digit,
// 8 bits at a time from the top (a histogram of the candidates that match the digits found so far,
// then the digit at which the count from the top reaches the number still wanted), and every key
// >= it is marked. Keys are distinct, so exactly `need` are kept. One block.
__global__ void __launch_bounds__(1024) select_top_k(const int32_t* cand, const double* w, WseState* st, char* sel) {
    __shared__ int hist[256];
    __shared__ int s_digit, s_rem;
    const long long need = st->need;
    const int nc = st->ncand;
    if (need <= 0 || nc <= need) return;
    unsigned long long thi = 0;  // digits found so far (key bits 95..32)
    unsigned tlo = 0;            // (key bits 31..0)
    if (threadIdx.x == 0) s_rem = (int)need;
    for (int p = 0; p < 12; ++p) {
        const int top = 95 - 8 * p;  // highest bit of this digit
        for (int q = threadIdx.x; q < 256; q += blockDim.x) hist[q] = 0;
        __syncthreads();
        for (int t = threadIdx.x; t < nc; t += blockDim.x) {
            const int32_t i = cand[t];
            const unsigned long long kh = (unsigned long long)__double_as_longlong(w[i]);
            const unsigned kl = (unsigned)i;
            // match the digits above this one
            bool match;
            if (top == 95) match = true;
            else if (top + 1 >= 32 + 64) match = true;
            else if (top + 1 > 32) match = (kh >> (top + 1 - 32)) == (thi >> (top + 1 - 32));
            else match = kh == thi && (top + 1 == 32 || (kl >> (top + 1)) == (tlo >> (top + 1)));
            if (!match) continue;
            const int d = top >= 32 ? (int)((kh >> (top - 7 - 32)) & 0xffull) : (int)((kl >> (top - 7)) & 0xffu);
            atomicAdd(&hist[d], 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int rem = s_rem, d = 255;
            for (; d > 0; --d) {
                if (hist[d] >= rem) break;
                rem -= hist[d];
            }
            s_digit = d;
            s_rem = rem;
        }
        __syncthreads();
        const unsigned dg = (unsigned)s_digit;
        if (top >= 32) thi |= (unsigned long long)dg << (top - 7 - 32);
        else tlo |= dg << (top - 7);
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
        const int32_t i = cand[t];
        const unsigned long long kh = (unsigned long long)__double_as_longlong(w[i]);
        const unsigned kl = (unsigned)i;
        sel[t] = (kh > thi || (kh == thi && kl >= tlo)) ? 1 : 0;
    }
    if (threadIdx.x == 0) st->selective = 1;
}

__global__ void remove_k(const int32_t* cand, const char* sel, const WseState* st, const int32_t* rp, const int32_t* nbr,
                         char* live, char* dirty) {
    if (st->need <= 0) return;
    const int nc = st->ncand;
    const bool selective = st->selective != 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nc; t += gridDim.x * blockDim.x) {
        if (selective && !sel[t]) continue;
        int32_t v = cand[t];
        live[v] = 0;
        for (int32_t p = rp[v]; p < rp[v + 1]; ++p) dirty[nbr[p]] = 1;
    }
}

__global__ void wse_round_end_k(WseState* st) {
    if (st->need <= 0) return;
    st->nlive -= st->selective ? st->need : (long long)st->ncand;
}

__global__ void live_flags_k(const char* live, int64_t n, int32_t* fl) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) fl[i] = live[i] ? 1 : 0;
}
__global__ void compact_live_k(const char* live, const int32_t* pos, int64_t n, int32_t* keep) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && live[i]) keep[pos[i]] = (int32_t)i;
}

void coarsen(const double* x, int64_t N, int64_t NH, int32_t* keep, cudaStream_t s, double* rmax_out) {
    REQUIRE(x && keep, "null array");
    REQUIRE(N >= 2 && N < 0x7fffffff, "N_fine must be in [2, 2^31)");
    REQUIRE(NH >= 1 && NH <= N, "N_coarse must be in [1, N_fine]");
    // mean nearest-neighbour distance, summed exactly in 2^-32 fixed point
    Temp<int32_t> idx2(2 * N, s);
    knn_device(x, N, x, N, 2, 1, idx2.get(), nullptr, s);
    Temp<unsigned long long> S(1, s);
    CK(cudaMemsetAsync(S.get(), 0, sizeof(unsigned long long), s));
    trace_mark(s, "  wse:knn2");
    nn_fixed_sum_k<<<grid_for(N, 256), 256, 0, s>>>(x, idx2.get(), N, S.get());
    CK_LAUNCH();
    Temp<double> prm(3, s);
    wse_params_k<<<1, 1, 0, s>>>(S.get(), N, NH, prm.get());
    CK_LAUNCH();
    double hp[3];
    to_host(hp, prm.get(), 3, s);
    if (rmax_out) *rmax_out = hp[2];
    if (NH == N) {
        iota_i32(keep, N, s);
        return;
    }
    Temp<int32_t> rp, nbr;
    Temp<double> f;
    trace_mark(s, "  wse:params");
    radius_graph(x, N, prm.get(), hp[0], rp, nbr, f, s);
    trace_mark(s, "  wse:radius");
    Temp<char> live(N, s), dirty(N, s), sel(N, s);
    Temp<double> w(N, s);
    Temp<int32_t> cand(N, s);
    Temp<WseState> st(1, s);
    WseState init{(long long)N, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(st.get(), &init, sizeof(WseState), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(live.get(), 1, N, s));
    CK(cudaMemsetAsync(dirty.get(), 0, N, s));
    weights_k<<<grid_for(N, 256), 256, 0, s>>>(rp.get(), nbr.get(), f.get(), live.get(), dirty.get(), N, 0, w.get());
    CK_LAUNCH();
    const unsigned grid = (unsigned)std::min<int64_t>(grid_for(N, 256), 152 * 8);
    // one elimination round: seven kernels that return at once when nothing is left to remove
    auto round_on = [&](cudaStream_t q) {
        wse_round_begin_k<<<1, 1, 0, q>>>(st.get(), (long long)NH);
        CK_LAUNCH();
        count_pos_k<<<grid, 256, 0, q>>>(live.get(), w.get(), N, st.get());
        CK_LAUNCH();
        candidates_k<<<grid, 256, 0, q>>>(rp.get(), nbr.get(), live.get(), w.get(), N, st.get(), cand.get());
        CK_LAUNCH();
        select_top_k<<<1, 1024, 0, q>>>(cand.get(), w.get(), st.get(), sel.get());
        CK_LAUNCH();
        remove_k<<<grid, 256, 0, q>>>(cand.get(), sel.get(), st.get(), rp.get(), nbr.get(), live.get(), dirty.get());
        CK_LAUNCH();
        weights_k<<<grid_for(N, 256), 256, 0, q>>>(rp.get(), nbr.get(), f.get(), live.get(), dirty.get(), N, 1, w.get());
        CK_LAUNCH();
        wse_round_end_k<<<1, 1, 0, q>>>(st.get());
        CK_LAUNCH();
    };
    // WSE_BATCH rounds captured once as a CUDA graph and replayed; the host reads the state between
    // replays (rounds after the last useful one are no-ops)
    GraphBatch gb;
    gb.capture([&](cudaStream_t q) {
        for (int r = 0; r < WSE_BATCH; ++r) round_on(q);
    });
    int64_t rounds_done = 0;
    for (int64_t batch = 0;; ++batch) {
        WseState h;
        to_host(&h, st.get(), 1, s);
        rounds_done = batch * WSE_BATCH;
        if (h.nlive <= NH) break;
        if (batch > 0 && h.ncand <= 0 && h.need > 0) fail(MGM_ERR_UNSUPPORTED, "elimination round without candidates");
        if (rounds_done > N + WSE_BATCH) fail(MGM_ERR_UNSUPPORTED, "elimination did not terminate");
        gb.launch(s);
    }
    if (trace_on()) std::fprintf(stderr, "[mgm setup] wse rounds: %lld\n", (long long)rounds_done);
    trace_mark(s, "  wse:rounds");
    Temp<int32_t> fl(N, s), pos(N + 1, s);
    live_flags_k<<<grid_for(N, 256), 256, 0, s>>>(live.get(), N, fl.get());
    CK_LAUNCH();
    exclusive_scan_i32(fl.get(), pos.get(), N, s);
    compact_live_k<<<grid_for(N, 256), 256, 0, s>>>(live.get(), pos.get(), N, keep);
    CK_LAUNCH();
}

}  // namespace mgm

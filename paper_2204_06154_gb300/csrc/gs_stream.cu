// Streamed multicolour Gauss-Seidel sweeps: one launch per sweep of a level, its matrix streamed
// through shared memory by bulk copies while the rows wait for their inputs.
//
// The forward multicolour sweep (eq. (smoother) in colour order, Alg. 3's smoother) updates the
// rows of one colour from the current values of all other rows; rows of one colour are
// independent. Launching one kernel per colour leaves each launch a thin wave bound by its chain
// of dependent loads. Here one cooperative launch runs every colour:
//
//  * Ownership. Block k owns the rows whose RCM index lies in band k = [ceil(k n / B),
//    ceil((k+1) n / B)); within each colour these rows are one contiguous solve-order range (a
//    colour keeps RCM order), its "slice", cut into chunks of at most 512 / G rows whose entries
//    fit one stage.
//  * Dependencies are local. A row reads only its matrix neighbours, and RCM keeps them within
//    D bands (D from the level's RCM bandwidth). Block k starts colour c once blocks k-D..k+D
//    have finished colours < c (per-block progress counters, release/acquire at GPU scope).
//    This also orders the upper-part reads of a full sweep (old values of later colours) before
//    those rows are rewritten: their owners wait for block k to finish its earlier colour.
//  * Streaming. One producer warp copies the chunks' columns and values (static data) with
//    cp.async.bulk into a ring of shared-memory stages, running ahead across colour boundaries,
//    so the HBM stream continues while the consumers wait on their neighbours. The 512 consumer
//    threads take each chunk together (G lanes a row): every consumer waits on every stage
//    phase in order (an mbarrier parity wait is only exact one phase ahead) and one thread
//    releases the stage after a barrier. A lane issues all gathers of its quads of entries
//    before the first product, so a chunk costs one round trip to L1/L2. Gathered vector
//    entries are ordinary loads; the acquire at each colour start makes other blocks' writes
//    visible.
//  * MODE 0 (first sweep from zero) reads lower parts only; with `resid` it then streams the
//    upper parts and writes the residual s = -U e (exact after a sweep from zero, since
//    (D + L_lower) e = b row by row), so pre-smoothing and the residual take one launch.
//    MODE 1 is a full sweep (lower parts with new values, upper parts with old ones).
//
// Progress counters are never reset: every launch advances every block by the same number of
// colour steps, so at a launch's start all counters are equal and each block reads its own as the
// base. Every wait is bounded (global timer); past the limit the block records MGM_ERR_TIMEOUT,
// leaves its loops, and the producer waits (bounded) for its copies in flight before exiting;
// the host then clears the error word and the counters.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "hier.cuh"

namespace mgm {

constexpr int SS_CONSUMERS = 512;                          // threads 0..511
constexpr int SS_THREADS = SS_CONSUMERS + 32;              // + the producer warp
constexpr int SS_MAXC = 128;                               // colours a streamed level may have
constexpr int SS_MAXSTAGES = 8;
constexpr int SS_SMEM_BUDGET = 200 * 1024;                 // stage ring
constexpr int SS_QB = 8;                                   // quads a lane gathers at once (FP32; FP64: 4)
constexpr unsigned long long SS_LIMIT_NS = 2000000000ull;  // 2 s a wait

template <class T>
struct StreamArgs {
    const int32_t* lo;
    const int32_t* up;
    const int32_t* sc;
    const T* sv;
    const T* dinv;
    const T* b;
    T* e;
    T* s;
    const int32_t* cchunk;  // B x (C + 1): first chunk of colour c in block k (block-relative)
    const int32_t* recptr;  // B + 1: first chunk of block k
    const int4* rec;        // per chunk {lo[r0], lo[r1], up[r0], up[r1]}
    const int2* rrow;       // per chunk {r0, r1}
    unsigned* prog;         // B
    int* err;
    int C, B, D, ns, sb;     // colours, blocks, dependency radius, stages, stage bytes
    int resid;               // MODE 0: also write s = -U e
    int n;                   // rows of the level
    int eres;                // resident form: bytes of shared memory holding e
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"r"(SS_CONSUMERS) : "memory"); }
// barrier of the consumer threads that also ORs a flag over them (the same answer in every thread)
__device__ __forceinline__ int consumer_sync_or(int v) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(v), "r"(SS_CONSUMERS)
        : "memory");
    return r;
}
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// bounded wait on an mbarrier phase; false if the block is aborting or the wait ran out
__device__ bool wait_phase(uint64_t* bar, unsigned parity, volatile int* abort, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (unsigned it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if ((it & 255) == 0) {
            if (*(volatile int*)err) { *abort = 1; return false; }
            if (gtimer() - t0 > SS_LIMIT_NS) {
                atomicOr(err, MGM_ERR_TIMEOUT);
                *abort = 1;
                return false;
            }
        }
    }
}

template <class T>
struct RowMeta {
    int32_t row = -1, lb = 0, le = 0, ub = 0, ue = 0;
    int4 rc = make_int4(0, 0, 0, 0);  // the chunk's record {lo[r0], lo[r1], up[r0], up[r1]}
    T bv = T(0), dv = T(0);
};

__device__ __forceinline__ float fmaT(float x, float y, float z) { return fmaf(x, y, z); }
__device__ __forceinline__ double fmaT(double x, double y, double z) { return fma(x, y, z); }

// acc += this lane's products of one row held in shared memory: the lane's quads of entries
// (columns cl, values vl) in [l0, l1) of the lower part, then in [u0, u1) of the upper part (cu,
// vu), lane gl of G taking every G-th quad. Gathers of up to QB quads are issued before their
// products; the products are added in the order of the quads.
template <class T, int G, int QB = (sizeof(T) == 4 ? SS_QB : SS_QB / 2)>
__device__ __forceinline__ T row_dot(const int32_t* cl, const T* vl, int32_t l0, int32_t l1, const int32_t* cu,
                                     const T* vu, int32_t u0, int32_t u1, int gl, const T* e, T acc) {
    // (a lane's gathers of up to QB quads are issued before their products)
    const int32_t nql = l1 > l0 + 4 * gl ? (l1 - l0 - 4 * gl + 4 * G - 1) / (4 * G) : 0;
    const int32_t nqu = u1 > u0 + 4 * gl ? (u1 - u0 - 4 * gl + 4 * G - 1) / (4 * G) : 0;
    const int32_t nq = nql + nqu;
    for (int32_t t0 = 0; t0 < nq; t0 += QB) {
        T x[QB][4];
#pragma unroll
        for (int t = 0; t < QB; ++t) {
            const int32_t q = t0 + t;
            if (q < nq) {
                const int32_t* c = q < nql ? cl + l0 + 4 * (gl + G * q) : cu + u0 + 4 * (gl + G * (q - nql));
                const int4 cc = *reinterpret_cast<const int4*>(c);
                x[t][0] = e[cc.x];
                x[t][1] = e[cc.y];
                x[t][2] = e[cc.z];
                x[t][3] = e[cc.w];
            }
        }
#pragma unroll
        for (int t = 0; t < QB; ++t) {
            const int32_t q = t0 + t;
            if (q < nq) {
                const T* v = q < nql ? vl + l0 + 4 * (gl + G * q) : vu + u0 + 4 * (gl + G * (q - nql));
                acc = fmaT(v[0], x[t][0], acc);
                acc = fmaT(v[1], x[t][1], acc);
                acc = fmaT(v[2], x[t][2], acc);
                acc = fmaT(v[3], x[t][3], acc);
            }
        }
    }
    return acc;
}

// RES: the resident form for a level small enough for one block: B = 1, the level's vector e
// lives in shared memory for the whole sweep (gathers from shared memory; loaded first for a full
// sweep, written back at the end), and colours are separated by the consumers' barrier alone.
template <int MODE, class T, int G, bool RES>
__global__ void __launch_bounds__(SS_THREADS, 1) gs_stream_k(const StreamArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + SS_MAXSTAGES;
    int32_t* chs = reinterpret_cast<int32_t*>(empty + SS_MAXSTAGES);  // C + 1 chunk starts
    volatile int* abort_flag = reinterpret_cast<volatile int*>(chs + SS_MAXC + 1);
    unsigned* base_s = reinterpret_cast<unsigned*>(chs + SS_MAXC + 2);
    T* es = reinterpret_cast<T*>(smem + 2048);                              // RES: e of the level
    unsigned char* stages = smem + 2048 + (RES ? a.eres : 0);
    const int tid = threadIdx.x;
    const int k = blockIdx.x;
    const int C = a.C, B = a.B, NS = a.ns;
    constexpr int TS = (int)sizeof(T);
    const int npass = (MODE == 0 && a.resid) ? 2 : 1;

    if (tid < NS) {
        mbar_init(full + tid, 1);
        mbar_init(empty + tid, 1);
    }
    for (int c = tid; c <= C; c += SS_THREADS) chs[c] = a.cchunk[(int64_t)k * (C + 1) + c];
    if (tid == 0) {
        *abort_flag = 0;
        *base_s = *(volatile unsigned*)(a.prog + k);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const unsigned base = *base_s;
    const int32_t rb = a.recptr[k], nrec = a.recptr[k + 1] - rb;

    if (tid >= SS_CONSUMERS) {
        // ------------------------------ producer warp ------------------------------------------
        const int lane = tid & 31;
        const uint64_t pol = evict_first_policy();
        unsigned q = 0;
        bool ok = true;
        for (int pass = 0; pass < npass && ok; ++pass) {
            const bool useL = !(MODE == 0 && pass == 1);
            const bool useU = MODE == 1 || pass == 1;
            for (int32_t r = 0; r < nrec && ok; r += 32) {
                int4 my = make_int4(0, 0, 0, 0);
                if (r + lane < nrec) my = a.rec[rb + r + lane];
                const int cnt = min(32, nrec - r);
                for (int t = 0; t < cnt; ++t) {
                    const int32_t a0 = __shfl_sync(0xffffffffu, my.x, t), a1 = __shfl_sync(0xffffffffu, my.y, t);
                    const int32_t u0 = __shfl_sync(0xffffffffu, my.z, t), u1 = __shfl_sync(0xffffffffu, my.w, t);
                    int go = 1;
                    if (lane == 0) {
                        const int st = (int)(q % (unsigned)NS);
                        const unsigned ph = (q / (unsigned)NS) & 1u;
                        if (!wait_phase(empty + st, ph ^ 1u, abort_flag, a.err)) {
                            go = 0;
                        } else {
                            const unsigned nL = useL ? (unsigned)(a1 - a0) : 0u, nU = useU ? (unsigned)(u1 - u0) : 0u;
                            unsigned char* stg = stages + (size_t)st * a.sb;
                            mbar_expect_tx(full + st, (nL + nU) * (4u + TS));
                            if (nL) {
                                bulk_copy(stg, a.sc + a0, nL * 4u, full + st, pol);
                                bulk_copy(stg + 4u * nL, a.sv + a0, nL * TS, full + st, pol);
                            }
                            if (nU) {
                                unsigned char* su = stg + (4u + TS) * nL;
                                bulk_copy(su, a.sc + u0, nU * 4u, full + st, pol);
                                bulk_copy(su + 4u * nU, a.sv + u0, nU * TS, full + st, pol);
                            }
                        }
                    }
                    go = __shfl_sync(0xffffffffu, go, 0);
                    if (!go) { ok = false; break; }
                    ++q;
                }
            }
        }
        if (!ok && lane == 0) {  // copies in flight land before the block's shared memory is released
            const unsigned first = q > (unsigned)NS ? q - (unsigned)NS : 0u;
            for (unsigned i = first; i < q; ++i) {
                const int st = (int)(i % (unsigned)NS);
                const unsigned long long t0 = gtimer();
                while (!mbar_try_wait(full + st, (i / (unsigned)NS) & 1u))
                    if (gtimer() - t0 > SS_LIMIT_NS) break;
            }
        }
        return;
    }

    // ------------------------------ consumers --------------------------------------------------
    const int ri = tid / G;  // row within the chunk
    const int gl = tid % G;  // lane within the row
    const int wlo = max(0, k - a.D), whi = min(B - 1, k + a.D);
    T* ev = RES ? es : a.e;  // the vector the sweep reads and writes
    if (RES) {  // a full sweep starts from the current e; a first sweep from zero (padding entries
                // of a row point at the row itself with value 0, so its slot must hold a number)
        for (int32_t i = tid; i < a.n; i += SS_CONSUMERS) es[i] = MODE == 1 ? a.e[i] : T(0);
        consumer_sync();
    }

    // row data of chunk ci (block-relative) for a pass
    auto load_meta = [&](int pass, int32_t ci) {
        RowMeta<T> m;
        const int2 rr = a.rrow[rb + ci];
        m.rc = a.rec[rb + ci];
        if (ri < rr.y - rr.x) {
            m.row = rr.x + ri;
            if (!(MODE == 0 && pass == 1)) { m.lb = a.lo[m.row]; m.le = a.lo[m.row + 1]; }
            if (MODE == 1 || pass == 1) { m.ub = a.up[m.row]; m.ue = a.up[m.row + 1]; }
            if (pass == 0) { m.bv = a.b[m.row]; m.dv = a.dinv[m.row]; }
        }
        return m;
    };
    // neighbours' progress >= target (bounded); the acquires make their writes visible to every
    // consumer after the barrier, which also agrees on whether to stop
    auto dep_wait = [&](unsigned target) {
        if (RES) return consumer_sync_or(*abort_flag);
        for (int kk = wlo + tid; kk <= whi; kk += SS_CONSUMERS) {
            unsigned long long t0 = 0;
            for (unsigned it = 0;; ++it) {
                if ((int)(ld_acq(a.prog + kk) - target) >= 0) break;
                if (*abort_flag) break;
                if ((it & 63) == 63) {
                    if (*(volatile int*)a.err) { *abort_flag = 1; break; }
                    const unsigned long long t = gtimer();
                    if (!t0) t0 = t;
                    else if (t - t0 > SS_LIMIT_NS) {
                        atomicOr(a.err, MGM_ERR_TIMEOUT);
                        *abort_flag = 1;
                        break;
                    }
                }
            }
        }
        return consumer_sync_or(*abort_flag);
    };

    unsigned q = 0;  // chunks consumed so far: stage and phase of the next one
    for (int pass = 0; pass < npass; ++pass) {
        const bool useL = !(MODE == 0 && pass == 1);
        const bool useU = MODE == 1 || pass == 1;
        RowMeta<T> m;
        if (nrec > 0) m = load_meta(pass, 0);
        for (int c = 0; c < C; ++c) {
            int stop = 0;
            if (pass == 0) stop = dep_wait(base + (unsigned)c);
            else if (c == 0) stop = dep_wait(base + (unsigned)C);
            if (stop) return;
            for (int32_t ci = chs[c]; ci < chs[c + 1]; ++ci) {
                RowMeta<T> mn;
                if (ci + 1 < nrec) mn = load_meta(pass, ci + 1);
                const int st = (int)(q % (unsigned)NS);
                const bool ready = wait_phase(full + st, (q / (unsigned)NS) & 1u, abort_flag, a.err);
                T acc = T(0);
                if (ready && m.row >= 0) {
                    const unsigned char* stg = stages + (size_t)st * a.sb;
                    const int32_t nL = useL ? m.rc.y - m.rc.x : 0;
                    const int32_t nU = useU ? m.rc.w - m.rc.z : 0;
                    const int32_t* cl = reinterpret_cast<const int32_t*>(stg);
                    const T* vl = reinterpret_cast<const T*>(stg + 4 * nL);
                    const int32_t* cu = reinterpret_cast<const int32_t*>(stg + (4 + TS) * nL);
                    const T* vu = reinterpret_cast<const T*>(stg + (4 + TS) * nL + 4 * nU);
                    acc = row_dot<T, G>(cl, vl, useL ? m.lb - m.rc.x : 0, useL ? m.le - m.rc.x : 0, cu, vu,
                                        useU ? m.ub - m.rc.z : 0, useU ? m.ue - m.rc.z : 0, gl, ev, acc);
                }
#pragma unroll
                for (int o = G / 2; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (ready && m.row >= 0 && gl == 0) {
                    if (pass == 0) ev[m.row] = (m.bv - acc) * m.dv;
                    else a.s[m.row] = -acc;
                }
                consumer_sync();                     // every consumer is done with the stage
                if (tid == 0) mbar_arrive(empty + st);
                ++q;
                m = mn;
            }
            // every row of colour c is written (the chunk loop ends with a barrier)
            if (!RES && pass == 0 && tid == 0) st_rel(a.prog + k, base + (unsigned)c + 1u);
        }
    }
    if (RES) {  // the sweep's e back to the level (every consumer passed the last barrier)
        consumer_sync();
        for (int32_t i = tid; i < a.n; i += SS_CONSUMERS) a.e[i] = es[i];
    }
}

// ------------------------------ set-up of a streamed level ------------------------------------
// split[c * (B + 1) + k] = first solve row of colour c whose RCM index is >= ceil(k n / B)
__global__ void ss_split_k(const int32_t* __restrict__ ord, const int32_t* __restrict__ cptr, int C, int B, int64_t n,
                           int32_t* split) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)C * (B + 1)) return;
    const int c = (int)(t / (B + 1)), kk = (int)(t % (B + 1));
    const int64_t bs = ((int64_t)kk * n + B - 1) / B;
    int32_t lo = cptr[c], hi = cptr[c + 1];
    while (lo < hi) {
        const int32_t md = lo + (hi - lo) / 2;
        if (ord[md] < bs) lo = md + 1; else hi = md;
    }
    split[t] = lo;
}
// Chunks of slice (k, c): consecutive rows, at most rmax rows and cap entries (both parts) each,
// formed greedily from the slice's first row. One thread per slice.
__device__ __forceinline__ int32_t chunk_end(const int32_t* lo, const int32_t* up, int32_t r0, int32_t s1, int rmax,
                                             int32_t cap) {
    const int32_t a0 = lo[r0], u0 = up[r0];
    int32_t r1 = r0;
    while (r1 < s1 && r1 - r0 < rmax && (lo[r1 + 1] - a0) + (up[r1 + 1] - u0) <= cap) ++r1;
    return r1;
}
__global__ void ss_count_k(const int32_t* __restrict__ split, int C, int B, int rmax, int32_t cap,
                           const int32_t* __restrict__ lo, const int32_t* __restrict__ up, int32_t* cnt, int* bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * C) return;
    const int kk = (int)(t / C), c = (int)(t % C);
    const int32_t s0 = split[(int64_t)c * (B + 1) + kk], s1 = split[(int64_t)c * (B + 1) + kk + 1];
    int32_t n = 0;
    for (int32_t r0 = s0; r0 < s1;) {
        const int32_t r1 = chunk_end(lo, up, r0, s1, rmax, cap);
        if (r1 == r0) { atomicOr(bad, 1); break; }  // one row exceeds a stage
        r0 = r1;
        ++n;
    }
    cnt[t] = n;
}
__global__ void ss_fill_k(const int32_t* __restrict__ split, int C, int B, int rmax, int32_t cap,
                          const int32_t* __restrict__ lo, const int32_t* __restrict__ up, const int32_t* __restrict__ off,
                          int4* rec, int2* rrow, int32_t* cchunk) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)B * C) return;
    const int kk = (int)(t / C), c = (int)(t % C);
    const int32_t s0 = split[(int64_t)c * (B + 1) + kk], s1 = split[(int64_t)c * (B + 1) + kk + 1];
    const int32_t kb = off[(int64_t)kk * C];
    int32_t w = off[t];
    cchunk[(int64_t)kk * (C + 1) + c] = w - kb;
    if (c == C - 1) cchunk[(int64_t)kk * (C + 1) + C] = off[t + 1] - kb;
    for (int32_t r0 = s0; r0 < s1;) {
        const int32_t r1 = chunk_end(lo, up, r0, s1, rmax, cap);
        rec[w] = make_int4(lo[r0], lo[r1], up[r0], up[r1]);
        rrow[w] = make_int2(r0, r1);
        ++w;
        r0 = r1;
    }
}
// largest band distance between a row and its columns (canonical CSR in RCM order, columns sorted)
__global__ void ss_radius_k(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n, int B, int* D) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int d = 0;
    if (i < n && rp[i + 1] > rp[i]) {
        const int64_t bi = i * B / n, b0 = (int64_t)ci[rp[i]] * B / n, b1 = (int64_t)ci[rp[i + 1] - 1] * B / n;
        d = (int)max(bi - b0, b1 - bi);
    }
    for (int o = 16; o; o >>= 1) d = max(d, __shfl_xor_sync(0xffffffffu, d, o));
    if ((threadIdx.x & 31) == 0 && d > 0) atomicMax(D, d);
}

template <int MODE, class T, bool RES>
static const void* stream_kernel_g(int G) {
    if (G == 1) return (const void*)gs_stream_k<MODE, T, 1, RES>;
    if (G == 2) return (const void*)gs_stream_k<MODE, T, 2, RES>;
    if (G == 4) return (const void*)gs_stream_k<MODE, T, 4, RES>;
    return (const void*)gs_stream_k<MODE, T, 8, RES>;
}

template <class T>
static const void* stream_kernel(int mode, int G, bool res) {
    if (mode == 0) return res ? stream_kernel_g<0, T, true>(G) : stream_kernel_g<0, T, false>(G);
    return res ? stream_kernel_g<1, T, true>(G) : stream_kernel_g<1, T, false>(G);
}

static int stream_smem(const Level& L) { return 2048 + L.sEres + L.sNS * L.sSB; }

// largest number of co-resident blocks of the streamed kernels with this stage ring (0: none)
template <class T>
static int stream_max_blocks(int smem) {
    int dev = 0, sms = 0, lo = 1 << 30;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int mode = 0; mode < 2; ++mode)
        for (int G : {1, 2, 4, 8}) {
            const void* k = stream_kernel<T>(mode, G, false);
            const void* kr = stream_kernel<T>(mode, G, true);
            CK(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, 2048 + SS_SMEM_BUDGET));
            CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 2048 + SS_SMEM_BUDGET));
            int per = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, SS_THREADS, smem));
            lo = std::min(lo, per);
        }
    return lo * sms;
}

// Tables of a streamed level for B blocks, G lanes a row (chunks of at most 512 / G rows) and NS
// stages. Returns false (level left to per-colour launches) when the level has too many colours
// or a row does not fit one stage.
bool stream_prepare(mgm_hierarchy* H, Level& L, int B, int G, int NS, cudaStream_t s, bool resident) {
    L.stream = 0;
    L.csched = 0;
    const int C = (int)L.cptr.size() - 1;
    if (C < 1 || C > SS_MAXC || L.n < 1 || !(G == 1 || G == 2 || G == 4 || G == 8) || NS < 2 || NS > SS_MAXSTAGES)
        return false;
    const int ts = H->precision == MGM_F32 ? 4 : 8;
    const int eres = resident ? (int)(((int64_t)L.n * ts + 127) / 128 * 128) : 0;
    if (resident && (eres > SS_SMEM_BUDGET / 2 || L.n > INT32_MAX)) return false;
    if (resident) B = 1;
    const int rmax = SS_CONSUMERS / G;
    const int sb = ((SS_SMEM_BUDGET - eres) / NS / 128) * 128;
    const int32_t cap = sb / (4 + ts);
    B = (int)std::max<int64_t>(1, std::min<int64_t>(B, L.n));
    const int smem = 2048 + eres + NS * sb;
    const int maxb = H->precision == MGM_F32 ? stream_max_blocks<float>(smem) : stream_max_blocks<double>(smem);
    if (maxb < B) return false;
    L.split.alloc((size_t)C * (B + 1));
    ss_split_k<<<grid_for((int64_t)C * (B + 1), 256), 256, 0, s>>>(L.ord.get(), L.cptr_dev.get(), C, B, L.n,
                                                                  L.split.get());
    CK_LAUNCH();
    const int64_t nsl = (int64_t)B * C;
    Temp<int32_t> cnt(nsl + 1, s), off(nsl + 1, s);
    Temp<int> mx(2, s);
    CK(cudaMemsetAsync(mx.get(), 0, 2 * sizeof(int), s));
    ss_count_k<<<grid_for(nsl, 128), 128, 0, s>>>(L.split.get(), C, B, rmax, cap, L.lo.get(), L.up.get(), cnt.get(),
                                                  mx.get());
    CK_LAUNCH();
    ss_radius_k<<<grid_for(L.n, 256), 256, 0, s>>>(L.rp.get(), L.ci.get(), L.n, B, mx.get() + 1);
    CK_LAUNCH();
    exclusive_scan_i32(cnt.get(), off.get(), nsl, s);
    int hm[2];
    to_host(hm, mx.get(), 2, s);
    if (hm[0]) return false;
    const int32_t total = read1(off.get() + nsl, s);
    L.rec.alloc(std::max(1, total));
    L.rrow.alloc(std::max(1, total));
    L.cchunk.alloc((size_t)B * (C + 1));
    ss_fill_k<<<grid_for(nsl, 128), 128, 0, s>>>(L.split.get(), C, B, rmax, cap, L.lo.get(), L.up.get(), off.get(),
                                                 L.rec.get(), L.rrow.get(), L.cchunk.get());
    CK_LAUNCH();
    std::vector<int32_t> ho(nsl + 1), hp(B + 1);
    to_host(ho.data(), off.get(), nsl + 1, s);
    for (int k = 0; k <= B; ++k) hp[k] = ho[(size_t)k * C];
    L.recptr.alloc(B + 1);
    CK(cudaMemcpyAsync(L.recptr.get(), hp.data(), sizeof(int32_t) * (B + 1), cudaMemcpyHostToDevice, s));
    L.prog.alloc(B);
    CK(cudaMemsetAsync(L.prog.get(), 0, sizeof(unsigned) * B, s));
    L.sB = B;
    L.sG = G;
    L.sD = hm[1];
    L.sNS = NS;
    L.sSB = sb;
    L.sEres = eres;
    L.stream = 1;
    return true;
}

// the co-resident block count of the streamed kernels (one block an SM)
int stream_blocks_limit(mgm_hierarchy* H) {
    return H->precision == MGM_F32 ? stream_max_blocks<float>(2048 + SS_SMEM_BUDGET)
                                   : stream_max_blocks<double>(2048 + SS_SMEM_BUDGET);
}

template <class T>
void stream_sweep(mgm_hierarchy* H, Level& L, int mode, bool resid, cudaStream_t s) {
    StreamArgs<T> a;
    a.lo = L.lo.get();
    a.up = L.up.get();
    a.sc = L.sc.get();
    if constexpr (sizeof(T) == 4) {
        a.sv = L.sv32.get(); a.dinv = L.dinv32.get(); a.b = L.b32.get(); a.e = L.e32.get(); a.s = L.s32.get();
    } else {
        a.sv = L.sv64.get(); a.dinv = L.dinv64.get(); a.b = L.b64.get(); a.e = L.e64.get(); a.s = L.s64.get();
    }
    a.cchunk = L.cchunk.get();
    a.recptr = L.recptr.get();
    a.rec = L.rec.get();
    a.rrow = L.rrow.get();
    a.prog = L.prog.get();
    a.err = H->err.get();
    a.C = (int)L.cptr.size() - 1;
    a.B = L.sB;
    a.D = L.sD;
    a.ns = L.sNS;
    a.sb = L.sSB;
    a.resid = resid ? 1 : 0;
    a.n = (int)L.n;
    a.eres = L.sEres;
    void* args[] = {(void*)&a};
    if (L.sEres) {  // one block: an ordinary launch
        CK(cudaLaunchKernel(stream_kernel<T>(mode, L.sG, true), dim3(1), dim3(SS_THREADS), args,
                            (size_t)stream_smem(L), s));
    } else {
        CK(cudaLaunchCooperativeKernel(stream_kernel<T>(mode, L.sG, false), dim3(L.sB), dim3(SS_THREADS), args,
                                       (size_t)stream_smem(L), s));
    }
    CK_LAUNCH();
}
template void stream_sweep<float>(mgm_hierarchy*, Level&, int, bool, cudaStream_t);
template void stream_sweep<double>(mgm_hierarchy*, Level&, int, bool, cudaStream_t);

// after a timeout the counters of the streamed levels no longer agree: start them again at zero
void stream_reset(mgm_hierarchy* H, cudaStream_t s) {
    for (auto& L : H->lv)
        if (L.stream) CK(cudaMemsetAsync(L.prog.get(), 0, sizeof(unsigned) * L.sB, s));
}

// ------------------------------ per-colour launches staged through shared memory -------------
// One kernel per colour as in the plain schedule, but each block owns one band's slice of the
// colour (the split table above), and before the programmatic-launch wait it copies the slice's
// columns and values into shared memory with cp.async.bulk and loads its rows' static data. The
// next colour's kernel is allowed to start as soon as every block of this one has started, so its
// blocks, where they fit beside this kernel's, fetch their slices while this colour computes; after
// the wait only the gathers of the vector remain. b is read after the wait (the kernel that writes
// it may still be running before it). MODE 0: lower parts (first sweep from zero); MODE 1: both.
constexpr int CS_THREADS = 256;
constexpr int CS_QB = 4;  // quads a lane gathers at once (FP64: 2)

template <class T>
struct ColourArgs {
    const int32_t* lo;
    const int32_t* up;
    const int32_t* sc;
    const T* sv;
    const T* dinv;
    const T* b;
    T* e;
    const int32_t* split;  // this colour's row of the split table: B + 1 slice bounds
    const int4* sl;        // this colour's slices: {lo[r0], lo[r1], up[r0], up[r1]} of each block
    int* err;
};

template <int MODE, class T, int G>
__global__ void __launch_bounds__(CS_THREADS, 4) gs_colour_k(const ColourArgs<T> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ int4 rg;  // {lo[r0], lo[r1], up[r0], up[r1]}
    pdl_trigger();
    const int tid = threadIdx.x;
    const int32_t r0 = a.split[blockIdx.x], r1 = a.split[blockIdx.x + 1];
    if (r0 >= r1) return;
    constexpr int TS = (int)sizeof(T);
    if (tid == 0) {
        int4 v = a.sl[blockIdx.x];
        if (MODE == 0) v.z = v.w = 0;
        rg = v;
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const unsigned nL = (unsigned)(v.y - v.x), nU = (unsigned)(v.w - v.z);
        const uint64_t pol = evict_first_policy();
        mbar_expect_tx(&bar, (nL + nU) * (4u + TS));
        if (nL) {
            bulk_copy(smem, a.sc + v.x, nL * 4u, &bar, pol);
            bulk_copy(smem + 4u * nL, a.sv + v.x, nL * TS, &bar, pol);
        }
        if (nU) {
            bulk_copy(smem + (4u + TS) * nL, a.sc + v.z, nU * 4u, &bar, pol);
            bulk_copy(smem + (4u + TS) * nL + 4u * nU, a.sv + v.z, nU * TS, &bar, pol);
        }
    }
    // this thread's first row: its static data (row starts, diagonal inverse) before the wait
    const int rpp = CS_THREADS / G;  // rows a pass
    const int gl = tid % G;
    int32_t row = r0 + tid / G;
    int32_t lb = 0, le = 0, ub = 0, ue = 0;
    T dv = T(0);
    if (row < r1) {
        lb = a.lo[row];
        le = a.lo[row + 1];
        if (MODE == 1) { ub = a.up[row]; ue = a.up[row + 1]; }
        dv = a.dinv[row];
    }
    __syncthreads();
    const int4 v = rg;
    const int32_t nL = v.y - v.x, nU = v.w - v.z;
    const int32_t* cl = reinterpret_cast<const int32_t*>(smem);
    const T* vl = reinterpret_cast<const T*>(smem + 4 * nL);
    const int32_t* cu = reinterpret_cast<const int32_t*>(smem + (4 + TS) * nL);
    const T* vu = reinterpret_cast<const T*>(smem + (4 + TS) * nL + 4 * nU);
    pdl_wait();
    // the slice's entries have landed (bounded wait; a timeout abandons the block's rows)
    bool ready = mbar_try_wait(&bar, 0);
    if (!ready) {
        const unsigned long long t0 = gtimer();
        while (!(ready = mbar_try_wait(&bar, 0)))
            if (gtimer() - t0 > SS_LIMIT_NS) { if (gl == 0) atomicOr(a.err, MGM_ERR_TIMEOUT); break; }
    }
    if (__syncthreads_or(!ready)) {  // copies still in flight land before the block exits
        if (tid == 0) {
            const unsigned long long t0 = gtimer();
            while (!mbar_try_wait(&bar, 0) && gtimer() - t0 < SS_LIMIT_NS) {}
        }
        __syncthreads();
        return;
    }
    constexpr int QB = sizeof(T) == 4 ? CS_QB : CS_QB / 2;
    for (int32_t base = r0; base < r1; base += rpp, row += rpp) {  // (uniform over the block: shuffles below)
        const bool act = row < r1;
        if (base > r0 && act) {  // rows of later passes
            lb = a.lo[row];
            le = a.lo[row + 1];
            if (MODE == 1) { ub = a.up[row]; ue = a.up[row + 1]; }
            dv = a.dinv[row];
        }
        T acc = T(0), bv = T(0);
        if (act) {
            bv = a.b[row];
            acc = row_dot<T, G, QB>(cl, vl, lb - v.x, le - v.x, cu, vu, MODE == 1 ? ub - v.z : 0,
                                    MODE == 1 ? ue - v.z : 0, gl, a.e, acc);
        }
#pragma unroll
        for (int o = G / 2; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (act && gl == 0) a.e[row] = (bv - acc) * dv;
    }
}

template <int MODE, class T>
static const void* colour_kernel_g(int G) {
    if (G == 1) return (const void*)gs_colour_k<MODE, T, 1>;
    if (G == 2) return (const void*)gs_colour_k<MODE, T, 2>;
    if (G == 4) return (const void*)gs_colour_k<MODE, T, 4>;
    return (const void*)gs_colour_k<MODE, T, 8>;
}
template <class T>
static const void* colour_kernel(int mode, int G) {
    return mode == 0 ? colour_kernel_g<0, T>(G) : colour_kernel_g<1, T>(G);
}

// slice table of the staged schedule: {lo[r0], lo[r1], up[r0], up[r1]} of colour c's rows in block
// k, and the largest slice of each colour: lower entries (x) and lower + upper entries (y)
__global__ void cs_slices_k(const int32_t* __restrict__ split, int C, int B, const int32_t* __restrict__ lo,
                            const int32_t* __restrict__ up, int4* sl, int2* mx) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)C * B) return;
    const int c = (int)(t / B), k = (int)(t % B);
    const int32_t s0 = split[(int64_t)c * (B + 1) + k], s1 = split[(int64_t)c * (B + 1) + k + 1];
    const int4 v = make_int4(lo[s0], lo[s1], up[s0], up[s1]);
    sl[t] = v;
    atomicMax(&mx[c].x, v.y - v.x);
    atomicMax(&mx[c].y, v.y - v.x + v.w - v.z);
}

// Tables of the staged per-colour schedule for B bands and G lanes a row. False when some slice
// does not fit the largest shared-memory allocation of a block.
bool colour_prepare(mgm_hierarchy* H, Level& L, int B, int G, cudaStream_t s) {
    L.stream = 0;
    L.csched = 0;
    const int C = (int)L.cptr.size() - 1;
    if (C < 1 || L.n < 1 || !(G == 1 || G == 2 || G == 4 || G == 8) || B < 1) return false;
    const int ts = H->precision == MGM_F32 ? 4 : 8;
    B = (int)std::max<int64_t>(1, std::min<int64_t>(B, L.n));
    L.split.alloc((size_t)C * (B + 1));
    ss_split_k<<<grid_for((int64_t)C * (B + 1), 256), 256, 0, s>>>(L.ord.get(), L.cptr_dev.get(), C, B, L.n,
                                                                  L.split.get());
    CK_LAUNCH();
    Temp<int2> mx(C, s);
    CK(cudaMemsetAsync(mx.get(), 0, sizeof(int2) * C, s));
    L.cslice.alloc((size_t)C * B);
    cs_slices_k<<<grid_for((int64_t)C * B, 256), 256, 0, s>>>(L.split.get(), C, B, L.lo.get(), L.up.get(),
                                                             L.cslice.get(), mx.get());
    CK_LAUNCH();
    std::vector<int2> h(C);
    to_host(h.data(), mx.get(), C, s);
    int dev = 0, optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int limit = optin - 1024;
    L.csm0.assign(C, 0);
    L.csm1.assign(C, 0);
    for (int c = 0; c < C; ++c) {
        L.csm0[c] = (int)std::max<int64_t>(16, (int64_t)h[c].x * (4 + ts));
        L.csm1[c] = (int)std::max<int64_t>(16, (int64_t)h[c].y * (4 + ts));
        if (L.csm1[c] > limit) return false;
    }
    {   // the kernels' shared-memory limit, once per device and precision for the process
        static std::mutex mu;
        static std::map<std::pair<int, int>, bool> done;
        std::lock_guard<std::mutex> lk(mu);
        bool& d = done[{dev, H->precision}];
        if (!d) {
            for (int mode = 0; mode < 2; ++mode)
                for (int gi = 0; gi < 4; ++gi) {
                    const void* k = H->precision == MGM_F32 ? colour_kernel<float>(mode, 1 << gi)
                                                            : colour_kernel<double>(mode, 1 << gi);
                    CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, limit));
                }
            d = true;
        }
    }
    L.sB = B;
    L.sG = G;
    L.csched = 1;
    return true;
}

template <class T>
void colour_sweep(mgm_hierarchy* H, Level& L, int mode, cudaStream_t s) {
    ColourArgs<T> a;
    a.lo = L.lo.get();
    a.up = L.up.get();
    a.sc = L.sc.get();
    if constexpr (sizeof(T) == 4) {
        a.sv = L.sv32.get(); a.dinv = L.dinv32.get(); a.b = L.b32.get(); a.e = L.e32.get();
    } else {
        a.sv = L.sv64.get(); a.dinv = L.dinv64.get(); a.b = L.b64.get(); a.e = L.e64.get();
    }
    a.err = H->err.get();
    const int C = (int)L.cptr.size() - 1;
    for (int c = 0; c < C; ++c) {
        if (L.cptr[c + 1] == L.cptr[c]) continue;
        a.split = L.split.get() + (int64_t)c * (L.sB + 1);
        a.sl = L.cslice.get() + (int64_t)c * L.sB;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(L.sB);
        cfg.blockDim = dim3(CS_THREADS);
        cfg.dynamicSmemBytes = (size_t)(mode == 0 ? L.csm0[c] : L.csm1[c]);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = pdl_off() ? 0 : 1;
        void* args[] = {(void*)&a};
        CK(cudaLaunchKernelExC(&cfg, colour_kernel<T>(mode, L.sG), args));
        CK_LAUNCH();
    }
}
template void colour_sweep<float>(mgm_hierarchy*, Level&, int, cudaStream_t);
template void colour_sweep<double>(mgm_hierarchy*, Level&, int, cudaStream_t);

// ------------------------------ schedules and the autotuner ----------------------------------
void sweep_config_get(const mgm_hierarchy* H, int j, mgm_sweep_config* out) {
    REQUIRE(H && out && j >= 0 && j < H->p, "bad argument");
    const Level& L = H->lv[j];
    out->kind = L.csched ? MGM_SCHEDULE_COLOUR
                         : (!L.stream ? MGM_SCHEDULE_LAUNCH : (L.sEres ? MGM_SCHEDULE_RESIDENT : MGM_SCHEDULE_STREAM));
    out->blocks = (L.stream || L.csched) ? L.sB : 0;
    out->lanes = (L.stream || L.csched) ? L.sG : 0;
    out->stages = L.stream ? L.sNS : 0;
    out->ms = L.tuned_ms;
}

static void apply_config(mgm_hierarchy* H, Level& L, const mgm_sweep_config& c, cudaStream_t s) {
    L.csched = 0;
    if (c.kind == MGM_SCHEDULE_STREAM || c.kind == MGM_SCHEDULE_RESIDENT) {
        if (!stream_prepare(H, L, c.blocks, c.lanes, c.stages, s, c.kind == MGM_SCHEDULE_RESIDENT))
            fail(MGM_ERR_UNSUPPORTED, "streamed schedule does not fit this level (colours, row length, blocks or size)");
    } else if (c.kind == MGM_SCHEDULE_COLOUR) {
        if (!colour_prepare(H, L, c.blocks, c.lanes, s))
            fail(MGM_ERR_UNSUPPORTED, "staged per-colour schedule: a slice does not fit shared memory");
    } else {
        L.stream = 0;
    }
}

void sweep_config_set(mgm_hierarchy* H, int j, const mgm_sweep_config* cfg, cudaStream_t s) {
    REQUIRE(H && cfg && j >= 0 && j + 1 < H->p, "bad argument (level must be smoothed)");
    REQUIRE(H->sweep_mode == MGM_SWEEP_LAUNCH || H->sweep_mode >= MGM_SWEEP_STREAM,
            "per-level schedules need persistent_sweeps 0, 3, 4 or 5");
    REQUIRE(cfg->kind >= MGM_SCHEDULE_LAUNCH && cfg->kind <= MGM_SCHEDULE_COLOUR, "unknown schedule kind");
    apply_config(H, H->lv[j], *cfg, s);
    H->lv[j].tuned_ms = 0.0f;
    if (H->lv[j].stream || H->lv[j].csched) H->persistent = true;  // the error word of the bounded waits is checked
    invalidate_graphs(H);
    CK(cudaStreamSynchronize(s));
}

// Tuning decisions are kept per level shape for the life of the process (levels of the same
// precision, smoothing counts, size, entries a row and colour count are timed once).
namespace {
using TuneKey = std::tuple<int, int, int, int64_t, int64_t, int64_t, int>;
std::map<TuneKey, mgm_sweep_config> g_tuned;
std::mutex g_tuned_mu;
}  // namespace

// For every smoothed level: time the level's smoothing in a V-cycle (pre-smoothing with its
// residual, post-smoothing) under each candidate schedule -- one launch per colour, or streamed
// with B blocks (the co-resident maximum and its halvings, at least n / 16384 and at most n / 64),
// G = 1, 2 or 4 lanes a row and 2 stages (3 as well at the largest B) -- and keep the fastest.
void autotune(mgm_hierarchy* H, int reps, bool use_cache, cudaStream_t s) {
    REQUIRE(H && reps >= 1, "bad argument");
    REQUIRE(H->sweep_mode == MGM_SWEEP_LAUNCH || H->sweep_mode >= MGM_SWEEP_STREAM,
            "the autotuner chooses among the schedules of persistent_sweeps 0, 3, 4 or 5");
    const int maxb = stream_blocks_limit(H);
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    H->persistent = true;  // candidates include streamed schedules
    for (int j = 0; j + 1 < H->p; ++j) {
        Level& L = H->lv[j];
        const int C = (int)L.cptr.size() - 1;
        const int64_t epr = (L.nlow + L.nupp + L.n / 2) / std::max<int64_t>(1, L.n);
        const int64_t lg = (int64_t)std::log2((double)std::max<int64_t>(1, L.n));
        const int64_t top = L.n >> std::max<int64_t>(0, lg - 3);  // n to 4 significant bits
        const TuneKey key{H->precision, H->nu1, H->nu2, lg, top, epr, (C + 3) / 4};
        if (use_cache) {
            std::lock_guard<std::mutex> lk(g_tuned_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                apply_config(H, L, it->second, s);
                L.tuned_ms = it->second.ms;
                continue;
            }
        }
        mgm_sweep_config best{MGM_SCHEDULE_LAUNCH, 0, 0, 0, 0.0f};
        L.stream = 0;
        L.csched = 0;
        best.ms = time_level_smoothing(H, j, reps, s);
        std::vector<int> bs;
        const int64_t bhi = std::min<int64_t>(maxb, std::max<int64_t>(1, L.n / 64));
        const int64_t blo = std::max<int64_t>(2, L.n / 16384);
        for (int64_t b = bhi; b >= blo && (int)bs.size() < 6; b /= 2) bs.push_back((int)b);
        for (int b : bs)
            for (int g : {1, 2, 4})
                for (int ns : {2, 3}) {
                    if (ns == 3 && b != bs.front()) continue;
                    if (!stream_prepare(H, L, b, g, ns, s)) continue;
                    const float ms = time_level_smoothing(H, j, reps, s);
                    if (ms < best.ms) best = mgm_sweep_config{MGM_SCHEDULE_STREAM, b, g, ns, ms};
                }
        for (int mult : {1, 2, 3, 4})  // staged per-colour launches, 1-4 bands an SM
            for (int g : {1, 2, 4, 8}) {
                const int b = (int)std::min<int64_t>((int64_t)mult * sms, std::max<int64_t>(1, L.n / 32));
                if (mult > 1 && b < (int64_t)mult * sms) continue;
                if (!colour_prepare(H, L, b, g, s)) continue;
                const float ms = time_level_smoothing(H, j, reps, s);
                if (ms < best.ms) best = mgm_sweep_config{MGM_SCHEDULE_COLOUR, b, g, 0, ms};
            }
        for (int g : {1, 2, 4})  // one block with the level's vector in shared memory
            for (int ns : {2, 4}) {
                if (!stream_prepare(H, L, 1, g, ns, s, true)) continue;
                const float ms = time_level_smoothing(H, j, reps, s);
                if (ms < best.ms) best = mgm_sweep_config{MGM_SCHEDULE_RESIDENT, 1, g, ns, ms};
            }
        apply_config(H, L, best, s);
        L.tuned_ms = best.ms;
        if (use_cache) {
            std::lock_guard<std::mutex> lk(g_tuned_mu);
            g_tuned[key] = best;
        }
    }
    invalidate_graphs(H);
    CK(cudaStreamSynchronize(s));
}

}  // namespace mgm

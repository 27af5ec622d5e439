// The coarse tail of the FP32 V-cycle (Alg. 3 on levels t..p-1) in one thread-block-cluster launch.
//
// On the coarse levels every colour of a sweep is a dependent step of a few hundred rows, and as a
// kernel launch each costs the launch chain's latency (about 0.9 us on GB300) plus a round trip to
// L2 for the gathers. Here one cluster of CL CTAs (16, or 8 where 16 cannot be co-scheduled) runs
// the whole sub-cycle from level t down to the coarsest and back:
//   level t..p-2: pre-smoothing sweep from zero (lower parts), residual -U e, restriction;
//   coarsest: e = L_p^-1 b (the explicit FP64 inverse, read from global memory);
//   level p-2..t: interpolation and correction, post-smoothing sweep.
// Every matrix entry, transfer weight and row datum a CTA needs stays in its shared memory for the
// whole launch (one bulk copy of a blob prepared at set-up), and each vector a step gathers from is
// replicated in every CTA's shared memory: a CTA computes its rows of a colour (a contiguous share
// of the colour's rows), writes each new value into all CTAs' copies through distributed shared
// memory, and the cluster barrier (release / acquire) separates the steps. The arithmetic is that
// of the staged per-colour sweep (Alg. 3's forward Gauss-Seidel in the multicolour order); sums of a
// row are in the order of its stored quads.
//
// Every CTA executes the same sequence of cluster barriers whatever happens, so no barrier can wait
// for a CTA that left. The one wait that depends on memory (the blob's bulk copy) is bounded; past
// it the CTA records MGM_ERR_TIMEOUT in the error word and skips its computations, but keeps taking
// part in every barrier.
#include <algorithm>
#include <cstring>
#include <vector>

#include "hier.cuh"

namespace mgm {

constexpr int TL_THREADS = 256;
constexpr int TL_G = 8;                       // lanes a row
constexpr int TL_RPP = TL_THREADS / TL_G;     // rows a pass
constexpr int TL_MAXLEV = 8;                  // tail levels
constexpr int TL_MAXCL = 16;
constexpr int TL_META = 8;                    // ints a row record
constexpr int TL_HDR = 8 + 8 * TL_MAXLEV;     // header ints: 8 global + 8 a level
constexpr unsigned long long TL_LIMIT_NS = 2000000000ull;

// header of a CTA's blob (ints): [0] ent_c, [1] ent_v, [2] rent_c, [3] rent_v (byte offsets in the
// blob); per level li at 8 + 8 li: [0] colour-table offset, [1] row-record offset, [2] own rows,
// [3] interpolation-block offset (per own row: m columns, then m weights)
struct TailArgs {
    const unsigned char* blob;
    unsigned long long stride;
    unsigned bytes[TL_MAXCL];
    int nlev, m, np;
    int n[TL_MAXLEV], C[TL_MAXLEV];
    int ve[TL_MAXLEV], vb[TL_MAXLEV], vs[TL_MAXLEV];  // byte offsets of the replicated vectors
    int bar_off, blob_off;
    const float* b_top;
    float* e_top;
    const double* Ainv;
    int* err;
};

__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cl_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned long long tl_timer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// v into element `loc` of every CTA's copy; lane gl of the row's TL_G lanes writes copies gl, gl + TL_G
__device__ __forceinline__ void bcast(float* loc, float v, int gl, unsigned rank, int CL) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(loc);
    for (int t = gl; t < CL; t += TL_G) {
        if ((unsigned)t == rank) {
            *loc = v;
        } else {
            uint32_t r;
            asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(t));
            asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(r), "f"(v) : "memory");
        }
    }
}

__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = TL_G / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the quads of [b, b + n) (entries in the blob's column / value arrays) of a * x[col],
// lane gl taking quads gl, gl + TL_G, ...
__device__ __forceinline__ float quads_dot(const int* ec, const float* ev, int b, int n, const float* x, int gl,
                                           float acc) {
    for (int q = gl; 4 * q < n; q += TL_G) {
        const int4 c = *reinterpret_cast<const int4*>(ec + b + 4 * q);
        const float4 v = *reinterpret_cast<const float4*>(ev + b + 4 * q);
        acc = fmaf(v.x, x[c.x], acc);
        acc = fmaf(v.y, x[c.y], acc);
        acc = fmaf(v.z, x[c.z], acc);
        acc = fmaf(v.w, x[c.w], acc);
    }
    return acc;
}

__global__ void __launch_bounds__(TL_THREADS) tail_k(const TailArgs a) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int tid = threadIdx.x, gl = tid % TL_G;
    const unsigned rank = cl_rank();
    int CL;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(CL));
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + a.bar_off);
    unsigned char* blob = sm + a.blob_off;
    __shared__ int ok_s;
    if (tid == 0) {
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(a.bytes[rank]) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                (uint32_t)__cvta_generic_to_shared(blob)),
            "l"(a.blob + a.stride * rank), "r"(a.bytes[rank]), "r"(b)
            : "memory");
    }
    // this CTA's copies of the vectors start at zero (e from zero, b and s written before read)
    for (int li = 0; li < a.nlev; ++li) {
        float* e = reinterpret_cast<float*>(sm + a.ve[li]);
        float* b = reinterpret_cast<float*>(sm + a.vb[li]);
        float* s = li + 1 < a.nlev ? reinterpret_cast<float*>(sm + a.vs[li]) : nullptr;
        for (int i = tid; i < a.n[li]; i += TL_THREADS) {
            e[i] = 0.0f;
            b[i] = 0.0f;
            if (s) s[i] = 0.0f;
        }
    }
    // the blob has landed (bounded wait)
    int ok = 1;
    if (tid == 0) {
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
        const unsigned long long t0 = tl_timer();
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(b)
                : "memory");
            if (done) break;
            if (tl_timer() - t0 > TL_LIMIT_NS) {
                ok = 0;
                atomicOr(a.err, MGM_ERR_TIMEOUT);
                break;
            }
        }
        ok_s = ok;
    }
    __syncthreads();
    ok = ok_s;
    const int* hdr = reinterpret_cast<const int*>(blob);
    const int* ec = reinterpret_cast<const int*>(blob + hdr[0]);
    const float* ev = reinterpret_cast<const float*>(blob + hdr[1]);
    const int* rc = reinterpret_cast<const int*>(blob + hdr[2]);
    const float* rv = reinterpret_cast<const float*>(blob + hdr[3]);
    auto meta = [&](int li) { return reinterpret_cast<const int*>(blob + hdr[8 + 8 * li + 1]); };
    auto nown = [&](int li) { return hdr[8 + 8 * li + 2]; };
    auto vec = [&](int off) { return reinterpret_cast<float*>(sm + off); };
    if (ok) {  // the top level's right-hand side, own rows
        const int* M = meta(0);
        for (int r = tid; r < nown(0); r += TL_THREADS) vec(a.vb[0])[M[TL_META * r]] = a.b_top[M[TL_META * r]];
    }
    cl_sync();  // every copy zeroed before any CTA writes into it
    const int last = a.nlev - 1;
    // one sweep of level li over its colours: mode 0 from zero (lower parts), 1 both parts
    auto sweep = [&](int li, int mode) {
        const int* ct = reinterpret_cast<const int*>(blob + hdr[8 + 8 * li]);
        const int* M = meta(li);
        float* e = vec(a.ve[li]);
        const float* b = vec(a.vb[li]);
        for (int c = 0; c < a.C[li]; ++c) {
            if (ok) {
                const int m0 = ct[2 * c], cnt = ct[2 * c + 1];
                for (int base = 0; base < cnt; base += TL_RPP) {  // uniform over the block
                    const int r = base + tid / TL_G;
                    const bool act = r < cnt;
                    float acc = 0.0f, bv = 0.0f, dv = 0.0f;
                    int row = 0;
                    if (act) {
                        const int* R = M + TL_META * (m0 + r);
                        row = R[0];
                        dv = __int_as_float(R[5]);
                        bv = b[row];
                        acc = quads_dot(ec, ev, R[1], R[2], e, gl, acc);
                        if (mode == 1) acc = quads_dot(ec, ev, R[3], R[4], e, gl, acc);
                    }
                    acc = group_sum(acc);
                    if (act) bcast(e + row, (bv - acc) * dv, gl, rank, CL);
                }
            }
            cl_sync();
        }
    };
    // down: pre-smoothing from zero, residual -U e, restriction
    for (int li = 0; li < last; ++li) {
        sweep(li, 0);
        if (ok) {  // s = -U e on the own rows
            const int* M = meta(li);
            const float* e = vec(a.ve[li]);
            float* s = vec(a.vs[li]);
            for (int base = 0; base < nown(li); base += TL_RPP) {
                const int r = base + tid / TL_G;
                const bool act = r < nown(li);
                float acc = 0.0f;
                int row = 0;
                if (act) {
                    const int* R = M + TL_META * r;
                    row = R[0];
                    acc = quads_dot(ec, ev, R[3], R[4], e, gl, acc);
                }
                acc = group_sum(acc);
                if (act) bcast(s + row, -acc, gl, rank, CL);
            }
        }
        cl_sync();
        if (ok) {  // b_{li+1} = R s on the next level's own rows (every copy for the coarsest)
            const int* M = meta(li + 1);
            const float* s = vec(a.vs[li]);
            float* b = vec(a.vb[li + 1]);
            for (int base = 0; base < nown(li + 1); base += TL_RPP) {
                const int r = base + tid / TL_G;
                const bool act = r < nown(li + 1);
                float acc = 0.0f;
                int row = 0;
                if (act) {
                    const int* R = M + TL_META * r;
                    row = R[0];
                    for (int q = gl; q < R[7]; q += TL_G) acc = fmaf(rv[R[6] + q], s[rc[R[6] + q]], acc);
                }
                acc = group_sum(acc);
                if (act) {
                    if (li + 1 == last) bcast(b + row, acc, gl, rank, CL);
                    else if (gl == 0) b[row] = acc;
                }
            }
        }
        cl_sync();
    }
    if (ok) {  // coarsest: e = A^-1 b (FP64 inverse and sums), own rows, into every copy
        const int* M = meta(last);
        const float* b = vec(a.vb[last]);
        float* e = vec(a.ve[last]);
        for (int base = 0; base < nown(last); base += TL_RPP) {
            const int r = base + tid / TL_G;
            const bool act = r < nown(last);
            double acc = 0.0;
            int row = 0;
            if (act) {
                row = M[TL_META * r];
                const double* arow = a.Ainv + (int64_t)row * a.np;
                for (int j = gl; j < a.np; j += TL_G) acc = fma(arow[j], (double)b[j], acc);
            }
#pragma unroll
            for (int o = TL_G / 2; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (act) bcast(e + row, (float)acc, gl, rank, CL);
        }
    }
    cl_sync();
    // up: interpolation and correction, post-smoothing
    for (int li = last - 1; li >= 0; --li) {
        if (ok) {
            const int* M = meta(li);
            const int* pb = reinterpret_cast<const int*>(blob + hdr[8 + 8 * li + 3]);
            const float* ec1 = vec(a.ve[li + 1]);
            float* e = vec(a.ve[li]);
            for (int base = 0; base < nown(li); base += TL_RPP) {
                const int r = base + tid / TL_G;
                const bool act = r < nown(li);
                float acc = 0.0f;
                int row = 0;
                if (act) {
                    row = M[TL_META * r];
                    const int* pc = pb + 2 * a.m * r;
                    const float* pv = reinterpret_cast<const float*>(pc + a.m);
                    for (int t = gl; t < a.m; t += TL_G) acc = fmaf(pv[t], ec1[pc[t]], acc);
                }
                acc = group_sum(acc);
                if (act) bcast(e + row, e[row] + acc, gl, rank, CL);
            }
        }
        cl_sync();
        sweep(li, 1);
    }
    if (ok) {  // the top level's e, own rows
        const int* M = meta(0);
        const float* e = vec(a.ve[0]);
        for (int r = tid; r < nown(0); r += TL_THREADS) a.e_top[M[TL_META * r]] = e[M[TL_META * r]];
    } else if (tid == 0) {  // a copy that outlived the first wait lands before the CTA exits (bounded)
        const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
        const unsigned long long t0 = tl_timer();
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(done)
                : "r"(b)
                : "memory");
            if (done || tl_timer() - t0 > TL_LIMIT_NS) break;
        }
    }
}

// ------------------------------ set-up -----------------------------------------------------------
namespace {
struct HostLevel {  // host copies of a tail level's solve-order data
    int n = 0;
    std::vector<int32_t> lo, up, sc, cptr;
    std::vector<float> sv, dinv;
    std::vector<int32_t> pc;  // interpolation to the next level (smoothed levels)
    std::vector<float> pv;
    std::vector<int32_t> rrp, rci;  // restriction from the previous level into this one (li >= 1)
    std::vector<float> rvv;
};

template <class T>
void fetch(std::vector<T>& h, const T* d, size_t n, cudaStream_t s) {
    h.resize(n);
    if (n) to_host(h.data(), d, n, s);
}

size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }

// FP32 weights rounded to their BF16 values (nearest, ties to even), the numbers the BF16-stored
// transfers of the launch path read
void round_bf16(std::vector<float>& w) {
    for (float& x : w) {
        uint32_t u;
        std::memcpy(&u, &x, 4);
        u = ((u + 0x7fffu + ((u >> 16) & 1u)) >> 16) << 16;
        std::memcpy(&x, &u, 4);
    }
}

// own rows of CTA k: a contiguous share of each colour (smoothed levels) or of all rows (coarsest)
std::vector<int> own_rows(const HostLevel& L, bool smoothed, int k, int CL, std::vector<int>* ctab) {
    std::vector<int> rows;
    if (smoothed) {
        const int C = (int)L.cptr.size() - 1;
        for (int c = 0; c < C; ++c) {
            const int c0 = L.cptr[c], cnt = L.cptr[c + 1] - c0;
            const int r0 = c0 + (int)((int64_t)cnt * k / CL), r1 = c0 + (int)((int64_t)cnt * (k + 1) / CL);
            ctab->push_back((int)rows.size());
            ctab->push_back(r1 - r0);
            for (int r = r0; r < r1; ++r) rows.push_back(r);
        }
    } else {
        const int r0 = (int)((int64_t)L.n * k / CL), r1 = (int)((int64_t)L.n * (k + 1) / CL);
        for (int r = r0; r < r1; ++r) rows.push_back(r);
    }
    return rows;
}

// CTA k's blob for tail levels hl (hl.back() the coarsest) with m interpolation entries a row
std::vector<unsigned char> build_blob(const std::vector<HostLevel>& hl, int m, int k, int CL) {
    const int nlev = (int)hl.size();
    std::vector<int> hdr(TL_HDR, 0);
    std::vector<std::vector<int>> ctab(nlev), meta(nlev), pblk(nlev);
    std::vector<int32_t> ecol, rcol;
    std::vector<float> eval, rval;
    for (int li = 0; li < nlev; ++li) {
        const HostLevel& L = hl[li];
        const bool smoothed = li + 1 < nlev;
        const std::vector<int> rows = own_rows(L, smoothed, k, CL, &ctab[li]);
        for (int row : rows) {
            int rec[TL_META] = {row, 0, 0, 0, 0, 0, 0, 0};
            if (smoothed) {
                rec[1] = (int)ecol.size();
                rec[2] = L.lo[row + 1] - L.lo[row];
                for (int q = L.lo[row]; q < L.lo[row + 1]; ++q) { ecol.push_back(L.sc[q]); eval.push_back(L.sv[q]); }
                rec[3] = (int)ecol.size();
                rec[4] = L.up[row + 1] - L.up[row];
                for (int q = L.up[row]; q < L.up[row + 1]; ++q) { ecol.push_back(L.sc[q]); eval.push_back(L.sv[q]); }
                float d = L.dinv[row];
                std::memcpy(&rec[5], &d, 4);
                for (int t = 0; t < m; ++t) pblk[li].push_back(L.pc[(size_t)row * m + t]);
                for (int t = 0; t < m; ++t) {
                    int bits;
                    std::memcpy(&bits, &L.pv[(size_t)row * m + t], 4);
                    pblk[li].push_back(bits);
                }
            }
            if (li >= 1) {
                rec[6] = (int)rcol.size();
                rec[7] = L.rrp[row + 1] - L.rrp[row];
                for (int q = L.rrp[row]; q < L.rrp[row + 1]; ++q) { rcol.push_back(L.rci[q]); rval.push_back(L.rvv[q]); }
            }
            meta[li].insert(meta[li].end(), rec, rec + TL_META);
        }
    }
    // layout: header | colour tables | row records | interpolation blocks | entries | restriction
    std::vector<unsigned char> out;
    auto put = [&](const void* p, size_t bytes) {
        const size_t off = up16(out.size());
        out.resize(off + up16(bytes), 0);
        if (bytes) std::memcpy(out.data() + off, p, bytes);
        return (int)off;
    };
    put(hdr.data(), hdr.size() * 4);  // placeholder, rewritten below
    for (int li = 0; li < nlev; ++li) {
        hdr[8 + 8 * li + 0] = put(ctab[li].data(), ctab[li].size() * 4);
        hdr[8 + 8 * li + 1] = put(meta[li].data(), meta[li].size() * 4);
        hdr[8 + 8 * li + 2] = (int)(meta[li].size() / TL_META);
        hdr[8 + 8 * li + 3] = put(pblk[li].data(), pblk[li].size() * 4);
    }
    hdr[0] = put(ecol.data(), ecol.size() * 4);
    hdr[1] = put(eval.data(), eval.size() * 4);
    hdr[2] = put(rcol.data(), rcol.size() * 4);
    hdr[3] = put(rval.data(), rval.size() * 4);
    std::memcpy(out.data(), hdr.data(), hdr.size() * 4);
    out.resize(up16(out.size()));
    return out;
}
}  // namespace

// Chooses the tail's top level (the highest level whose vectors and per-CTA data, from there down,
// fit one CTA's shared memory) and builds the CTAs' blobs. FP32 V(1,1)-cycles of unconstrained
// hierarchies only; otherwise (or when nothing fits) the tail stays off.
void tail_prepare(mgm_hierarchy* H, cudaStream_t s) {
    H->tail_top = 0;
    H->tail_cl = 0;
    const int p = H->p;
    if (H->precision != MGM_F32 || H->bordered || H->cycle != MGM_CYCLE_V || H->nu1 != 1 || H->nu2 != 1 || p < 3) return;
    if (H->m > 8) return;
    int dev = 0, optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t limit = (size_t)optin - 1024;  // (the kernel's static shared memory)
    CK(cudaFuncSetAttribute(tail_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit));
    CK(cudaFuncSetAttribute(tail_k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    int CL = 0;
    for (int cl : {16, 8}) {  // the largest cluster that can be resident
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(TL_THREADS);
        cfg.dynamicSmemBytes = limit;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, tail_k, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            nc = 0;
        }
        if (nc >= 1) {
            CL = cl;
            break;
        }
    }
    if (!CL) return;
    // host copies of the coarse levels, coarsest first, while they fit
    for (int t = 1; t + 1 < p; ++t) {
        const int nlev = p - t;
        if (nlev > TL_MAXLEV) continue;
        size_t vbytes = 16;  // mbarrier
        for (int j = t; j < p; ++j) vbytes += up16(4 * (size_t)H->lv[j].n) * (j + 1 < p ? 3 : 2);
        if (vbytes + 16 >= limit) continue;
        std::vector<HostLevel> hl(nlev);
        for (int li = 0; li < nlev; ++li) {
            const int j = t + li;
            Level& L = H->lv[j];
            HostLevel& h = hl[li];
            h.n = (int)L.n;
            if (li + 1 < nlev) {
                fetch(h.lo, L.lo.get(), L.n + 1, s);
                fetch(h.up, L.up.get(), L.n + 1, s);
                fetch(h.sc, L.sc.get(), (size_t)L.snnz, s);
                fetch(h.sv, L.sv32.get(), (size_t)L.snnz, s);
                fetch(h.dinv, L.dinv32.get(), L.n, s);
                h.cptr = L.cptr;
                fetch(h.pc, L.pc.get(), (size_t)L.n * L.pw, s);
                fetch(h.pv, L.pv32.get(), (size_t)L.n * L.pw, s);
                if (H->transfer_bf16) round_bf16(h.pv);
            }
            if (li >= 1) {
                Level& F = H->lv[j - 1];
                fetch(h.rrp, F.r_rp.get(), L.n + 1, s);
                fetch(h.rci, F.r_ci.get(), (size_t)std::max<int64_t>(F.pnnz, 1), s);
                fetch(h.rvv, F.r_v32.get(), (size_t)std::max<int64_t>(F.pnnz, 1), s);
                if (H->transfer_bf16) round_bf16(h.rvv);
            }
        }
        std::vector<std::vector<unsigned char>> blobs(CL);
        size_t maxb = 0;
        for (int k = 0; k < CL; ++k) {
            blobs[k] = build_blob(hl, H->lv[t].pw, k, CL);
            maxb = std::max(maxb, blobs[k].size());
        }
        if (vbytes + maxb > limit || maxb >= (1u << 20)) continue;
        H->tail_stride = maxb;
        H->tail_bytes.assign(CL, 0);
        std::vector<unsigned char> all((size_t)CL * maxb, 0);
        for (int k = 0; k < CL; ++k) {
            std::memcpy(all.data() + (size_t)k * maxb, blobs[k].data(), blobs[k].size());
            H->tail_bytes[k] = (unsigned)blobs[k].size();
        }
        H->tail_blob.alloc(all.size());
        CK(cudaMemcpyAsync(H->tail_blob.get(), all.data(), all.size(), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        H->tail_smem = vbytes + maxb;
        H->tail_cl = CL;
        H->tail_top = t;
        return;
    }
}

void tail_launch(mgm_hierarchy* H, cudaStream_t s) {
    const int t = H->tail_top, p = H->p, nlev = p - t;
    TailArgs a = {};
    a.blob = H->tail_blob.get();
    a.stride = H->tail_stride;
    for (int k = 0; k < H->tail_cl; ++k) a.bytes[k] = H->tail_bytes[k];
    a.nlev = nlev;
    a.m = H->lv[t].pw;
    a.np = (int)H->np;
    int off = 0;
    for (int li = 0; li < nlev; ++li) {
        const Level& L = H->lv[t + li];
        a.n[li] = (int)L.n;
        a.C[li] = li + 1 < nlev ? (int)L.cptr.size() - 1 : 0;
        const int vb = (int)up16(4 * (size_t)L.n);
        a.ve[li] = off; off += vb;
        a.vb[li] = off; off += vb;
        if (li + 1 < nlev) { a.vs[li] = off; off += vb; }
    }
    a.bar_off = off;
    a.blob_off = off + 16;
    a.b_top = H->lv[t].b32.get();
    a.e_top = H->lv[t].e32.get();
    a.Ainv = H->Ainv.get();
    a.err = H->err.get();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(H->tail_cl);
    cfg.blockDim = dim3(TL_THREADS);
    cfg.dynamicSmemBytes = H->tail_smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = H->tail_cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, tail_k, a));
    CK_LAUNCH();
}

}  // namespace mgm

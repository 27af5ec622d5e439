// extern "C" entry points of libmgm (declared in include/mgm.h): argument checks, translation of
// internal failures into status codes, and nothing else.
#include "hier.cuh"

namespace mgm {
void knn_device(const double* data, int64_t nd, const double* query, int64_t nq, int k, int self_first, int32_t* idx_out,
                double* d2_out, cudaStream_t s);
void stencil_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, const mgm_stencil_params* sp,
                     double* w, cudaStream_t s);
void assemble(int64_t N, int n, const int32_t* idx, const double* w, double mu, int poisson, int32_t* rp, int32_t* col,
              double* val, cudaStream_t s);
void build_stencils(const double* xyz, const double* nrm, int64_t N, const mgm_stencil_params* sp, int32_t* idx_out,
                    double* w_out, int32_t* rp, int32_t* col, double* val, cudaStream_t s);
void coarsen(const double* x, int64_t N, int64_t NH, int32_t* keep, cudaStream_t s, double* rmax_out);
int64_t interp(const double* xf, int64_t nf, const double* xc, int64_t nc, int m, int32_t* rp, int32_t* col, double* val,
               cudaStream_t s);
int64_t spgemm_symbolic(int64_t nA, const int32_t* arp, const int32_t* aci, const int32_t* brp, const int32_t* bci,
                        int32_t* crp, cudaStream_t s);
void spgemm_numeric(int64_t nA, const int32_t* arp, const int32_t* aci, const double* av, const int32_t* brp,
                    const int32_t* bci, const double* bv, const int32_t* crp, int32_t* cci, double* cv, cudaStream_t s);
void rcm(int64_t N, const int32_t* rp, const int32_t* ci, int32_t* perm, cudaStream_t s);
void color(int64_t N, const int32_t* rp, const int32_t* ci, uint64_t seed, int32_t* colour, int32_t* ncolors,
           cudaStream_t s);
mgm_hierarchy* setup(const double* xyz, int64_t N, const int32_t* rp, const int32_t* ci, const double* v,
                     const mgm_params* prm, cudaStream_t s);
void vcycle_api(mgm_hierarchy* H, const void* r, void* z, int dtype, cudaStream_t s);
void hierarchy_level(const mgm_hierarchy* H, int j, int32_t* perm, int32_t* keep, double* xyz, int32_t* lrp, int32_t* lci,
                     double* lv, int32_t* prp, int32_t* pci, double* pv, int32_t* colour, cudaStream_t s);
// stencil.cu: first derivatives (heat method)
void gradient_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx, const mgm_stencil_params* sp,
                      double* wx, double* wy, cudaStream_t s);
void surface_gradient(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx, const double* wy,
                      const double* u, double* g, int normalize, cudaStream_t s);
void surface_divergence(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx, const double* wy,
                        const double* eta, double* d, cudaStream_t s);
// learned.cu
void learned_attach(mgm_hierarchy* H, const double* xyz, const double* nrm, const int32_t* idx, const double* w, int n,
                    cudaStream_t s);
void learned_features(mgm_hierarchy* H, const double* r, float* feat, float* rho, cudaStream_t s);
void learned_cycle_residual(mgm_hierarchy* H, const double* r, double* rout, cudaStream_t s);
double learned_loss(mgm_hierarchy* H, const mgm_mlp* M, const double* r, float* grad, cudaStream_t s);
double learned_train_step(mgm_hierarchy* H, mgm_mlp* M, const double* r, float lr, cudaStream_t s);
void learned_enable(mgm_hierarchy* H, const mgm_mlp* M, cudaStream_t s);
void learned_correction(mgm_hierarchy* H, const double* r, double* delta, cudaStream_t s);
mgm_mlp* mlp_create(int n, uint64_t seed);
void mlp_destroy(mgm_mlp* M);
void mlp_get(const mgm_mlp* M, float* W);
void mlp_set(mgm_mlp* M, const float* W);
int64_t mlp_size(int n);
void mlp_forward_api(const mgm_mlp* M, const float* feat, int64_t B, float* out, cudaStream_t s);
void mlp_vjp_api(const mgm_mlp* M, const float* feat, const float* gout, int64_t B, float* grad, cudaStream_t s);
}  // namespace mgm

using namespace mgm;

static inline cudaStream_t S(mgm_stream s) { return reinterpret_cast<cudaStream_t>(s); }

// heavy entry points: run, then trim the scratch pool's cached memory to the cache budget, so a
// call that needed more hands the excess back while the next call of the same size maps nothing
template <class F>
static mgm_status guarded_trim(F&& body) {
    const mgm_status st = guarded(std::forward<F>(body));
    scratch_trim(cache_budget());
    return st;
}

extern "C" {

mgm_status mgm_knn(const double* data, int64_t nd, const double* query, int64_t nq, int k, int self_first,
                   int32_t* idx_out, mgm_stream stream) {
    return guarded_trim([&] {
        REQUIRE(data && query && idx_out, "null array");
        REQUIRE(nd >= 1 && nq >= 0, "sizes out of range");
        knn_device(data, nd, query, nq, k, self_first, idx_out, nullptr, S(stream));
    });
}

mgm_status mgm_stencil_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx,
                               const mgm_stencil_params* sp, double* w_out, mgm_stream stream) {
    return guarded_trim([&] {
        REQUIRE(sp && idx, "null argument");
        REQUIRE(N >= 1 && sp->n >= 1, "sizes out of range");
        validate_index(idx, N * (int64_t)sp->n, N, "stencil indices", S(stream));
        stencil_weights(xyz, nrm, N, idx, sp, w_out, S(stream));
    });
}

mgm_status mgm_assemble(int64_t N, int n, const int32_t* idx, const double* w, double mu, int poisson,
                        int32_t* rowptr_out, int32_t* col_out, double* val_out, mgm_stream stream) {
    return guarded([&] {
        REQUIRE(idx && N >= 1 && n >= 1, "bad argument");
        validate_index(idx, N * (int64_t)n, N, "stencil indices", S(stream));
        assemble(N, n, idx, w, mu, poisson, rowptr_out, col_out, val_out, S(stream));
    });
}

mgm_status mgm_build_stencils(const double* xyz, const double* nrm, int64_t N, const mgm_stencil_params* sp,
                              int32_t* idx_out, double* w_out, int32_t* rowptr_out, int32_t* col_out, double* val_out,
                              mgm_stream stream) {
    return guarded_trim([&] {
        REQUIRE(xyz && nrm && rowptr_out && col_out && val_out, "null array");
        build_stencils(xyz, nrm, N, sp, idx_out, w_out, rowptr_out, col_out, val_out, S(stream));
    });
}

mgm_status mgm_coarsen(const double* xyz, int64_t N_fine, int64_t N_coarse, uint64_t seed, int32_t* keep_out,
                       mgm_stream stream) {
    return guarded_trim([&] {
        REQUIRE(seed == 0, "seed is reserved and must be 0");
        coarsen(xyz, N_fine, N_coarse, keep_out, S(stream), nullptr);
    });
}

mgm_status mgm_interp(const double* xf, int64_t Nf, const double* xc, int64_t Nc, int m, int32_t* rowptr_out,
                      int32_t* col_out, double* val_out, int64_t* nnz_out, mgm_stream stream) {
    return guarded_trim([&] {
        REQUIRE(Nc >= 1, "N_c must be >= 1");
        int64_t nnz = interp(xf, Nf, xc, Nc, m, rowptr_out, col_out, val_out, S(stream));
        if (nnz_out) *nnz_out = nnz;
    });
}

mgm_status mgm_transpose(int64_t nrows, int64_t ncols, const int32_t* rowptr, const int32_t* col, const double* val,
                         int32_t* trowptr, int32_t* tcol, double* tval, mgm_stream stream) {
    return guarded([&] {
        REQUIRE(rowptr && col && trowptr && tcol, "null array");
        REQUIRE(nrows >= 0 && ncols >= 0 && nrows < 0x7fffffff && ncols < 0x7fffffff, "sizes out of range");
        validate_csr(nrows, ncols, rowptr, col, "transpose input", S(stream));
        csr_transpose(nrows, ncols, rowptr, col, val, trowptr, tcol, tval, S(stream));
    });
}

mgm_status mgm_spgemm(int64_t nA, int64_t nB, int64_t ncolsB, const int32_t* a_rowptr, const int32_t* a_col, const double* a_val,
                      const int32_t* b_rowptr, const int32_t* b_col, const double* b_val, int32_t* c_rowptr,
                      int32_t* c_col, double* c_val, int64_t* nnz_out, mgm_stream stream) {
    return guarded([&] {
        REQUIRE(a_rowptr && a_col && b_rowptr && b_col && c_rowptr, "null array");
        REQUIRE(nA >= 0 && nA < 0x7fffffff && nB >= 0 && nB < 0x7fffffff && ncolsB >= 0 && ncolsB < 0x7fffffff,
                "sizes out of range");
        validate_csr(nA, nB, a_rowptr, a_col, "spgemm A", S(stream));
        validate_csr(nB, ncolsB, b_rowptr, b_col, "spgemm B", S(stream));
        if (!c_col) {
            int64_t nnz = spgemm_symbolic(nA, a_rowptr, a_col, b_rowptr, b_col, c_rowptr, S(stream));
            if (nnz_out) *nnz_out = nnz;
        } else {
            REQUIRE(a_val && b_val && c_val, "null value array");
            spgemm_numeric(nA, a_rowptr, a_col, a_val, b_rowptr, b_col, b_val, c_rowptr, c_col, c_val, S(stream));
            if (nnz_out) *nnz_out = csr_nnz(c_rowptr, nA, S(stream));
        }
    });
}

mgm_status mgm_rcm(int64_t N, const int32_t* rowptr, const int32_t* col, int32_t* perm_out, mgm_stream stream) {
    return guarded([&] {
        REQUIRE(rowptr && col && N >= 1, "bad argument");
        validate_csr(N, N, rowptr, col, "rcm input", S(stream));
        rcm(N, rowptr, col, perm_out, S(stream));
    });
}

mgm_status mgm_color(int64_t N, const int32_t* rowptr, const int32_t* col, uint64_t seed, int32_t* color_out,
                     int32_t* ncolors_out, mgm_stream stream) {
    return guarded([&] {
        REQUIRE(ncolors_out && rowptr && col && N >= 1, "bad argument");
        validate_csr(N, N, rowptr, col, "colouring input", S(stream));
        color(N, rowptr, col, seed, color_out, ncolors_out, S(stream));
    });
}

mgm_status mgm_setup(const double* xyz, int64_t N, const int32_t* rowptr, const int32_t* col, const double* val,
                     const mgm_params* params, mgm_hierarchy** out, mgm_stream stream) {
    return guarded_trim([&] {
        REQUIRE(out, "null output handle");
        *out = nullptr;
        REQUIRE(rowptr && col && N >= 1, "bad argument");
        validate_csr(N, N, rowptr, col, "operator", S(stream));
        *out = setup(xyz, N, rowptr, col, val, params, S(stream));
    });
}

mgm_status mgm_vcycle(mgm_hierarchy* H, const void* r, void* z, int dtype, mgm_stream stream) {
    return guarded([&] { vcycle_api(H, r, z, dtype, S(stream)); });
}

mgm_status mgm_solve(mgm_hierarchy* H, const double* f, double* u, const mgm_solve_params* sp, mgm_solve_info* info,
                     mgm_stream stream) {
    return guarded([&] { solve(H, f, u, sp, info, S(stream)); });
}

mgm_status mgm_solve_multi(mgm_hierarchy* H, int nrhs, const double* F, double* U, const mgm_solve_params* sp,
                           mgm_solve_info* info, mgm_stream stream) {
    return guarded([&] { solve_multi(H, nrhs, F, U, sp, info, S(stream)); });
}

mgm_status mgm_solve_batched(mgm_hierarchy* const* H, int nprob, const double* const* F, double* const* U, int nrhs,
                             const mgm_solve_params* sp, mgm_solve_info* info, mgm_status* status_out,
                             mgm_stream stream) {
    return guarded_trim([&] { solve_batched(H, nprob, F, U, nrhs, sp, info, status_out, S(stream)); });
}

mgm_status mgm_eigs(mgm_hierarchy* H, int nev, int b, int s, int max_cycles, double tol, const mgm_solve_params* sp,
                    uint64_t seed, double* lam_re, double* lam_im, double* resid, double* evec, int* nconv,
                    int* nsolves, mgm_stream stream) {
    return guarded_trim([&] {
        eigs(H, nev, b, s, max_cycles, tol, sp, seed, lam_re, lam_im, evec, resid, nconv, nsolves, S(stream));
    });
}

mgm_status mgm_reaction_steps(mgm_hierarchy* Hu, mgm_hierarchy* Hv, int model, const double* prm, double dt, double* u,
                              double* v, int steps, const mgm_solve_params* sp, int* iters_out, mgm_stream stream) {
    return guarded([&] { reaction_steps(Hu, Hv, model, prm, dt, u, v, steps, sp, iters_out, S(stream)); });
}

mgm_status mgm_reaction_rhs(int model, int scheme, int64_t N, const double* u, const double* v, const double* u_prev,
                            const double* v_prev, const double* prm, double dt, double* ru, double* rv,
                            mgm_stream stream) {
    return guarded([&] { reaction_rhs(model, scheme, N, u, v, u_prev, v_prev, prm, dt, ru, rv, S(stream)); });
}

mgm_status mgm_hierarchy_stats_get(const mgm_hierarchy* H, mgm_hierarchy_stats* out) {
    return guarded([&] {
        REQUIRE(H && out, "null argument");
        *out = mgm_hierarchy_stats{};
        out->p = H->p;
        out->precision = H->precision;
        for (int j = 0; j < H->p && j < 16; ++j) {
            out->n[j] = H->lv[j].n;
            out->nnz[j] = H->lv[j].nnz;
            out->ncolors[j] = H->lv[j].ncolors;
        }
        out->device_bytes = H->device_bytes;
    });
}

mgm_status mgm_hierarchy_level(const mgm_hierarchy* H, int j, int32_t* perm, int32_t* keep, double* xyz,
                               int32_t* l_rowptr, int32_t* l_col, double* l_val, int32_t* p_rowptr, int32_t* p_col,
                               double* p_val, int32_t* colour, mgm_stream stream) {
    return guarded([&] {
        hierarchy_level(H, j, perm, keep, xyz, l_rowptr, l_col, l_val, p_rowptr, p_col, p_val, colour, S(stream));
    });
}

mgm_status mgm_hierarchy_pnnz(const mgm_hierarchy* H, int j, int64_t* nnz_out) {
    return guarded([&] {
        REQUIRE(H && nnz_out && j >= 0 && j < H->p, "bad argument");
        *nnz_out = H->lv[j].pnnz;
    });
}

mgm_status mgm_profile(mgm_hierarchy* H, int reps, mgm_profile_info* out, mgm_stream stream) {
    return guarded([&] {
        REQUIRE(H && out && reps >= 1, "bad argument");
        *out = mgm_profile_info{};
        profile_vcycle(H, reps, out, S(stream));
        profile_spmv(H, reps, out, S(stream));
    });
}

mgm_status mgm_vcycle_floor(mgm_hierarchy* H, double chain_us, double gbs, double* floor_ms, double* bytes_ms,
                            double* chain_ms) {
    return guarded([&] {
        REQUIRE(H && floor_ms && chain_us >= 0.0 && gbs > 0.0, "bad argument");
        *floor_ms = vcycle_floor_ms(H, chain_us, gbs, bytes_ms, chain_ms);
    });
}

mgm_status mgm_sweep_config_set(mgm_hierarchy* H, int j, const mgm_sweep_config* cfg, mgm_stream stream) {
    return guarded([&] { sweep_config_set(H, j, cfg, S(stream)); });
}

mgm_status mgm_sweep_config_get(const mgm_hierarchy* H, int j, mgm_sweep_config* out) {
    return guarded([&] { sweep_config_get(H, j, out); });
}

mgm_status mgm_tail_info(const mgm_hierarchy* H, int* top_out, int* cluster_out) {
    return guarded([&] {
        REQUIRE(H && top_out && cluster_out, "bad argument");
        *top_out = H->tail_top;
        *cluster_out = H->tail_cl;
    });
}

mgm_status mgm_level_smoothing_bytes(const mgm_hierarchy* H, int j, int64_t* bytes_out) {
    return guarded([&] {
        REQUIRE(H && bytes_out && j >= 0 && j + 1 < H->p, "bad argument");
        *bytes_out = level_smoothing_bytes(H, j);
    });
}

mgm_status mgm_profile_level(mgm_hierarchy* H, int j, int reps, float* ms_out, mgm_stream stream) {
    return guarded([&] {
        REQUIRE(H && ms_out && reps >= 1 && j >= 0 && j + 1 < H->p, "bad argument");
        *ms_out = time_level_smoothing(H, j, reps, S(stream));
    });
}

mgm_status mgm_autotune(mgm_hierarchy* H, int reps, int use_cache, mgm_stream stream) {
    return guarded([&] { autotune(H, reps, use_cache != 0, S(stream)); });
}

// FP64 multiply-add rate: every thread runs 8 independent chains of fused multiply-adds (values
// stay bounded: x <- x * a + b with |a| < 1)
__global__ void fp64_fma_probe_k(double* out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-3 + q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += x[q];
    if (s == 12345.678) out[0] = s;  // keeps the chains live
}

mgm_status mgm_probe_fp64_fma(int reps, double* gflops_out, mgm_stream stream) {
    return guarded([&] {
        REQUIRE(reps >= 1 && gflops_out, "bad argument");
        cudaStream_t s = S(stream);
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        Temp<double> out(1, s);
        const int blocks = sms * 8, threads = 256, iters = 4096;
        fp64_fma_probe_k<<<blocks, threads, 0, s>>>(out.get(), iters, 0.999, 1e-3);  // warm-up
        CK_LAUNCH();
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, s));
        for (int t = 0; t < reps; ++t) {
            fp64_fma_probe_k<<<blocks, threads, 0, s>>>(out.get(), iters, 0.999, 1e-3);
            CK_LAUNCH();
        }
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const double flops = 2.0 * 8.0 * iters * (double)blocks * threads * reps;
        *gflops_out = flops / (ms * 1e-3) / 1e9;
    });
}

// dependent-launch latency: each kernel waits for its predecessor, then block 0 advances a counter
// the predecessor wrote (a real read-after-write dependency between consecutive launches)
__global__ void chain_probe_k(unsigned* p) {
    pdl_trigger();
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) p[0] += 1u;
}

mgm_status mgm_probe_launch_chain(int blocks, int threads, int launches, int pdl, int reps, double* us_out,
                                  mgm_stream stream) {
    return guarded([&] {
        REQUIRE(blocks >= 1 && threads >= 32 && threads <= 1024 && launches >= 1 && launches <= 100000 &&
                    reps >= 1 && us_out, "bad argument");
        cudaStream_t s = S(stream);
        Temp<unsigned> cnt(1, s);
        CK(cudaMemsetAsync(cnt.get(), 0, sizeof(unsigned), s));
        cudaStream_t c = nullptr;
        CK(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        auto cleanup = [&] {
            if (ge) cudaGraphExecDestroy(ge);
            if (g) cudaGraphDestroy(g);
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            cudaStreamDestroy(c);
        };
        try {
            const bool was = pdl_off();
            pdl_off() = pdl == 0;
            CK(cudaStreamBeginCapture(c, cudaStreamCaptureModeThreadLocal));
            try {
                for (int k = 0; k < launches; ++k) launch_pdl(chain_probe_k, (unsigned)blocks, (unsigned)threads, c, cnt.get());
            } catch (...) {
                pdl_off() = was;
                cudaGraph_t junk = nullptr;
                cudaStreamEndCapture(c, &junk);
                if (junk) cudaGraphDestroy(junk);
                throw;
            }
            pdl_off() = was;
            CK(cudaStreamEndCapture(c, &g));
            CK(cudaGraphInstantiate(&ge, g, 0));
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaGraphLaunch(ge, s));  // warm-up
            CK(cudaEventRecord(e0, s));
            for (int t = 0; t < reps; ++t) CK(cudaGraphLaunch(ge, s));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            note_launch((int64_t)launches * (reps + 1));
            *us_out = 1e3 * (double)ms / ((double)reps * launches);
        } catch (...) {
            cleanup();
            throw;
        }
        cleanup();
    });
}

int64_t mgm_kernel_launches(void) { return launches(); }

mgm_status mgm_check_bounded_wait(int nblocks, int64_t spin_limit, int* status_out, mgm_stream stream) {
    return guarded([&] {
        REQUIRE(status_out && nblocks >= 1 && nblocks <= 152 && spin_limit >= 1, "bad argument");
        int e = barrier_timeout_probe(nblocks, (unsigned long long)spin_limit, S(stream));
        *status_out = e ? MGM_ERR_TIMEOUT : MGM_OK;
    });
}

void mgm_destroy(mgm_hierarchy* H) {
    if (!H) return;
    cudaDeviceSynchronize();
    {  // the hierarchy's blocks stay mapped for the next one, within the cache budget
        BufCacheScope keep;
        delete H;
    }
    buf_cache_trim(cache_budget());
}

void mgm_release_cached_memory(void) { release_cached_memory(); }

const char* mgm_status_string(mgm_status s) {
    switch (s) {
        case MGM_OK: return "MGM_OK";
        case MGM_ERR_INVALID_ARG: return "MGM_ERR_INVALID_ARG";
        case MGM_ERR_SINGULAR_STENCIL: return "MGM_ERR_SINGULAR_STENCIL";
        case MGM_ERR_NOT_CONVERGED: return "MGM_ERR_NOT_CONVERGED";
        case MGM_ERR_BREAKDOWN: return "MGM_ERR_BREAKDOWN";
        case MGM_ERR_TIMEOUT: return "MGM_ERR_TIMEOUT";
        case MGM_ERR_CUDA: return "MGM_ERR_CUDA";
        case MGM_ERR_OOM: return "MGM_ERR_OOM";
        case MGM_ERR_UNSUPPORTED: return "MGM_ERR_UNSUPPORTED";
    }
    return "unknown status";
}

const char* mgm_last_error_message(void) { return error_message(); }
int64_t mgm_last_error_row(void) { return bad_row(); }
int64_t mgm_last_weights_fp64_rows(void) { return fp64_rows(); }

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// learned correction
// ---------------------------------------------------------------------------------------------
int64_t mgm_mlp_size(int n) { return mlp_size(n); }

mgm_status mgm_mlp_create(int n, uint64_t seed, mgm_mlp** out) {
    return guarded([&] {
        REQUIRE(out, "null argument");
        *out = nullptr;
        *out = mlp_create(n, seed);
    });
}

void mgm_mlp_destroy(mgm_mlp* M) {
    if (!M) return;
    cudaDeviceSynchronize();
    mlp_destroy(M);
}

mgm_status mgm_mlp_get(const mgm_mlp* M, float* W_host) { return guarded([&] { mlp_get(M, W_host); }); }
mgm_status mgm_mlp_set(mgm_mlp* M, const float* W_host) { return guarded([&] { mlp_set(M, W_host); }); }

mgm_status mgm_mlp_forward(const mgm_mlp* M, const float* feat, int64_t B, float* out, mgm_stream stream) {
    return guarded([&] { mlp_forward_api(M, feat, B, out, S(stream)); });
}

mgm_status mgm_mlp_vjp(const mgm_mlp* M, const float* feat, const float* gout, int64_t B, float* grad, mgm_stream stream) {
    return guarded([&] { mlp_vjp_api(M, feat, gout, B, grad, S(stream)); });
}

mgm_status mgm_learned_attach(mgm_hierarchy* H, const double* xyz, const double* nrm, const int32_t* idx, const double* w,
                              int n, mgm_stream stream) {
    return guarded([&] { learned_attach(H, xyz, nrm, idx, w, n, S(stream)); });
}

mgm_status mgm_learned_features(mgm_hierarchy* H, const double* r, float* feat, float* rho, mgm_stream stream) {
    return guarded([&] { learned_features(H, r, feat, rho, S(stream)); });
}

mgm_status mgm_learned_cycle_residual(mgm_hierarchy* H, const double* r, double* r_out, mgm_stream stream) {
    return guarded([&] { learned_cycle_residual(H, r, r_out, S(stream)); });
}

mgm_status mgm_learned_loss(mgm_hierarchy* H, const mgm_mlp* M, const double* r, double* loss, float* grad,
                            mgm_stream stream) {
    return guarded([&] {
        REQUIRE(loss, "null argument");
        *loss = learned_loss(H, M, r, grad, S(stream));
    });
}

mgm_status mgm_learned_train_step(mgm_hierarchy* H, mgm_mlp* M, const double* r, float lr, double* loss,
                                  mgm_stream stream) {
    return guarded([&] {
        double J = learned_train_step(H, M, r, lr, S(stream));
        if (loss) *loss = J;
    });
}

mgm_status mgm_learned_enable(mgm_hierarchy* H, const mgm_mlp* M, mgm_stream stream) {
    return guarded([&] { learned_enable(H, M, S(stream)); });
}

mgm_status mgm_learned_correction(mgm_hierarchy* H, const double* r, double* delta, mgm_stream stream) {
    return guarded([&] { learned_correction(H, r, delta, S(stream)); });
}

mgm_status mgm_learned_info(const mgm_hierarchy* H, int* enabled, int64_t* fallbacks) {
    return guarded([&] {
        REQUIRE(H, "null hierarchy");
        if (enabled) *enabled = H->learned ? 1 : 0;
        if (fallbacks) *fallbacks = H->learned_fallbacks;
    });
}

// ---------------------------------------------------------------------------------------------
// surface gradient and divergence (heat method)
// ---------------------------------------------------------------------------------------------
mgm_status mgm_gradient_weights(const double* xyz, const double* nrm, int64_t N, const int32_t* idx,
                                const mgm_stencil_params* sp, double* wx_out, double* wy_out, mgm_stream stream) {
    return guarded_trim([&] {
        REQUIRE(sp && idx, "null argument");
        validate_index(idx, N * (int64_t)sp->n, N, "stencil indices", S(stream));
        gradient_weights(xyz, nrm, N, idx, sp, wx_out, wy_out, S(stream));
    });
}

mgm_status mgm_surface_gradient(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx,
                                const double* wy, const double* u, double* g_out, int normalize, mgm_stream stream) {
    return guarded([&] { surface_gradient(nrm, N, idx, n, wx, wy, u, g_out, normalize, S(stream)); });
}

mgm_status mgm_surface_divergence(const double* nrm, int64_t N, const int32_t* idx, int n, const double* wx,
                                  const double* wy, const double* eta, double* div_out, mgm_stream stream) {
    return guarded([&] { surface_divergence(nrm, N, idx, n, wx, wy, eta, div_out, S(stream)); });
}

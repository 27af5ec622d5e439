// Internal layout of an MGM hierarchy on the device (not part of the public ABI).
//
// Every level j keeps its canonical data in its own RCM order (paper Alg. 2): points, the FP64
// operator L_j (CSR), the RCM permutation, the coarsening survivors and the interpolation I_{j+1}^j.
// Levels that are smoothed (all but the coarsest) also carry a "solve order": rows grouped by
// colour (RCM order inside a colour), so that one multicolour Gauss-Seidel step is a contiguous
// row range. In that order the off-diagonal entries are stored in two regions of the same arrays:
//   [ lower parts of rows 0..n-1 (columns of earlier colours) | upper parts of rows 0..n-1 ]
// each row's part padded to a multiple of 4 entries with (own row, 0), so that every part starts
// 16-byte aligned (int4 / float4 loads) and a range of rows' parts is one contiguous block (one
// bulk copy). The diagonal is kept apart (value and inverse). Interpolation rows are stored as fixed-width ELL (width m) and the
// restriction as CSR, both indexed in the solve orders of the two levels.
#pragma once
#include <vector>

#include "common.cuh"

namespace mgm {

struct Level {
    int64_t n = 0, nnz = 0;
    // canonical data (RCM order, FP64)
    Buf<double> X;
    Buf<int32_t> rp, ci;
    Buf<double> v;
    Buf<int32_t> perm, keep;
    Buf<int32_t> P_rp, P_ci;
    Buf<double> P_v;
    int64_t pnnz = 0;
    Buf<int32_t> colour;
    int ncolors = 0;
    // solve order
    Buf<int32_t> ord, inv;     // ord[s] = RCM index of solve row s; inv = ord^-1
    std::vector<int32_t> cptr; // host: colour c = solve rows [cptr[c], cptr[c+1])
    Buf<int32_t> cptr_dev;     // the same on the device (persistent sweeps)
    Buf<unsigned> bar;         // grid-barrier counter of this level's persistent sweeps
    Buf<int32_t> gptr;         // dependency-driven sweeps: row groups (<= 4 rows of one colour)
    int32_t ngroups = 0;
    Buf<int> flag;             // per-row ready flags of the current sweep
    Buf<float> eold32;         // e before a full sweep (read for the upper-part columns)
    Buf<double> eold64;
    Buf<int32_t> lo, up;       // row s: lower part [lo[s], lo[s+1]), upper part [up[s], up[s+1]); up[0] = lo[n]
    Buf<int32_t> sc;           // padded columns (solve order of this level)
    Buf<float> sv32, diag32, dinv32;
    Buf<double> sv64, diag64, dinv64;
    int64_t snnz = 0;          // padded entry count (both regions)
    int64_t nl_pad = 0;        // padded entries of the lower region
    // streamed sweeps (gs_stream.cu): B blocks, block k owns the rows whose RCM index lies in its band;
    // split[c * (B + 1) + k] = first solve row of colour c in band k; per block, per colour, its
    // chunks of consecutive rows: rows {r0, r1} (rrow) and entry ranges {lo[r0], lo[r1], up[r0],
    // up[r1]} (rec); cchunk[k * (C + 1) + c] = first chunk of colour c, relative to recptr[k]
    int sB = 0, sD = 0, sG = 0, sNS = 0, sSB = 0;  // blocks, dependency radius, lanes a row, stages, stage bytes
    int sEres = 0;             // resident form (one block): shared-memory bytes holding the level's e
    int csched = 0;            // staged per-colour launches (sB bands, sG lanes a row)
    std::vector<int> csm0, csm1;  // their shared memory a block per colour: lower parts / both parts
    Buf<int32_t> split, recptr, cchunk;
    Buf<int4> rec;
    Buf<int4> cslice;          // staged schedule: C x sB slices {lo[r0], lo[r1], up[r0], up[r1]}
    Buf<int2> rrow;
    Buf<unsigned> prog;        // per block: colour steps completed (monotone over launches)
    int stream = 0;            // this level's sweeps run streamed
    float tuned_ms = 0.0f;     // the autotuner's time of the chosen schedule (0: not tuned)
    int64_t nlow = 0, nupp = 0; // unpadded lower / upper off-diagonal counts
    // transfers in solve orders
    int pw = 0;                // ELL width of the interpolation (= m)
    Buf<int32_t> pc;           // n * pw
    Buf<float> pv32;
    Buf<uint16_t> pv16, r_v16;  // BF16 bit patterns of pv32 / r_v32 (transfer_bf16)
    Buf<double> pv64;
    Buf<int32_t> r_rp, r_ci;   // restriction: rows = next level's solve order
    Buf<float> r_v32;
    Buf<double> r_v64;
    // work vectors: b = right-hand side of the level, e = its solution, s = residual (on the
    // coarsest level of a constrained hierarchy b and e carry one more entry: the constraint
    // residual and the multiplier)
    Buf<float> b32, e32, s32;
    Buf<double> b64, e64, s64;
    // constrained (bordered) hierarchies: the border vector c_j of this level (c_0 = 1,
    // c_{j+1} = R_j c_j), in the level's vector order
    Buf<double> c64;
    Buf<float> c32;
};

}  // namespace mgm

struct mgm_hierarchy {
    int p = 0;
    int cycle = 0;     // MGM_CYCLE_V / W / F
    bool transfer_bf16 = false;  // FP32 cycle: BF16-stored P and R weights
    int precision = MGM_F32;
    int nu1 = 1, nu2 = 1, m = 3;
    uint64_t seed = 0;
    int64_t N = 0;
    std::vector<mgm::Level> lv;
    mgm::Buf<double> Ainv;      // explicit inverse of L_p (RCM order), FP64; bordered: of [L_p c; c^T 0]
    int64_t np = 0;
    int64_t nb = 0;             // dimension of Ainv: np, or np + 1 for a constrained hierarchy
    bool bordered = false;      // mean-zero constrained surface Poisson (Sec. 4.4)
    mgm::Buf<double> sres;      // constraint residual per level (bordered cycle)
    mgm::Buf<double> bpart;     // partial sums of the bordered cycle's dot products
    mgm::Buf<int32_t> ord_caller;  // level-0 solve index -> caller index
    // persistent multicolour sweeps (one cooperative launch per sweep) instead of one launch
    // per colour; error word of their bounded waits
    int sweep_mode = 0;         // 0: a launch per colour, 1: grid barriers, 2: per-row ready flags
    bool persistent = false;    // sweep_mode != 0
    mgm::Buf<int> err;
    // cluster-resident coarse tail of the FP32 V-cycle (tail.cu): levels tail_top..p-1 in one
    // thread-block-cluster launch (0: none)
    int tail_top = 0;
    int tail_cl = 0;                 // CTAs of the cluster
    size_t tail_smem = 0;            // dynamic shared memory a CTA
    size_t tail_stride = 0;          // bytes between the CTAs' blobs
    std::vector<unsigned> tail_bytes;  // each CTA's blob size
    mgm::Buf<unsigned char> tail_blob;
    // V-cycle graph (captured lazily)
    cudaGraphExec_t vgraph = nullptr;
    int64_t graph_kernels = 0;  // kernel nodes in vgraph
    cudaStream_t cap_stream = nullptr;
    // Krylov workspace (allocated on first solve)
    int krylov_m = 0;
    mgm::Buf<double> V, f, u, w, r, part, hbuf;
    mgm::Buf<float> Z32;
    mgm::Buf<double> zd;        // FP64 copy of an FP32 z_k for the outer product (mixed mode)
    mgm::Buf<double> Z64;
    mgm::Buf<double> ydev;
    double* hhost = nullptr;    // pinned
    // FGMRES driven on the device (graph with WHILE conditional nodes; krylov.cu)
    cudaGraphExec_t sgraph = nullptr;
    int sgraph_m = 0, sgraph_maxit = 0;
    mgm::Buf<double> gsd, ghist;  // scalars, Hessenberg, rotations, y; estimates per iteration
    mgm::Buf<int> gsi;            // k, iterations, convergence flag, maxit, estimates recorded
    void* multi = nullptr;      // workspace of the many-right-hand-side solve (multi.cu)
    // learned correction after the V-cycle (learned.cu); level-0 solve order throughout
    int ln = 0;                          // stencil size of the attached features (0: not attached)
    mgm::Buf<int32_t> lnbr;              // N x n stencil members, centre first
    mgm::Buf<float> lgeo;                // N x n x 3: xh/s, yh/s, c s^2
    mgm::Buf<uint16_t> lhg;              // N x 64 FP16: first layer applied to the geometric features
    mgm::Buf<uint16_t> lw;               // BF16 [n x 64 residual columns of W1 | W2 | w3]
    mgm::Buf<int32_t> lrp, lci, ltrp, ltci;  // L_0 and L_0^T as plain CSR (training)
    mgm::Buf<float> lval, ltval;
    bool learned = false;                // correction enabled
    bool learned_active = true;          // cleared by a solve that falls back to the plain cycle
    int64_t learned_fallbacks = 0;
    cudaGraphExec_t lgraph = nullptr;    // V-cycle + correction
    int64_t lgraph_kernels = 0;
    int64_t device_bytes = 0;
    ~mgm_hierarchy();
};

namespace mgm {
// vcycle.cu
void vcycle_core(mgm_hierarchy* H, cudaStream_t s);          // b_0 -> e_0 (graph if captured)
void vcycle_plain(mgm_hierarchy* H, cudaStream_t s);         // the same without the learned correction
void vcycle_prepare(mgm_hierarchy* H);                       // capture the graph
void vcycle_enqueue(mgm_hierarchy* H, cudaStream_t s);       // the plain cycle's launches (for captures)
void invalidate_graphs(mgm_hierarchy* H);
float time_level_smoothing(mgm_hierarchy* H, int j, int reps, cudaStream_t s);
void load_input(mgm_hierarchy* H, const void* src, int src_dtype, const int32_t* gather, cudaStream_t s);
void store_output(mgm_hierarchy* H, void* dst, int dst_dtype, const int32_t* scatter, cudaStream_t s);
void alloc_work(mgm_hierarchy* H);
void check_device_error(mgm_hierarchy* H, cudaStream_t s);
int barrier_timeout_probe(int nblocks, unsigned long long limit, cudaStream_t s);
void profile_vcycle(mgm_hierarchy* H, int reps, mgm_profile_info* out, cudaStream_t s);
double vcycle_floor_ms(const mgm_hierarchy* H, double chain_us, double gbs, double* bytes_ms, double* chain_ms);
int64_t level_smoothing_bytes(const mgm_hierarchy* H, int j);
// cluster-resident coarse tail (tail.cu)
void tail_prepare(mgm_hierarchy* H, cudaStream_t s);
void tail_launch(mgm_hierarchy* H, cudaStream_t s);
// krylov.cu
bool solve_graph_supported(const mgm_hierarchy* H, const mgm_solve_params* sp);
void reaction_steps(mgm_hierarchy* Hu, mgm_hierarchy* Hv, int model, const double* prm, double dt, double* u, double* v,
                    int steps, const mgm_solve_params* sp, int* iters_out, cudaStream_t s);
void profile_spmv(mgm_hierarchy* H, int reps, mgm_profile_info* out, cudaStream_t s);
void solve(mgm_hierarchy* H, const double* f, double* u, const mgm_solve_params* sp, mgm_solve_info* info,
           cudaStream_t s);
// gs_stream.cu
bool stream_prepare(mgm_hierarchy* H, Level& L, int B, int G, int NS, cudaStream_t s, bool resident = false);
int stream_blocks_limit(mgm_hierarchy* H);
template <class T>
void stream_sweep(mgm_hierarchy* H, Level& L, int mode, bool resid, cudaStream_t s);
void stream_reset(mgm_hierarchy* H, cudaStream_t s);
bool colour_prepare(mgm_hierarchy* H, Level& L, int B, int G, cudaStream_t s);
template <class T>
void colour_sweep(mgm_hierarchy* H, Level& L, int mode, cudaStream_t s);
void sweep_config_set(mgm_hierarchy* H, int j, const mgm_sweep_config* cfg, cudaStream_t s);
void sweep_config_get(const mgm_hierarchy* H, int j, mgm_sweep_config* out);
void autotune(mgm_hierarchy* H, int reps, bool use_cache, cudaStream_t s);
// learned.cu
void learned_correct(mgm_hierarchy* H, cudaStream_t s);     // e_0 += correction from s_0 = b_0 - L_0 e_0
// multi.cu
void solve_multi(mgm_hierarchy* H, int nrhs, const double* F, double* U, const mgm_solve_params* sp, mgm_solve_info* info,
                 cudaStream_t s);
void free_multi(mgm_hierarchy* H);
void solve_batched(mgm_hierarchy* const* H, int nprob, const double* const* F, double* const* U, int nrhs,
                   const mgm_solve_params* sp, mgm_solve_info* info, mgm_status* status, cudaStream_t s);
// pattern.cu
void reaction_rhs(int model, int scheme, int64_t n, const double* u, const double* v, const double* up, const double* vp,
                  const double* prm, double dt, double* ru, double* rv, cudaStream_t s);
// eigs.cu
void eigs(mgm_hierarchy* H, int nev, int b, int s_steps, int max_cycles, double tol, const mgm_solve_params* sp,
          uint64_t seed, double* lam_re, double* lam_im, double* evec, double* resid, int* nconv, int* nsolves,
          cudaStream_t s);
}  // namespace mgm

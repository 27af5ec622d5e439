// Internal helpers of libmgm: error state, stream-ordered device buffers, warp reductions,
// device-wide scans. Not part of the public ABI (see include/mgm.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/mgm.h"

namespace mgm {

// ---------------------------------------------------------------------------------------------
// error state (thread-local, read through mgm_last_error_message / mgm_last_error_row)
// ---------------------------------------------------------------------------------------------
void set_error(const std::string& msg);
void set_bad_row(int64_t row);
const char* error_message();
int64_t bad_row();
void set_fp64_rows(int64_t n);
int64_t fp64_rows();

struct Fail {
    mgm_status st;
};

[[noreturn]] void fail(mgm_status st, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define CK(call) ::mgm::check_cuda((call), #call, __FILE__, __LINE__)
// every kernel launch site is followed by exactly one CK_LAUNCH, which also counts the launch
void note_launch(int64_t n = 1);
int64_t launches();         // all threads of the process
int64_t thread_launches();  // launches made by the calling thread (graph capture counts)
#define CK_LAUNCH() (::mgm::note_launch(), ::mgm::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__))
#define REQUIRE(cond, msg)                                              \
    do {                                                                \
        if (!(cond)) ::mgm::fail(MGM_ERR_INVALID_ARG, std::string(msg)); \
    } while (0)

// run body, translating Fail into a status (C-ABI boundary)
template <class F>
mgm_status guarded(F&& body) {
    try {
        body();
        return MGM_OK;
    } catch (const Fail& f) {
        return f.st;
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return MGM_ERR_OOM;
    }
}

// ---------------------------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------------------------
// set-up tracing (util.cu): with MGM_TRACE set, synchronise and print the time since the last mark
bool trace_on();
void trace_mark(cudaStream_t s, const char* what, int level = -1);

// Persistent device blocks (util.cu): buf_alloc takes the smallest cached block of the current
// device that fits (up to twice the size asked for) or calls cudaMalloc (on failure it hands the
// caches back and tries once more, then fails with MGM_ERR_OOM); buf_free calls cudaFree, or,
// inside a BufCacheScope, keeps the block for reuse. A scope is opened only after a device
// synchronisation (mgm_destroy), so no work in flight uses a cached block. buf_cache_trim frees
// cached blocks, largest first, down to keep_bytes; buf_cache_flush frees them all.
// cache_budget: what the scratch pool and the block cache may each keep mapped on the current
// device between calls (1/32 of its memory). release_cached_memory: synchronise the device and
// hand both back.
void* buf_alloc(size_t bytes);
void buf_free(void* p);
void buf_cache_trim(size_t keep_bytes);
void buf_cache_flush();
size_t cache_budget();
void release_cached_memory();
// the library's stream-ordered scratch pool on the current device (util.cu), and a release of its
// cached memory down to keep_bytes
cudaMemPool_t scratch_pool();
void scratch_trim(size_t keep_bytes = 0);

// Temp<T>: stream-ordered scratch (from the scratch pool, freed with cudaFreeAsync) owned by one call.
template <class T>
struct Temp {
    T* p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    Temp() = default;
    Temp(size_t count, cudaStream_t st) { alloc(count, st); }
    void alloc(size_t count, cudaStream_t st) {
        release();
        s = st;
        n = count;
        if (count) {
            cudaError_t e = cudaMallocFromPoolAsync((void**)&p, count * sizeof(T), scratch_pool(), st);
            if (e != cudaSuccess) {  // hand the caches back to the device and try once more
                (void)cudaGetLastError();
                release_cached_memory();
                e = cudaMallocFromPoolAsync((void**)&p, count * sizeof(T), scratch_pool(), st);
            }
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                p = nullptr;
                fail(MGM_ERR_OOM, "stream-ordered allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
            }
        }
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        n = 0;
    }
    ~Temp() { release(); }
    Temp(const Temp&) = delete;
    Temp& operator=(const Temp&) = delete;
    Temp(Temp&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
    Temp& operator=(Temp&& o) noexcept {
        release();
        p = o.p; n = o.n; s = o.s;
        o.p = nullptr; o.n = 0;
        return *this;
    }
    T* get() const { return p; }
};

struct BufCacheScope {
    BufCacheScope();
    ~BufCacheScope();
};

// Buf<T>: persistent device memory owned by a hierarchy.
template <class T>
struct Buf {
    T* p = nullptr;
    size_t n = 0;
    Buf() = default;
    explicit Buf(size_t count) { alloc(count); }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) p = (T*)buf_alloc(count * sizeof(T));
    }
    void release() {
        if (p) buf_free(p);
        p = nullptr;
        n = 0;
    }
    ~Buf() { release(); }
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
    Buf(Buf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    Buf& operator=(Buf&& o) noexcept {
        release();
        p = o.p; n = o.n;
        o.p = nullptr; o.n = 0;
        return *this;
    }
    T* get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

inline unsigned grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 0x7fffffff) g = 0x7fffffff;
    return (unsigned)g;
}

// the calling thread's pinned host buffer of HOST_STAGE_BYTES (util.cu; nullptr if it cannot be
// allocated), through which to_host reads small results
constexpr size_t HOST_STAGE_BYTES = 64 * 1024;
void* host_stage();
template <class T>
inline void to_host(T* dst, const T* src, size_t count, cudaStream_t s) {
    if (!count) return;
    const size_t bytes = count * sizeof(T);
    void* stage = bytes <= HOST_STAGE_BYTES ? host_stage() : nullptr;
    if (stage) {  // small reads through the calling thread's pinned buffer (no pageable staging)
        CK(cudaMemcpyAsync(stage, src, bytes, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        std::memcpy(dst, stage, bytes);
        return;
    }
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
}
template <class T>
inline T read1(const T* src, cudaStream_t s) {
    T v;
    to_host(&v, src, 1, s);
    return v;
}

// ---------------------------------------------------------------------------------------------
// device-wide primitives (util.cu)
// ---------------------------------------------------------------------------------------------
// exclusive scan of n int32 counts into out (n+1 entries, out[n] = total as int64 is returned
// through total_dev if non-null). in and out may alias. Totals must fit int32 (checked).
void exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);
// same for int64
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);
// fill
void fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s);
void iota_i32(int32_t* p, int64_t n, cudaStream_t s);
// inverse permutation: inv[perm[i]] = i
void invert_perm(const int32_t* perm, int32_t* inv, int64_t n, cudaStream_t s);
// gather rows of an N x 3 double array: out[i] = in[idx[i]]
void gather_xyz(const double* in, const int32_t* idx, double* out, int64_t n, cudaStream_t s);
// CSR transpose with columns ascending (deterministic)
void csr_transpose(int64_t nrows, int64_t ncols, const int32_t* rp, const int32_t* ci, const double* v,
                   int32_t* trp, int32_t* tci, double* tv, cudaStream_t s);
// B = A[perm][:, perm] (perm[new] = old), rows sorted by column; brp must have N+1 entries,
// bci/bv nnz entries.
void csr_permute(int64_t N, const int32_t* rp, const int32_t* ci, const double* v, const int32_t* perm,
                 int32_t* brp, int32_t* bci, double* bv, cudaStream_t s);
// symmetrised pattern of A (A + A^T without the diagonal), rows ascending. Returns arrays via Temp.
void sym_pattern(int64_t N, const int32_t* rp, const int32_t* ci, Temp<int32_t>& srp, Temp<int32_t>& sci,
                 cudaStream_t s);
// nnz of a CSR from its last row pointer (synchronises)
int64_t csr_nnz(const int32_t* rp, int64_t nrows, cudaStream_t s);
// argument validation (synchronise): all a[i] in [0, hi); CSR row pointers monotone from 0
void validate_index(const int32_t* a, int64_t cnt, int64_t hi, const char* what, cudaStream_t s);
void validate_csr(int64_t nrows, int64_t ncols, const int32_t* rp, const int32_t* ci, const char* what, cudaStream_t s);

// A fixed sequence of launches captured once on a private stream and replayed as a CUDA graph.
// Captured launches are not counted; each replay counts them.
struct GraphBatch {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
    template <class F>
    void capture(F&& body) {
        cudaStream_t cs = nullptr;
        CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        const int64_t before = thread_launches();
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            try {
                body(cs);
            } catch (...) {
                cudaStreamEndCapture(cs, &g);
                if (g) cudaGraphDestroy(g);
                cudaStreamDestroy(cs);
                throw;
            }
            e = cudaStreamEndCapture(cs, &g);
        }
        kernels = thread_launches() - before;
        note_launch(-kernels);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        CK(e);
    }
    void launch(cudaStream_t s) {
        CK(cudaGraphLaunch(exec, s));
        note_launch(kernels);
    }
    ~GraphBatch() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

// Blocks of `kernel` (with `threads` threads and `smem` dynamic shared memory) that can be
// co-resident on the current device, at most `per_sm_cap` an SM (0: no cap); cached per device and
// configuration. MGM_ERR_UNSUPPORTED when not even one block fits an SM (a cooperative launch of it
// could never start).
int coresident_blocks(const void* kernel, int threads, size_t smem, int per_sm_cap);

// kNN (knn.cu)
void knn_device(const double* data, int64_t nd, const double* query, int64_t nq, int k, int self_first,
                int32_t* idx_out, double* d2_out, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier of a cooperative launch: a monotone arrival counter in global memory (`target` =
// blocks x barriers passed so far). Each wait is bounded: past `limit` polls the block records
// MGM_ERR_TIMEOUT in `err`; a block that sees `err` set stops waiting. Returns false (for every
// thread of the block) in either case, and the caller leaves the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, unsigned long long limit, int* err, int* ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        unsigned long long it = 0;
        int good = 1;
        while (ld_acquire_u32(bar) < target) {
            if (*(volatile int*)err) { good = 0; break; }
            if (++it > limit) { atomicOr(err, MGM_ERR_TIMEOUT); good = 0; break; }
            __nanosleep(32);
        }
        __threadfence();
        *ok = good;
    }
    __syncthreads();
    return *ok != 0;
}

// Programmatic dependent launch: a kernel launched with launch_pdl may be scheduled while its
// predecessor in the stream is still running. pdl_trigger lets the successor start; pdl_wait blocks
// until the predecessor has completed and its memory is visible (it returns at once when the
// kernel was not launched programmatically).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// off for the calling thread while it captures kernels into a graph that does not admit programmatic
// dependencies (the bodies of conditional nodes); launches are then stream-ordered as usual
bool& pdl_off();

template <class... KArgs, class... Args>
inline void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_off() ? 0 : 1;
    CK(cudaLaunchKernelEx(&cfg, kern, args...));
    CK_LAUNCH();
}

__device__ __forceinline__ double warp_max_d(double v) {
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace mgm

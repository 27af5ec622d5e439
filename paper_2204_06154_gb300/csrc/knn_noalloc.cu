// mgm_knn_noalloc: the k-nearest-neighbour search of mgm_knn for callers that cannot allocate
// device memory. Same kernels, same results; the grid scratch lives in one file-scope device
// array instead of cudaMallocAsync'd temporaries, and the cell-count scan is a single-block
// kernel that needs no temporary either. Built with --fmad=false like knn.cu.
#include <mutex>

#include "knn_grid.cuh"

namespace mgm {

constexpr int64_t NOALLOC_MAX_POINTS = MGM_KNN_NOALLOC_MAX_POINTS;
constexpr int64_t NOALLOC_CELLS = 2 * NOALLOC_MAX_POINTS;  // grid cells for the largest cloud
constexpr int NOALLOC_PARTS = 1024;                        // bounding-box partial results

// scratch layout (byte offsets, each 256-aligned)
constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t OFF_GRID = 0;
constexpr size_t OFF_ERR = al256(OFF_GRID + sizeof(Grid));
constexpr size_t OFF_PART = al256(OFF_ERR + sizeof(int));
constexpr size_t OFF_CNT = al256(OFF_PART + sizeof(double) * 6 * NOALLOC_PARTS);
constexpr size_t OFF_START = al256(OFF_CNT + sizeof(int32_t) * (NOALLOC_CELLS + 1));
constexpr size_t OFF_CELLOF = al256(OFF_START + sizeof(int32_t) * (NOALLOC_CELLS + 1));
constexpr size_t OFF_SIDX = al256(OFF_CELLOF + sizeof(int32_t) * NOALLOC_MAX_POINTS);
constexpr size_t OFF_SXYZ = al256(OFF_SIDX + sizeof(int32_t) * NOALLOC_MAX_POINTS);
constexpr size_t SCRATCH_BYTES = al256(OFF_SXYZ + sizeof(double) * 3 * NOALLOC_MAX_POINTS);

// Held by every GPU that loads the library, for the life of the process (about 12.6 MB).
static __device__ __align__(256) unsigned char g_knn_scratch[SCRATCH_BYTES];

// Device address of g_knn_scratch on the current device, looked up once per device. In host code
// the array's name is only a host-side stand-in; a kernel must be given this address instead.
static unsigned char* scratch_on_current_device() {
    static std::mutex mu;
    static unsigned char* ptr[128] = {nullptr};
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) fail(MGM_ERR_UNSUPPORTED, "device ordinal above 127");
    std::lock_guard<std::mutex> lock(mu);
    if (!ptr[dev]) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_knn_scratch));
        ptr[dev] = static_cast<unsigned char*>(p);
    }
    return ptr[dev];
}

// exclusive scan of cnt[0..n) into out[0..n] by one block (no temporaries)
__global__ void __launch_bounds__(1024) scan_one_block_k(const int32_t* cnt, int32_t* out, int64_t n) {
    __shared__ int64_t part[1024];
    const int64_t per = (n + 1023) / 1024;
    const int64_t b = threadIdx.x * per, e = min(n, b + per);
    int64_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += cnt[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int t = 0; t < 1024; ++t) { int64_t v = part[t]; part[t] = acc; acc += v; }
        out[n] = (int32_t)acc;
    }
    __syncthreads();
    int64_t acc = part[threadIdx.x];
    for (int64_t i = b; i < e; ++i) { out[i] = (int32_t)acc; acc += cnt[i]; }
}

void knn_noalloc(const double* data, int64_t nd, const double* query, int64_t nq, int k, int self_first,
                 int32_t* idx_out, cudaStream_t s) {
    REQUIRE(data && query && idx_out, "null array");
    REQUIRE(k >= 1 && k <= 256, "k must be in [1, 256]");
    REQUIRE(nd >= k, "k exceeds the number of data points");
    REQUIRE(nq >= 0 && nq < 0x7fffffff, "query count out of range");
    REQUIRE(!self_first || (data == query && nd == nq), "self_first requires query == data");
    if (nd > NOALLOC_MAX_POINTS)
        fail(MGM_ERR_UNSUPPORTED, "mgm_knn_noalloc: " + std::to_string(nd) + " data points exceed the maximum of " +
                                      std::to_string(NOALLOC_MAX_POINTS) + " (use mgm_knn)");
    unsigned char* base = scratch_on_current_device();
    Grid* g = reinterpret_cast<Grid*>(base + OFF_GRID);
    int* err = reinterpret_cast<int*>(base + OFF_ERR);
    double* part = reinterpret_cast<double*>(base + OFF_PART);
    int32_t* cnt = reinterpret_cast<int32_t*>(base + OFF_CNT);
    int32_t* start = reinterpret_cast<int32_t*>(base + OFF_START);
    int32_t* cell_of = reinterpret_cast<int32_t*>(base + OFF_CELLOF);
    int32_t* sidx = reinterpret_cast<int32_t*>(base + OFF_SIDX);
    double* sxyz = reinterpret_cast<double*>(base + OFF_SXYZ);
    if (nq == 0) return;
    const int64_t cells = 2 * nd;
    // the array keeps the previous call's contents: zero what accumulates
    CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (cells + 1), s));
    const int nparts = (int)std::min<int64_t>(grid_for(nd, 256), NOALLOC_PARTS);
    bbox_partial_k<<<nparts, 256, 0, s>>>(data, nd, part);
    CK_LAUNCH();
    grid_params_k<<<1, GRID_PARAMS_THREADS, 0, s>>>(part, nparts, cells, 0.0, g);
    CK_LAUNCH();
    cell_count_k<<<grid_for(nd, 256), 256, 0, s>>>(data, nd, g, cnt, cell_of);
    CK_LAUNCH();
    scan_one_block_k<<<1, 1024, 0, s>>>(cnt, start, cells);
    CK_LAUNCH();
    CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (cells + 1), s));
    cell_place_k<<<grid_for(nd, 256), 256, 0, s>>>(data, nd, cell_of, start, cnt, sidx, sxyz, nullptr);
    CK_LAUNCH();
    const size_t smem = (sizeof(double) + sizeof(int)) * KNN_WARPS * KNN_CAP;
    CK(cudaFuncSetAttribute(knn_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    knn_k<<<grid_for(nq, KNN_WARPS), KNN_WARPS * 32, smem, s>>>(g, start, sidx, sxyz, query, nq, k, self_first, idx_out,
                                                               nullptr, err);
    CK_LAUNCH();
    int e = 0;
    CK(cudaMemcpyAsync(&e, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (e & 2) fail(MGM_ERR_INVALID_ARG, "fewer than k data points");
    if (e) fail(MGM_ERR_UNSUPPORTED, "kNN search failed");
}

}  // namespace mgm

extern "C" mgm_status mgm_knn_noalloc(const double* data, int64_t nd, const double* query, int64_t nq, int k,
                                      int self_first, int32_t* idx_out, mgm_stream stream) {
    return mgm::guarded([&] {
        mgm::knn_noalloc(data, nd, query, nq, k, self_first, idx_out, reinterpret_cast<cudaStream_t>(stream));
    });
}

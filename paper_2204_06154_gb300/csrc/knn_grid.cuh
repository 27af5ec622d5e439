// Uniform-grid kNN building blocks shared by the kNN entry points (kernels defined in knn.cu).
#pragma once
#include "common.cuh"

namespace mgm {

constexpr int KNN_WARPS = 4;
constexpr int GRID_PARAMS_THREADS = 256;  // block size grid_params_k must be launched with
constexpr int KNN_CAP = 1024;  // candidate buffer per warp (>= k + 32 for k <= 256: compaction keeps k)

struct Grid {
    double x0, y0, z0, h;
    int nx, ny, nz;
    int64_t ncells;
};

__global__ void bbox_partial_k(const double* x, int64_t n, double* part);
__global__ void grid_params_k(const double* part, int nparts, int64_t cells, double h_min, Grid* g);
__global__ void cell_count_k(const double* x, int64_t n, const Grid* gp, int32_t* cnt, int32_t* cell_of);
__global__ void cell_place_k(const double* x, int64_t n, const int32_t* cell_of, const int32_t* start, int32_t* fill,
                             int32_t* sidx, double* sxyz);
__global__ void knn_k(const Grid* gp, const int32_t* start, const int32_t* sidx, const double* sxyz, const double* q,
                      int64_t nq, int k, int self_first, int32_t* idx_out, double* d2_out, int* err);

}  // namespace mgm

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
    double amax;  // largest |coordinate| of the data points (infinite when one is not finite)
};

__global__ void bbox_partial_k(const double* x, int64_t n, double* part);
__global__ void grid_params_k(const double* part, int nparts, int64_t cells, double h_min, Grid* g);
__global__ void cell_count_k(const double* x, int64_t n, const Grid* gp, int32_t* cnt, int32_t* cell_of);
__global__ void cell_place_k(const double* x, int64_t n, const int32_t* cell_of, const int32_t* start, int32_t* fill,
                             int32_t* sidx, double* sxyz, float4* s32);

// FP32 culling of distance tests. A candidate whose FP32 squared distance (from coordinates
// rounded to FP32, differences, squares and sums rounded in FP32, with or without contraction)
// exceeds far_sq_f32(D, A) is farther than D from the query: each rounded coordinate is within
// 2^-24 |x| of the exact one and each FP32 operation adds a relative 2^-24, so the FP32 difference
// vector is within 2^-24 |d| + 1.74 * 2^-24 A of the exact one (A >= |query coordinate| + |data
// coordinate|) and its rounded squared norm within 3 * 2^-24 relative; the threshold uses 2^-22
// in place of 2^-24 throughout, so it also clears the FP64 rounding of the exact test by a wide
// margin. Such a candidate fails the exact FP64 test, which therefore need not run. A NaN or
// infinite D or A gives an infinite or NaN threshold, which culls nothing, and so does a NaN
// coordinate (a NaN distance compares false).
__device__ __forceinline__ float far_sq_f32(double D, double A) {
    const double u = 0x1p-22;
    const double r = (1.0 + 2.0 * u) * D + 16.0 * u * A + 1e-36;  // (the last: subnormal coordinates)
    // 2^-140: the absolute error of squares and sums that fall into FP32's subnormal range
    return __double2float_ru(r * r * (1.0 + 8.0 * u) + 0x1p-140);
}
__device__ __forceinline__ float d2_f32(float px, float py, float pz, float4 q) {
    const float dx = px - q.x, dy = py - q.y, dz = pz - q.z;
    return (dx * dx + dy * dy) + dz * dz;
}
__global__ void knn_k(const Grid* gp, const int32_t* start, const int32_t* sidx, const double* sxyz, const double* q,
                      int64_t nq, int k, int self_first, int32_t* idx_out, double* d2_out, int* err);

}  // namespace mgm

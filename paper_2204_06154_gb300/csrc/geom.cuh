// Tangent-plane geometry of a stencil (paper Sec. 2.1), shared by the stencil-weight kernels and
// the learned correction's features.
#pragma once
#include <stdint.h>

namespace mgm {

__device__ __forceinline__ double dot3d(const double* a, const double* b) { return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2]; }

// Sec. 2.1: orthonormal t1, t2 of T_x M; t1 from the coordinate axis of smallest |n_a| (first on ties)
__device__ inline void tangent_basis(const double* nin, double* t1, double* t2) {
    double nn = sqrt((nin[0] * nin[0] + nin[1] * nin[1]) + nin[2] * nin[2]);
    double n[3] = {nin[0] / nn, nin[1] / nn, nin[2] / nn};
    int a = 0;
    if (fabs(n[1]) < fabs(n[a])) a = 1;
    if (fabs(n[2]) < fabs(n[a])) a = 2;
    double v[3] = {-n[a] * n[0], -n[a] * n[1], -n[a] * n[2]};
    v[a] = 1.0 + v[a];
    double vn = sqrt((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    t1[0] = v[0] / vn; t1[1] = v[1] / vn; t1[2] = v[2] / vn;
    t2[0] = n[1] * t1[2] - n[2] * t1[1];
    t2[1] = n[2] * t1[0] - n[0] * t1[2];
    t2[2] = n[0] * t1[1] - n[1] * t1[0];
}

__device__ inline double project_support(const double* xyz, const double* nrm, int64_t i, const int32_t* id, int n,
                                         double* xh, double* yh) {
    double t1[3], t2[3];
    tangent_basis(nrm + 3 * i, t1, t2);
    const double* xc = xyz + 3 * i;
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
        const double* xj = xyz + 3 * (int64_t)id[j];
        double d[3] = {xj[0] - xc[0], xj[1] - xc[1], xj[2] - xc[2]};
        double u = dot3d(t1, d), v = dot3d(t2, d);
        if (xh) { xh[j] = u; yh[j] = v; }
        double r = sqrt(u * u + v * v);
        if (r > s) s = r;
    }
    return s;
}

}  // namespace mgm

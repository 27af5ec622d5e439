// Right-hand sides of the semi-implicit reaction-diffusion steps (paper Sec. 6.2), one fused pass
// over the points: the reaction terms at the current (and, for SBDF2, the previous) step and the
// combination the scheme solves for, so the step reads each state vector once.
//   Gierer-Meinhardt, eq. (turing): f = A - B u + u^2 / (v (1 + C u^2)), g = u^2 - v.
//   Schnakenberg: f = gamma (a - u + u^2 v), g = gamma (b - u^2 v).
//   IMEX Euler:  r_w = w^n + dt r^n, for (I - dt D_w Lap) w^{n+1} = r_w.
//   SBDF2:       r_w = (4 w^n - w^{n-1}) / 3 + (2/3) dt (2 r^n - r^{n-1}),
//                for (I - (2/3) dt D_w Lap) w^{n+1} = r_w.
#include "hier.cuh"

namespace mgm {

__device__ __forceinline__ void reactions(int model, double p0, double p1, double p2, double u, double v, double& f,
                                          double& g) {
    if (model == MGM_RD_GIERER_MEINHARDT) {
        f = p0 - p1 * u + u * u / (v * (1.0 + p2 * u * u));
        g = u * u - v;
    } else {
        f = p0 * (p1 - u + u * u * v);
        g = p0 * (p2 - u * u * v);
    }
}

__global__ void reaction_rhs_k(int model, int scheme, int64_t n, const double* __restrict__ u,
                               const double* __restrict__ v, const double* __restrict__ up,
                               const double* __restrict__ vp, double p0, double p1, double p2, double dt, double* ru,
                               double* rv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ui = u[i], vi = v[i];
    double f, g;
    reactions(model, p0, p1, p2, ui, vi, f, g);
    if (scheme == MGM_RD_EULER) {
        ru[i] = ui + dt * f;
        rv[i] = vi + dt * g;
    } else {
        const double upi = up[i], vpi = vp[i];
        double fp, gp;
        reactions(model, p0, p1, p2, upi, vpi, fp, gp);
        const double c = (2.0 / 3.0) * dt;
        ru[i] = (4.0 * ui - upi) / 3.0 + c * (2.0 * f - fp);
        rv[i] = (4.0 * vi - vpi) / 3.0 + c * (2.0 * g - gp);
    }
}

void reaction_rhs(int model, int scheme, int64_t n, const double* u, const double* v, const double* up, const double* vp,
                  const double* prm, double dt, double* ru, double* rv, cudaStream_t s) {
    REQUIRE(model == MGM_RD_GIERER_MEINHARDT || model == MGM_RD_SCHNAKENBERG, "unknown reaction model");
    REQUIRE(scheme == MGM_RD_EULER || scheme == MGM_RD_SBDF2, "unknown time-stepping scheme");
    REQUIRE(n >= 1 && u && v && ru && rv && prm, "bad argument");
    REQUIRE(scheme == MGM_RD_EULER || (up && vp), "SBDF2 needs the previous step");
    reaction_rhs_k<<<grid_for(n, 256), 256, 0, s>>>(model, scheme, n, u, v, up, vp, prm[0], prm[1], prm[2], dt, ru, rv);
    CK_LAUNCH();
}

}  // namespace mgm

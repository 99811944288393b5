// Per-edge geometry and angular/radial features shared by the edge kernels.
//
//   d = fl64(fl64(x_j - x_i) + n L) rounded to FP32 (the tensor-core path forms
//   it from FP32 position pairs instead, within one FP32 rounding of this),
//   r = |d|, u = d / r
//   e_k(r) = sqrt(2 / r_c) sin(k pi r / r_c) / r,  k = 1..8
//   u_env(x) = 1 - (p+1)(p+2)/2 x^p + p(p+2) x^(p+1) - p(p+1)/2 x^(p+2)
//   eps_k = e_k u_env,  and d eps_k / d r for the adjoint
//   real spherical harmonics, component normalisation (sum_m Y_lm^2 = 2l+1),
//   order Y0; Y1 = sqrt3 (x, y, z);
//   Y2 = (sqrt15 xy, sqrt15 yz, sqrt5/2 (3z^2-1), sqrt15 xz, sqrt15/2 (x^2-y^2))
#pragma once

#include "common.cuh"

namespace mp {

struct EdgeConst {
    double L[3];
    float rc, inv_rc, pref;     // pref = sqrt(2 / r_c)
    float c1, c2, c3;           // envelope coefficients
    int p;
    float inv_navg;
    float rep_eps, rep_sig12;   // eps_rep, sigma_rep^12 (rep_eps = 0: off)
};

inline EdgeConst make_edge_const(const mp_model_desc& d, const double box[3]) {
    EdgeConst k;
    for (int a = 0; a < 3; ++a) k.L[a] = box[a];
    k.rc = (float)d.r_cut;
    k.inv_rc = (float)(1.0 / d.r_cut);
    k.pref = (float)sqrt(2.0 / d.r_cut);
    double p = d.p_env;
    k.c1 = (float)((p + 1) * (p + 2) / 2.0);
    k.c2 = (float)(p * (p + 2));
    k.c3 = (float)(p * (p + 1) / 2.0);
    k.p = d.p_env;
    k.inv_navg = (float)(1.0 / d.n_avg);
    k.rep_eps = (float)d.rep_eps;
    k.rep_sig12 = (float)pow(d.rep_sigma, 12.0);
    return k;
}

// One component of fl64(fl64(x_j - x_i) + n L) for n in {-1, 0, 1}: n L is
// selected rather than multiplied, and the addition is skipped for n = 0 (the
// common case; adding +0 would not change the nonzero difference).  FP64 runs
// at a small fraction of the FP32 rate here, so this halves the FP64 work of
// an edge vector without changing a bit of it.
__device__ __forceinline__ float image_diff(double xj, double xi, int n, double L) {
    const double a = __dsub_rn(xj, xi);
    return (float)(n == 0 ? a : __dadd_rn(a, n > 0 ? L : -L));
}

__device__ __forceinline__ void edge_vector(const double* __restrict__ x, int64_t i, int64_t j,
                                            int code, const EdgeConst& k, float d[3]) {
    const int n0 = code / 9 - 1, n1 = (code / 3) % 3 - 1, n2 = code % 3 - 1;
    d[0] = image_diff(x[3 * j], x[3 * i], n0, k.L[0]);
    d[1] = image_diff(x[3 * j + 1], x[3 * i + 1], n1, k.L[1]);
    d[2] = image_diff(x[3 * j + 2], x[3 * i + 2], n2, k.L[2]);
}

// r = |d| and the unit vector u = d / r in FP32 (the reciprocal taken once).
__device__ __forceinline__ float edge_unit(const float d[3], float u[3]) {
    const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const float ir = 1.f / r;
    u[0] = d[0] * ir;
    u[1] = d[1] * ir;
    u[2] = d[2] * ir;
    return r;
}

// Envelope u(x) and du/dr; exactly 0 for x >= 1, so an edge of a skin list
// beyond r_c gives eps = d eps/dr = 0, hence R = dR/dr = 0 (the radial MLP is
// bias free and silu(0) = 0) and adds exact zeros everywhere.
__device__ __forceinline__ void envelope(float r, const EdgeConst& k, float& u, float& du_dr) {
    const float x = r * k.inv_rc;
    float xpm1 = 1.f;
    for (int q = 0; q < k.p - 1; ++q) xpm1 *= x;
    const float xp = xpm1 * x;
    u = 1.f - k.c1 * xp + k.c2 * xp * x - k.c3 * xp * x * x;
    du_dr = (-k.c1 * (float)k.p * xpm1 + k.c2 * (float)(k.p + 1) * xp -
             k.c3 * (float)(k.p + 2) * xp * x) * k.inv_rc;
    if (!(x < 1.f)) {
        u = 0.f;
        du_dr = 0.f;
    }
}

// eps_k(r) (and d eps_k / dr when DERIV); sin/cos(k pi x) by the angle-sum
// recurrence from one sincospi call.
template <bool DERIV>
__device__ __forceinline__ void radial_basis(float r, const EdgeConst& k, float eps[kNB],
                                             float deps[kNB], float& u, float& du) {
    envelope(r, k, u, du);
    const float x = r * k.inv_rc;
    float s1, c1;
    sincospif(x, &s1, &c1);
    const float inv_r = 1.f / r;
    float sp = 0.f, cp = 1.f, s = s1, c = c1;
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
        const float e = k.pref * s * inv_r;
        eps[q] = e * u;
        if (DERIV) {
            const float kpi = (float)(q + 1) * 3.14159265358979f * k.inv_rc;
            const float de = k.pref * (kpi * c - s * inv_r) * inv_r;
            deps[q] = de * u + e * du;
        }
        const float sn = 2.f * c1 * s - sp, cn = 2.f * c1 * c - cp;
        sp = s;
        cp = c;
        s = sn;
        c = cn;
    }
}

template <int LMAX>
__device__ __forceinline__ void sph_harm(const float u[3], float* Y) {
    Y[0] = 1.f;
    const float s3 = 1.7320508075688772f;
    Y[1] = s3 * u[0];
    Y[2] = s3 * u[1];
    Y[3] = s3 * u[2];
    if (LMAX >= 2) {
        const float s15 = 3.872983346207417f, s5h = 1.118033988749895f;
        Y[4] = s15 * u[0] * u[1];
        Y[5] = s15 * u[1] * u[2];
        Y[6] = s5h * (3.f * u[2] * u[2] - 1.f);
        Y[7] = s15 * u[0] * u[2];
        Y[8] = 0.5f * s15 * (u[0] * u[0] - u[1] * u[1]);
    }
}

// v = sum_lm gY_lm dY_lm/du (gY indexed like Y, entry 0 unused).
template <int LMAX, class T = float>
__device__ __forceinline__ void sph_grad(const T u[3], const T* gY, T v[3]) {
    const T s3 = (T)1.7320508075688772;
    v[0] = s3 * gY[1];
    v[1] = s3 * gY[2];
    v[2] = s3 * gY[3];
    if (LMAX >= 2) {
        const T s15 = (T)3.872983346207417, s5 = (T)2.23606797749979;
        v[0] += s15 * (gY[4] * u[1] + gY[7] * u[2] + gY[8] * u[0]);
        v[1] += s15 * (gY[4] * u[0] + gY[5] * u[2] - gY[8] * u[1]);
        v[2] += s15 * (gY[5] * u[1] + gY[7] * u[0]) + (T)3 * s5 * gY[6] * u[2];
    }
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

}  // namespace mp

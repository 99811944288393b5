// Tangent (forward-mode) pass of the layers along a displacement field v:
// dh^(t) = sum_k (d h^(t) / d r_k) v_k, used for the force term of the
// correction-head loss (its gradient needs J v, J = d h^(K) / d r).
//
// Edge (i <- j), d = r_j - r_i + n L, dd = v_j - v_i:
//   dr   = u . dd
//   dY_l = grad_u Y_l . (dd - (u . dd) u) / r
//   dR   = (dR / dr) dr          (dR/dr propagated forward through the MLP)
//   dA0_i   += dR0 h0_j + R0 dh0_j
//   dAl_i,m += dRla h0_j Y_lm + Rla dh0_j Y_lm + Rla h0_j dY_lm
//              + dRlb hl_j,m + Rlb dhl_j,m             (all / N_avg)
// Node: ds = W0 dA0 + sum_l Ul dBl with dBl = 2 sum_m Al,m dAl,m;
//   dh0' = dh0 + silu'(S) ds;  dhl' = dhl + Vl dAl.
// FP32 on CUDA cores; receiver rows owned by one block, no atomics.
#include "kernels.h"

namespace mp {

namespace {

constexpr int CT = 8;     // edges per chunk
constexpr int RPBT = 4;   // rows per block

__device__ __forceinline__ int find_row_tg(const int64_t* rp, int nrows, int64_t e) {
    int lr = 0;
    while (lr + 1 < nrows && rp[lr + 1] <= e) ++lr;
    return lr;
}

template <int F, int LMAX>
struct TanSmem {
    static constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    float eps[CT][kNB], deps[CT][kNB];
    float Y[CT][NLM], dY[CT][NLM];
    float dr[CT];
    float a1[kH][CT], da1[kH][CT], a2[kH][CT], da2[kH][CT];
    int row[CT], col[CT];
    int64_t rp[RPBT + 1];
};

template <int F, int LMAX, bool FIRST>
__global__ void __launch_bounds__(F) k_edge_tangent(TangentArgs a, const float* __restrict__ W1,
                                                    const float* __restrict__ W2T,
                                                    const float* __restrict__ W3T) {
    constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    constexpr int P = F * (1 + 2 * LMAX);
    constexpr int NP = 1 + 2 * LMAX;
    constexpr int EG = CT * kH / F;
    __shared__ TanSmem<F, LMAX> s;
    const int c = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * RPBT;
    const int nrows = (int)min((int64_t)RPBT, a.n - r0);
    if (c <= nrows) s.rp[c] = a.row_ptr[r0 + c];
    __syncthreads();
    const int64_t e_beg = s.rp[0], e_end = s.rp[nrows];
    float acc[NLM];
#pragma unroll
    for (int q = 0; q < NLM; ++q) acc[q] = 0.f;
    int cur = -1, next = 0;
    auto write_row = [&](int lr, bool zero) {
        float* o = a.dAout + ((r0 + lr) * NLM) * F + c;
#pragma unroll
        for (int q = 0; q < NLM; ++q) o[q * F] = zero ? 0.f : acc[q] * a.k.inv_navg;
    };

    for (int64_t cb = e_beg; cb < e_end; cb += CT) {
        if (c < CT) {
            const int64_t e = cb + c;
            float eps[kNB], deps[kNB], Y[NLM], dY[NLM], drv = 0.f;
            if (e < e_end) {
                const int lr = find_row_tg(s.rp, nrows, e);
                const int64_t i = r0 + lr;
                const int j = a.col[e];
                float d[3];
                edge_vector(a.x, i, j, a.shift[e], a.k, d);
                const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                const float ir = 1.f / r;
                const float u[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
                float env, denv;
                radial_basis<true>(r, a.k, eps, deps, env, denv);
                sph_harm<LMAX>(u, Y);
                const float dd[3] = {a.v[3 * j] - a.v[3 * i], a.v[3 * j + 1] - a.v[3 * i + 1],
                                     a.v[3 * j + 2] - a.v[3 * i + 2]};
                drv = u[0] * dd[0] + u[1] * dd[1] + u[2] * dd[2];
                const float wv[3] = {(dd[0] - drv * u[0]) * ir, (dd[1] - drv * u[1]) * ir,
                                     (dd[2] - drv * u[2]) * ir};
                // dY_lm = grad_u Y_lm . w
                const float s3 = 1.7320508075688772f;
                dY[0] = 0.f;
                dY[1] = s3 * wv[0];
                dY[2] = s3 * wv[1];
                dY[3] = s3 * wv[2];
                if (LMAX >= 2) {
                    const float s15 = 3.872983346207417f, s5 = 2.23606797749979f;
                    dY[4] = s15 * (u[1] * wv[0] + u[0] * wv[1]);
                    dY[5] = s15 * (u[2] * wv[1] + u[1] * wv[2]);
                    dY[6] = 3.f * s5 * u[2] * wv[2];
                    dY[7] = s15 * (u[2] * wv[0] + u[0] * wv[2]);
                    dY[8] = s15 * (u[0] * wv[0] - u[1] * wv[1]);
                }
                s.row[c] = lr;
                s.col[c] = j;
            } else {
#pragma unroll
                for (int q = 0; q < kNB; ++q) eps[q] = deps[q] = 0.f;
#pragma unroll
                for (int q = 0; q < NLM; ++q) Y[q] = dY[q] = 0.f;
                s.row[c] = -1;
                s.col[c] = 0;
            }
#pragma unroll
            for (int q = 0; q < kNB; ++q) {
                s.eps[c][q] = eps[q];
                s.deps[c][q] = deps[q];
            }
#pragma unroll
            for (int q = 0; q < NLM; ++q) {
                s.Y[c][q] = Y[q];
                s.dY[c][q] = dY[q];
            }
            s.dr[c] = drv;
        }
        __syncthreads();
        for (int o = c; o < kH * CT; o += F) {
            const int kk = o / CT, e = o % CT;
            float z = 0.f, dz = 0.f;
#pragma unroll
            for (int b = 0; b < kNB; ++b) {
                const float wv = __ldg(&W1[kk * kNB + b]);
                z = fmaf(wv, s.eps[e][b], z);
                dz = fmaf(wv, s.deps[e][b], dz);
            }
            s.a1[kk][e] = silu(z);
            s.da1[kk][e] = silu_grad(z) * dz;
        }
        __syncthreads();
        {
            const int kk = c % kH, e0 = (c / kH) * EG;
            float z[EG], dz[EG];
#pragma unroll
            for (int q = 0; q < EG; ++q) z[q] = dz[q] = 0.f;
            for (int jj = 0; jj < kH; ++jj) {
                const float wv = __ldg(&W2T[jj * kH + kk]);
#pragma unroll
                for (int q = 0; q < EG; ++q) {
                    z[q] = fmaf(wv, s.a1[jj][e0 + q], z[q]);
                    dz[q] = fmaf(wv, s.da1[jj][e0 + q], dz[q]);
                }
            }
#pragma unroll
            for (int q = 0; q < EG; ++q) {
                s.a2[kk][e0 + q] = silu(z[q]);
                s.da2[kk][e0 + q] = silu_grad(z[q]) * dz[q];
            }
        }
        __syncthreads();
        // R and dR/dr for this thread's channel, all radial paths
        float R[NP][CT], dR[NP][CT];
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
            for (int e = 0; e < CT; ++e) R[q][e] = dR[q][e] = 0.f;
        for (int kk = 0; kk < kH; ++kk) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float wv = __ldg(&W3T[kk * P + q * F + c]);
#pragma unroll
                for (int e = 0; e < CT; ++e) {
                    R[q][e] = fmaf(wv, s.a2[kk][e], R[q][e]);
                    dR[q][e] = fmaf(wv, s.da2[kk][e], dR[q][e]);
                }
            }
        }
#pragma unroll
        for (int e = 0; e < CT; ++e) {
            const int lr = s.row[e];
            if (lr < 0) break;
            if (lr != cur) {
                if (cur >= 0) {
                    write_row(cur, false);
                    next = cur + 1;
                }
                for (int q = next; q < lr; ++q) write_row(q, true);
                next = lr;
                cur = lr;
#pragma unroll
                for (int q = 0; q < NLM; ++q) acc[q] = 0.f;
            }
            const int64_t jb = ((int64_t)s.col[e] * NLM) * F + c;
            const float dr = s.dr[e];
            const float h0 = a.Hin[jb];
            const float dh0 = FIRST ? 0.f : a.dHin[jb];
            acc[0] += dR[0][e] * dr * h0 + R[0][e] * dh0;
#pragma unroll
            for (int l = 1; l <= LMAX; ++l) {
                const int la = 2 * l - 1, lb = 2 * l;
                const float ta = dR[la][e] * dr * h0 + R[la][e] * dh0;   // d(Rla h0)
                const float pa = R[la][e] * h0;
#pragma unroll
                for (int m = 0; m < 2 * l + 1; ++m) {
                    const int q = l * l + m;
                    float v = ta * s.Y[e][q] + pa * s.dY[e][q];
                    if (!FIRST) v += dR[lb][e] * dr * a.Hin[jb + q * F] + R[lb][e] * a.dHin[jb + q * F];
                    acc[q] += v;
                }
            }
        }
        __syncthreads();
    }
    if (cur >= 0) {
        write_row(cur, false);
        next = cur + 1;
    }
    for (int q = next; q < nrows; ++q) write_row(q, true);
}

// Node tangent: thread d = output channel, TA atoms per block.
constexpr int TAN = 8;

template <int F, int LMAX, bool LAST>
__global__ void __launch_bounds__(F) k_node_tangent(TangentArgs a, const float* __restrict__ W0T,
                                                    const float* __restrict__ U1T,
                                                    const float* __restrict__ U2T,
                                                    const float* __restrict__ V1T,
                                                    const float* __restrict__ V2T) {
    constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    __shared__ float sdA[TAN][NLM][F];
    __shared__ float sdB[TAN][LMAX][F];
    const int d = threadIdx.x;
    const int64_t a0 = (int64_t)blockIdx.x * TAN;
    const int na = (int)min((int64_t)TAN, a.n - a0);
#pragma unroll
    for (int t = 0; t < TAN; ++t)
#pragma unroll
        for (int q = 0; q < NLM; ++q)
            sdA[t][q][d] = t < na ? a.dA[((a0 + t) * NLM + q) * F + d] : 0.f;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < TAN; ++t) {
        const int64_t base = ((a0 + t) * NLM) * F + d;
        float b1 = 0.f, b2 = 0.f;
        if (t < na) {
#pragma unroll
            for (int m = 1; m < 4; ++m) b1 += 2.f * a.A[base + m * F] * sdA[t][m][d];
            if (LMAX >= 2) {
#pragma unroll
                for (int m = 4; m < 9; ++m) b2 += 2.f * a.A[base + m * F] * sdA[t][m][d];
            }
        }
        sdB[t][0][d] = b1;
        if (LMAX >= 2) sdB[t][1][d] = b2;
    }
    __syncthreads();
    float ds[TAN], dv[TAN][NLM - 1];
#pragma unroll
    for (int t = 0; t < TAN; ++t) {
        ds[t] = 0.f;
#pragma unroll
        for (int q = 0; q < NLM - 1; ++q) dv[t][q] = 0.f;
    }
    for (int c = 0; c < F; ++c) {
        const float w0 = __ldg(&W0T[c * F + d]);
        const float u1 = __ldg(&U1T[c * F + d]);
        const float u2 = LMAX >= 2 ? __ldg(&U2T[c * F + d]) : 0.f;
        const float v1 = LAST ? 0.f : __ldg(&V1T[c * F + d]);
        const float v2 = (LAST || LMAX < 2) ? 0.f : __ldg(&V2T[c * F + d]);
#pragma unroll
        for (int t = 0; t < TAN; ++t) {
            ds[t] += w0 * sdA[t][0][c] + u1 * sdB[t][0][c];
            if (LMAX >= 2) ds[t] += u2 * sdB[t][1][c];
            if (!LAST) {
#pragma unroll
                for (int m = 1; m < 4; ++m) dv[t][m - 1] += v1 * sdA[t][m][c];
                if (LMAX >= 2) {
#pragma unroll
                    for (int m = 4; m < 9; ++m) dv[t][m - 1] += v2 * sdA[t][m][c];
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < TAN; ++t) {
        if (t >= na) break;
        const int64_t base = ((a0 + t) * NLM) * F + d;
        const float dh0 = a.first ? 0.f : a.dHin[base];
        a.dHout[base] = dh0 + silu_grad(a.S[(a0 + t) * F + d]) * ds[t];
        if (!LAST) {
#pragma unroll
            for (int q = 1; q < NLM; ++q)
                a.dHout[base + q * F] = (a.first ? 0.f : a.dHin[base + q * F]) + dv[t][q - 1];
        }
    }
}

template <int F, int LMAX>
int tangent_impl(const TangentArgs& a, cudaStream_t st) {
    if (a.n == 0) return MP_OK;
    const LayerW& w = *a.w;
    const unsigned ge = (unsigned)((a.n + RPBT - 1) / RPBT);
    if (a.first)
        k_edge_tangent<F, LMAX, true><<<ge, F, 0, st>>>(a, w.W1, w.W2T, w.W3T);
    else
        k_edge_tangent<F, LMAX, false><<<ge, F, 0, st>>>(a, w.W1, w.W2T, w.W3T);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

template <int F, int LMAX>
int node_tangent_impl(const TangentArgs& a, cudaStream_t st) {
    if (a.n == 0) return MP_OK;
    const LayerW& w = *a.w;
    const unsigned gn = (unsigned)((a.n + TAN - 1) / TAN);
    const float* U2T = LMAX >= 2 ? w.UT[1] : w.UT[0];
    const float* V2T = LMAX >= 2 ? w.VT[1] : w.VT[0];
    if (a.last)
        k_node_tangent<F, LMAX, true><<<gn, F, 0, st>>>(a, w.W0T, w.UT[0], U2T, w.VT[0], V2T);
    else
        k_node_tangent<F, LMAX, false><<<gn, F, 0, st>>>(a, w.W0T, w.UT[0], U2T, w.VT[0], V2T);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int launch_edge_tangent_f32(const Model& m, const TangentArgs& a, cudaStream_t st) {
    if (m.d.F == 128 && m.d.lmax == 2) return tangent_impl<128, 2>(a, st);
    if (m.d.F == 64 && m.d.lmax == 1) return tangent_impl<64, 1>(a, st);
    return MP_ERR_UNSUPPORTED;
}

int launch_node_tangent_f32(const Model& m, const TangentArgs& a, cudaStream_t st) {
    if (m.d.F == 128 && m.d.lmax == 2) return node_tangent_impl<128, 2>(a, st);
    if (m.d.F == 64 && m.d.lmax == 1) return node_tangent_impl<64, 1>(a, st);
    return MP_ERR_UNSUPPORTED;
}

}  // namespace mp

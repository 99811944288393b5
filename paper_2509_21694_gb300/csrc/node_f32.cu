// Node update of one layer and its adjoint, FP32 on CUDA cores.
//
// Forward:  S  = W0 A0 + sum_l Ul Bl + b,   Bl[c] = sum_m Al[c, m]^2
//           h0' = h0 + silu(S),             hl' = hl + Vl Al  (Vl on channels)
// Adjoint:  gS  = G0' * silu'(S)
//           dE/dA0 = W0^T gS,  dE/dBl = Ul^T gS
//           dE/dAl[., m] = Vl^T Gl'[., m] + 2 Al[., m] * dE/dBl
//           alpha = dE/dA / N_avg   (coefficient of the raw message sums)
// A block handles TA atoms; a thread owns one output channel (forward) or
// one input channel (adjoint) and streams the weight rows coalesced.
#include "kernels.h"

namespace mp {

namespace {

constexpr int TA = 8;

template <int F, int LMAX, bool LAST>
__global__ void __launch_bounds__(F) k_node_fwd(NodeArgs a, const float* __restrict__ W0T,
                                                const float* __restrict__ U1T,
                                                const float* __restrict__ U2T,
                                                const float* __restrict__ bias,
                                                const float* __restrict__ V1T,
                                                const float* __restrict__ V2T) {
    constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    __shared__ __align__(16) float sA[TA][NLM][F];
    __shared__ __align__(16) float sB[TA][LMAX][F];
    const int d = threadIdx.x;
    const int64_t a0 = (int64_t)blockIdx.x * TA;
    const int na = (int)min((int64_t)TA, a.n - a0);
#pragma unroll
    for (int t = 0; t < TA; ++t)
#pragma unroll
        for (int q = 0; q < NLM; ++q)
            sA[t][q][d] = t < na ? a.A[((a0 + t) * NLM + q) * F + d] : 0.f;
    __syncthreads();
#pragma unroll
    for (int t = 0; t < TA; ++t) {
        float b1 = 0.f;
#pragma unroll
        for (int m = 1; m < 4; ++m) b1 = fmaf(sA[t][m][d], sA[t][m][d], b1);
        sB[t][0][d] = b1;
        if (LMAX >= 2) {
            float b2 = 0.f;
#pragma unroll
            for (int m = 4; m < 9; ++m) b2 = fmaf(sA[t][m][d], sA[t][m][d], b2);
            sB[t][1][d] = b2;
        }
    }
    __syncthreads();
    float s[TA], hv[TA][NLM - 1];
    const float bd = bias[d];
#pragma unroll
    for (int t = 0; t < TA; ++t) {
        s[t] = bd;
#pragma unroll
        for (int q = 0; q < NLM - 1; ++q) hv[t][q] = 0.f;
    }
    // four input channels per step: the shared-memory reads are float4
    for (int c4 = 0; c4 < F; c4 += 4) {
        float w0[4], u1[4], u2[4], v1[4], v2[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = c4 + k;
            w0[k] = __ldg(&W0T[c * F + d]);
            u1[k] = __ldg(&U1T[c * F + d]);
            u2[k] = LMAX >= 2 ? __ldg(&U2T[c * F + d]) : 0.f;
            v1[k] = LAST ? 0.f : __ldg(&V1T[c * F + d]);
            v2[k] = (LAST || LMAX < 2) ? 0.f : __ldg(&V2T[c * F + d]);
        }
#pragma unroll
        for (int t = 0; t < TA; ++t) {
            const float4 a0v = *reinterpret_cast<const float4*>(&sA[t][0][c4]);
            const float4 b1v = *reinterpret_cast<const float4*>(&sB[t][0][c4]);
            float acc = s[t];
            acc = fmaf(w0[0], a0v.x, acc); acc = fmaf(u1[0], b1v.x, acc);
            acc = fmaf(w0[1], a0v.y, acc); acc = fmaf(u1[1], b1v.y, acc);
            acc = fmaf(w0[2], a0v.z, acc); acc = fmaf(u1[2], b1v.z, acc);
            acc = fmaf(w0[3], a0v.w, acc); acc = fmaf(u1[3], b1v.w, acc);
            if (LMAX >= 2) {
                const float4 b2v = *reinterpret_cast<const float4*>(&sB[t][1][c4]);
                acc = fmaf(u2[0], b2v.x, acc); acc = fmaf(u2[1], b2v.y, acc);
                acc = fmaf(u2[2], b2v.z, acc); acc = fmaf(u2[3], b2v.w, acc);
            }
            s[t] = acc;
            if (!LAST) {
#pragma unroll
                for (int q = 1; q < NLM; ++q) {
                    const float4 av = *reinterpret_cast<const float4*>(&sA[t][q][c4]);
                    const float* v = q < 4 ? v1 : v2;
                    float h = hv[t][q - 1];
                    h = fmaf(v[0], av.x, h);
                    h = fmaf(v[1], av.y, h);
                    h = fmaf(v[2], av.z, h);
                    h = fmaf(v[3], av.w, h);
                    hv[t][q - 1] = h;
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < TA; ++t) {
        if (t >= na) break;
        const int64_t base = ((a0 + t) * NLM) * F + d;
        a.S[(a0 + t) * F + d] = s[t];
        a.Hout[base] = a.Hin[base] + silu(s[t]);
        if (!LAST) {
#pragma unroll
            for (int q = 1; q < NLM; ++q)
                a.Hout[base + q * F] = (a.first ? 0.f : a.Hin[base + q * F]) + hv[t][q - 1];
        }
    }
}

template <int F, int LMAX, bool LAST>
__global__ void __launch_bounds__(F) k_node_bwd(NodeArgs a, const float* __restrict__ W0,
                                                const float* __restrict__ U1,
                                                const float* __restrict__ U2,
                                                const float* __restrict__ V1,
                                                const float* __restrict__ V2) {
    constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    __shared__ float gs[TA][F];
    __shared__ float sG[LAST ? 1 : TA][LAST ? 1 : NLM - 1][F];
    const int c = threadIdx.x;
    const int64_t a0 = (int64_t)blockIdx.x * TA;
    const int na = (int)min((int64_t)TA, a.n - a0);
#pragma unroll
    for (int t = 0; t < TA; ++t) {
        const int64_t base = ((a0 + t) * NLM) * F + c;
        gs[t][c] = t < na ? a.Gout[base] * silu_grad(a.S[(a0 + t) * F + c]) : 0.f;
        if (!LAST) {
#pragma unroll
            for (int q = 1; q < NLM; ++q) sG[t][q - 1][c] = t < na ? a.Gout[base + q * F] : 0.f;
        }
    }
    __syncthreads();
    float dA0[TA], dB[TA][LMAX], dAl[TA][NLM - 1];
#pragma unroll
    for (int t = 0; t < TA; ++t) {
        dA0[t] = 0.f;
#pragma unroll
        for (int l = 0; l < LMAX; ++l) dB[t][l] = 0.f;
#pragma unroll
        for (int q = 0; q < NLM - 1; ++q) dAl[t][q] = 0.f;
    }
#pragma unroll 2
    for (int dd = 0; dd < F; ++dd) {
        const float w0 = __ldg(&W0[dd * F + c]);
        const float u1 = __ldg(&U1[dd * F + c]);
        const float u2 = LMAX >= 2 ? __ldg(&U2[dd * F + c]) : 0.f;
        const float v1 = LAST ? 0.f : __ldg(&V1[dd * F + c]);
        const float v2 = (LAST || LMAX < 2) ? 0.f : __ldg(&V2[dd * F + c]);
#pragma unroll
        for (int t = 0; t < TA; ++t) {
            const float g = gs[t][dd];
            dA0[t] = fmaf(w0, g, dA0[t]);
            dB[t][0] = fmaf(u1, g, dB[t][0]);
            if (LMAX >= 2) dB[t][1] = fmaf(u2, g, dB[t][1]);
            if (!LAST) {
#pragma unroll
                for (int m = 1; m < 4; ++m) dAl[t][m - 1] = fmaf(v1, sG[t][m - 1][dd], dAl[t][m - 1]);
                if (LMAX >= 2) {
#pragma unroll
                    for (int m = 4; m < 9; ++m) dAl[t][m - 1] = fmaf(v2, sG[t][m - 1][dd], dAl[t][m - 1]);
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < TA; ++t) {
        if (t >= na) break;
        const int64_t base = ((a0 + t) * NLM) * F + c;
        a.Alpha[base] = dA0[t] * a.inv_navg;
#pragma unroll
        for (int q = 1; q < NLM; ++q) {
            const int l = q < 4 ? 0 : 1;
            const float v = dAl[t][q - 1] + 2.f * a.A[base + q * F] * dB[t][l];
            a.Alpha[base + q * F] = v * a.inv_navg;
        }
    }
}

template <int F, int LMAX>
int node_fwd_impl(const NodeArgs& a, cudaStream_t st) {
    if (a.n == 0) return MP_OK;
    const LayerW& w = *a.w;
    dim3 grid((unsigned)((a.n + TA - 1) / TA));
    const float* U2T = LMAX >= 2 ? w.UT[1] : w.UT[0];
    const float* V2T = LMAX >= 2 ? w.VT[1] : w.VT[0];
    if (a.last)
        k_node_fwd<F, LMAX, true><<<grid, F, 0, st>>>(a, w.W0T, w.UT[0], U2T, w.b, w.VT[0], V2T);
    else
        k_node_fwd<F, LMAX, false><<<grid, F, 0, st>>>(a, w.W0T, w.UT[0], U2T, w.b, w.VT[0], V2T);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

template <int F, int LMAX>
int node_bwd_impl(const NodeArgs& a, cudaStream_t st) {
    if (a.n == 0) return MP_OK;
    const LayerW& w = *a.w;
    dim3 grid((unsigned)((a.n + TA - 1) / TA));
    const float* U2 = LMAX >= 2 ? w.U[1] : w.U[0];
    const float* V2 = LMAX >= 2 ? w.V[1] : w.V[0];
    if (a.last)
        k_node_bwd<F, LMAX, true><<<grid, F, 0, st>>>(a, w.W0, w.U[0], U2, w.V[0], V2);
    else
        k_node_bwd<F, LMAX, false><<<grid, F, 0, st>>>(a, w.W0, w.U[0], U2, w.V[0], V2);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int launch_node_fwd_f32(const Model& m, const NodeArgs& a, cudaStream_t st) {
    if (m.d.F == 128 && m.d.lmax == 2) return node_fwd_impl<128, 2>(a, st);
    if (m.d.F == 64 && m.d.lmax == 1) return node_fwd_impl<64, 1>(a, st);
    return MP_ERR_UNSUPPORTED;
}

int launch_node_bwd_f32(const Model& m, const NodeArgs& a, cudaStream_t st) {
    if (m.d.F == 128 && m.d.lmax == 2) return node_bwd_impl<128, 2>(a, st);
    if (m.d.F == 64 && m.d.lmax == 1) return node_bwd_impl<64, 1>(a, st);
    return MP_ERR_UNSUPPORTED;
}

}  // namespace mp

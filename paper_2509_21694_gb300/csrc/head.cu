// Training of the per-atom correction head on energies and forces of a
// reference (teacher) model, with the message-passing backbone frozen.
//
// Student: E = E_backbone(K layers) + sum_i head(h_i), head(h) = w2 .
// silu(W1 h + b1) + b2, h_i = h0_i^(K); F = -grad E through the library's
// adjoint.  Loss per snapshot of N atoms:
//   L = (dE / N)^2 + lambda / (3N) sum_k |dF_k|^2,  dE = E - E_ref, dF = F - F_ref.
// Gradient: the energy term gives 2 dE / N^2 sum_i d head(h_i) / d theta; the
// force term is -2 lambda / (3N) sum_i d Q_i / d theta with
// Q_i = g_i(theta) . t_i, g_i = d head / d h_i and t_i = J_i dF the tangent of
// h_i along the displacement field dF (forward-mode pass of the backbone).
// With z = W1 h + b1, u = W1 t, s1 = silu'(z), s2 = silu''(z):
//   dQ/dW1[k][c] = w2_k (s2_k u_k h_c + s1_k t_c),  dQ/db1_k = w2_k s2_k u_k,
//   dQ/dw2_k = s1_k u_k,  dQ/db2 = 0.
// Reductions over atoms run in a fixed order (deterministic).
#include <cmath>

#include "kernels.h"

namespace mp {

int reduce_sum(const double* v, int64_t n, double* out, DevBuf& tmp, cudaStream_t st);

namespace {

__device__ __forceinline__ float silu_grad2(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f - s) * (2.f + z * (1.f - 2.f * s));
}

// dF in cell order (the tangent direction) and |dF|^2 per atom.
__global__ void k_force_residual(int64_t n, const int32_t* __restrict__ perm,
                                 const float* __restrict__ f, const float* __restrict__ f_ref,
                                 float* __restrict__ v, double* __restrict__ sq) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm[s];
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float d = f[3 * i + q] - f_ref[3 * i + q];
        v[3 * s + q] = d;
        acc += (double)d * (double)d;
    }
    sq[s] = acc;
}

// loss = (dE/N)^2 + lambda/(3N) sum |dF|^2 ; coefficients cE = 2 dE / N^2,
// cF = -2 lambda / (3N).
__global__ void k_loss(const double* __restrict__ e, const double* __restrict__ e_ref,
                       const double* __restrict__ sqsum, int64_t n, double lambda,
                       double* __restrict__ loss, double* __restrict__ coef) {
    const double dE = *e - *e_ref;
    const double N = (double)n;
    *loss = (dE / N) * (dE / N) + lambda / (3.0 * N) * *sqsum;
    coef[0] = 2.0 * dE / (N * N);
    coef[1] = -2.0 * lambda / (3.0 * N);
}

// Per atom (warp per atom, lane = hidden unit k): alpha_k (coefficient of
// h_c), beta_k (of t_c), and the b1 and w2 contributions.
__global__ void k_head_coef(int64_t n, int F, int NLM, const float* __restrict__ H,
                            const float* __restrict__ dH, const float* __restrict__ head,
                            const double* __restrict__ coef, float* __restrict__ out) {
    extern __shared__ float sh[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= n) return;
    float* h = sh + wib * 2 * F;
    float* t = h + F;
    for (int c = lane; c < F; c += 32) {
        h[c] = H[(i * NLM) * F + c];
        t[c] = dH[(i * NLM) * F + c];
    }
    __syncwarp();
    const float* W1 = head;
    const float* b1 = head + kHeadH * F;
    const float* w2 = b1 + kHeadH;
    float z = b1[lane], u = 0.f;
    for (int c = 0; c < F; ++c) {
        z = fmaf(W1[lane * F + c], h[c], z);
        u = fmaf(W1[lane * F + c], t[c], u);
    }
    const float cE = (float)coef[0], cF = (float)coef[1];
    const float s1 = silu_grad(z), s2 = silu_grad2(z), wk = w2[lane];
    float* o = out + i * 4 * kHeadH;
    o[lane] = cE * wk * s1 + cF * wk * s2 * u;            // alpha_k, also d/db1_k
    o[kHeadH + lane] = cF * wk * s1;                     // beta_k
    o[2 * kHeadH + lane] = cE * silu(z) + cF * s1 * u;   // d/dw2_k
}

// grad W1[k][c] = sum_i alpha_ik h_ic + beta_ik t_ic  (block = k, thread = c);
// the last block sums the b1, w2 and b2 parts.
__global__ void k_head_reduce(int64_t n, int F, int NLM, const float* __restrict__ H,
                              const float* __restrict__ dH, const float* __restrict__ co,
                              const double* __restrict__ coef, double* __restrict__ grad) {
    const int k = blockIdx.x;
    if (k < kHeadH) {
        for (int c = threadIdx.x; c < F; c += blockDim.x) {
            double acc = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                const float* o = co + i * 4 * kHeadH;
                acc += (double)o[k] * (double)H[(i * NLM) * F + c] +
                       (double)o[kHeadH + k] * (double)dH[(i * NLM) * F + c];
            }
            grad[(int64_t)k * F + c] = acc;
        }
    } else {
        for (int q = threadIdx.x; q < 2 * kHeadH + 1; q += blockDim.x) {
            double acc = 0.0;
            if (q < 2 * kHeadH) {
                const int off = q < kHeadH ? q : 2 * kHeadH + (q - kHeadH);
                for (int64_t i = 0; i < n; ++i) acc += (double)co[i * 4 * kHeadH + off];
            } else {
                acc = coef[0] * (double)n;                 // d/db2
            }
            grad[(int64_t)kHeadH * F + q] = acc;
        }
    }
}

__global__ void k_adam(int64_t np, float* __restrict__ p, float* __restrict__ m,
                       float* __restrict__ v, const double* __restrict__ g, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    const float gq = (float)g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

}  // namespace

int64_t head_param_count(const Model& m) { return (int64_t)kHeadH * m.d.F + 2 * kHeadH + 1; }

// Loss and gradient of the head parameters for one snapshot (whole graph,
// no partitions).  Runs the student evaluation (backbone + head, forward and
// adjoint), then the tangent pass of the backbone along dF, then the
// per-atom gradient terms and their fixed-order sums.  The evaluation's
// workspace (cell-ordered positions, per-layer features, messages and
// pre-activations of the unpartitioned graph) is read after it returns.
int head_loss_grad(mp_ctx* ctx, const double* d_pos, const int32_t* d_species, const Graph& g,
                   int K, int precision, const double* d_e_ref, const float* d_f_ref,
                   double lambda, double* d_loss, double* d_grad) {
    const Model& m = ctx->model;
    if (!d_e_ref || !d_f_ref || !d_loss || K < 1) return MP_ERR_ARG;
    cudaStream_t st = ctx->stream;
    Workspace& ws = ctx->ws;
    const int64_t n = g.n;
    const int F = m.d.F, NLM = m.NLM;
    const int64_t feat = n * NLM * F;
    const int64_t np = head_param_count(m);
    DevBuf& hb = ws.headbuf;
    // scratch: energy (1), coef (2), sqsum (1), |dF|^2 [n], forces [n][3] f32,
    // v [n][3] f32, per-atom coefficients [n][4][32] f32, grad [np] if needed
    const size_t bytes = sizeof(double) * (8 + n + np) + sizeof(float) * (9 * n + 4 * kHeadH * n);
    MP_TRY(hb.reserve(bytes + 256));
    double* e_s = hb.as<double>();
    double* coef = e_s + 1;
    double* sqsum = coef + 2;
    double* sq = e_s + 8;
    double* grad_tmp = sq + n;
    float* f_s = reinterpret_cast<float*>(grad_tmp + np);
    float* v = f_s + 3 * n;
    float* co = v + 3 * n;
    MP_TRY(evaluate(ctx, d_pos, d_species, g, nullptr, K, precision, 1, e_s, f_s, nullptr));
    k_force_residual<<<grid_for(n, 256), 256, 0, st>>>(n, g.perm.as<int32_t>(), f_s, d_f_ref, v, sq);
    note_launch();
    MP_TRY(reduce_sum(sq, n, sqsum, ws.red, st));
    k_loss<<<1, 1, 0, st>>>(e_s, d_e_ref, sqsum, n, lambda, d_loss, coef);
    note_launch();
    if (!d_grad) {
        MP_CUDA_TRY(cudaGetLastError());
        return MP_OK;
    }
    // tangent pass along dF: dH ping-pongs between two buffers, dA reuses alpha
    float* dH[2] = {ws.G0.as<float>(), ws.G1.as<float>()};
    const EdgeConst kc = make_edge_const(m.d, g.box);
    TangentArgs ta{};
    ta.n = n;
    ta.row_ptr = g.row_ptr.as<int64_t>();
    ta.col = g.col.as<int32_t>();
    ta.shift = g.shift.as<int8_t>();
    ta.x = ws.xw.as<double>();
    ta.v = v;
    ta.k = kc;
    for (int t = 0; t < K; ++t) {
        ta.w = &m.layers[t];
        ta.first = t == 0;
        ta.last = t == K - 1;
        ta.Hin = ws.H.as<float>() + t * feat;
        ta.dHin = dH[t & 1];
        ta.dAout = ws.alpha.as<float>();
        MP_TRY(launch_edge_tangent_f32(m, ta, st));
        ta.A = ws.A.as<float>() + t * feat;
        ta.dA = ws.alpha.as<float>();
        ta.S = ws.S.as<float>() + t * n * F;
        ta.dHout = dH[(t + 1) & 1];
        MP_TRY(launch_node_tangent_f32(m, ta, st));
    }
    const float* HK = ws.H.as<float>() + (int64_t)K * feat;
    const float* dHK = dH[K & 1];
    const int wpb = 4;
    k_head_coef<<<grid_for(n, wpb), 32 * wpb, sizeof(float) * 2 * F * wpb, st>>>(
        n, F, NLM, HK, dHK, m.head, coef, co);
    note_launch();
    k_head_reduce<<<kHeadH + 1, 128, 0, st>>>(n, F, NLM, HK, dHK, co, coef, d_grad);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int head_adam(mp_ctx* ctx, const double* d_grad, double lr, double beta1, double beta2,
              double eps, int64_t step) {
    const Model& m = ctx->model;
    if (!d_grad || step < 1 || !(lr > 0)) return MP_ERR_ARG;
    const int64_t np = head_param_count(m);
    DevBuf& ad = ctx->ws.adam;
    if (ad.bytes < sizeof(float) * 2 * np || step == 1) {
        MP_TRY(ad.reserve(sizeof(float) * 2 * np));
        MP_CUDA_TRY(cudaMemsetAsync(ad.p, 0, sizeof(float) * 2 * np, ctx->stream));
    }
    float* mm = ad.as<float>();
    const float c1 = (float)(1.0 - pow(beta1, (double)step));
    const float c2 = (float)(1.0 - pow(beta2, (double)step));
    k_adam<<<grid_for(np, 256), 256, 0, ctx->stream>>>(np, m.head, mm, mm + np, d_grad, (float)lr,
                                                      (float)beta1, (float)beta2, (float)eps, c1, c2);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace mp

// Layer diagnostics (Methods, "Mean Feature Shift and Linear CKA") on the
// scalar features h0 of every layer of one unpartitioned evaluation:
//   centred features  H~ = H - (1/N) 1 1^T H
//   MFS(t -> t+1)     = (1/N) || H~(t+1) - H~(t) ||_F
//   CKA(t -> t+1)     = || H~(t)^T H~(t+1) ||_F^2
//                       / ( || H~(t)^T H~(t) ||_F || H~(t+1)^T H~(t+1) ||_F )
// The column means, the squared shift and the F x F Gram matrices are summed
// in FP64 in a fixed order (per-block partials, then an ordered sum), so the
// results are deterministic; the Frobenius norms and ratios are taken on the
// host.  The Gram matrices are dense contractions over the atoms, but FP64
// is kept: the CKA is a ratio of nearly equal quantities when layers are
// similar, and the diagnostic is not on the MD path.
#include <cmath>
#include <vector>

#include "kernels.h"

namespace mp {

namespace {

constexpr int kTile = 32;      // channels per Gram tile edge
constexpr int kChunk = 64;     // atoms staged in shared memory at a time
constexpr int kSplits = 64;    // atom ranges, one partial Gram tile each
constexpr int kRedBlock = 256;

// Column means of h0 of one layer: block c sums channel c over all atoms.
__global__ void __launch_bounds__(kRedBlock) k_col_mean(const float* __restrict__ H, int64_t n,
                                                        int F, int NLM, double* __restrict__ mean) {
    __shared__ double sh[kRedBlock];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kRedBlock) s += (double)H[i * NLM * F + c];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kRedBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[c] = sh[0] / (double)n;
}

// Per-block partial sums of sum_c ((hb - mb) - (ha - ma))^2 over a strided
// set of atoms.
__global__ void __launch_bounds__(kRedBlock) k_shift_partial(
    const float* __restrict__ Ha, const float* __restrict__ Hb, const double* __restrict__ ma,
    const double* __restrict__ mb, int64_t n, int F, int NLM, double* __restrict__ part) {
    __shared__ double sh[kRedBlock];
    double s = 0.0;
    const int64_t total = n * F;
    for (int64_t q = (int64_t)blockIdx.x * kRedBlock + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * kRedBlock) {
        const int64_t i = q / F;
        const int c = (int)(q % F);
        const double d = ((double)Hb[i * NLM * F + c] - mb[c]) - ((double)Ha[i * NLM * F + c] - ma[c]);
        s += d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kRedBlock / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// Tile (blockIdx.x, blockIdx.y) of H~a^T H~b summed over atom range
// blockIdx.z: thread (r, q) accumulates row r, columns 4 q .. 4 q + 3.
__global__ void __launch_bounds__(256) k_gram_partial(
    const float* __restrict__ Ha, const float* __restrict__ Hb, const double* __restrict__ ma,
    const double* __restrict__ mb, int64_t n, int F, int NLM, double* __restrict__ part) {
    __shared__ double xs[kChunk][kTile], ys[kChunk][kTile];
    const int ca0 = blockIdx.x * kTile, cb0 = blockIdx.y * kTile, sp = blockIdx.z;
    const int r = threadIdx.x >> 3, q = threadIdx.x & 7;
    const int64_t i_beg = n * sp / kSplits, i_end = n * (sp + 1) / kSplits;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t i0 = i_beg; i0 < i_end; i0 += kChunk) {
        for (int t = threadIdx.x; t < kChunk * kTile; t += 256) {
            const int k = t / kTile, c = t % kTile;
            const int64_t i = i0 + k;
            const bool ok = i < i_end;
            xs[k][c] = ok ? (double)Ha[i * NLM * F + ca0 + c] - ma[ca0 + c] : 0.0;
            ys[k][c] = ok ? (double)Hb[i * NLM * F + cb0 + c] - mb[cb0 + c] : 0.0;
        }
        __syncthreads();
        for (int k = 0; k < kChunk; ++k) {
            const double x = xs[k][r];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = fma(x, ys[k][4 * q + j], acc[j]);
        }
        __syncthreads();
    }
    double* out = part + (size_t)sp * F * F;
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(size_t)(ca0 + r) * F + cb0 + 4 * q + j] = acc[j];
}

// Ordered sum of the partials: out[k] = sum_s part[s][k].
__global__ void k_ordered_sum(const double* __restrict__ part, int n_parts, int64_t len,
                              double* __restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    double s = 0.0;
    for (int p = 0; p < n_parts; ++p) s += part[(size_t)p * len + k];
    out[k] = s;
}

double frob(const std::vector<double>& g) {
    double s = 0.0;
    for (double v : g) s += v * v;
    return std::sqrt(s);
}

}  // namespace

int layer_stats(mp_ctx* ctx, const double* d_pos, const int32_t* d_species, const Graph& g, int K,
                int precision, double* h_mfs, double* h_cka) {
    const Model& m = ctx->model;
    if (K < 1 || K > m.d.n_layers_full || !h_mfs || !h_cka) return MP_ERR_ARG;
    const int F = m.d.F, NLM = m.NLM;
    if (F % kTile != 0) return MP_ERR_UNSUPPORTED;
    const int64_t n = g.n;
    cudaStream_t st = ctx->stream;
    DevBuf ef, stats;
    BufGuard guard{&ef, &stats};
    MP_TRY(ef.reserve(sizeof(double) + sizeof(float) * 3 * n + 64));
    MP_TRY(evaluate(ctx, d_pos, d_species, g, nullptr, K, precision, 0, ef.as<double>(),
                    reinterpret_cast<float*>(ef.as<double>() + 1), nullptr));
    // layer t's h0 (rows in cell order; every statistic is order independent)
    const int64_t feat = n * NLM * F;
    const float* H = ctx->ws.H.as<float>();
    const int n_shift_blocks = 2 * ctx->num_sms;
    const size_t FF = (size_t)F * F;
    // means [K+1][F], shift partials, Gram partials [kSplits][F][F], Gram [F][F]
    MP_TRY(stats.reserve(sizeof(double) * ((K + 1) * F + n_shift_blocks + 1 +
                                           kSplits * FF + FF)));
    double* mean = stats.as<double>();
    double* spart = mean + (size_t)(K + 1) * F;
    double* ssum = spart + n_shift_blocks;
    double* gpart = ssum + 1;
    double* gram = gpart + kSplits * FF;
    for (int t = 0; t <= K; ++t) {
        k_col_mean<<<F, kRedBlock, 0, st>>>(H + t * feat, n, F, NLM, mean + (size_t)t * F);
        note_launch();
    }
    auto gram_norm = [&](int a, int b, std::vector<double>& host) -> int {
        dim3 grid(F / kTile, F / kTile, kSplits);
        k_gram_partial<<<grid, 256, 0, st>>>(H + a * feat, H + b * feat, mean + (size_t)a * F,
                                            mean + (size_t)b * F, n, F, NLM, gpart);
        note_launch();
        k_ordered_sum<<<grid_for((int64_t)FF, 256), 256, 0, st>>>(gpart, kSplits, (int64_t)FF, gram);
        note_launch();
        host.resize(FF);
        MP_CUDA_TRY(cudaMemcpyAsync(host.data(), gram, sizeof(double) * FF, cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        return MP_OK;
    };
    std::vector<double> g_self_prev, g_self, g_cross;
    MP_TRY(gram_norm(0, 0, g_self_prev));
    for (int t = 0; t < K; ++t) {
        k_shift_partial<<<n_shift_blocks, kRedBlock, 0, st>>>(H + t * feat, H + (t + 1) * feat,
                                                               mean + (size_t)t * F,
                                                               mean + (size_t)(t + 1) * F, n, F,
                                                               NLM, spart);
        note_launch();
        k_ordered_sum<<<1, 32, 0, st>>>(spart, n_shift_blocks, 1, ssum);
        note_launch();
        double shift = 0.0;
        MP_CUDA_TRY(cudaMemcpyAsync(&shift, ssum, sizeof(double), cudaMemcpyDeviceToHost, st));
        MP_TRY(gram_norm(t, t + 1, g_cross));
        MP_TRY(gram_norm(t + 1, t + 1, g_self));
        h_mfs[t] = std::sqrt(shift) / (double)n;
        const double c = frob(g_cross);
        h_cka[t] = c * c / (frob(g_self_prev) * frob(g_self));
        g_self_prev.swap(g_self);
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace mp

using namespace mp;

extern "C" int mp_layer_stats(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                              const mp_graph* g, int n_layers, int precision, double* h_mfs,
                              double* h_cka) {
    if (!ctx || !g || !d_pos || !d_species) return MP_ERR_ARG;
    return layer_stats(ctx, d_pos, d_species, g->g, n_layers, precision, h_mfs, h_cka);
}

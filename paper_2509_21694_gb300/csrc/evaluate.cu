// Energy and forces of the first K layers (the pruned model), whole graph or
// partition by partition.
//
// Per sub-system (the whole graph, or one partition's extended set with its
// local CSR): embedding -> K x (edge forward, node update) -> readout
// E_i = w_out . h0^(K) + e0[z_i] (+ head) (+ pair term) -> adjoint seeded
// with s_i (1 on roots, 0 on halo atoms) -> K x (node adjoint, edge
// adjoint) accumulating F.  Partition results are combined in partition
// order: root energies are written once each, forces are summed (Methods,
// "Global Output Integration": E = sum of root energies, F = sum over
// partitions of the gradients of root energies).
#include "kernels.h"

namespace mp {

namespace {

constexpr int kErrSpecies = 8;   // error word: a species index outside 0..S-1

// Positions in cell order, wrapped into the box (wrap != 0), or as given: a
// skin list reused between builds keeps the image shifts of its build, so
// the positions must continue without jumps by a box length until the next
// build wraps them.
__global__ void k_gather_pos(const double* __restrict__ pos, const int32_t* __restrict__ species,
                             const int32_t* __restrict__ perm, int64_t n, double L0, double L1,
                             double L2, int n_species, int wrap, double* __restrict__ xs,
                             int32_t* __restrict__ sp, int* __restrict__ err) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm[s];
    const double L[3] = {L0, L1, L2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double x = pos[3 * i + a];
        double w = x;
        if (wrap) {
            w = __dsub_rn(x, __dmul_rn(L[a], floor(__ddiv_rn(x, L[a]))));
            if (w >= L[a]) w = __dsub_rn(w, L[a]);
        }
        xs[3 * s + a] = w;
    }
    int z = species[i];
    if (z < 0 || z >= n_species) {   // reported after the evaluation; never indexes out of range
        atomicOr(err, kErrSpecies);
        z = 0;
    }
    sp[s] = z;
}

__global__ void k_gather_local(const int32_t* __restrict__ gid, int64_t n,
                               const double* __restrict__ xs, const int32_t* __restrict__ sp,
                               double* __restrict__ xl, int32_t* __restrict__ spl) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int64_t s = gid[l];
    xl[3 * l] = xs[3 * s];
    xl[3 * l + 1] = xs[3 * s + 1];
    xl[3 * l + 2] = xs[3 * s + 2];
    spl[l] = sp[s];
}

// h0 of layer 0 from the species embedding.  The l >= 1 features of layer 0
// are zero and are not stored: every reader of layer 0 skips them.
__global__ void k_embed(const int32_t* __restrict__ sp, int64_t n, int F, int NLM,
                        const float* __restrict__ emb, float* __restrict__ H) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * F) return;
    const int c = (int)(idx % F);
    const int64_t i = idx / F;
    H[i * NLM * F + c] = emb[(int64_t)sp[i] * F + c];
}

// Readout and adjoint seed: E_i = w_out . h0 + e0[z] (+ head), warp per atom.
// The head E^head_i = W2 . silu(W1 h0 + b1) + b2 has hidden width 32 = one
// lane per hidden unit.  G0 = s_i (w_out + dE^head/dh0); higher l: 0.
__global__ void k_readout(int64_t n, int F, int NLM, const float* __restrict__ H,
                          const int32_t* __restrict__ sp, const float* __restrict__ w_out,
                          const float* __restrict__ e0, const float* __restrict__ head,
                          const uint8_t* __restrict__ seed, double* __restrict__ Ei,
                          float* __restrict__ G) {
    extern __shared__ float sh_h[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= n) return;
    float* h = sh_h + wib * F;
    const float* hi = H + (i * NLM) * F;
    float e = 0.f;
    for (int c = lane; c < F; c += 32) {
        h[c] = hi[c];
        e = fmaf(w_out[c], h[c], e);
    }
    __syncwarp();
    float gk = 0.f, eh = 0.f;
    if (head) {
        const float* W1 = head;
        const float* b1 = head + kHeadH * F;
        const float* W2 = b1 + kHeadH;
        float z = b1[lane];
        for (int c = 0; c < F; ++c) z = fmaf(W1[lane * F + c], h[c], z);
        eh = W2[lane] * silu(z);
        gk = W2[lane] * silu_grad(z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        eh += __shfl_xor_sync(0xffffffffu, eh, o);
    }
    const float s = seed ? (float)seed[i] : 1.f;
    for (int c = lane; c < F; c += 32) {
        float g = w_out[c];
        if (head) {
            for (int k = 0; k < kHeadH; ++k)
                g = fmaf(head[k * F + c], __shfl_sync(0xffffffffu, gk, k), g);
        }
        G[(i * NLM) * F + c] = s * g;
        for (int q = 1; q < NLM; ++q) G[(i * NLM + q) * F + c] = 0.f;
    }
    if (lane == 0) {
        double v = (double)e + (double)e0[sp[i]];
        if (head) v += (double)eh + (double)head[kHeadH * F + 2 * kHeadH];
        Ei[i] = v;
    }
}

// Pair term phi(r) = eps (sigma/r)^12 u(r/r_c): E_i += 1/2 sum_row phi and
// F_k += sum_i 1/2 (s_k + s_i) phi'(r) u_hat (both directed edges of a pair
// carry half of phi).  Warp per row.
__global__ void k_pair_term(int64_t n, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col, const int8_t* __restrict__ shift,
                            const double* __restrict__ x, EdgeConst k,
                            const uint8_t* __restrict__ seed, double* __restrict__ Ei,
                            double* __restrict__ frc, double* __restrict__ vir,
                            int64_t vir_stride) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    float ei = 0.f, f[3] = {0.f, 0.f, 0.f};
    double vr[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};    // sum_e (g d) (x) d, when vir
    const float si = seed ? (float)seed[i] : 1.f;
    for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
        const int j = col[e];
        float d[3];
        edge_vector(x, i, j, shift[e], k, d);
        const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        float u, du;
        envelope(r, k, u, du);
        const float ir = 1.f / r, ir2 = ir * ir, ir4 = ir2 * ir2;
        const float s12 = k.rep_sig12 * ir4 * ir4 * ir4;
        ei += 0.5f * k.rep_eps * s12 * u;
        const float dphi = k.rep_eps * s12 * (du - 12.f * ir * u);
        const float sj = seed ? (float)seed[j] : 1.f;
        const float g = 0.5f * (si + sj) * dphi * ir;
        f[0] += g * d[0];
        f[1] += g * d[1];
        f[2] += g * d[2];
        if (vir) {
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
                for (int q = 0; q < 3; ++q) vr[3 * p + q] += (double)(g * d[p]) * (double)d[q];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ei += __shfl_xor_sync(0xffffffffu, ei, o);
#pragma unroll
        for (int q = 0; q < 3; ++q) f[q] += __shfl_xor_sync(0xffffffffu, f[q], o);
    }
    if (vir) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            double v = vr[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) vir[q * vir_stride + i] += v;
        }
    }
    if (lane == 0) {
        if (si != 0.f) Ei[i] += (double)ei;   // energies of non-roots are never read
#pragma unroll
        for (int q = 0; q < 3; ++q) frc[3 * i + q] += (double)f[q];
    }
}

__global__ void k_scatter(int64_t n, const int32_t* __restrict__ gid,
                          const uint8_t* __restrict__ is_root, const double* __restrict__ Ei,
                          const double* __restrict__ floc, double* __restrict__ e_sorted,
                          double* __restrict__ f_sorted) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int64_t s = gid ? gid[l] : l;
    if (!is_root || is_root[l]) e_sorted[s] = Ei[l];
#pragma unroll
    for (int q = 0; q < 3; ++q) f_sorted[3 * s + q] += floc[3 * l + q];
}

// Caller-order outputs: FP32 forces and/or the FP64 sums themselves (the
// partial forces of a range of partitions, summed across ranks by the caller).
__global__ void k_finalize(int64_t n, const int32_t* __restrict__ perm,
                           const double* __restrict__ e_sorted, const double* __restrict__ f_sorted,
                           float* __restrict__ forces, double* __restrict__ forces64,
                           double* __restrict__ e_atom) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm[s];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (forces) forces[3 * i + q] = (float)f_sorted[3 * s + q];
        if (forces64) forces64[3 * i + q] = f_sorted[3 * s + q];
    }
    if (e_atom) e_atom[i] = e_sorted[s];
}

// Deterministic FP64 sum: fixed per-block tree, then one block over partials.
constexpr int kRedThreads = 256;
constexpr int kRedItems = 8;

__global__ void k_sum_partial(const double* __restrict__ v, int64_t n, double* __restrict__ part) {
    __shared__ double sm[kRedThreads];
    const int64_t base = (int64_t)blockIdx.x * kRedThreads * kRedItems;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < kRedItems; ++q) {
        const int64_t idx = base + (int64_t)q * kRedThreads + threadIdx.x;
        if (idx < n) acc += v[idx];
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_sum_final(const double* __restrict__ part, int64_t m, double* __restrict__ out) {
    __shared__ double sm[kRedThreads];
    double acc = 0.0;
    for (int64_t idx = threadIdx.x; idx < m; idx += kRedThreads) acc += part[idx];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

}  // namespace

__global__ void k_add9(double* __restrict__ acc, const double* __restrict__ v) {
    if (threadIdx.x < 9) acc[threadIdx.x] += v[threadIdx.x];
}

// sigma = scale * vtot (scale = 1 / (2 V): every pair is visited from both rows)
__global__ void k_stress_final(const double* __restrict__ vtot, double scale,
                               double* __restrict__ stress) {
    if (threadIdx.x < 9) stress[threadIdx.x] = vtot[threadIdx.x] * scale;
}

int reduce_sum(const double* v, int64_t n, double* out, DevBuf& tmp, cudaStream_t st) {
    const int64_t per = (int64_t)kRedThreads * kRedItems;
    const int64_t blocks = n > 0 ? (n + per - 1) / per : 1;
    MP_TRY(tmp.reserve(sizeof(double) * blocks));
    if (n > 0) {
        k_sum_partial<<<(unsigned)blocks, kRedThreads, 0, st>>>(v, n, tmp.as<double>());
        note_launch();
    } else
        MP_CUDA_TRY(cudaMemsetAsync(tmp.as<double>(), 0, sizeof(double), st));
    k_sum_final<<<1, kRedThreads, 0, st>>>(tmp.as<double>(), blocks, out); note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

namespace {

struct EvalBufs {
    double* xs;       // sorted wrapped positions
    int32_t* sp;      // sorted species
    double* e_sorted;
    double* f_sorted;
    double* xl;
    int32_t* spl;
    float* H;         // (K+1) feature arrays
    float* A;         // K message arrays
    float* S;         // K pre-activation arrays
    float* alpha;
    float* G[2];
    double* floc;
    double* eloc;
    double* vloc;     // stress only: per-row virial [9][n_max]; else null
    double* vsum;     // [9] one sub-system's virial
    double* vtot;     // [9] all sub-systems', in sub-system order
    float4* geo;      // BF16: per edge (u, r) of the current sub-system
    float4* split;    // BF16: the sub-system's positions as FP32 pairs (2 n)
    float* vfirst;    // BF16 layer 0 by hidden unit: G or V [n][S][NLM][kH], or null
};

// Rows a pass must cover: atoms within `hops` hops of a root (a prefix of
// the local numbering for partitions, all atoms otherwise), and their edges.
struct Prefix {
    const SubSys& ss;
    int64_t rows(int hops) const {
        if (ss.n_le.empty()) return ss.n;
        const int kp = (int)ss.n_le.size() - 1;
        return ss.n_le[hops < 0 ? 0 : (hops > kp ? kp : hops)];
    }
    int64_t edges(int hops) const {
        if (ss.e_le.empty()) return ss.n_edges;
        const int kp = (int)ss.e_le.size() - 1;
        return ss.e_le[hops < 0 ? 0 : (hops > kp ? kp : hops)];
    }
    // edges whose two ends are both in class `hops` (zero for the whole graph)
    int64_t same(int hops) const {
        if (ss.e_same.empty() || hops < 0 || hops >= (int)ss.e_same.size()) return 0;
        return ss.e_same[hops];
    }
};

int run_subsystem(mp_ctx* ctx, const SubSys& ss, const EvalBufs& b, const EdgeConst& kc, int K,
                  int precision, int use_head) {
    const Model& m = ctx->model;
    cudaStream_t st = ctx->stream;
    const int F = m.d.F, NLM = m.NLM;
    const int64_t n = ss.n;
    if (n == 0) return MP_OK;
    const int64_t feat = n * NLM * F;
    const int64_t row_f = (int64_t)NLM * F;   // floats per atom in a feature array
    const Prefix pre{ss};
    const double* x = b.xs;
    const int32_t* sp = b.sp;
    if (ss.gid) {
        k_gather_local<<<grid_for(n, 256), 256, 0, st>>>(ss.gid, n, b.xs, b.sp, b.xl, b.spl);
        note_launch();
        x = b.xl;
        sp = b.spl;
    }
    k_embed<<<grid_for(n * F, 256), 256, 0, st>>>(sp, n, F, NLM, m.emb, b.H);
    note_launch();
    EdgeArgs ea{};
    ea.row_ptr = ss.row_ptr;
    ea.col = ss.col;
    ea.shift = ss.shift;
    ea.x = x;
    ea.k = kc;
    ea.seed = ss.is_root;
    ea.err = ctx->ws.err.as<int>();
    ea.vir = b.vloc;
    ea.vir_stride = n;
    if (b.vloc) MP_CUDA_TRY(cudaMemsetAsync(b.vloc, 0, sizeof(double) * 9 * n, st));
    ea.sched = ctx->ws.sched.as<int>();
    ea.species = sp;
    ea.emb = m.emb;
    ea.n_species = m.d.n_species;
    ea.vfirst = b.vfirst;
    if (precision == MP_BF16) {   // edge geometry once for all of this sub-system's passes
        ea.geo = b.geo;
        TimerScope ts(ctx, MP_TIMER_PARTITION, ss.n_edges, n);
        MP_TRY(launch_edge_geometry(n, ss.row_ptr, ss.col, ss.shift, x, kc, b.geo, b.split, st));
    }
    NodeArgs na{};
    na.inv_navg = kc.inv_navg;
    na.err = ctx->ws.err.as<int>();
    // Forward: layer t only needs outputs within K-1-t hops of a root; the
    // rest of the next feature array is set to zero (never multiplied by a
    // nonzero coefficient, but kept finite).
    for (int t = 0; t < K; ++t) {
        const int64_t rows = pre.rows(K - 1 - t);
        ea.n = rows;
        ea.w = &m.layers[t];
        ea.first = t == 0;
        ea.Hin = b.H + t * feat;
        ea.Aout = b.A + t * feat;
        {
            TimerScope ts(ctx, t == 0 ? MP_TIMER_EDGE_FWD_L0 : MP_TIMER_EDGE_FWD,
                          pre.edges(K - 1 - t), rows);
            if (precision == MP_BF16)
                MP_TRY(launch_edge_fwd_bf16(m, ea, st, ctx->num_sms));
            else
                MP_TRY(launch_edge_fwd_f32(m, ea, st));
        }
        na.n = rows;
        na.w = &m.layers[t];
        na.A = b.A + t * feat;
        na.Hin = b.H + t * feat;
        na.Hout = b.H + (t + 1) * feat;
        na.S = b.S + t * n * F;
        na.first = t == 0;
        na.last = t == K - 1;
        {
            TimerScope ts(ctx, t == 0 ? MP_TIMER_NODE_FWD_L0 : MP_TIMER_NODE_FWD, 0, rows);
            if (precision == MP_BF16)
                MP_TRY(launch_node_fwd_bf16(m, na, st, ctx->num_sms));
            else
                MP_TRY(launch_node_fwd_f32(m, na, st));
        }
        if (rows < n)
            MP_CUDA_TRY(cudaMemsetAsync(b.H + (t + 1) * feat + rows * row_f, 0,
                                        sizeof(float) * (n - rows) * row_f, st));
    }
    // Readout on roots; adjoint seeds of every other atom are zero.
    const int64_t n_roots = pre.rows(0);   // may be 0: a slab without atoms
    if (n_roots > 0) {
        const int wpb = 4;
        k_readout<<<grid_for(n_roots, wpb), 32 * wpb, sizeof(float) * F * wpb, st>>>(
            n_roots, F, NLM, b.H + (int64_t)K * feat, sp, m.w_out, m.e0,
            use_head ? m.head : nullptr, ss.is_root, b.eloc, b.G[K & 1]);
        note_launch();
    }
    if (n_roots < n)
        MP_CUDA_TRY(cudaMemsetAsync(b.G[K & 1] + n_roots * row_f, 0,
                                    sizeof(float) * (n - n_roots) * row_f, st));
    MP_CUDA_TRY(cudaMemsetAsync(b.floc, 0, sizeof(double) * 3 * n, st));
    if (m.d.rep_eps != 0.0) {
        const int wpb = 8;
        // atoms beyond one hop of a root have no root neighbour: zero force
        const int64_t n_pair = pre.rows(1);
        if (n_pair > 0) {
            k_pair_term<<<grid_for(n_pair, wpb), 32 * wpb, 0, st>>>(
                n_pair, ss.row_ptr, ss.col, ss.shift, x, kc, ss.is_root, b.eloc, b.floc, b.vloc, n);
            note_launch();
        }
    }
    // Adjoint: alpha of layer t is nonzero only within K-1-t hops (node pass
    // there, zero beyond); the edge pass covers rows within K-t hops, and the
    // rows beyond it keep dE/dh = the layer output's (zero there).
    for (int t = K - 1; t >= 0; --t) {
        float* Gout = b.G[(t + 1) & 1];
        float* Gin = b.G[t & 1];
        const int64_t nrows = pre.rows(K - 1 - t);
        na.n = nrows;
        na.w = &m.layers[t];
        na.A = b.A + t * feat;
        na.S = b.S + t * n * F;
        na.Gout = Gout;
        na.Alpha = b.alpha;
        na.last = t == K - 1;
        {
            TimerScope ts(ctx, t == 0 ? MP_TIMER_NODE_BWD_L0 : MP_TIMER_NODE_BWD, 0, nrows);
            if (precision == MP_BF16)
                MP_TRY(launch_node_bwd_bf16(m, na, st, ctx->num_sms));
            else
                MP_TRY(launch_node_bwd_f32(m, na, st));
        }
        if (nrows < n)
            MP_CUDA_TRY(cudaMemsetAsync(b.alpha + nrows * row_f, 0,
                                        sizeof(float) * (n - nrows) * row_f, st));
        const int64_t erows = pre.rows(K - t);
        ea.n = erows;
        ea.w = &m.layers[t];
        ea.first = t == 0;
        ea.Hin = b.H + t * feat;
        ea.Alpha = b.alpha;
        ea.Gout = Gout;
        ea.Gin = t == 0 ? nullptr : Gin;
        ea.frc = b.floc;
        // rows nrows..erows-1 (the outermost class of this layer) receive no
        // messages at layer t, so their adjoints are zero and an edge between
        // two of them contributes exactly nothing: the adjoint kernels skip
        // those edges
        ea.n_recv = nrows < erows ? nrows : 0;
        {
            const int64_t e_work = pre.edges(K - t) - (nrows < erows ? pre.same(K - t) : 0);
            TimerScope ts(ctx, t == 0 ? MP_TIMER_EDGE_BWD_L0 : MP_TIMER_EDGE_BWD, e_work, erows);
            if (precision == MP_BF16)
                MP_TRY(launch_edge_bwd_bf16(m, ea, st, ctx->num_sms));
            else
                MP_TRY(launch_edge_bwd_f32(m, ea, st));
        }
        if (t > 0 && erows < n)
            MP_CUDA_TRY(cudaMemcpyAsync(Gin + erows * row_f, Gout + erows * row_f,
                                        sizeof(float) * (n - erows) * row_f,
                                        cudaMemcpyDeviceToDevice, st));
    }
    k_scatter<<<grid_for(n, 256), 256, 0, st>>>(n, ss.gid, ss.is_root, b.eloc, b.floc, b.e_sorted,
                                                b.f_sorted);
    note_launch();
    if (b.vloc) {   // this sub-system's virial, summed in a fixed order
        for (int q = 0; q < 9; ++q)
            MP_TRY(reduce_sum(b.vloc + (int64_t)q * n, n, b.vsum + q, ctx->ws.red, st));
        k_add9<<<1, 32, 0, st>>>(b.vtot, b.vsum);
        note_launch();
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int evaluate(mp_ctx* ctx, const double* d_pos, const int32_t* d_species, const Graph& g,
             const Plan* plan, int K, int precision, int use_head, double* d_energy,
             float* d_forces, double* d_e_atom, double* d_stress, int part_begin, int part_end,
             double* d_forces64, bool wrap_pos) {
    const Model& m = ctx->model;
    if (!d_pos || !d_species || !d_energy || (!d_forces && !d_forces64)) return MP_ERR_ARG;
    if (K < 0 || K > m.d.n_layers_full) return MP_ERR_ARG;
    if (precision != MP_FP32 && precision != MP_BF16) return MP_ERR_ARG;
    if (plan && plan->n != g.n) return MP_ERR_ARG;
    const int n_plan_parts = plan ? (int)plan->parts.size() : 1;
    if (part_end < 0) part_end = n_plan_parts;
    if (part_begin < 0 || part_begin > part_end || part_end > n_plan_parts) return MP_ERR_ARG;
    cudaStream_t st = ctx->stream;
    Workspace& ws = ctx->ws;
    const int64_t n = g.n;
    const int F = m.d.F, NLM = m.NLM;

    std::vector<SubSys> subs;
    if (!plan) {
        subs.push_back(SubSys{n, g.n_edges, g.row_ptr.as<int64_t>(), g.col.as<int32_t>(),
                              g.shift.as<int8_t>(), nullptr, nullptr, {}, {}, {}});
    } else {
        // partitions part_begin .. part_end - 1 (all of them by default); the
        // energy and force sums then hold only those partitions' shares
        for (int p = part_begin; p < part_end; ++p) {
            const Part& P = plan->parts[p];
            if (P.n_root > 0)   // a slab without roots contributes nothing
                subs.push_back(SubSys{P.n_ext, P.n_edges, P.row_ptr.as<int64_t>(),
                                      P.col.as<int32_t>(), P.shift.as<int8_t>(),
                                      P.gid.as<int32_t>(), P.is_root.as<uint8_t>(), P.n_le,
                                      P.e_le, P.e_same});
        }
    }
    int64_t nmax = 0, emax = 0;
    for (const SubSys& s : subs) {
        nmax = s.n > nmax ? s.n : nmax;
        emax = s.n_edges > emax ? s.n_edges : emax;
    }
    const int64_t feat = nmax * NLM * F;

    MP_TRY(ws.xw.reserve(sizeof(double) * 3 * n));
    MP_TRY(ws.sp.reserve(sizeof(int32_t) * 2 * n + 64));
    MP_TRY(ws.esum.reserve(sizeof(double) * n));
    MP_TRY(ws.fsum.reserve(sizeof(double) * 3 * n));
    MP_TRY(ws.xl.reserve(sizeof(double) * 3 * nmax + sizeof(int32_t) * nmax + 64));
    MP_TRY(ws.H.reserve(sizeof(float) * (K + 1) * feat));
    MP_TRY(ws.A.reserve(sizeof(float) * (K > 0 ? K : 1) * feat));
    MP_TRY(ws.S.reserve(sizeof(float) * (K > 0 ? K : 1) * nmax * F));
    MP_TRY(ws.alpha.reserve(sizeof(float) * feat));
    MP_TRY(ws.G0.reserve(sizeof(float) * feat));
    MP_TRY(ws.G1.reserve(sizeof(float) * feat));
    MP_TRY(ws.floc.reserve(sizeof(double) * 3 * nmax));
    MP_TRY(ws.eatom.reserve(sizeof(double) * nmax));
    MP_TRY(ws.err.reserve(64));
    MP_TRY(ws.sched.reserve(64));
    MP_CUDA_TRY(cudaMemsetAsync(ws.err.as<int>(), 0, sizeof(int), st));

    EvalBufs b;
    b.xs = ws.xw.as<double>();
    b.sp = ws.sp.as<int32_t>();
    b.e_sorted = ws.esum.as<double>();
    b.f_sorted = ws.fsum.as<double>();
    b.xl = ws.xl.as<double>();
    b.spl = reinterpret_cast<int32_t*>(b.xl + 3 * nmax);
    b.H = ws.H.as<float>();
    b.A = ws.A.as<float>();
    b.S = ws.S.as<float>();
    b.alpha = ws.alpha.as<float>();
    b.G[0] = ws.G0.as<float>();
    b.G[1] = ws.G1.as<float>();
    b.floc = ws.floc.as<double>();
    b.eloc = ws.eatom.as<double>();
    b.vloc = b.vsum = b.vtot = nullptr;
    b.geo = b.split = nullptr;
    b.vfirst = nullptr;
    if (precision == MP_BF16) {
        MP_TRY(ws.geo.reserve(sizeof(float4) * (emax + 1 + 2 * nmax)));
        b.geo = ws.geo.as<float4>();
        b.split = b.geo + emax + 1;
        if (F == 128 && m.d.lmax == 2) {
            MP_TRY(ws.vfirst.reserve(sizeof(float) * (size_t)nmax * m.d.n_species * NLM * kH));
            b.vfirst = ws.vfirst.as<float>();
        }
    }
    if (d_stress) {
        MP_TRY(ws.vir.reserve(sizeof(double) * (9 * nmax + 18)));
        b.vloc = ws.vir.as<double>();
        b.vsum = b.vloc + 9 * nmax;
        b.vtot = b.vsum + 9;
        MP_CUDA_TRY(cudaMemsetAsync(b.vtot, 0, sizeof(double) * 9, st));
    }

    k_gather_pos<<<grid_for(n, 256), 256, 0, st>>>(d_pos, d_species, g.perm.as<int32_t>(), n,
                                                   g.box[0], g.box[1], g.box[2], m.d.n_species,
                                                   wrap_pos ? 1 : 0, b.xs, b.sp, ws.err.as<int>());
    note_launch();
    MP_CUDA_TRY(cudaMemsetAsync(b.f_sorted, 0, sizeof(double) * 3 * n, st));
    MP_CUDA_TRY(cudaMemsetAsync(b.e_sorted, 0, sizeof(double) * n, st));
    const EdgeConst kc = make_edge_const(m.d, g.box);
    for (const SubSys& s : subs) MP_TRY(run_subsystem(ctx, s, b, kc, K, precision, use_head));
    k_finalize<<<grid_for(n, 256), 256, 0, st>>>(n, g.perm.as<int32_t>(), b.e_sorted, b.f_sorted,
                                                 d_forces, d_forces64, d_e_atom); note_launch();
    MP_TRY(reduce_sum(b.e_sorted, n, d_energy, ws.red, st));
    if (d_stress) {
        k_stress_final<<<1, 32, 0, st>>>(b.vtot, 0.5 / (g.box[0] * g.box[1] * g.box[2]), d_stress);
        note_launch();
    }
    MP_CUDA_TRY(cudaGetLastError());
    // error word: invalid species; bounded-wait timeouts of the tensor-core kernels
    int herr = 0;
    MP_CUDA_TRY(cudaMemcpyAsync(&herr, ws.err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr & kErrSpecies) return MP_ERR_ARG;
    if (herr) return MP_ERR_TIMEOUT;
    return MP_OK;
}

}  // namespace mp

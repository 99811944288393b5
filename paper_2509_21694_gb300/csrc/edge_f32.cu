// FP32 edge kernels on CUDA cores: one message-passing layer forward
// (messages summed by receiver) and its adjoint.
//
// A block owns RPB consecutive receiver rows of the CSR and walks their
// edges in chunks of CE.  Per chunk the block computes the edge geometry,
// the Bessel basis with envelope and the spherical harmonics, then the
// radial MLP R = W3 silu(W2 silu(W1 eps)); thread c then owns channel c and
// walks the chunk's edges in order, keeping the receiver's running sums in
// registers.  A row is owned by exactly one block and summed in a fixed
// order: no atomics, deterministic results.
//
// Adjoint (forces): the symmetric-pair form.  Row k visits each neighbour
// i once and handles both directed edges of the pair: (k <- i) with
// displacement d and (i <- k) with -d.  R(|d|) is shared and
// Y_l(-u) = (-1)^l Y_l(u), so row k gathers alpha_i = dE/dA_i and h_i and
// forms (a) dE/dh_k as a sender, (b) dE/dR summed over both directions,
// pushed once through the radial MLP's transpose, and (c) g = dE_pair/dd;
// F_k = sum_i g.  Nothing is scattered to another row.
#include "kernels.h"

namespace mp {

namespace {

constexpr int CE = 16;   // edges per chunk
constexpr int RPB = 4;   // receiver rows per block

template <int LMAX, bool FIRST>
struct Paths {
    // Radial outputs kept in registers: layer 0 never needs R_lb (its l >= 1
    // inputs are zero).
    static constexpr int NP = FIRST ? 1 + LMAX : 1 + 2 * LMAX;
    __host__ __device__ static constexpr int block(int q) { return FIRST ? (q == 0 ? 0 : 2 * q - 1) : q; }
    __host__ __device__ static constexpr int sla(int l) { return FIRST ? l : 2 * l - 1; }
    __host__ __device__ static constexpr int slb(int l) { return 2 * l; }
};

__device__ __forceinline__ int find_row(const int64_t* s_rp, int nrows, int64_t e) {
    int lr = 0;
    while (lr + 1 < nrows && s_rp[lr + 1] <= e) ++lr;
    return lr;
}

// R[q][e] = sum_k W3[block(q) F + c][k] a2[k][e]
template <int F, int LMAX, bool FIRST>
__device__ __forceinline__ void radial_out(const float* __restrict__ W3T, const float (*s_a2)[CE],
                                           int c, float R[][CE]) {
    using PP = Paths<LMAX, FIRST>;
    constexpr int P = F * (1 + 2 * LMAX);
#pragma unroll
    for (int q = 0; q < PP::NP; ++q)
#pragma unroll
        for (int e = 0; e < CE; ++e) R[q][e] = 0.f;
#pragma unroll 2
    for (int kk = 0; kk < kH; ++kk) {
        float wv[PP::NP];
#pragma unroll
        for (int q = 0; q < PP::NP; ++q) wv[q] = __ldg(&W3T[kk * P + PP::block(q) * F + c]);
        float av[CE];
#pragma unroll
        for (int e4 = 0; e4 < CE / 4; ++e4) {
            float4 v = reinterpret_cast<const float4*>(s_a2[kk])[e4];
            av[4 * e4] = v.x;
            av[4 * e4 + 1] = v.y;
            av[4 * e4 + 2] = v.z;
            av[4 * e4 + 3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < PP::NP; ++q)
#pragma unroll
            for (int e = 0; e < CE; ++e) R[q][e] = fmaf(wv[q], av[e], R[q][e]);
    }
}

// a2 = silu(W2 a1) (and silu' when DERIV) for the CE edges of a chunk.
template <int F, bool DERIV>
__device__ __forceinline__ void hidden2(const float* __restrict__ W2T, const float (*s_a1)[CE],
                                        float (*s_a2)[CE], float (*s_sp2)[CE], int c) {
    constexpr int EG = CE * kH / F;
    const int kk = c % kH, e0 = (c / kH) * EG;
    float z[EG];
#pragma unroll
    for (int q = 0; q < EG; ++q) z[q] = 0.f;
#pragma unroll 4
    for (int jj = 0; jj < kH; ++jj) {
        const float wv = __ldg(&W2T[jj * kH + kk]);
#pragma unroll
        for (int q = 0; q < EG; ++q) z[q] = fmaf(wv, s_a1[jj][e0 + q], z[q]);
    }
#pragma unroll
    for (int q = 0; q < EG; ++q) {
        s_a2[kk][e0 + q] = silu(z[q]);
        if (DERIV) s_sp2[kk][e0 + q] = silu_grad(z[q]);
    }
}

template <int F, int LMAX, bool FIRST>
__global__ void __launch_bounds__(F) k_edge_fwd(EdgeArgs a, const float* __restrict__ W1,
                                                const float* __restrict__ W2T,
                                                const float* __restrict__ W3T) {
    using PP = Paths<LMAX, FIRST>;
    constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    __shared__ __align__(16) float s_eps[CE][kNB];
    __shared__ float s_Y[CE][NLM];
    __shared__ __align__(16) float s_a1[kH][CE];
    __shared__ __align__(16) float s_a2[kH][CE];
    __shared__ int s_row[CE];
    __shared__ int s_col[CE];
    __shared__ int64_t s_rp[RPB + 1];

    const int c = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * RPB;
    const int nrows = (int)min((int64_t)RPB, a.n - r0);
    if (c <= nrows) s_rp[c] = a.row_ptr[r0 + c];
    __syncthreads();
    const int64_t e_beg = s_rp[0], e_end = s_rp[nrows];

    float acc[NLM];
#pragma unroll
    for (int q = 0; q < NLM; ++q) acc[q] = 0.f;
    int cur = -1, next = 0;
    auto write_row = [&](int lr, bool zero) {
        float* o = a.Aout + ((r0 + lr) * NLM) * F + c;
#pragma unroll
        for (int q = 0; q < NLM; ++q) o[q * F] = zero ? 0.f : acc[q] * a.k.inv_navg;
    };

    for (int64_t cb = e_beg; cb < e_end; cb += CE) {
        if (c < CE) {
            const int64_t e = cb + c;
            float eps[kNB], Y[NLM];
            if (e < e_end) {
                const int lr = find_row(s_rp, nrows, e);
                const int j = a.col[e];
                float d[3];
                edge_vector(a.x, r0 + lr, j, a.shift[e], a.k, d);
                const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                const float u[3] = {d[0] / r, d[1] / r, d[2] / r};
                float dd[kNB], env, denv;
                radial_basis<false>(r, a.k, eps, dd, env, denv);
                sph_harm<LMAX>(u, Y);
                s_row[c] = lr;
                s_col[c] = j;
            } else {
#pragma unroll
                for (int q = 0; q < kNB; ++q) eps[q] = 0.f;
#pragma unroll
                for (int q = 0; q < NLM; ++q) Y[q] = 0.f;
                s_row[c] = -1;
                s_col[c] = 0;
            }
#pragma unroll
            for (int q = 0; q < kNB; ++q) s_eps[c][q] = eps[q];
#pragma unroll
            for (int q = 0; q < NLM; ++q) s_Y[c][q] = Y[q];
        }
        __syncthreads();
        for (int o = c; o < kH * CE; o += F) {
            const int kk = o / CE, e = o % CE;
            float z = 0.f;
#pragma unroll
            for (int b = 0; b < kNB; ++b) z = fmaf(__ldg(&W1[kk * kNB + b]), s_eps[e][b], z);
            s_a1[kk][e] = silu(z);
        }
        __syncthreads();
        hidden2<F, false>(W2T, s_a1, s_a2, nullptr, c);
        __syncthreads();
        float R[PP::NP][CE];
        radial_out<F, LMAX, FIRST>(W3T, s_a2, c, R);
#pragma unroll
        for (int e = 0; e < CE; ++e) {
            const int lr = s_row[e];
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
            const float* hj = a.Hin + ((int64_t)s_col[e] * NLM) * F + c;
            const float h0 = __ldg(hj);
            acc[0] = fmaf(R[0][e], h0, acc[0]);
            const float t1 = R[PP::sla(1)][e] * h0;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                acc[1 + m] = fmaf(t1, s_Y[e][1 + m], acc[1 + m]);
                if (!FIRST) acc[1 + m] = fmaf(R[PP::slb(1)][e], hj[(1 + m) * F], acc[1 + m]);
            }
            if (LMAX >= 2) {
                const float t2 = R[PP::sla(2)][e] * h0;
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    acc[4 + m] = fmaf(t2, s_Y[e][4 + m], acc[4 + m]);
                    if (!FIRST) acc[4 + m] = fmaf(R[PP::slb(2)][e], hj[(4 + m) * F], acc[4 + m]);
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

// ---------------------------------------------------------------- adjoint --

constexpr int CB = 8;    // edges per chunk in the adjoint

template <int F, int LMAX>
struct BwdSmem {
    static constexpr int NLM = (LMAX + 1) * (LMAX + 1);
    static constexpr int NQ = NLM;           // q = 0: dE/dr partial, 1..: dE/dY_lm partials
    float eps[CB][kNB];
    float deps[CB][kNB];
    float Y[CB][NLM];
    float u[CB][4];          // unit vector, r
    float a1[kH][CB], da1[kH][CB], a2[kH][CB], da2[kH][CB];
    float part[CB][NQ][F + 1];
    double red[CB][NQ];
    double frow[RPB][3];
    double vrow[RPB][9];     // per-row virial sum_e g_e (x) d_e (when requested)
    int row[CB], col[CB];
    int64_t rp[RPB + 1];
    int klist[4 * F];        // kept edges of a window of raw edges (offsets from its start)
    int kwarp[F / 32];
};

// R (value) and dR/dr (tangent) of the radial MLP's last layer for CB edges,
// one pass over W3.
template <int F, int LMAX, bool FIRST>
__device__ __forceinline__ void radial_out2(const float* __restrict__ W3T,
                                            const float (*s_a2)[CB], const float (*s_da2)[CB],
                                            int c, float R[][CB], float dR[][CB]) {
    using PP = Paths<LMAX, FIRST>;
    constexpr int P = F * (1 + 2 * LMAX);
#pragma unroll
    for (int q = 0; q < PP::NP; ++q)
#pragma unroll
        for (int e = 0; e < CB; ++e) R[q][e] = dR[q][e] = 0.f;
#pragma unroll 2
    for (int kk = 0; kk < kH; ++kk) {
        float wv[PP::NP];
#pragma unroll
        for (int q = 0; q < PP::NP; ++q) wv[q] = __ldg(&W3T[kk * P + PP::block(q) * F + c]);
        float av[CB], dv[CB];
#pragma unroll
        for (int e4 = 0; e4 < CB / 4; ++e4) {
            const float4 v = reinterpret_cast<const float4*>(s_a2[kk])[e4];
            const float4 w = reinterpret_cast<const float4*>(s_da2[kk])[e4];
            av[4 * e4] = v.x; av[4 * e4 + 1] = v.y; av[4 * e4 + 2] = v.z; av[4 * e4 + 3] = v.w;
            dv[4 * e4] = w.x; dv[4 * e4 + 1] = w.y; dv[4 * e4 + 2] = w.z; dv[4 * e4 + 3] = w.w;
        }
#pragma unroll
        for (int q = 0; q < PP::NP; ++q)
#pragma unroll
            for (int e = 0; e < CB; ++e) {
                R[q][e] = fmaf(wv[q], av[e], R[q][e]);
                dR[q][e] = fmaf(wv[q], dv[e], dR[q][e]);
            }
    }
}

// Compensated (Kahan) sum of n floats with stride 1, result in double.
__device__ __forceinline__ double kahan_sum(const float* v, int n) {
    float s = 0.f, comp = 0.f;
    for (int q = 0; q < n; ++q) {
        const float y = v[q] - comp;
        const float t = s + y;
        comp = (t - s) - y;
        s = t;
    }
    return (double)s - (double)comp;
}

// Adjoint of one layer.  dE/dr of an edge pair is sum_q dE/dR_q dR_q/dr with
// dR/dr propagated forward through the radial MLP (it depends on the
// geometry only).  Per-edge sums over channels (dE/dr, dE/dY) go through
// shared memory and a compensated FP32 sum per (edge, quantity).
template <int F, int LMAX, bool FIRST>
__global__ void __launch_bounds__(F) k_edge_bwd(EdgeArgs a, const float* __restrict__ W1,
                                                const float* __restrict__ W2T,
                                                const float* __restrict__ W3T) {
    using PP = Paths<LMAX, FIRST>;
    using SM = BwdSmem<F, LMAX>;
    constexpr int NLM = SM::NLM, NQ = SM::NQ;
    constexpr int EG = CB * kH / F;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SM& s = *reinterpret_cast<SM*>(smem_raw);

    const int c = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * RPB;
    const int nrows = (int)min((int64_t)RPB, a.n - r0);
    if (c <= nrows) s.rp[c] = a.row_ptr[r0 + c];
    if (c < RPB * 3) s.frow[c / 3][c % 3] = 0.0;
    if (a.vir && c < RPB * 9) s.vrow[c / 9][c % 9] = 0.0;
    __syncthreads();
    const int64_t e_beg = s.rp[0], e_end = s.rp[nrows];

    float gacc[NLM], ak[NLM], hk[NLM];
#pragma unroll
    for (int q = 0; q < NLM; ++q) gacc[q] = ak[q] = hk[q] = 0.f;
    int cur = -1, next = 0;
    auto flush = [&](int lr, bool with_acc) {
        if (FIRST) return;
        const int64_t base = ((r0 + lr) * NLM) * F + c;
#pragma unroll
        for (int q = 0; q < NLM; ++q)
            a.Gin[base + q * F] = a.Gout[base + q * F] + (with_acc ? gacc[q] : 0.f);
    };

    // Rows >= n_recv receive no messages at this layer: their adjoints are
    // zero and an edge between two of them adds exact zeros, so the block's
    // edges are compacted (in order) without those edges, 4 F at a time.
    const bool compact = a.n_recv > 0 && r0 + nrows > a.n_recv;
    const int lane = c & 31, wid = c >> 5;
    for (int64_t wb = e_beg; wb < e_end;) {
        const int64_t we = compact ? min(wb + (int64_t)(4 * F), e_end) : e_end;
        int64_t nk = we - wb;
        if (compact) {
            int keep[4], cnt = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t e = wb + 4 * c + q;
                keep[q] = 0;
                if (e < we) {
                    const int lr = find_row(s.rp, nrows, e);
                    keep[q] = !(r0 + lr >= a.n_recv && (int64_t)a.col[e] >= a.n_recv);
                }
                cnt += keep[q];
            }
            int inc = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) s.kwarp[wid] = inc;
            __syncthreads();
            int off = inc - cnt;
            for (int q = 0; q < wid; ++q) off += s.kwarp[q];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (keep[q]) s.klist[off++] = 4 * c + q;
            nk = 0;
            for (int q = 0; q < F / 32; ++q) nk += s.kwarp[q];
            __syncthreads();
        }
        for (int64_t cb = 0; cb < nk; cb += CB) {
            if (c < CB) {
                const int64_t v = cb + c;
                const int64_t e = v < nk ? wb + (compact ? (int64_t)s.klist[v] : v) : e_end;
                float eps[kNB], deps[kNB], Y[NLM], u4[4] = {0.f, 0.f, 0.f, 1.f};
                if (e < e_end) {
                    const int lr = find_row(s.rp, nrows, e);
                    const int j = a.col[e];
                    float d[3];
                    edge_vector(a.x, r0 + lr, j, a.shift[e], a.k, d);
                    const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    u4[0] = d[0] / r;
                    u4[1] = d[1] / r;
                    u4[2] = d[2] / r;
                    u4[3] = r;
                    float env, denv;
                    radial_basis<true>(r, a.k, eps, deps, env, denv);
                    sph_harm<LMAX>(u4, Y);
                    s.row[c] = lr;
                    s.col[c] = j;
                } else {
#pragma unroll
                    for (int q = 0; q < kNB; ++q) eps[q] = deps[q] = 0.f;
#pragma unroll
                    for (int q = 0; q < NLM; ++q) Y[q] = 0.f;
                    s.row[c] = -1;
                    s.col[c] = 0;
                }
#pragma unroll
                for (int q = 0; q < kNB; ++q) {
                    s.eps[c][q] = eps[q];
                    s.deps[c][q] = deps[q];
                }
#pragma unroll
                for (int q = 0; q < NLM; ++q) s.Y[c][q] = Y[q];
#pragma unroll
                for (int q = 0; q < 4; ++q) s.u[c][q] = u4[q];
            }
            __syncthreads();
            for (int o = c; o < kH * CB; o += F) {
                const int kk = o / CB, e = o % CB;
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
#pragma unroll 4
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
            float R[PP::NP][CB], dR[PP::NP][CB];
            radial_out2<F, LMAX, FIRST>(W3T, s.a2, s.da2, c, R, dR);

#pragma unroll
            for (int e = 0; e < CB; ++e) {
                const int lr = s.row[e];
                if (lr < 0) {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) s.part[e][q][c] = 0.f;
                    continue;
                }
                if (lr != cur) {
                    if (cur >= 0) {
                        flush(cur, true);
                        next = cur + 1;
                    }
                    for (int q = next; q < lr; ++q) flush(q, false);
                    next = lr;
                    cur = lr;
                    const int64_t base = ((r0 + lr) * NLM) * F + c;
#pragma unroll
                    for (int q = 0; q < NLM; ++q) {
                        gacc[q] = 0.f;
                        ak[q] = a.Alpha[base + q * F];
                        hk[q] = (FIRST && q > 0) ? 0.f : a.Hin[base + q * F];
                    }
                }
                const int64_t jb = ((int64_t)s.col[e] * NLM) * F + c;
                float aj[NLM], hj[NLM];
#pragma unroll
                for (int q = 0; q < NLM; ++q) {
                    aj[q] = a.Alpha[jb + q * F];
                    hj[q] = (FIRST && q > 0) ? 0.f : a.Hin[jb + q * F];
                }
                float Y[NLM];
#pragma unroll
                for (int q = 0; q < NLM; ++q) Y[q] = s.Y[e][q];
                // (a) dE/dh_k as the sender of the reverse edge (i <- k)
                if (!FIRST) {
                    float g0 = R[0][e] * aj[0];
                    float sm1 = 0.f;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        sm1 = fmaf(aj[1 + m], Y[1 + m], sm1);
                        gacc[1 + m] = fmaf(R[PP::slb(1)][e], aj[1 + m], gacc[1 + m]);
                    }
                    g0 = fmaf(-R[PP::sla(1)][e], sm1, g0);
                    if (LMAX >= 2) {
                        float sm2 = 0.f;
#pragma unroll
                        for (int m = 0; m < 5; ++m) {
                            sm2 = fmaf(aj[4 + m], Y[4 + m], sm2);
                            gacc[4 + m] = fmaf(R[PP::slb(2)][e], aj[4 + m], gacc[4 + m]);
                        }
                        g0 = fmaf(R[PP::sla(2)][e], sm2, g0);
                    }
                    gacc[0] += g0;
                }
                // (b) dE/dR of both directions contracted with dR/dr; (c) dE/dY
                float gr = (ak[0] * hj[0] + aj[0] * hk[0]) * dR[0][e];
                {
                    float g1a = 0.f, g1b = 0.f;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const float t = ak[1 + m] * hj[0] - aj[1 + m] * hk[0];
                        g1a = fmaf(Y[1 + m], t, g1a);
                        s.part[e][1 + m][c] = R[PP::sla(1)][e] * t;
                        if (!FIRST) g1b += ak[1 + m] * hj[1 + m] + aj[1 + m] * hk[1 + m];
                    }
                    gr = fmaf(g1a, dR[PP::sla(1)][e], gr);
                    if (!FIRST) gr = fmaf(g1b, dR[PP::slb(1)][e], gr);
                }
                if (LMAX >= 2) {
                    float g2a = 0.f, g2b = 0.f;
#pragma unroll
                    for (int m = 0; m < 5; ++m) {
                        const float t = ak[4 + m] * hj[0] + aj[4 + m] * hk[0];
                        g2a = fmaf(Y[4 + m], t, g2a);
                        s.part[e][4 + m][c] = R[PP::sla(2)][e] * t;
                        if (!FIRST) g2b += ak[4 + m] * hj[4 + m] + aj[4 + m] * hk[4 + m];
                    }
                    gr = fmaf(g2a, dR[PP::sla(2)][e], gr);
                    if (!FIRST) gr = fmaf(g2b, dR[PP::slb(2)][e], gr);
                }
                s.part[e][0][c] = gr;
            }
            __syncthreads();
            for (int t = c; t < CB * NQ; t += F) s.red[t / NQ][t % NQ] = kahan_sum(s.part[t / NQ][t % NQ], F);
            __syncthreads();
            if (c < CB && s.row[c] >= 0) {
                const int e = c;
                const double gr = s.red[e][0];
                double gY[NLM];
                gY[0] = 0.0;
#pragma unroll
                for (int q = 1; q < NLM; ++q) gY[q] = s.red[e][q];
                const double u[3] = {s.u[e][0], s.u[e][1], s.u[e][2]};
                const double ir = 1.0 / (double)s.u[e][3];
                double v[3];
                sph_grad<LMAX, double>(u, gY, v);
                const double vu = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
#pragma unroll
                for (int q = 0; q < 3; ++q) s.red[e][q] = gr * u[q] + (v[q] - vu * u[q]) * ir;
            }
            __syncthreads();
            // one thread per output component, each summing the chunk's edges in order
            if (c < 3) {
                for (int e = 0; e < CB; ++e) {
                    const int lr = s.row[e];
                    if (lr < 0) break;
                    s.frow[lr][c] += s.red[e][c];
                }
            } else if (a.vir && c < 12) {
                const int p = (c - 3) / 3, q = (c - 3) % 3;
                for (int e = 0; e < CB; ++e) {
                    const int lr = s.row[e];
                    if (lr < 0) break;
                    s.vrow[lr][3 * p + q] += s.red[e][p] * ((double)s.u[e][q] * (double)s.u[e][3]);
                }
            }
            __syncthreads();
        }
        wb = we;
    }
    if (cur >= 0) {
        flush(cur, true);
        next = cur + 1;
    }
    for (int q = next; q < nrows; ++q) flush(q, false);
    __syncthreads();
    if (c < nrows * 3) a.frc[(r0 + c / 3) * 3 + c % 3] += s.frow[c / 3][c % 3];
    if (a.vir && c < nrows * 9) a.vir[(int64_t)(c % 9) * a.vir_stride + r0 + c / 9] += s.vrow[c / 9][c % 9];
}

template <int F, int LMAX>
int fwd_impl(const Model& m, const EdgeArgs& a, cudaStream_t st) {
    if (a.n == 0) return MP_OK;
    const LayerW& w = *a.w;
    dim3 grid((unsigned)((a.n + RPB - 1) / RPB));
    if (a.first)
        k_edge_fwd<F, LMAX, true><<<grid, F, 0, st>>>(a, w.W1, w.W2T, w.W3T);
    else
        k_edge_fwd<F, LMAX, false><<<grid, F, 0, st>>>(a, w.W1, w.W2T, w.W3T);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

template <int F, int LMAX>
int bwd_impl(const Model& m, const EdgeArgs& a, cudaStream_t st) {
    if (a.n == 0) return MP_OK;
    const LayerW& w = *a.w;
    dim3 grid((unsigned)((a.n + RPB - 1) / RPB));
    const size_t sm = sizeof(BwdSmem<F, LMAX>);
    if (a.first) {
        MP_CUDA_TRY(cudaFuncSetAttribute(k_edge_bwd<F, LMAX, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_edge_bwd<F, LMAX, true><<<grid, F, sm, st>>>(a, w.W1, w.W2T, w.W3T); note_launch();
    } else {
        MP_CUDA_TRY(cudaFuncSetAttribute(k_edge_bwd<F, LMAX, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_edge_bwd<F, LMAX, false><<<grid, F, sm, st>>>(a, w.W1, w.W2T, w.W3T); note_launch();
    }
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int launch_edge_fwd_f32(const Model& m, const EdgeArgs& a, cudaStream_t st) {
    if (m.d.F == 128 && m.d.lmax == 2) return fwd_impl<128, 2>(m, a, st);
    if (m.d.F == 64 && m.d.lmax == 1) return fwd_impl<64, 1>(m, a, st);
    return MP_ERR_UNSUPPORTED;
}

int launch_edge_bwd_f32(const Model& m, const EdgeArgs& a, cudaStream_t st) {
    if (m.d.F == 128 && m.d.lmax == 2) return bwd_impl<128, 2>(m, a, st);
    if (m.d.F == 64 && m.d.lmax == 1) return bwd_impl<64, 1>(m, a, st);
    return MP_ERR_UNSUPPORTED;
}

}  // namespace mp

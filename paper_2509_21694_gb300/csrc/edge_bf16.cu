// Edge kernels with the radial MLP's dense contractions on tcgen05 tensor
// cores (BF16 operands, FP32 accumulation in tensor memory).  Geometry, the
// first radial layer (K = 8), messages, adjoint sums and forces stay FP32 on
// CUDA cores.  Shapes compiled: F = 128, lmax = 2, H = 64.
//
// A CTA holds one copy of the W2 / W3 operand tiles and runs four
// independent warpgroups; each warpgroup owns a stream of receiver-row
// groups, 128 tensor-memory columns, an mbarrier and a named barrier, so one
// warpgroup's MMAs overlap the others' CUDA-core work.
// Per chunk of edges (rows owned by the warpgroup):
//   1. CUDA cores: geometry, eps (and d eps/dr), a1 = silu(W1 eps) -> BF16
//      K-major tile B1 (rows = edges; adjoint: edges, then their r-tangents).
//   2. MMA1: D1[128 x 16] = W2pad[128 x 64] . B1^T  (rows 0..63 = hidden).
//   3. warps 0-1 read D1 from tensor memory: a2 = silu(z2) (adjoint also
//      da2 = silu'(z2) dz2) -> BF16 tile B2.
//   4. MMA2: D2_q[128 x 16] = W3_q[128 x 64] . B2^T for each radial path q
//      (lane = channel, column = edge: R, and dR/dr in the adjoint).
//   5. thread = channel reads its row of D2 and runs the message (forward)
//      or symmetric-pair adjoint (backward) epilogue.  In the adjoint each
//      channel forms its own share of dE_pair/dd and accumulates it over the
//      receiver row (compensated); the sum over channels happens once per
//      row (FP64 warp sums), F_k = sum_e sum_c g_c(e).
// One thread issues the MMAs; completion is signalled through an mbarrier
// whose waits are bounded: on a timeout the CTA sets an error bit, drains,
// frees its tensor memory and returns.
#include "kernels.h"
#include "tc.cuh"

namespace mp {

namespace {

constexpr int TF = 128, TLMAX = 2, TNLM = 9;
constexpr int NWG = 4;             // warpgroups per CTA, each an independent row stream
constexpr int NTH = 128 * NWG;     // threads per CTA
constexpr int WG_COLS = 128;       // tensor-memory columns per warpgroup
constexpr int TM_COLS = 512;       // allocated per CTA
constexpr int RPG = 8;             // receiver rows per row group
constexpr int CEF = 16;            // edges per forward chunk (MMA N = 16)
constexpr int CEB = 8;             // edges per adjoint chunk (+ 8 tangent columns, N = 16)
constexpr int kErrTimeout = 2;

template <bool FIRST>
struct TPaths {
    static constexpr int NP = FIRST ? 3 : 5;
    __host__ __device__ static constexpr int block(int q) { return FIRST ? (q == 0 ? 0 : 2 * q - 1) : q; }
    __host__ __device__ static constexpr int sla(int l) { return FIRST ? l : 2 * l - 1; }
    __host__ __device__ static constexpr int slb(int l) { return 2 * l; }
};

struct alignas(1024) Tiles {
    __nv_bfloat16 W3[5][128 * 64];   // 5 x 16 KB, one 128-row tile per radial path
    __nv_bfloat16 W2[128 * 64];      // 16 KB, rows 64..127 zero
};

// Per-warpgroup state.  B tiles hold 16 rows of 64 BF16 (two 1 KB atoms).
struct alignas(1024) WgState {
    __nv_bfloat16 B1[16 * 64];
    __nv_bfloat16 B2[16 * 64];
    float eps[16][kNB];
    float deps[CEB][kNB];
    float Y[16][TNLM];
    float u[16][4];
    double fpart[RPG][4][3];         // per-row, per-warp force partial sums
    int row[16], col[16];
    int64_t rp[RPG + 1];
    uint64_t mbar;
    int abort;
};

struct SmemTC {
    Tiles t;
    WgState wg[NWG];
    uint32_t taddr;
};

__device__ __forceinline__ SmemTC& smem_tc(unsigned char* raw) {
    uintptr_t p = (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023);
    return *reinterpret_cast<SmemTC*>(p);
}

__device__ __forceinline__ void wg_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(128) : "memory");
}

__device__ __forceinline__ int find_row_t(const int64_t* rp, int nrows, int64_t e) {
    int lr = 0;
    while (lr + 1 < nrows && rp[lr + 1] <= e) ++lr;
    return lr;
}

__device__ __forceinline__ void st_bf16(__nv_bfloat16* tile, int row, int k, float v) {
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(tile) +
                                      tc::sw128_off(row, k)) = __float2bfloat16_rn(v);
}

// D[tmem, 128 x 16] = A(128 x 64 tile) . B(16 x 64 tile)^T, four K = 16 steps.
__device__ __forceinline__ void mma_tile16(uint32_t d, const __nv_bfloat16* A, const __nv_bfloat16* B) {
    const uint64_t ad = tc::desc_sw128(tc::smem_u32(A));
    const uint64_t bd = tc::desc_sw128(tc::smem_u32(B));
    constexpr uint32_t idesc = tc::idesc_bf16(128, 16);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc, kk > 0 ? 1u : 0u);
}

// Bounded wait of one warpgroup on its mbarrier; uniform result.
__device__ __forceinline__ bool wg_wait(WgState& w, uint32_t& phase, int g) {
    const bool ok = tc::mbar_wait(&w.mbar, phase);
    if (ok)
        phase ^= 1u;
    else
        w.abort = 1;
    wg_sync(g);
    tc::fence_after_sync();
    return w.abort == 0;
}

__device__ __forceinline__ void tc_setup(SmemTC& s, const LayerW& wl, int np, bool first, int tid) {
    const uint4* src2 = reinterpret_cast<const uint4*>(wl.W2sw);
    uint4* dst2 = reinterpret_cast<uint4*>(s.t.W2);
    for (int q = tid; q < 128 * 64 * 2 / 16; q += NTH) dst2[q] = __ldg(&src2[q]);
    for (int p = 0; p < np; ++p) {
        const int blk = first ? (p == 0 ? 0 : 2 * p - 1) : p;
        const uint4* src = reinterpret_cast<const uint4*>(wl.W3sw + (size_t)blk * 128 * 64);
        uint4* dst = reinterpret_cast<uint4*>(s.t.W3[p]);
        for (int q = tid; q < 128 * 64 * 2 / 16; q += NTH) dst[q] = __ldg(&src[q]);
    }
    if ((tid & 127) == 0) {
        tc::mbar_init(&s.wg[tid >> 7].mbar, 1);
        s.wg[tid >> 7].abort = 0;
    }
    if ((tid >> 5) == 0) tc::tmem_alloc<TM_COLS>(&s.taddr);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

__device__ __forceinline__ void tc_teardown(SmemTC& s, uint32_t phase, int* err, int tid) {
    WgState& w = s.wg[tid >> 7];
    if (w.abort) {
        // drain: give in-flight MMAs of this warpgroup a bounded chance to land
        tc::mbar_wait(&w.mbar, phase, 1u << 16);
        if ((tid & 127) == 0) atomicOr(err, kErrTimeout);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if ((tid >> 5) == 0) tc::tmem_dealloc<TM_COLS>(s.taddr);
}

// Geometry of one chunk edge: eps (and d eps/dr), Y, unit vector and r.
template <bool DERIV>
__device__ __forceinline__ void chunk_geometry(const EdgeArgs& a, WgState& w, int lt, int64_t cb,
                                               int64_t e_end, int64_t r0, int nrows) {
    const int64_t e = cb + lt;
    float eps[kNB], deps[kNB], Y[TNLM], u4[4] = {0.f, 0.f, 0.f, 1.f};
    if (e < e_end) {
        const int lr = find_row_t(w.rp, nrows, e);
        const int j = a.col[e];
        float d[3];
        edge_vector(a.x, r0 + lr, j, a.shift[e], a.k, d);
        const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        u4[0] = d[0] / r;
        u4[1] = d[1] / r;
        u4[2] = d[2] / r;
        u4[3] = r;
        float env, denv;
        radial_basis<DERIV>(r, a.k, eps, deps, env, denv);
        sph_harm<TLMAX>(u4, Y);
        w.row[lt] = lr;
        w.col[lt] = j;
    } else {
#pragma unroll
        for (int q = 0; q < kNB; ++q) eps[q] = deps[q] = 0.f;
#pragma unroll
        for (int q = 0; q < TNLM; ++q) Y[q] = 0.f;
        w.row[lt] = -1;
        w.col[lt] = 0;
    }
#pragma unroll
    for (int q = 0; q < kNB; ++q) w.eps[lt][q] = eps[q];
    if (DERIV) {
#pragma unroll
        for (int q = 0; q < kNB; ++q) w.deps[lt][q] = deps[q];
    }
#pragma unroll
    for (int q = 0; q < TNLM; ++q) w.Y[lt][q] = Y[q];
#pragma unroll
    for (int q = 0; q < 4; ++q) w.u[lt][q] = u4[q];
}

// ------------------------------------------------------------------ forward --

template <bool FIRST>
__global__ void __launch_bounds__(NTH, 1) k_edge_fwd_tc(EdgeArgs a, LayerW wl, int64_t n_groups,
                                                        int* err) {
    using PP = TPaths<FIRST>;
    extern __shared__ unsigned char smem_raw[];
    SmemTC& s = smem_tc(smem_raw);
    const int tid = threadIdx.x, g = tid >> 7, lt = tid & 127, warp = tid >> 5;
    const int c = lt;
    WgState& w = s.wg[g];
    tc_setup(s, wl, PP::NP, FIRST, tid);
    const uint32_t tb = s.taddr + WG_COLS * g;
    const uint32_t tl = tb + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t phase = 0;
    bool alive = true;

    for (int64_t grp = (int64_t)blockIdx.x * NWG + g; grp < n_groups && alive;
         grp += (int64_t)gridDim.x * NWG) {
        const int64_t r0 = grp * RPG;
        const int nrows = (int)min((int64_t)RPG, a.n - r0);
        if (lt <= nrows) w.rp[lt] = a.row_ptr[r0 + lt];
        wg_sync(g);
        const int64_t e_beg = w.rp[0], e_end = w.rp[nrows];
        float acc[TNLM];
#pragma unroll
        for (int q = 0; q < TNLM; ++q) acc[q] = 0.f;
        int cur = -1, next = 0;
        auto write_row = [&](int lr, bool zero) {
            float* o = a.Aout + ((r0 + lr) * TNLM) * TF + c;
#pragma unroll
            for (int q = 0; q < TNLM; ++q) o[q * TF] = zero ? 0.f : acc[q] * a.k.inv_navg;
        };
        for (int64_t cb = e_beg; cb < e_end; cb += CEF) {
            if (lt < CEF) chunk_geometry<false>(a, w, lt, cb, e_end, r0, nrows);
            wg_sync(g);
            {   // a1 = silu(W1 eps) -> B1 (row = edge)
                const int kk = lt & 63, e0 = (lt >> 6) * 8;
                float w1[kNB];
#pragma unroll
                for (int b = 0; b < kNB; ++b) w1[b] = __ldg(&wl.W1[kk * kNB + b]);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float z = 0.f;
#pragma unroll
                    for (int b = 0; b < kNB; ++b) z = fmaf(w1[b], w.eps[e0 + q][b], z);
                    st_bf16(w.B1, e0 + q, kk, silu(z));
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            wg_sync(g);
            if (lt == 0) {
                tc::fence_after_sync();
                mma_tile16(tb, s.t.W2, w.B1);
                tc::mma_commit(&w.mbar);
            }
            if (!wg_wait(w, phase, g)) { alive = false; break; }
            if ((warp & 3) < 2) {   // lanes 0..63 = hidden units
                float z[16];
                tc::tmem_ld16(tl, z);
                tc::tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < CEF; ++e) st_bf16(w.B2, e, lt, silu(z[e]));
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            wg_sync(g);
            if (lt == 0) {
                tc::fence_after_sync();
#pragma unroll
                for (int q = 0; q < PP::NP; ++q) mma_tile16(tb + 16 + 16 * q, s.t.W3[q], w.B2);
                tc::mma_commit(&w.mbar);
            }
            if (!wg_wait(w, phase, g)) { alive = false; break; }
#pragma unroll 1
            for (int eb = 0; eb < CEF / 8; ++eb) {
                float R[PP::NP][8];
#pragma unroll
                for (int q = 0; q < PP::NP; ++q) tc::tmem_ld8(tl + 16 + 16 * q + 8 * eb, R[q]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int e8 = 0; e8 < 8; ++e8) {
                    const int e = eb * 8 + e8;
                    const int lr = w.row[e];
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
                        for (int q = 0; q < TNLM; ++q) acc[q] = 0.f;
                    }
                    const float* hj = a.Hin + ((int64_t)w.col[e] * TNLM) * TF + c;
                    const float h0 = hj[0];
                    acc[0] = fmaf(R[0][e8], h0, acc[0]);
                    const float t1 = R[PP::sla(1)][e8] * h0;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        acc[1 + m] = fmaf(t1, w.Y[e][1 + m], acc[1 + m]);
                        if (!FIRST) acc[1 + m] = fmaf(R[PP::slb(1)][e8], hj[(1 + m) * TF], acc[1 + m]);
                    }
                    const float t2 = R[PP::sla(2)][e8] * h0;
#pragma unroll
                    for (int m = 0; m < 5; ++m) {
                        acc[4 + m] = fmaf(t2, w.Y[e][4 + m], acc[4 + m]);
                        if (!FIRST) acc[4 + m] = fmaf(R[PP::slb(2)][e8], hj[(4 + m) * TF], acc[4 + m]);
                    }
                }
            }
            tc::fence_before_sync();
            wg_sync(g);
        }
        if (!alive) break;
        if (cur >= 0) {
            write_row(cur, false);
            next = cur + 1;
        }
        for (int q = next; q < nrows; ++q) write_row(q, true);
        wg_sync(g);
    }
    tc_teardown(s, phase, err, tid);
}

// ------------------------------------------------------------------ adjoint --

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool FIRST>
__global__ void __launch_bounds__(NTH, 1) k_edge_bwd_tc(EdgeArgs a, LayerW wl, int64_t n_groups,
                                                        int* err) {
    using PP = TPaths<FIRST>;
    extern __shared__ unsigned char smem_raw[];
    SmemTC& s = smem_tc(smem_raw);
    const int tid = threadIdx.x, g = tid >> 7, lt = tid & 127, warp = tid >> 5, lane = tid & 31;
    const int c = lt;
    WgState& w = s.wg[g];
    tc_setup(s, wl, PP::NP, FIRST, tid);
    const uint32_t tb = s.taddr + WG_COLS * g;
    const uint32_t tl = tb + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t phase = 0;
    bool alive = true;

    for (int64_t grp = (int64_t)blockIdx.x * NWG + g; grp < n_groups && alive;
         grp += (int64_t)gridDim.x * NWG) {
        const int64_t r0 = grp * RPG;
        const int nrows = (int)min((int64_t)RPG, a.n - r0);
        if (lt <= nrows) w.rp[lt] = a.row_ptr[r0 + lt];
        if (lt < RPG * 12) (&w.fpart[0][0][0])[lt] = 0.0;
        wg_sync(g);
        const int64_t e_beg = w.rp[0], e_end = w.rp[nrows];
        float gacc[TNLM], ak[TNLM], hk[TNLM];
        float fk[3] = {0.f, 0.f, 0.f}, fc[3] = {0.f, 0.f, 0.f};   // compensated row force
#pragma unroll
        for (int q = 0; q < TNLM; ++q) gacc[q] = ak[q] = hk[q] = 0.f;
        int cur = -1, next = 0;
        auto flush = [&](int lr, bool with_acc) {
            if (!FIRST) {
                const int64_t base = ((r0 + lr) * TNLM) * TF + c;
#pragma unroll
                for (int q = 0; q < TNLM; ++q)
                    a.Gin[base + q * TF] = a.Gout[base + q * TF] + (with_acc ? gacc[q] : 0.f);
            }
            if (with_acc) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const double v = warp_sum_d((double)fk[q] - (double)fc[q]);
                    if (lane == 0) w.fpart[lr][warp & 3][q] = v;
                }
            }
        };
        for (int64_t cb = e_beg; cb < e_end; cb += CEB) {
            if (lt < CEB) chunk_geometry<true>(a, w, lt, cb, e_end, r0, nrows);
            wg_sync(g);
            {   // a1 and its r-tangent -> B1 rows [0,8) and [8,16)
                const int kk = lt & 63, e0 = (lt >> 6) * 4;
                float w1[kNB];
#pragma unroll
                for (int b = 0; b < kNB; ++b) w1[b] = __ldg(&wl.W1[kk * kNB + b]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float z = 0.f, dz = 0.f;
#pragma unroll
                    for (int b = 0; b < kNB; ++b) {
                        z = fmaf(w1[b], w.eps[e0 + q][b], z);
                        dz = fmaf(w1[b], w.deps[e0 + q][b], dz);
                    }
                    st_bf16(w.B1, e0 + q, kk, silu(z));
                    st_bf16(w.B1, CEB + e0 + q, kk, silu_grad(z) * dz);
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            wg_sync(g);
            if (lt == 0) {
                tc::fence_after_sync();
                mma_tile16(tb, s.t.W2, w.B1);
                tc::mma_commit(&w.mbar);
            }
            if (!wg_wait(w, phase, g)) { alive = false; break; }
            if ((warp & 3) < 2) {
                float z[16];
                tc::tmem_ld16(tl, z);     // columns 0..7: z2, 8..15: dz2
                tc::tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < CEB; ++e) {
                    st_bf16(w.B2, e, lt, silu(z[e]));
                    st_bf16(w.B2, CEB + e, lt, silu_grad(z[e]) * z[CEB + e]);
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            wg_sync(g);
            if (lt == 0) {
                tc::fence_after_sync();
#pragma unroll
                for (int q = 0; q < PP::NP; ++q) mma_tile16(tb + 16 + 16 * q, s.t.W3[q], w.B2);
                tc::mma_commit(&w.mbar);
            }
            if (!wg_wait(w, phase, g)) { alive = false; break; }
            float R[PP::NP][8], dR[PP::NP][8];
#pragma unroll
            for (int q = 0; q < PP::NP; ++q) {
                tc::tmem_ld8(tl + 16 + 16 * q, R[q]);
                tc::tmem_ld8(tl + 16 + 16 * q + CEB, dR[q]);
            }
            tc::tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < CEB; ++e) {
                const int lr = w.row[e];
                if (lr < 0) break;
                if (lr != cur) {
                    if (cur >= 0) {
                        flush(cur, true);
                        next = cur + 1;
                    }
                    for (int q = next; q < lr; ++q) flush(q, false);
                    next = lr;
                    cur = lr;
                    const int64_t base = ((r0 + lr) * TNLM) * TF + c;
#pragma unroll
                    for (int q = 0; q < TNLM; ++q) {
                        gacc[q] = 0.f;
                        ak[q] = a.Alpha[base + q * TF];
                        hk[q] = (FIRST && q > 0) ? 0.f : a.Hin[base + q * TF];
                    }
#pragma unroll
                    for (int q = 0; q < 3; ++q) fk[q] = fc[q] = 0.f;
                }
                const int64_t jb = ((int64_t)w.col[e] * TNLM) * TF + c;
                float aj[TNLM], hj[TNLM], Y[TNLM];
#pragma unroll
                for (int q = 0; q < TNLM; ++q) {
                    aj[q] = a.Alpha[jb + q * TF];
                    hj[q] = (FIRST && q > 0) ? 0.f : a.Hin[jb + q * TF];
                    Y[q] = w.Y[e][q];
                }
                if (!FIRST) {
                    float g0 = R[0][e] * aj[0];
                    float sm1 = 0.f, sm2 = 0.f;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        sm1 = fmaf(aj[1 + m], Y[1 + m], sm1);
                        gacc[1 + m] = fmaf(R[PP::slb(1)][e], aj[1 + m], gacc[1 + m]);
                    }
#pragma unroll
                    for (int m = 0; m < 5; ++m) {
                        sm2 = fmaf(aj[4 + m], Y[4 + m], sm2);
                        gacc[4 + m] = fmaf(R[PP::slb(2)][e], aj[4 + m], gacc[4 + m]);
                    }
                    g0 = fmaf(-R[PP::sla(1)][e], sm1, g0);
                    g0 = fmaf(R[PP::sla(2)][e], sm2, g0);
                    gacc[0] += g0;
                }
                // this channel's share of dE_pair/dd: radial part (dE/dR . dR/dr)
                // along u plus the angular part through dE/dY
                float gr = (ak[0] * hj[0] + aj[0] * hk[0]) * dR[0][e];
                float gy[TNLM];
                gy[0] = 0.f;
                {
                    float g1a = 0.f, g1b = 0.f;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        const float t = ak[1 + m] * hj[0] - aj[1 + m] * hk[0];
                        g1a = fmaf(Y[1 + m], t, g1a);
                        gy[1 + m] = R[PP::sla(1)][e] * t;
                        if (!FIRST) g1b += ak[1 + m] * hj[1 + m] + aj[1 + m] * hk[1 + m];
                    }
                    gr = fmaf(g1a, dR[PP::sla(1)][e], gr);
                    if (!FIRST) gr = fmaf(g1b, dR[PP::slb(1)][e], gr);
                }
                {
                    float g2a = 0.f, g2b = 0.f;
#pragma unroll
                    for (int m = 0; m < 5; ++m) {
                        const float t = ak[4 + m] * hj[0] + aj[4 + m] * hk[0];
                        g2a = fmaf(Y[4 + m], t, g2a);
                        gy[4 + m] = R[PP::sla(2)][e] * t;
                        if (!FIRST) g2b += ak[4 + m] * hj[4 + m] + aj[4 + m] * hk[4 + m];
                    }
                    gr = fmaf(g2a, dR[PP::sla(2)][e], gr);
                    if (!FIRST) gr = fmaf(g2b, dR[PP::slb(2)][e], gr);
                }
                const float u[3] = {w.u[e][0], w.u[e][1], w.u[e][2]};
                const float ir = 1.f / w.u[e][3];
                float v[3];
                sph_grad<TLMAX, float>(u, gy, v);
                const float vu = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float gq = gr * u[q] + (v[q] - vu * u[q]) * ir;
                    const float y = gq - fc[q];
                    const float t = fk[q] + y;
                    fc[q] = (t - fk[q]) - y;
                    fk[q] = t;
                }
            }
            tc::fence_before_sync();
            wg_sync(g);
        }
        if (!alive) break;
        if (cur >= 0) {
            flush(cur, true);
            next = cur + 1;
        }
        for (int q = next; q < nrows; ++q) flush(q, false);
        wg_sync(g);
        if (lt < nrows * 3) {
            const int lr = lt / 3, q = lt % 3;
            const double f = w.fpart[lr][0][q] + w.fpart[lr][1][q] + w.fpart[lr][2][q] + w.fpart[lr][3][q];
            a.frc[(r0 + lr) * 3 + q] += f;
        }
        wg_sync(g);
    }
    tc_teardown(s, phase, err, tid);
}

template <class K>
int launch_tc(K kernel, const EdgeArgs& a, int num_sms, cudaStream_t st) {
    const int64_t groups = (a.n + RPG - 1) / RPG;
    const size_t smem = sizeof(SmemTC) + 1024;
    MP_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    int64_t grid = (int64_t)num_sms;   // one CTA (and one 512-column TMEM allocation) per SM
    const int64_t need = (groups + NWG - 1) / NWG;
    if (grid > need) grid = need;
    kernel<<<(unsigned)grid, NTH, smem, st>>>(a, *a.w, groups, a.err);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int launch_edge_fwd_bf16(const Model& m, const EdgeArgs& a, cudaStream_t st, int num_sms) {
    if (!(m.d.F == TF && m.d.lmax == TLMAX) || !a.w->W3sw || !a.err) return MP_ERR_UNSUPPORTED;
    if (a.n == 0) return MP_OK;
    return a.first ? launch_tc(k_edge_fwd_tc<true>, a, num_sms, st)
                   : launch_tc(k_edge_fwd_tc<false>, a, num_sms, st);
}

int launch_edge_bwd_bf16(const Model& m, const EdgeArgs& a, cudaStream_t st, int num_sms) {
    if (!(m.d.F == TF && m.d.lmax == TLMAX) || !a.w->W3sw || !a.err) return MP_ERR_UNSUPPORTED;
    if (a.n == 0) return MP_OK;
    return a.first ? launch_tc(k_edge_bwd_tc<true>, a, num_sms, st)
                   : launch_tc(k_edge_bwd_tc<false>, a, num_sms, st);
}

}  // namespace mp

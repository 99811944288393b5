// Edge kernels with the radial MLP's dense contractions on tcgen05 tensor
// cores (BF16 operands, FP32 accumulation in tensor memory).  Geometry, the
// first radial layer (K = 8), messages, adjoint sums and forces stay FP32 on
// CUDA cores.  Shapes compiled: F = 128, lmax = 2, H = 64.
//
// Per chunk of edges (rows owned by the CTA, as in the FP32 kernels):
//   1. CUDA cores: geometry, eps (and d eps/dr), a1 = silu(W1 eps) -> BF16
//      K-major tile B1 (rows = edges; adjoint: edges, then their r-tangents).
//   2. MMA1: D1[128 x 32] = W2pad[128 x 64] . B1^T  (rows 0..63 = hidden).
//   3. warps 0-1 read D1 from tensor memory: a2 = silu(z2) (adjoint also
//      da2 = silu'(z2) dz2) -> BF16 tile B2.
//   4. MMA2: D2_q[128 x 32] = W3_q[128 x 64] . B2^T for each radial path q
//      (lane = channel, column = edge: R, and dR/dr in the adjoint).
//   5. thread = channel reads its row of D2 and runs the message (forward)
//      or symmetric-pair adjoint (backward) epilogue.
// One thread issues the MMAs; completion is signalled through an mbarrier
// whose waits are bounded: on a timeout the CTA sets an error bit, drains,
// frees its tensor memory and returns.
#include "kernels.h"
#include "tc.cuh"

namespace mp {

namespace {

constexpr int TF = 128, TLMAX = 2, TNLM = 9, TP = 640;
constexpr int NT = 128;            // threads per CTA (= channels)
constexpr int RPBT = 8;            // receiver rows per row group
constexpr int CF = 32;             // edges per forward chunk
constexpr int CBW = 16;            // edges per adjoint chunk (+16 tangent columns)
constexpr int NCOLS = 256;         // tensor-memory columns per CTA
constexpr int kErrTimeout = 2;

template <bool FIRST>
struct TPaths {
    static constexpr int NP = FIRST ? 3 : 5;
    __host__ __device__ static constexpr int block(int q) { return FIRST ? (q == 0 ? 0 : 2 * q - 1) : q; }
    __host__ __device__ static constexpr int sla(int l) { return FIRST ? l : 2 * l - 1; }
    __host__ __device__ static constexpr int slb(int l) { return 2 * l; }
};

struct alignas(1024) TileSmem {
    __nv_bfloat16 W3[5][128 * 64];   // 5 x 16 KB
    __nv_bfloat16 W2[128 * 64];      // 16 KB
    __nv_bfloat16 B1[32 * 64];       // 4 KB
    __nv_bfloat16 B2[32 * 64];       // 4 KB
};

struct FwdSmemT {
    TileSmem t;
    float eps[CF][kNB];
    float Y[CF][TNLM];
    int row[CF], col[CF];
    int64_t rp[RPBT + 1];
    uint64_t mbar;
    uint32_t taddr;
    int abort;
};

struct BwdSmemT {
    TileSmem t;
    float eps[CBW][kNB], deps[CBW][kNB];
    float Y[CBW][TNLM];
    float u[CBW][4];
    float part[CBW][TNLM][TF + 1];
    double red[CBW][TNLM];
    double frow[RPBT][3];
    int row[CBW], col[CBW];
    int64_t rp[RPBT + 1];
    uint64_t mbar;
    uint32_t taddr;
    int abort;
};

template <class S>
__device__ __forceinline__ S& aligned_smem(unsigned char* raw) {
    uintptr_t p = (reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023);
    return *reinterpret_cast<S*>(p);
}

__device__ __forceinline__ void copy16(void* dst, const void* src, int bytes, int tid) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (int q = tid; q < bytes / 16; q += NT) d[q] = __ldg(&s[q]);
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

// Issue D[tmem] = A(tile 128 x 64) . B(tile 32 x 64)^T as four K = 16 steps.
__device__ __forceinline__ void mma_tile(uint32_t d, const __nv_bfloat16* A, const __nv_bfloat16* B) {
    const uint64_t ad = tc::desc_sw128(tc::smem_u32(A));
    const uint64_t bd = tc::desc_sw128(tc::smem_u32(B));
    constexpr uint32_t idesc = tc::idesc_bf16(128, 32);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc, kk > 0 ? 1u : 0u);
}

// Wait for the next MMA batch; returns false (uniformly) if any thread of
// the CTA timed out.
template <class S>
__device__ __forceinline__ bool wait_mma(S& s, uint32_t& phase) {
    const bool ok = tc::mbar_wait(&s.mbar, phase);
    if (ok)
        phase ^= 1u;
    else
        s.abort = 1;
    __syncthreads();
    tc::fence_after_sync();
    return s.abort == 0;
}

template <class S>
__device__ __forceinline__ void tc_setup(S& s, const LayerW& wl, int np, bool first, int tid) {
    copy16(s.t.W2, wl.W2sw, 128 * 64 * 2, tid);
    for (int q = 0; q < np; ++q) {
        const int blk = first ? (q == 0 ? 0 : 2 * q - 1) : q;
        copy16(s.t.W3[q], wl.W3sw + (size_t)blk * 128 * 64, 128 * 64 * 2, tid);
    }
    if (tid == 0) {
        tc::mbar_init(&s.mbar, 1);
        s.abort = 0;
    }
    if ((tid >> 5) == 0) tc::tmem_alloc<NCOLS>(&s.taddr);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

template <class S>
__device__ __forceinline__ void tc_teardown(S& s, uint32_t phase, int* err, int tid) {
    tc::fence_before_sync();
    __syncthreads();
    if (s.abort) {
        // drain: give in-flight MMAs a bounded chance to land before freeing
        tc::mbar_wait(&s.mbar, phase, 1u << 16);
        if (tid == 0) atomicOr(err, kErrTimeout);
    }
    __syncthreads();
    if ((tid >> 5) == 0) tc::tmem_dealloc<NCOLS>(s.taddr);
}

// ------------------------------------------------------------------ forward --

template <bool FIRST>
__global__ void __launch_bounds__(NT, 1) k_edge_fwd_tc(EdgeArgs a, LayerW wl, int64_t n_groups,
                                                       int* err) {
    using PP = TPaths<FIRST>;
    extern __shared__ unsigned char smem_raw[];
    FwdSmemT& s = aligned_smem<FwdSmemT>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int c = tid;
    tc_setup(s, wl, PP::NP, FIRST, tid);
    const uint32_t tbase = s.taddr;
    const uint32_t tlane = tbase + ((uint32_t)(32 * warp) << 16);
    uint32_t phase = 0;
    bool alive = true;

    for (int64_t grp = blockIdx.x; grp < n_groups && alive; grp += gridDim.x) {
        const int64_t r0 = grp * RPBT;
        const int nrows = (int)min((int64_t)RPBT, a.n - r0);
        if (tid <= nrows) s.rp[tid] = a.row_ptr[r0 + tid];
        __syncthreads();
        const int64_t e_beg = s.rp[0], e_end = s.rp[nrows];
        float acc[TNLM];
#pragma unroll
        for (int q = 0; q < TNLM; ++q) acc[q] = 0.f;
        int cur = -1, next = 0;
        auto write_row = [&](int lr, bool zero) {
            float* o = a.Aout + ((r0 + lr) * TNLM) * TF + c;
#pragma unroll
            for (int q = 0; q < TNLM; ++q) o[q * TF] = zero ? 0.f : acc[q] * a.k.inv_navg;
        };
        for (int64_t cb = e_beg; cb < e_end; cb += CF) {
            if (tid < CF) {
                const int64_t e = cb + tid;
                float eps[kNB], Y[TNLM];
                if (e < e_end) {
                    const int lr = find_row_t(s.rp, nrows, e);
                    const int j = a.col[e];
                    float d[3];
                    edge_vector(a.x, r0 + lr, j, a.shift[e], a.k, d);
                    const float r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                    const float u[3] = {d[0] / r, d[1] / r, d[2] / r};
                    float dd[kNB], env, denv;
                    radial_basis<false>(r, a.k, eps, dd, env, denv);
                    sph_harm<TLMAX>(u, Y);
                    s.row[tid] = lr;
                    s.col[tid] = j;
                } else {
#pragma unroll
                    for (int q = 0; q < kNB; ++q) eps[q] = 0.f;
#pragma unroll
                    for (int q = 0; q < TNLM; ++q) Y[q] = 0.f;
                    s.row[tid] = -1;
                    s.col[tid] = 0;
                }
#pragma unroll
                for (int q = 0; q < kNB; ++q) s.eps[tid][q] = eps[q];
#pragma unroll
                for (int q = 0; q < TNLM; ++q) s.Y[tid][q] = Y[q];
            }
            __syncthreads();
            {   // a1 = silu(W1 eps) -> B1 (row = edge)
                const int kk = tid & 63, e0 = (tid >> 6) * 16;
                float w1[kNB];
#pragma unroll
                for (int b = 0; b < kNB; ++b) w1[b] = __ldg(&wl.W1[kk * kNB + b]);
#pragma unroll 4
                for (int q = 0; q < 16; ++q) {
                    float z = 0.f;
#pragma unroll
                    for (int b = 0; b < kNB; ++b) z = fmaf(w1[b], s.eps[e0 + q][b], z);
                    st_bf16(s.t.B1, e0 + q, kk, silu(z));
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                mma_tile(tbase, s.t.W2, s.t.B1);
                tc::mma_commit(&s.mbar);
            }
            if (!wait_mma(s, phase)) { alive = false; break; }
            if (warp < 2) {   // lanes 0..63 = hidden units
                float z[32];
                tc::tmem_ld16(tlane + 0, z);
                tc::tmem_ld16(tlane + 16, z + 16);
                tc::tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < CF; ++e) st_bf16(s.t.B2, e, tid, silu(z[e]));
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
#pragma unroll
                for (int q = 0; q < PP::NP; ++q) mma_tile(tbase + 32 + 32 * q, s.t.W3[q], s.t.B2);
                tc::mma_commit(&s.mbar);
            }
            if (!wait_mma(s, phase)) { alive = false; break; }
            // epilogue: thread c = TMEM lane c
#pragma unroll 1
            for (int eb = 0; eb < CF / 8; ++eb) {
                float R[PP::NP][8];
#pragma unroll
                for (int q = 0; q < PP::NP; ++q) tc::tmem_ld8(tlane + 32 + 32 * q + 8 * eb, R[q]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int e8 = 0; e8 < 8; ++e8) {
                    const int e = eb * 8 + e8;
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
                        for (int q = 0; q < TNLM; ++q) acc[q] = 0.f;
                    }
                    const float* hj = a.Hin + ((int64_t)s.col[e] * TNLM) * TF + c;
                    const float h0 = hj[0];
                    acc[0] = fmaf(R[0][e8], h0, acc[0]);
                    const float t1 = R[PP::sla(1)][e8] * h0;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        acc[1 + m] = fmaf(t1, s.Y[e][1 + m], acc[1 + m]);
                        if (!FIRST) acc[1 + m] = fmaf(R[PP::slb(1)][e8], hj[(1 + m) * TF], acc[1 + m]);
                    }
                    const float t2 = R[PP::sla(2)][e8] * h0;
#pragma unroll
                    for (int m = 0; m < 5; ++m) {
                        acc[4 + m] = fmaf(t2, s.Y[e][4 + m], acc[4 + m]);
                        if (!FIRST) acc[4 + m] = fmaf(R[PP::slb(2)][e8], hj[(4 + m) * TF], acc[4 + m]);
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
        }
        if (!alive) break;
        if (cur >= 0) {
            write_row(cur, false);
            next = cur + 1;
        }
        for (int q = next; q < nrows; ++q) write_row(q, true);
        __syncthreads();
    }
    tc_teardown(s, phase, err, tid);
}

// ------------------------------------------------------------------ adjoint --

__device__ __forceinline__ double kahan_sum_t(const float* v, int n) {
    float s = 0.f, comp = 0.f;
    for (int q = 0; q < n; ++q) {
        const float y = v[q] - comp;
        const float t = s + y;
        comp = (t - s) - y;
        s = t;
    }
    return (double)s - (double)comp;
}

template <bool FIRST>
__global__ void __launch_bounds__(NT, 1) k_edge_bwd_tc(EdgeArgs a, LayerW wl, int64_t n_groups,
                                                       int* err) {
    using PP = TPaths<FIRST>;
    extern __shared__ unsigned char smem_raw[];
    BwdSmemT& s = aligned_smem<BwdSmemT>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int c = tid;
    tc_setup(s, wl, PP::NP, FIRST, tid);
    const uint32_t tbase = s.taddr;
    const uint32_t tlane = tbase + ((uint32_t)(32 * warp) << 16);
    uint32_t phase = 0;
    bool alive = true;

    for (int64_t grp = blockIdx.x; grp < n_groups && alive; grp += gridDim.x) {
        const int64_t r0 = grp * RPBT;
        const int nrows = (int)min((int64_t)RPBT, a.n - r0);
        if (tid <= nrows) s.rp[tid] = a.row_ptr[r0 + tid];
        if (tid < RPBT * 3) s.frow[tid / 3][tid % 3] = 0.0;
        __syncthreads();
        const int64_t e_beg = s.rp[0], e_end = s.rp[nrows];
        float gacc[TNLM], ak[TNLM], hk[TNLM];
#pragma unroll
        for (int q = 0; q < TNLM; ++q) gacc[q] = ak[q] = hk[q] = 0.f;
        int cur = -1, next = 0;
        auto flush = [&](int lr, bool with_acc) {
            if (FIRST) return;
            const int64_t base = ((r0 + lr) * TNLM) * TF + c;
#pragma unroll
            for (int q = 0; q < TNLM; ++q)
                a.Gin[base + q * TF] = a.Gout[base + q * TF] + (with_acc ? gacc[q] : 0.f);
        };
        for (int64_t cb = e_beg; cb < e_end; cb += CBW) {
            if (tid < CBW) {
                const int64_t e = cb + tid;
                float eps[kNB], deps[kNB], Y[TNLM], u4[4] = {0.f, 0.f, 0.f, 1.f};
                if (e < e_end) {
                    const int lr = find_row_t(s.rp, nrows, e);
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
                    sph_harm<TLMAX>(u4, Y);
                    s.row[tid] = lr;
                    s.col[tid] = j;
                } else {
#pragma unroll
                    for (int q = 0; q < kNB; ++q) eps[q] = deps[q] = 0.f;
#pragma unroll
                    for (int q = 0; q < TNLM; ++q) Y[q] = 0.f;
                    s.row[tid] = -1;
                    s.col[tid] = 0;
                }
#pragma unroll
                for (int q = 0; q < kNB; ++q) {
                    s.eps[tid][q] = eps[q];
                    s.deps[tid][q] = deps[q];
                }
#pragma unroll
                for (int q = 0; q < TNLM; ++q) s.Y[tid][q] = Y[q];
#pragma unroll
                for (int q = 0; q < 4; ++q) s.u[tid][q] = u4[q];
            }
            __syncthreads();
            {   // a1 and its r-tangent -> B1 rows [0,16) and [16,32)
                const int kk = tid & 63, e0 = (tid >> 6) * 8;
                float w1[kNB];
#pragma unroll
                for (int b = 0; b < kNB; ++b) w1[b] = __ldg(&wl.W1[kk * kNB + b]);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    float z = 0.f, dz = 0.f;
#pragma unroll
                    for (int b = 0; b < kNB; ++b) {
                        z = fmaf(w1[b], s.eps[e0 + q][b], z);
                        dz = fmaf(w1[b], s.deps[e0 + q][b], dz);
                    }
                    st_bf16(s.t.B1, e0 + q, kk, silu(z));
                    st_bf16(s.t.B1, CBW + e0 + q, kk, silu_grad(z) * dz);
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                mma_tile(tbase, s.t.W2, s.t.B1);
                tc::mma_commit(&s.mbar);
            }
            if (!wait_mma(s, phase)) { alive = false; break; }
            if (warp < 2) {
                float z[32];
                tc::tmem_ld16(tlane + 0, z);        // z2 of the 16 edges
                tc::tmem_ld16(tlane + 16, z + 16);  // their r-tangents dz2
                tc::tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < CBW; ++e) {
                    st_bf16(s.t.B2, e, tid, silu(z[e]));
                    st_bf16(s.t.B2, CBW + e, tid, silu_grad(z[e]) * z[CBW + e]);
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
#pragma unroll
                for (int q = 0; q < PP::NP; ++q) mma_tile(tbase + 32 + 32 * q, s.t.W3[q], s.t.B2);
                tc::mma_commit(&s.mbar);
            }
            if (!wait_mma(s, phase)) { alive = false; break; }
#pragma unroll 1
            for (int eb = 0; eb < CBW / 8; ++eb) {
                float R[PP::NP][8], dR[PP::NP][8];
#pragma unroll
                for (int q = 0; q < PP::NP; ++q) {
                    tc::tmem_ld8(tlane + 32 + 32 * q + 8 * eb, R[q]);
                    tc::tmem_ld8(tlane + 32 + 32 * q + CBW + 8 * eb, dR[q]);
                }
                tc::tmem_wait_ld();
#pragma unroll
                for (int e8 = 0; e8 < 8; ++e8) {
                    const int e = eb * 8 + e8;
                    const int lr = s.row[e];
                    if (lr < 0) {
#pragma unroll
                        for (int q = 0; q < TNLM; ++q) s.part[e][q][c] = 0.f;
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
                        const int64_t base = ((r0 + lr) * TNLM) * TF + c;
#pragma unroll
                        for (int q = 0; q < TNLM; ++q) {
                            gacc[q] = 0.f;
                            ak[q] = a.Alpha[base + q * TF];
                            hk[q] = (FIRST && q > 0) ? 0.f : a.Hin[base + q * TF];
                        }
                    }
                    const int64_t jb = ((int64_t)s.col[e] * TNLM) * TF + c;
                    float aj[TNLM], hj[TNLM], Y[TNLM];
#pragma unroll
                    for (int q = 0; q < TNLM; ++q) {
                        aj[q] = a.Alpha[jb + q * TF];
                        hj[q] = (FIRST && q > 0) ? 0.f : a.Hin[jb + q * TF];
                        Y[q] = s.Y[e][q];
                    }
                    if (!FIRST) {
                        float g0 = R[0][e8] * aj[0];
                        float sm1 = 0.f, sm2 = 0.f;
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            sm1 = fmaf(aj[1 + m], Y[1 + m], sm1);
                            gacc[1 + m] = fmaf(R[PP::slb(1)][e8], aj[1 + m], gacc[1 + m]);
                        }
#pragma unroll
                        for (int m = 0; m < 5; ++m) {
                            sm2 = fmaf(aj[4 + m], Y[4 + m], sm2);
                            gacc[4 + m] = fmaf(R[PP::slb(2)][e8], aj[4 + m], gacc[4 + m]);
                        }
                        g0 = fmaf(-R[PP::sla(1)][e8], sm1, g0);
                        g0 = fmaf(R[PP::sla(2)][e8], sm2, g0);
                        gacc[0] += g0;
                    }
                    float gr = (ak[0] * hj[0] + aj[0] * hk[0]) * dR[0][e8];
                    {
                        float g1a = 0.f, g1b = 0.f;
#pragma unroll
                        for (int m = 0; m < 3; ++m) {
                            const float t = ak[1 + m] * hj[0] - aj[1 + m] * hk[0];
                            g1a = fmaf(Y[1 + m], t, g1a);
                            s.part[e][1 + m][c] = R[PP::sla(1)][e8] * t;
                            if (!FIRST) g1b += ak[1 + m] * hj[1 + m] + aj[1 + m] * hk[1 + m];
                        }
                        gr = fmaf(g1a, dR[PP::sla(1)][e8], gr);
                        if (!FIRST) gr = fmaf(g1b, dR[PP::slb(1)][e8], gr);
                    }
                    {
                        float g2a = 0.f, g2b = 0.f;
#pragma unroll
                        for (int m = 0; m < 5; ++m) {
                            const float t = ak[4 + m] * hj[0] + aj[4 + m] * hk[0];
                            g2a = fmaf(Y[4 + m], t, g2a);
                            s.part[e][4 + m][c] = R[PP::sla(2)][e8] * t;
                            if (!FIRST) g2b += ak[4 + m] * hj[4 + m] + aj[4 + m] * hk[4 + m];
                        }
                        gr = fmaf(g2a, dR[PP::sla(2)][e8], gr);
                        if (!FIRST) gr = fmaf(g2b, dR[PP::slb(2)][e8], gr);
                    }
                    s.part[e][0][c] = gr;
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            for (int t = tid; t < CBW * TNLM; t += NT)
                s.red[t / TNLM][t % TNLM] = kahan_sum_t(s.part[t / TNLM][t % TNLM], TF);
            __syncthreads();
            if (tid < CBW && s.row[tid] >= 0) {
                const int e = tid;
                const double gr = s.red[e][0];
                double gY[TNLM];
                gY[0] = 0.0;
#pragma unroll
                for (int q = 1; q < TNLM; ++q) gY[q] = s.red[e][q];
                const double u[3] = {s.u[e][0], s.u[e][1], s.u[e][2]};
                const double ir = 1.0 / (double)s.u[e][3];
                double v[3];
                sph_grad<TLMAX, double>(u, gY, v);
                const double vu = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
#pragma unroll
                for (int q = 0; q < 3; ++q) s.red[e][q] = gr * u[q] + (v[q] - vu * u[q]) * ir;
            }
            __syncthreads();
            if (tid == 0) {
                for (int e = 0; e < CBW; ++e) {
                    const int lr = s.row[e];
                    if (lr < 0) break;
#pragma unroll
                    for (int q = 0; q < 3; ++q) s.frow[lr][q] += s.red[e][q];
                }
            }
            __syncthreads();
        }
        if (!alive) break;
        if (cur >= 0) {
            flush(cur, true);
            next = cur + 1;
        }
        for (int q = next; q < nrows; ++q) flush(q, false);
        __syncthreads();
        if (tid < nrows * 3) a.frc[(r0 + tid / 3) * 3 + tid % 3] += s.frow[tid / 3][tid % 3];
        __syncthreads();
    }
    tc_teardown(s, phase, err, tid);
}

template <class K>
int launch_tc(K kernel, size_t smem, const EdgeArgs& a, int num_sms, cudaStream_t st) {
    const int64_t groups = (a.n + RPBT - 1) / RPBT;
    MP_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    int per_sm = 0;
    MP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem));
    if (per_sm < 1) return MP_ERR_UNSUPPORTED;
    // tensor memory: at most 512 / NCOLS resident CTAs per SM may allocate
    per_sm = per_sm > 512 / NCOLS ? 512 / NCOLS : per_sm;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > groups) grid = groups;
    kernel<<<(unsigned)grid, NT, smem, st>>>(a, *a.w, groups, a.err);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int launch_edge_fwd_bf16(const Model& m, const EdgeArgs& a, cudaStream_t st, int num_sms) {
    if (!(m.d.F == TF && m.d.lmax == TLMAX) || !a.w->W3sw || !a.err) return MP_ERR_UNSUPPORTED;
    if (a.n == 0) return MP_OK;
    const size_t smem = sizeof(FwdSmemT) + 1024;
    return a.first ? launch_tc(k_edge_fwd_tc<true>, smem, a, num_sms, st)
                   : launch_tc(k_edge_fwd_tc<false>, smem, a, num_sms, st);
}

int launch_edge_bwd_bf16(const Model& m, const EdgeArgs& a, cudaStream_t st, int num_sms) {
    if (!(m.d.F == TF && m.d.lmax == TLMAX) || !a.w->W3sw || !a.err) return MP_ERR_UNSUPPORTED;
    if (a.n == 0) return MP_OK;
    const size_t smem = sizeof(BwdSmemT) + 1024;
    return a.first ? launch_tc(k_edge_bwd_tc<true>, smem, a, num_sms, st)
                   : launch_tc(k_edge_bwd_tc<false>, smem, a, num_sms, st);
}

}  // namespace mp

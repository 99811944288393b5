// Node update of one layer with the F x F contractions on tcgen05 tensor
// cores: BF16 operands, FP32 accumulation in tensor memory.  Shapes
// compiled: F = 128, lmax = 2.  Same equations as the FP32 kernel:
//   S = W0 A0 + U1 B1 + U2 B2 + b,  B_l = sum_m A_lm^2,
//   h0' = h0 + silu(S),  h_lm' = h_lm + V_l A_lm.
// (The adjoint stays FP32: it is linear in dE/dh', and rounding the
// per-partition adjoints to BF16 would not commute with their sum over
// partitions, so partitioned forces would no longer equal unpartitioned
// ones to FP32 rounding.  Each atom's forward, in contrast, sees identical
// inputs in every partition that needs it.)
//
// Orientation: output channels are the MMA's M = 128 rows (tensor-memory
// lanes), a tile of 16 atoms its N = 16 columns, input channels its K:
//   D_S  = [W0 | U1 | U2] . [A0 | B1 | B2]^T   (K = 384)
//   D_lm = V_l . A_lm^T                         (K = 128, lm = 1..8)
// so that in the epilogue a warp reads and writes 32 consecutive channels
// of one atom (coalesced).
//
// One CTA per SM keeps the five 128 x 128 weight images in shared memory
// (160 KB) and loops over atom tiles.  Per tile: every thread loads one
// atom's four channels of all nine (l, m) rows (float4), forms B_l and
// rounds to BF16 into the swizzled operand tiles; one thread issues the
// MMAs into one of two tensor-memory buffers; meanwhile the threads
// prefetch the next tile's inputs and write the previous tile's outputs
// from the other buffer.  The MMA completion wait is bounded: on a timeout
// the kernel sets an error bit, frees its tensor memory and returns.
#include "kernels.h"
#include "tc.cuh"

namespace mp {

namespace {

constexpr int NF = 128;          // channels
constexpr int NLM9 = 9;          // (l, m) rows per atom
constexpr int NT = 16;           // atoms per tile (MMA N)
constexpr int NTHR = 512;        // threads per CTA: 16 atoms x 32 channel quads
constexpr int BUF_COLS = 256;    // tensor-memory columns per buffer
constexpr int kErrTimeout = 4;

// Shared memory of a node kernel: NW weight images, NX operand tiles.
template <int NW, int NX>
struct alignas(1024) NodeSmemT {
    __nv_bfloat16 W[NW][2][128 * 64];   // weight images: matrix, K-block (16 KB each)
    __nv_bfloat16 X[NX][2][NT * 64];    // operand tiles: tile, K-block (2 KB each)
    uint64_t mbar;
    uint32_t taddr;
    int abort;
};
using NodeSmemF = NodeSmemT<5, 11>;     // forward: W0, U1, U2, V1, V2; A0, B1, B2, A_lm
using NodeSmemA = NodeSmemT<3, 3>;      // adjoint, W0^T, U1^T, U2^T against gS (3 parts)
using NodeSmemV = NodeSmemT<2, 24>;     // adjoint, V1^T, V2^T against G'_lm (3 parts each)

// Dynamic shared memory rounded up to 1024 bytes by offsetting the __shared__
// pointer itself (no integer round trip), so accesses stay shared-space.
template <class S>
__device__ __forceinline__ S& node_smem(unsigned char* raw) {
    const uint32_t pad = (1024u - (tc::smem_u32(raw) & 1023u)) & 1023u;
    return *reinterpret_cast<S*>(raw + pad);
}

// Byte offset of channels 4 q4 .. 4 q4 + 3 of atom row `row` in an operand
// tile (two K-blocks of 64 channels, 128-byte swizzle).
__device__ __forceinline__ uint32_t x4_off(int row, int q4) {
    const int kq = q4 & 15;                        // quad within the K-block
    return row * 128 + ((((kq >> 1) ^ (row & 7)) & 7) << 4) + ((kq & 1) << 3);
}

__device__ __forceinline__ void st_bf16x4(__nv_bfloat16 (*x)[NT * 64], int row, int q4,
                                          __nv_bfloat162 lo, __nv_bfloat162 hi) {
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&lo);
    u.y = *reinterpret_cast<uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(reinterpret_cast<unsigned char*>(x[q4 >> 4]) + x4_off(row, q4)) = u;
}

// Store channels 4 q4 .. 4 q4 + 3 of atom row `row` into operand tile x.
__device__ __forceinline__ void st_x4(__nv_bfloat16 (*x)[NT * 64], int row, int q4, float4 v) {
    st_bf16x4(x, row, q4, __floats2bfloat162_rn(v.x, v.y), __floats2bfloat162_rn(v.z, v.w));
}

// Split v = p0 + p1 + p2 (+ a remainder below 2^-24 |v|) into three BF16 parts,
// each the rounding of what the previous parts leave (differences are exact
// in FP32), and store them in three operand tiles.  A product with BF16
// weights accumulated in FP32 over the three parts is then linear in v to
// FP32 rounding.
__device__ __forceinline__ void st_x4_split3(__nv_bfloat16 (*x0)[NT * 64],
                                             __nv_bfloat16 (*x1)[NT * 64],
                                             __nv_bfloat16 (*x2)[NT * 64], int row, int q4,
                                             float4 v) {
    float r[4] = {v.x, v.y, v.z, v.w};
    __nv_bfloat162 p[3][2];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            p[k][h] = __floats2bfloat162_rn(r[2 * h], r[2 * h + 1]);
            r[2 * h] -= __low2float(p[k][h]);
            r[2 * h + 1] -= __high2float(p[k][h]);
        }
    }
    st_bf16x4(x0, row, q4, p[0][0], p[0][1]);
    st_bf16x4(x1, row, q4, p[1][0], p[1][1]);
    st_bf16x4(x2, row, q4, p[2][0], p[2][1]);
}

// D[128 x 16] (+)= W[g] (128 x 128) . X[x]^T (16 x 128), two K-blocks of 4 steps.
template <class S>
__device__ __forceinline__ void mma_k128(uint32_t d, S& s, int g, int x, bool accumulate) {
    constexpr uint32_t idesc = tc::idesc_bf16(128, NT);
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
        const uint64_t ad = tc::desc_sw128(tc::smem_u32(s.W[g][kb]));
        const uint64_t bd = tc::desc_sw128(tc::smem_u32(s.X[x][kb]));
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc,
                         (accumulate || kb > 0 || kk > 0) ? 1u : 0u);
    }
}

// Copy the weight images (all NW matrices, contiguous from img) to shared
// memory, set up the mbarrier and allocate the tensor memory.
template <class S, int NW>
__device__ __forceinline__ void node_setup(S& s, const __nv_bfloat16* img, int tid) {
    const uint4* src = reinterpret_cast<const uint4*>(img);
    uint4* dst = reinterpret_cast<uint4*>(&s.W[0][0][0]);
    for (int q = tid; q < NW * 2 * 128 * 64 * 2 / 16; q += NTHR) dst[q] = __ldg(&src[q]);
    if (tid == 0) {
        tc::mbar_init(&s.mbar, 1);
        s.abort = 0;
    }
    if ((tid >> 5) == 0) tc::tmem_alloc<2 * BUF_COLS>(&s.taddr);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

template <class S>
__device__ __forceinline__ void node_teardown(S& s, uint32_t phase, int* err, int tid) {
    if (s.abort) {
        tc::mbar_wait(&s.mbar, phase, 20000000LL);
        if (tid == 0) atomicOr(err, kErrTimeout);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if ((tid >> 5) == 0) tc::tmem_dealloc<2 * BUF_COLS>(s.taddr);
}

// All threads wait for the MMAs of the previous commit (bounded); uniform result.
template <class S>
__device__ __forceinline__ bool node_wait(S& s, uint32_t& phase) {
    if (tc::mbar_wait(&s.mbar, phase))
        phase ^= 1u;
    else
        s.abort = 1;
    __syncthreads();
    tc::fence_after_sync();
    return s.abort == 0;
}

// ------------------------------------------------------------------ forward --

template <bool LAST>
__global__ void __launch_bounds__(NTHR, 1) k_node_fwd_tc(NodeArgs a, LayerW wl, int64_t n_tiles) {
    extern __shared__ unsigned char smem_raw[];
    NodeSmemF& s = node_smem<NodeSmemF>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ia = tid >> 5, q4 = tid & 31;                 // load phase: atom, channel quad
    const int lq = warp & 3, ag = warp >> 2;                // epilogue: lane quarter, atom group
    const int c = 32 * lq + lane;
    node_setup<NodeSmemF, 5>(s, wl.NswF, tid);
    const float bc = wl.b[c];
    uint32_t phase = 0;

    float4 av[NLM9];
    auto load = [&](int64_t tile) {
        const int64_t i = tile * NT + ia;
        const bool ok = tile < n_tiles && i < a.n;
        const float4* src = reinterpret_cast<const float4*>(a.A + i * NLM9 * NF) + q4;
#pragma unroll
        for (int q = 0; q < NLM9; ++q) av[q] = ok ? __ldg(src + q * (NF / 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto epilogue = [&](int64_t tile, int buf) {
        const uint32_t tcol = s.taddr + ((uint32_t)(32 * lq) << 16) + buf * BUF_COLS + 4 * ag;
        const int64_t i0 = tile * NT + 4 * ag;
        float hin[LAST ? 1 : NLM9][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const bool ok = i0 + r < a.n;
#pragma unroll
            for (int q = 0; q < (LAST ? 1 : NLM9); ++q)
                hin[q][r] = (ok && (q == 0 || !a.first)) ? __ldg(a.Hin + ((i0 + r) * NLM9 + q) * NF + c) : 0.f;
        }
        float d[4];
        tc::tmem_ld4(tcol, d);
        tc::tmem_wait_ld();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (i0 + r >= a.n) break;
            const float sv = d[r] + bc;
            a.S[(i0 + r) * NF + c] = sv;
            a.Hout[((i0 + r) * NLM9) * NF + c] = hin[0][r] + silu(sv);
        }
        if (!LAST) {
#pragma unroll
            for (int lm = 1; lm < NLM9; ++lm) {
                tc::tmem_ld4(tcol + 16 * lm, d);
                tc::tmem_wait_ld();
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    if (i0 + r >= a.n) break;
                    a.Hout[((i0 + r) * NLM9 + lm) * NF + c] = hin[LAST ? 0 : lm][r] + d[r];
                }
            }
        }
        tc::fence_before_sync();
    };

    int64_t tile = blockIdx.x, prev = -1;
    int it = 0;
    load(tile);
    for (; tile < n_tiles; tile += gridDim.x, ++it) {
        if (it > 0 && !node_wait(s, phase)) break;   // previous MMAs done: X is free
        {   // operand tiles of this tile
            float4 b1 = make_float4(0.f, 0.f, 0.f, 0.f), b2 = b1;
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                b1.x = fmaf(av[q].x, av[q].x, b1.x); b1.y = fmaf(av[q].y, av[q].y, b1.y);
                b1.z = fmaf(av[q].z, av[q].z, b1.z); b1.w = fmaf(av[q].w, av[q].w, b1.w);
            }
#pragma unroll
            for (int q = 4; q < 9; ++q) {
                b2.x = fmaf(av[q].x, av[q].x, b2.x); b2.y = fmaf(av[q].y, av[q].y, b2.y);
                b2.z = fmaf(av[q].z, av[q].z, b2.z); b2.w = fmaf(av[q].w, av[q].w, b2.w);
            }
            st_x4(s.X[0], ia, q4, av[0]);
            st_x4(s.X[1], ia, q4, b1);
            st_x4(s.X[2], ia, q4, b2);
            if (!LAST) {
#pragma unroll
                for (int q = 1; q < NLM9; ++q) st_x4(s.X[2 + q], ia, q4, av[q]);
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t d0 = s.taddr + (it & 1) * BUF_COLS;
            mma_k128(d0, s, 0, 0, false);
            mma_k128(d0, s, 1, 1, true);
            mma_k128(d0, s, 2, 2, true);
            if (!LAST) {
#pragma unroll 1
                for (int lm = 1; lm < NLM9; ++lm) mma_k128(d0 + 16 * lm, s, lm < 4 ? 3 : 4, 2 + lm, false);
            }
            tc::mma_commit(&s.mbar);
        }
        load(tile + gridDim.x);                       // prefetch the next tile
        if (prev >= 0) epilogue(prev, (it - 1) & 1);
        prev = tile;
    }
    if (prev >= 0 && !s.abort && node_wait(s, phase)) epilogue(prev, (it - 1) & 1);
    node_teardown(s, phase, a.err, tid);
}

// ------------------------------------------------------------------ adjoint --
// Part 1: gS = G0' silu'(S) against W0^T, U1^T, U2^T (columns 0, 16, 32):
// alpha_0 = W0^T gS / N_avg and alpha_lm = 2 A_lm (U_l^T gS) / N_avg; part 2
// adds V_l^T G'_lm / N_avg (not at the last layer, whose G'_lm are zero).

__global__ void __launch_bounds__(NTHR, 1) k_node_bwd_a_tc(NodeArgs a, LayerW wl, int64_t n_tiles) {
    extern __shared__ unsigned char smem_raw[];
    NodeSmemA& s = node_smem<NodeSmemA>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ia = tid >> 5, q4 = tid & 31;
    const int lq = warp & 3, ag = warp >> 2;
    const int c = 32 * lq + lane;
    node_setup<NodeSmemA, 3>(s, wl.NswB, tid);
    const float inv = a.inv_navg;
    uint32_t phase = 0;

    float4 gv, sv;
    auto load = [&](int64_t tile) {
        const int64_t i = tile * NT + ia;
        const bool ok = tile < n_tiles && i < a.n;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        gv = ok ? __ldg(reinterpret_cast<const float4*>(a.Gout + i * NLM9 * NF) + q4) : z;
        sv = ok ? __ldg(reinterpret_cast<const float4*>(a.S + i * NF) + q4) : z;
    };
    auto epilogue = [&](int64_t tile, int buf) {
        const uint32_t tcol = s.taddr + ((uint32_t)(32 * lq) << 16) + buf * BUF_COLS + 4 * ag;
        const int64_t i0 = tile * NT + 4 * ag;
        float am[NLM9 - 1][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const bool ok = i0 + r < a.n;
#pragma unroll
            for (int q = 1; q < NLM9; ++q)
                am[q - 1][r] = ok ? __ldg(a.A + ((i0 + r) * NLM9 + q) * NF + c) : 0.f;
        }
        float d0[4], db1[4], db2[4];
        tc::tmem_ld4(tcol, d0);
        tc::tmem_ld4(tcol + 16, db1);
        tc::tmem_ld4(tcol + 32, db2);
        tc::tmem_wait_ld();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (i0 + r >= a.n) break;
            float* al = a.Alpha + ((i0 + r) * NLM9) * NF + c;
            al[0] = d0[r] * inv;
#pragma unroll
            for (int q = 1; q < NLM9; ++q)
                al[q * NF] = 2.f * am[q - 1][r] * (q < 4 ? db1[r] : db2[r]) * inv;
        }
        tc::fence_before_sync();
    };

    int64_t tile = blockIdx.x, prev = -1;
    int it = 0;
    load(tile);
    for (; tile < n_tiles; tile += gridDim.x, ++it) {
        if (it > 0 && !node_wait(s, phase)) break;
        {
            float4 g;
            g.x = gv.x * silu_grad(sv.x);
            g.y = gv.y * silu_grad(sv.y);
            g.z = gv.z * silu_grad(sv.z);
            g.w = gv.w * silu_grad(sv.w);
            st_x4_split3(s.X[0], s.X[1], s.X[2], ia, q4, g);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t d0 = s.taddr + (it & 1) * BUF_COLS;
#pragma unroll
            for (int gm = 0; gm < 3; ++gm)
#pragma unroll
                for (int part = 0; part < 3; ++part) mma_k128(d0 + 16 * gm, s, gm, part, part > 0);
            tc::mma_commit(&s.mbar);
        }
        load(tile + gridDim.x);
        if (prev >= 0) epilogue(prev, (it - 1) & 1);
        prev = tile;
    }
    if (prev >= 0 && !s.abort && node_wait(s, phase)) epilogue(prev, (it - 1) & 1);
    node_teardown(s, phase, a.err, tid);
}

__global__ void __launch_bounds__(NTHR, 1) k_node_bwd_v_tc(NodeArgs a, LayerW wl, int64_t n_tiles) {
    extern __shared__ unsigned char smem_raw[];
    NodeSmemV& s = node_smem<NodeSmemV>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ia = tid >> 5, q4 = tid & 31;
    const int lq = warp & 3, ag = warp >> 2;
    const int c = 32 * lq + lane;
    node_setup<NodeSmemV, 2>(s, wl.NswB + (size_t)3 * 2 * 128 * 64, tid);   // V1^T, V2^T
    const float inv = a.inv_navg;
    uint32_t phase = 0;

    float4 gv[NLM9 - 1];
    auto load = [&](int64_t tile) {
        const int64_t i = tile * NT + ia;
        const bool ok = tile < n_tiles && i < a.n;
        const float4* src = reinterpret_cast<const float4*>(a.Gout + i * NLM9 * NF) + q4;
#pragma unroll
        for (int q = 1; q < NLM9; ++q)
            gv[q - 1] = ok ? __ldg(src + q * (NF / 4)) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    // columns: V_l^T G'_lm of component lm at 16 (lm - 1)
    auto epilogue = [&](int64_t tile, int buf) {
        const uint32_t tcol = s.taddr + ((uint32_t)(32 * lq) << 16) + buf * BUF_COLS + 4 * ag;
        const int64_t i0 = tile * NT + 4 * ag;
        float al[NLM9 - 1][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const bool ok = i0 + r < a.n;
#pragma unroll
            for (int q = 1; q < NLM9; ++q)
                al[q - 1][r] = ok ? a.Alpha[((i0 + r) * NLM9 + q) * NF + c] : 0.f;
        }
#pragma unroll
        for (int q = 1; q < NLM9; ++q) {
            float d[4];
            tc::tmem_ld4(tcol + 16 * (q - 1), d);
            tc::tmem_wait_ld();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (i0 + r >= a.n) break;
                a.Alpha[((i0 + r) * NLM9 + q) * NF + c] = fmaf(d[r], inv, al[q - 1][r]);
            }
        }
        tc::fence_before_sync();
    };

    int64_t tile = blockIdx.x, prev = -1;
    int it = 0;
    load(tile);
    for (; tile < n_tiles; tile += gridDim.x, ++it) {
        if (it > 0 && !node_wait(s, phase)) break;
#pragma unroll
        for (int q = 1; q < NLM9; ++q)
            st_x4_split3(s.X[3 * (q - 1)], s.X[3 * (q - 1) + 1], s.X[3 * (q - 1) + 2], ia, q4,
                         gv[q - 1]);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t d0 = s.taddr + (it & 1) * BUF_COLS;
#pragma unroll 1
            for (int q = 1; q < NLM9; ++q)
#pragma unroll
                for (int part = 0; part < 3; ++part)
                    mma_k128(d0 + 16 * (q - 1), s, q < 4 ? 0 : 1, 3 * (q - 1) + part, part > 0);
            tc::mma_commit(&s.mbar);
        }
        load(tile + gridDim.x);
        if (prev >= 0) epilogue(prev, (it - 1) & 1);
        prev = tile;
    }
    if (prev >= 0 && !s.abort && node_wait(s, phase)) epilogue(prev, (it - 1) & 1);
    node_teardown(s, phase, a.err, tid);
}

template <class S, class K>
int launch_node_tc(K kernel, const NodeArgs& a, int num_sms, cudaStream_t st) {
    const int64_t tiles = (a.n + NT - 1) / NT;
    const size_t smem = sizeof(S) + 1024;
    MP_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t grid = num_sms;   // one CTA (160 KB of weights, 512 TMEM columns) per SM
    if (grid > tiles) grid = tiles;
    kernel<<<(unsigned)grid, NTHR, smem, st>>>(a, *a.w, tiles);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

int launch_node_bwd_bf16(const Model& m, const NodeArgs& a, cudaStream_t st, int num_sms) {
    if (!(m.d.F == NF && m.d.lmax == 2) || !a.w->NswB || !a.err) return MP_ERR_UNSUPPORTED;
    if (a.n == 0) return MP_OK;
    MP_TRY(launch_node_tc<NodeSmemA>(k_node_bwd_a_tc, a, num_sms, st));
    if (!a.last) MP_TRY(launch_node_tc<NodeSmemV>(k_node_bwd_v_tc, a, num_sms, st));
    return MP_OK;
}

int launch_node_fwd_bf16(const Model& m, const NodeArgs& a, cudaStream_t st, int num_sms) {
    if (!(m.d.F == NF && m.d.lmax == 2) || !a.w->NswF || !a.err) return MP_ERR_UNSUPPORTED;
    if (a.n == 0) return MP_OK;
    return a.last ? launch_node_tc<NodeSmemF>(k_node_fwd_tc<true>, a, num_sms, st)
                  : launch_node_tc<NodeSmemF>(k_node_fwd_tc<false>, a, num_sms, st);
}

}  // namespace mp

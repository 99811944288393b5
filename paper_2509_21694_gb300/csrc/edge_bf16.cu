// Edge kernels with the radial MLP's three contractions on tcgen05 tensor
// cores (BF16 operands, FP32 accumulation in tensor memory).  Geometry, the
// radial basis, messages, adjoint sums and forces stay FP32 on CUDA cores.
// Shapes compiled: F = 128, lmax = 2, H = 64.
//
// A CTA holds one copy of the W1 / W2 / W3 operand tiles and runs
// independent warpgroups (six or five in the forward, four in the
// later-layer adjoint, whose per-thread state needs more registers); each
// warpgroup owns a stream of receiver-row groups, its tensor-memory columns
// (80 / 96 forward, 128 adjoint), an mbarrier and a named barrier, so one
// warpgroup's MMAs overlap the others' CUDA-core work.  The geometry (unit
// vector and r of every edge) is formed once per sub-system by
// k_edge_geometry and read here.
//
// Per super-chunk of edges of the warpgroup's rows (128 edges forward; 64
// edges plus their r-tangents in the adjoint):
//   1. thread = edge: geometry, eps (and d eps/dr), spherical harmonics;
//      the basis rows (adjoint: eps and d eps/dr of each edge in adjacent
//      rows) -> BF16 K-major tile B as two-term splits (K = 32, see
//      st_basis_row; the first layer to about 16 significant bits).
//   2. MMA0: D0[128 x 64] = B . W1^T (two K = 16 instructions); thread =
//      tile row reads its row: a1 = silu(z1) (tangent rows: silu'(z1) dz1,
//      with z1 taken from the value row's lane) -> tile B (128 x 64).
//   3. MMA1: D1[128 x 64] = B . W2^T; a2 = silu(z2) (tangent rows:
//      silu'(z2) dz2) -> the same tile B, rewritten in place.
//   4. per 16-row slice of B: MMA2 D2_q[128 x 16] = W3_q . slice^T for each
//      radial path q (lane = channel, column = edge: R, and dR/dr in the
//      adjoint, where rows / columns alternate edge and tangent).  D0, D1
//      and D2 share the warpgroup's tensor-memory columns.
//   5. thread = channel runs the message (forward) or symmetric-pair adjoint
//      (backward) epilogue on the slice.  In the adjoint each channel forms
//      its own share of dE_pair/dd and accumulates it over the receiver row
//      (FP32 over a slice, compensated across slices); channels are summed
//      once per row as FP32 two-sum pairs across a warp's lanes, then the
//      four warps' pairs in FP64,
//      F_k = sum_e sum_c g_c(e).
// The adjoint of a layer first compacts each row group's edges, in order,
// without those between two atoms of the layer's outermost hop class (their
// terms are exact zeros).  The epilogues gather sender features ahead of
// the edge being computed: the adjoint the next edge's, the later-layer
// forward three edges ahead (a ring of four edges' features), the layer-0
// forward, which gathers one value per edge, a whole slice's at once.  They
// read the radial outputs from tensor memory four (layer-0 forward), two
// (later-layer forward) or one (adjoint) edges at a time.
// The MLP's hidden activations use the hardware tanh for the sigmoid: they
// are rounded to BF16 for the next contraction anyway.
// Layer 0 runs by hidden unit instead (k_v_first and k_edge_bwd0_tc for the
// adjoint, k_edge_fwd0_tc and k_a_first_tc for the forward, below): there
// the senders' features are species embeddings, so its channel sums factor
// through the last radial layer.  The channel-wise forward above still
// serves layer 0 for more than three species; the channel-wise adjoint
// serves the later layers only.
// One thread issues the MMAs; completion is signalled through an mbarrier
// whose waits are bounded (clock64): on a timeout the warpgroup sets an
// error bit, stops, and the CTA frees its tensor memory and returns.
#include <type_traits>

#include "kernels.h"
#include "tc.cuh"

namespace mp {

namespace {

constexpr int TF = 128, TLMAX = 2, TNLM = 9;
// Forward: its per-thread state is smaller, so more warpgroups hide more of
// the gathers' latency: six for layer 0 (one gathered value per edge), five
// for the later layers (96 registers, which also hold a ring of the next
// three edges' sender features); D1 (64 columns) and a slice's D2 (3 or 5
// paths x 16 columns) share 80 or 96 columns per warpgroup.
template <bool FIRST>
struct FwdCfg {
    static constexpr int NWG = FIRST ? 6 : 5;
    static constexpr int NTH = 128 * NWG;
    static constexpr int COLS = FIRST ? 80 : 96;
    static constexpr int PD = FIRST ? 0 : 3;   // later layers: sender prefetch distance
    static constexpr int RB = FIRST ? 4 : 2;   // edges per tensor-memory load of R
};
constexpr int TM_COLS = 512;       // allocated per CTA
// Receiver rows per row group.  All warpgroups of the GPU work on
// consecutive groups, so the group size sets the span of rows in flight and
// with it the sender features that must stay in L2 (measured on 1M atoms:
// 4 rows for the adjoint and 8 for the forward beat 16 by 13 % and 4 %).
constexpr int RPG_F = 8;           // forward
constexpr int RPG_B = 4;           // adjoint
constexpr int RPG = RPG_F > RPG_B ? RPG_F : RPG_B;   // row-group storage
constexpr int SCF = 128;           // forward super-chunk: 128 edges, slices of 16
constexpr int SCB = 64;            // adjoint super-chunk: 64 edges + 64 tangents, slices of 8 + 8
constexpr int KWIN = 512;          // adjoint: raw edges compacted at a time (4 per thread)
constexpr int kErrTimeout = 2;

template <bool FIRST>
struct TPaths {
    static constexpr int NP = FIRST ? 3 : 5;
    __host__ __device__ static constexpr int sla(int l) { return FIRST ? l : 2 * l - 1; }
    __host__ __device__ static constexpr int slb(int l) { return 2 * l; }
};

// Weight tiles of one layer: NP radial paths (3 at layer 0, whose l >= 1
// inputs are zero, else 5).
template <int NP>
struct alignas(1024) Tiles {
    static constexpr int NPATH = NP;
    __nv_bfloat16 W3[NP][128 * 64];  // NP x 16 KB, one 128-row tile per radial path
    __nv_bfloat16 W2[64 * 64];       // W2 (out, in), K-major
    __nv_bfloat16 W1[64 * 64];       // [W1_hi | W1_hi | W1_lo | 0] (out, K), K-major
};

// Sigmoid from the hardware tanh (PTX tanh.approx.f32, relative error about
// 2^-11): its absolute error, at most about 2.4e-4, stays below the BF16
// rounding (2^-9 relative) that the MLP activations get next.
__device__ __forceinline__ float sigmoid_fast(float z) {
    float t;   // sigmoid(z) = (1 + tanh(z / 2)) / 2 with the hardware tanh
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
    return fmaf(0.5f, t, 0.5f);
}

// The adjoint's warpgroup state; the virial partials exist with STRESS, the
// per-thread compensated force sums with FKS.
template <bool STRESS, bool FKS>
struct alignas(1024) WgState {
    __nv_bfloat16 B[128 * 64];       // basis rows, then the a1 and a2 tiles, of the super-chunk
    float Y[SCB][TNLM - 1];          // Y_lm for lm = 1..8 (Y_00 = 1)
    float u[SCB][4];                 // unit vector, r
    int row[SCB], col[SCB];
    int klist[KWIN];                 // adjoint: kept edges of a window (offsets from its start)
    int kwarp[4];
    float2 fpart[RPG_B][4][3];       // per-row, per-warp force partial sums (hi, lo)
    float2 vpart[RPG_B][4][STRESS ? 9 : 1];   // per-row, per-warp virial partial sums
    float fkc[FKS ? 6 : 1][128];     // per thread: compensated row force sums (fk, fc)
    int64_t rp[RPG_B + 1];
    int64_t next_grp;                // next row group, fetched by the leader
    uint64_t mbar;
    int abort;
};


// The forward's warpgroup state: the adjoint's fields it does not use are
// left out so that five warpgroups fit.
struct alignas(1024) WgStateF {
    __nv_bfloat16 B[128 * 64];       // a1 tile, then a2 tile, of the super-chunk
    float Y[SCF][TNLM - 1];          // Y_lm for lm = 1..8 (Y_00 = 1)
    int row[SCF], col[SCF];
    int64_t rp[RPG + 1];
    int64_t next_grp;
    uint64_t mbar;
    int abort;
};

// Adjoint of the later layers (channel-wise): four warpgroups at up to 128
// registers, 128 tensor-memory columns each.
template <bool STRESS>
struct BwdCfg {
    static constexpr int NWG = 4;
    static constexpr int NTH = 128 * NWG;
    static constexpr int COLS = 128;
};

template <int NP, class WG, int N>
struct SmemT {
    Tiles<NP> t;
    WG wg[N];
    uint32_t taddr;
};
template <bool STRESS>
using SmemB = SmemT<5, WgState<STRESS, false>, BwdCfg<STRESS>::NWG>;   // adjoint, later layers
template <bool FIRST>
using SmemF = SmemT<FIRST ? 3 : 5, WgStateF, FwdCfg<FIRST>::NWG>;          // forward
template <class S>
constexpr bool smem_fits() { return sizeof(S) + 1024 <= 232448; }
static_assert(smem_fits<SmemB<false>>() && smem_fits<SmemB<true>>(),
              "shared memory of the edge adjoint");
static_assert(smem_fits<SmemF<true>>() && smem_fits<SmemF<false>>(),
              "shared memory of the edge forward");
static_assert(BwdCfg<false>::NWG * BwdCfg<false>::COLS <= TM_COLS &&
              FwdCfg<true>::NWG * FwdCfg<true>::COLS <= TM_COLS &&
              FwdCfg<false>::NWG * FwdCfg<false>::COLS <= TM_COLS, "tensor memory");

// The dynamic shared memory rounded up to a 1024-byte boundary (the swizzled
// tiles need it).  The padding is added to the __shared__ pointer itself, not
// through an integer round trip, so the compiler still knows every access
// below is to shared memory and emits shared-space loads and stores.
template <class S>
__device__ __forceinline__ S& smem_as(unsigned char* raw) {
    const uint32_t pad = (1024u - (tc::smem_u32(raw) & 1023u)) & 1023u;
    return *reinterpret_cast<S*>(raw + pad);
}

__device__ __forceinline__ void wg_sync(int g) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "n"(128) : "memory");
}

// Row groups are handed out dynamically: each warpgroup starts at its own
// index and then takes the next unclaimed group from a global counter, so
// warpgroups that drew light groups keep working until the list is done.
template <int N, class W>
__device__ __forceinline__ int64_t next_group(W& w, const EdgeArgs& a, int g, int lt) {
    if (lt == 0) w.next_grp = (int64_t)gridDim.x * N + atomicAdd(a.sched, 1);
    wg_sync(g);
    return w.next_grp;
}

__device__ __forceinline__ int find_row_t(const int64_t* rp, int nrows, int64_t e) {
    int lo = 0, hi = nrows - 1;       // last row with rp[row] <= e
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rp[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Store 8 consecutive BF16 values (k = 8 j .. 8 j + 7) of tile row `row`.
__device__ __forceinline__ void st_row_chunk(__nv_bfloat16* tile, int row, int j, const float v[8]) {
    __nv_bfloat162 p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) p[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(tile) + row * 128 +
                              (((j ^ (row & 7)) & 7) << 4)) = *reinterpret_cast<uint4*>(p);
}

// D[tmem, 128 x N] = A(128 x 64 tile) . B(N x 64 tile)^T, four K = 16 steps.
template <int N>
__device__ __forceinline__ void mma_k64(uint32_t d, const __nv_bfloat16* A, const __nv_bfloat16* B) {
    const uint64_t ad = tc::desc_sw128(tc::smem_u32(A));
    const uint64_t bd = tc::desc_sw128(tc::smem_u32(B));
    constexpr uint32_t idesc = tc::idesc_bf16(128, N);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc, kk > 0 ? 1u : 0u);
}

// D[tmem, 128 x 64] = A(128 x 32, the first four K chunks of a tile) .
// W1(64 x 32)^T: the first radial layer, K = 8 in two-term BF16 splits
// (two K = 16 instructions).
__device__ __forceinline__ void mma_k32(uint32_t d, const __nv_bfloat16* A, const __nv_bfloat16* B) {
    const uint64_t ad = tc::desc_sw128(tc::smem_u32(A));
    const uint64_t bd = tc::desc_sw128(tc::smem_u32(B));
    constexpr uint32_t idesc = tc::idesc_bf16(128, 64);
    tc::mma_bf16(d, ad, bd, idesc, 0u);
    tc::mma_bf16(d, ad + 2, bd + 2, idesc, 1u);
}

// A radial basis row of the first layer's A operand: K chunks
// [eps_hi | eps_lo | eps_hi | 0] of tile row `row` (eps = eps_hi + eps_lo,
// eps_hi its BF16 rounding).
__device__ __forceinline__ void st_basis_row(__nv_bfloat16* tile, int row, const float eps[kNB]) {
    float hi[kNB], lo[kNB];
#pragma unroll
    for (int q = 0; q < kNB; ++q) {
        hi[q] = __bfloat162float(__float2bfloat16_rn(eps[q]));
        lo[q] = eps[q] - hi[q];
    }
    st_row_chunk(tile, row, 0, hi);
    st_row_chunk(tile, row, 1, lo);
    st_row_chunk(tile, row, 2, hi);
    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(tile) + row * 128 +
                              (((3 ^ (row & 7)) & 7) << 4)) = make_uint4(0u, 0u, 0u, 0u);
}

// Bounded wait of one warpgroup on its mbarrier; uniform result.
template <class W>
__device__ __forceinline__ bool wg_wait(W& w, uint32_t& phase, int g) {
    const bool ok = tc::mbar_wait(&w.mbar, phase);
    if (ok)
        phase ^= 1u;
    else
        w.abort = 1;
    wg_sync(g);
    tc::fence_after_sync();
    return w.abort == 0;
}

template <int NT, class S>
__device__ __forceinline__ void tc_setup(S& s, const LayerW& wl, int np, bool first, int tid) {
    const uint4* src2 = reinterpret_cast<const uint4*>(wl.W2sw);
    uint4* dst2 = reinterpret_cast<uint4*>(s.t.W2);
    for (int q = tid; q < 64 * 64 * 2 / 16; q += NT) dst2[q] = __ldg(&src2[q]);
    if constexpr (decltype(s.t)::NPATH > 0) {
        for (int p = 0; p < np; ++p) {
            const int blk = first ? (p == 0 ? 0 : 2 * p - 1) : p;
            const uint4* src = reinterpret_cast<const uint4*>(wl.W3sw + (size_t)blk * 128 * 64);
            uint4* dst = reinterpret_cast<uint4*>(s.t.W3[p]);
            for (int q = tid; q < 128 * 64 * 2 / 16; q += NT) dst[q] = __ldg(&src[q]);
        }
    }
    // W1 (64 x 8, FP32) as a BF16 K-major 128-byte-swizzled tile of two-term
    // splits W1 = W1_hi + W1_lo: K chunks [W1_hi | W1_hi | W1_lo | 0], against
    // basis rows [eps_hi | eps_lo | eps_hi | 0] (the first radial layer's MMA
    // reads K = 0..31), so that the product is W1_hi eps_hi + W1_hi eps_lo +
    // W1_lo eps_hi: the first layer to about 16 significant bits
    for (int q = tid; q < 64 * 64; q += NT) {
        const int h = q >> 6, k = q & 63, part = k >> 3;
        float v = 0.f;
        if (part < 3) {
            const float w1 = __ldg(&wl.W1[h * kNB + (k & 7)]);
            const float hi = __bfloat162float(__float2bfloat16_rn(w1));
            v = part < 2 ? hi : w1 - hi;
        }
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(s.t.W1) + h * 128 +
                                          (((part ^ (h & 7)) & 7) << 4) + (k & 7) * 2) =
            __float2bfloat16_rn(v);
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

template <class S>
__device__ __forceinline__ void tc_teardown(S& s, uint32_t phase, int* err, int tid) {
    auto& w = s.wg[tid >> 7];
    if (w.abort) {
        // drain: give in-flight MMAs of this warpgroup a bounded chance to land
        tc::mbar_wait(&w.mbar, phase, 20000000LL);
        if ((tid & 127) == 0) atomicOr(err, kErrTimeout);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if ((tid >> 5) == 0) tc::tmem_dealloc<TM_COLS>(s.taddr);
}

// Geometry of edge e: eps (and d eps/dr), Y_lm (lm >= 1), unit vector, 1 / r.
template <bool DERIV>
__device__ __forceinline__ int edge_geometry(const EdgeArgs& a, const int64_t* rp, int64_t e,
                                             int64_t e_end, int64_t r0, int nrows, float eps[kNB],
                                             float deps[kNB], float Y[TNLM], float u4[4], int& col) {
    if (e >= e_end) {
#pragma unroll
        for (int q = 0; q < kNB; ++q) eps[q] = deps[q] = 0.f;
#pragma unroll
        for (int q = 0; q < TNLM; ++q) Y[q] = 0.f;
        u4[0] = u4[1] = u4[2] = 0.f;
        u4[3] = 1.f;   // 1 / r
        col = 0;
        return -1;
    }
    const int lr = find_row_t(rp, nrows, e);
    col = a.col[e];
    const float4 q = a.geo[e];   // (u, r), formed once per evaluation
    const float r = q.w;
    const float ir = 1.f / r;
    u4[0] = q.x;
    u4[1] = q.y;
    u4[2] = q.z;
    u4[3] = ir;
    float env, denv;
    radial_basis<DERIV>(r, a.k, eps, deps, env, denv);
    sph_harm<TLMAX>(u4, Y);
    return lr;
}

// ------------------------------------------------------------------ forward --

template <bool FIRST>
__global__ void __launch_bounds__(FwdCfg<FIRST>::NTH, 1)
    k_edge_fwd_tc(EdgeArgs a, LayerW wl, int64_t n_groups, int* err) {
    using PP = TPaths<FIRST>;
    using Cfg = FwdCfg<FIRST>;
    extern __shared__ unsigned char smem_raw[];
    SmemF<FIRST>& s = smem_as<SmemF<FIRST>>(smem_raw);
    const int tid = threadIdx.x, g = tid >> 7, lt = tid & 127, warp = tid >> 5;
    const int c = lt;
    WgStateF& w = s.wg[g];
    const float* __restrict__ Hin = a.Hin;
    float* __restrict__ Aout = a.Aout;
    tc_setup<Cfg::NTH>(s, wl, PP::NP, FIRST, tid);
    const uint32_t tb = s.taddr + Cfg::COLS * g;
    const uint32_t tl = tb + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t phase = 0;
    bool alive = true;

    for (int64_t grp = (int64_t)blockIdx.x * Cfg::NWG + g; grp < n_groups && alive;
         grp = next_group<Cfg::NWG>(w, a, g, lt)) {
        const int64_t r0 = grp * RPG_F;
        const int nrows = (int)min((int64_t)RPG_F, a.n - r0);
        if (lt <= nrows) w.rp[lt] = a.row_ptr[r0 + lt];
        wg_sync(g);
        const int64_t e_beg = w.rp[0], e_end = w.rp[nrows];
        float acc[TNLM];
#pragma unroll
        for (int q = 0; q < TNLM; ++q) acc[q] = 0.f;
        int cur = -1, next = 0;
        auto write_row = [&](int lr, bool zero) {
            float* __restrict__ o = Aout + ((r0 + lr) * TNLM) * TF + c;
#pragma unroll
            for (int q = 0; q < TNLM; ++q) o[q * TF] = zero ? 0.f : acc[q] * a.k.inv_navg;
        };
        for (int64_t sc = e_beg; sc < e_end && alive; sc += SCF) {
            {   // geometry of edge lt; its radial basis -> tile row lt
                float eps[kNB], deps[kNB], Y[TNLM], u4[4];
                int col;
                const int lr = edge_geometry<false>(a, w.rp, sc + lt, e_end, r0, nrows, eps, deps,
                                                    Y, u4, col);
                w.row[lt] = lr;
                w.col[lt] = col;
#pragma unroll
                for (int q = 1; q < TNLM; ++q) w.Y[lt][q - 1] = Y[q];
                st_basis_row(w.B, lt, eps);
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            wg_sync(g);
            if (lt == 0) {   // MMA0: z1 = eps . W1^T
                tc::fence_after_sync();
                mma_k32(tb, w.B, s.t.W1);
                tc::mma_commit(&w.mbar);
            }
            if (!wg_wait(w, phase, g)) { alive = false; break; }
#pragma unroll
            for (int h = 0; h < 4; ++h) {   // a1 = silu(z1): lane lt holds tile row lt
                float z[16];
                tc::tmem_ld16(tl + 16 * h, z);
                tc::tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) z[q] = z[q] * sigmoid_fast(z[q]);
                st_row_chunk(w.B, lt, 2 * h, z);
                st_row_chunk(w.B, lt, 2 * h + 1, z + 8);
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            wg_sync(g);
            if (lt == 0) {
                tc::fence_after_sync();
                mma_k64<64>(tb, w.B, s.t.W2);
                tc::mma_commit(&w.mbar);
            }
            if (!wg_wait(w, phase, g)) { alive = false; break; }
#pragma unroll
            for (int h = 0; h < 4; ++h) {   // a2 = silu(z2): lane lt holds tile row lt
                float z[16];
                tc::tmem_ld16(tl + 16 * h, z);
                tc::tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) z[q] = z[q] * sigmoid_fast(z[q]);
                st_row_chunk(w.B, lt, 2 * h, z);
                st_row_chunk(w.B, lt, 2 * h + 1, z + 8);
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            wg_sync(g);
            if (lt == 0) {
                tc::fence_after_sync();
#pragma unroll
                for (int q = 0; q < PP::NP; ++q) mma_k64<16>(tb + 16 * q, s.t.W3[q], w.B);
                tc::mma_commit(&w.mbar);
            }
            for (int sl = 0; sl < SCF / 16; ++sl) {
                // prefetch the first edges' sender features before waiting for
                // the slice's MMA (col is 0, a valid row, for slots past the end)
                // later layers: a ring of PD + 1 edges' features, edge i + PD
                // requested while edge i computes (the ring index is static: the
                // slice loop is unrolled)
                float hr[FIRST ? 1 : Cfg::PD + 1][TNLM];
                // layer 0 gathers one value per edge (h0 of the sender): all 16 of
                // the slice are requested at once, so their latency overlaps
                float hb[FIRST ? 16 : 1];
                if (FIRST) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        hb[i] = __ldg(Hin + ((int64_t)w.col[sl * 16 + i] * TNLM) * TF + c);
                } else {
#pragma unroll
                    for (int d = 0; d < Cfg::PD; ++d) {
                        const float* __restrict__ hp =
                            Hin + ((int64_t)w.col[sl * 16 + d] * TNLM) * TF + c;
#pragma unroll
                        for (int q = 0; q < TNLM; ++q) hr[d][q] = __ldg(hp + q * TF);
                    }
                }
                if (!wg_wait(w, phase, g)) { alive = false; break; }
                constexpr int RB = Cfg::RB;
                float Rb[PP::NP][RB];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int e = sl * 16 + i;
                    const int lr = w.row[e];
                    if (lr < 0) break;
                    if ((i & (RB - 1)) == 0) {   // radial outputs of RB edges per path at once
#pragma unroll
                        for (int q = 0; q < PP::NP; ++q) {
                            if (RB == 4)
                                tc::tmem_ld4(tl + 16 * q + i, Rb[q]);
                            else
                                tc::tmem_ld2(tl + 16 * q + i, Rb[q]);
                        }
                    }
                    float R[PP::NP];
#pragma unroll
                    for (int q = 0; q < PP::NP; ++q) R[q] = Rb[q][i & (RB - 1)];
                    if (!FIRST && i + Cfg::PD < 16) {
                        const float* __restrict__ hp =
                            Hin + ((int64_t)w.col[e + Cfg::PD] * TNLM) * TF + c;
#pragma unroll
                        for (int q = 0; q < TNLM; ++q)
                            hr[FIRST ? 0 : (i + Cfg::PD) % (Cfg::PD + 1)][q] = __ldg(hp + q * TF);
                    }
                    const float* hjc = hr[FIRST ? 0 : i % (Cfg::PD + 1)];
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
                    tc::tmem_wait_ld();
                    const float h0 = FIRST ? hb[FIRST ? i : 0] : hjc[0];
                    acc[0] = fmaf(R[0], h0, acc[0]);
                    const float t1 = R[PP::sla(1)] * h0;
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        acc[1 + m] = fmaf(t1, w.Y[e][m], acc[1 + m]);
                        if (!FIRST) acc[1 + m] = fmaf(R[PP::slb(1)], hjc[1 + m], acc[1 + m]);
                    }
                    const float t2 = R[PP::sla(2)] * h0;
#pragma unroll
                    for (int m = 0; m < 5; ++m) {
                        acc[4 + m] = fmaf(t2, w.Y[e][3 + m], acc[4 + m]);
                        if (!FIRST) acc[4 + m] = fmaf(R[PP::slb(2)], hjc[4 + m], acc[4 + m]);
                    }
                }
                tc::fence_before_sync();
                wg_sync(g);
                if (lt == 0 && sl + 1 < SCF / 16) {
                    tc::fence_after_sync();
#pragma unroll
                    for (int q = 0; q < PP::NP; ++q)
                        mma_k64<16>(tb + 16 * q, s.t.W3[q], w.B + (sl + 1) * 16 * 64);
                    tc::mma_commit(&w.mbar);
                }
            }
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

// v = sum_lm gY_lm dY_lm/du (lmax = 2) with the harmonics' constant factors
// already in the operand: g_lm = sqrt3 gY_lm for l = 1 and sqrt15 gY_lm for
// l = 2 (entry 0 unused).  The gradient of Y_20 = sqrt5/2 (3 z^2 - 1) is
// 3 sqrt5 z = sqrt15 (sqrt3 z), and sqrt3 z is Y_1z, passed as y1z.
__device__ __forceinline__ void sph_grad_prescaled(const float u[3], float y1z, const float* g,
                                                   float v[3]) {
    v[0] = fmaf(g[4], u[1], fmaf(g[7], u[2], fmaf(g[8], u[0], g[1])));
    v[1] = fmaf(g[4], u[0], fmaf(g[5], u[2], fmaf(-g[8], u[1], g[2])));
    v[2] = fmaf(g[5], u[1], fmaf(g[7], u[0], fmaf(g[6], y1z, g[3])));
}
constexpr float kS3 = 1.7320508075688772f, kS15 = 3.872983346207417f;

// Sum over the warp's lanes of values held as unevaluated FP32 pairs
// hi + lo, without FP64 arithmetic (whose rate on this GPU is a small
// fraction of FP32's).  Each butterfly step adds two pairs with Knuth's
// two-sum (s + e = a + b exactly), adds the low parts into e and
// renormalises with a fast two-sum, so the pair keeps about 44 significant
// bits; two-sum gives the same s and e for either operand order, so every
// lane ends with the same pair.
__device__ __forceinline__ void warp_sum_pair(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const float s = __fadd_rn(hi, h2);
        const float bb = __fsub_rn(s, hi);
        float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
        e = __fadd_rn(e, __fadd_rn(lo, l2));
        hi = __fadd_rn(s, e);
        lo = __fsub_rn(e, __fsub_rn(hi, s));
    }
}

// Adjoint tile rows: row 2 e holds edge e, row 2 e + 1 its r-tangent, so a
// 16-row slice is 8 edges and D2 columns (2 i, 2 i + 1) are (R, dR/dr).
template <bool STRESS>
__global__ void __launch_bounds__((BwdCfg<STRESS>::NTH), 1)
    k_edge_bwd_tc(EdgeArgs a, LayerW wl, int64_t n_groups, int* err) {
    using PP = TPaths<false>;
    using Cfg = BwdCfg<STRESS>;
    extern __shared__ unsigned char smem_raw[];
    auto& s = smem_as<SmemB<STRESS>>(smem_raw);
    const int tid = threadIdx.x, g = tid >> 7, lt = tid & 127, warp = tid >> 5, lane = tid & 31;
    const int c = lt;
    auto& w = s.wg[g];
    const float* __restrict__ Hin = a.Hin;
    const float* __restrict__ Alpha = a.Alpha;
    const float* __restrict__ Gout = a.Gout;
    float* __restrict__ Gin = a.Gin;
    tc_setup<Cfg::NTH>(s, wl, PP::NP, false, tid);
    const uint32_t tb = s.taddr + Cfg::COLS * g;
    const uint32_t tl = tb + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t phase = 0;
    bool alive = true;

    for (int64_t grp = (int64_t)blockIdx.x * Cfg::NWG + g; grp < n_groups && alive;
         grp = next_group<Cfg::NWG>(w, a, g, lt)) {
        const int64_t r0 = grp * RPG_B;
        const int nrows = (int)min((int64_t)RPG_B, a.n - r0);
        if (lt <= nrows) w.rp[lt] = a.row_ptr[r0 + lt];
        for (int q = lt; q < RPG_B * 12; q += 128) (&w.fpart[0][0][0])[q] = make_float2(0.f, 0.f);
        if (STRESS)
            for (int q = lt; q < RPG_B * 36; q += 128)
                (&w.vpart[0][0][0])[q] = make_float2(0.f, 0.f);
        wg_sync(g);
        const int64_t e_beg = w.rp[0], e_end = w.rp[nrows];
        float gacc[TNLM], ak[TNLM], hk[TNLM];
        // this channel's share of the row force: FP32 partial sums over a slice
        // (fs), folded into a compensated row sum (fk, fc) once per slice
        float fk_r[3] = {0.f, 0.f, 0.f}, fc_r[3] = {0.f, 0.f, 0.f}, fs[3] = {0.f, 0.f, 0.f};
        auto FK = [&](int q) -> float& { return fk_r[q]; };
        auto FC = [&](int q) -> float& { return fc_r[q]; };
        // with STRESS: this channel's share of the row's virial sum_e g_e (x) d_e
        // (a global sum, so plain FP32 per row suffices)
        float va[STRESS ? 9 : 1];
#pragma unroll
        for (int q = 0; q < (STRESS ? 9 : 1); ++q) va[q] = 0.f;
        auto fold = [&]() {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float fkq = FK(q), fcq = FC(q);
                const float y = fs[q] - fcq;
                const float t = fkq + y;
                FC(q) = (t - fkq) - y;
                FK(q) = t;
                fs[q] = 0.f;
            }
        };
#pragma unroll
        for (int q = 0; q < TNLM; ++q) gacc[q] = ak[q] = hk[q] = 0.f;
        int cur = -1, next = 0;
        auto flush = [&](int lr, bool with_acc) {
            {
                const int64_t base = ((r0 + lr) * TNLM) * TF + c;
#pragma unroll
                for (int q = 0; q < TNLM; ++q)
                    Gin[base + q * TF] = __ldg(Gout + base + q * TF) + (with_acc ? gacc[q] : 0.f);
            }
            if (with_acc) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {   // this channel's share is fk - fc
                    float hi = FK(q), lo = -FC(q);
                    warp_sum_pair(hi, lo);
                    if (lane == 0) w.fpart[lr][warp & 3][q] = make_float2(hi, lo);
                }
                if (STRESS) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        float hi = va[q], lo = 0.f;
                        warp_sum_pair(hi, lo);
                        if (lane == 0) w.vpart[lr][warp & 3][q] = make_float2(hi, lo);
                    }
                }
            }
        };
        // Rows >= n_recv receive no messages at this layer, so their adjoints
        // are zero and an edge between two of them adds exact zeros to every
        // sum: when the group holds such rows its edges are compacted, in
        // order, into a list without those edges, a window at a time.
        const bool compact = a.n_recv > 0 && r0 + nrows > a.n_recv;
        for (int64_t wb = e_beg; wb < e_end && alive;) {
            const int64_t we = compact ? min(wb + (int64_t)KWIN, e_end) : e_end;
            int64_t nk = we - wb;
            if (compact) {
                int keep[4], cnt = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t e = wb + 4 * lt + q;
                    keep[q] = 0;
                    if (e < we) {
                        const int lr = find_row_t(w.rp, nrows, e);
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
                if (lane == 31) w.kwarp[warp & 3] = inc;
                wg_sync(g);
                int off = inc - cnt;
                for (int q = 0; q < (warp & 3); ++q) off += w.kwarp[q];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (keep[q]) w.klist[off++] = 4 * lt + q;
                nk = w.kwarp[0] + w.kwarp[1] + w.kwarp[2] + w.kwarp[3];
                wg_sync(g);
            }
            for (int64_t kc = 0; kc < nk && alive; kc += SCB) {
                if (lt < SCB) {
                    float eps[kNB], deps[kNB], Y[TNLM], u4[4];
                    int col;
                    const int64_t v = kc + lt;
                    const int64_t e = v < nk ? wb + (compact ? (int64_t)w.klist[v] : v) : e_end;
                    const int lr = edge_geometry<true>(a, w.rp, e, e_end, r0, nrows, eps, deps,
                                                       Y, u4, col);
                    w.row[lt] = lr;
                    w.col[lt] = col;
#pragma unroll
                    for (int q = 1; q < TNLM; ++q) w.Y[lt][q - 1] = Y[q];
#pragma unroll
                    for (int q = 0; q < 4; ++q) w.u[lt][q] = u4[q];
                    // tile rows 2 e (the basis of edge e) and 2 e + 1 (its r-derivative)
                    st_basis_row(w.B, 2 * lt, eps);
                    st_basis_row(w.B, 2 * lt + 1, deps);
                }
                tc::fence_proxy_async();
                tc::fence_before_sync();
                wg_sync(g);
                if (lt == 0) {   // MMA0: z1 = eps . W1^T, dz1 = (d eps/dr) . W1^T
                    tc::fence_after_sync();
                    mma_k32(tb, w.B, s.t.W1);
                    tc::mma_commit(&w.mbar);
                }
                if (!wg_wait(w, phase, g)) { alive = false; break; }
#pragma unroll
                for (int h = 0; h < 4; ++h) {   // value rows: silu(z1); tangent rows: silu'(z1) dz1
                    float z[16];
                    tc::tmem_ld16(tl + 16 * h, z);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float zv = __shfl_sync(0xffffffffu, z[q], lane & ~1);
                        const float sg = sigmoid_fast(zv);
                        z[q] = (lane & 1) ? sg * fmaf(zv, 1.f - sg, 1.f) * z[q] : zv * sg;
                    }
                    st_row_chunk(w.B, lt, 2 * h, z);
                    st_row_chunk(w.B, lt, 2 * h + 1, z + 8);
                }
                tc::fence_proxy_async();
                tc::fence_before_sync();
                wg_sync(g);
                if (lt == 0) {
                    tc::fence_after_sync();
                    mma_k64<64>(tb, w.B, s.t.W2);
                    tc::mma_commit(&w.mbar);
                }
                if (!wg_wait(w, phase, g)) { alive = false; break; }
#pragma unroll
                for (int h = 0; h < 4; ++h) {   // value rows: silu(z2); tangent rows: silu'(z2) dz2
                    float z[16];
                    tc::tmem_ld16(tl + 16 * h, z);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float zv = __shfl_sync(0xffffffffu, z[q], lane & ~1);
                        const float sg = sigmoid_fast(zv);
                        z[q] = (lane & 1) ? sg * fmaf(zv, 1.f - sg, 1.f) * z[q] : zv * sg;
                    }
                    st_row_chunk(w.B, lt, 2 * h, z);
                    st_row_chunk(w.B, lt, 2 * h + 1, z + 8);
                }
                tc::fence_proxy_async();
                tc::fence_before_sync();
                wg_sync(g);
                if (lt == 0) {
                    tc::fence_after_sync();
#pragma unroll
                    for (int q = 0; q < PP::NP; ++q) mma_k64<16>(tb + 16 * q, s.t.W3[q], w.B);
                    tc::mma_commit(&w.mbar);
                }
                for (int sl = 0; sl < SCB / 8; ++sl) {
                    // the slice's first sender gathers go out before the wait for
                    // its MMA, so their latency overlaps it (col is 0, a valid
                    // row, for slots past the end)
                    float ajc[TNLM], hjc[TNLM], ajn[TNLM], hjn[TNLM];
                    {
                        const int64_t jb = ((int64_t)w.col[sl * 8] * TNLM) * TF + c;
#pragma unroll
                        for (int q = 0; q < TNLM; ++q) {
                            ajc[q] = __ldg(Alpha + jb + q * TF);
                            hjc[q] = __ldg(Hin + jb + q * TF);
                        }
                    }
                    if (!wg_wait(w, phase, g)) { alive = false; break; }
                    // one edge of the slice: gathers of edge i in (ajc, hjc); those of
                    // edge i + 1 are fetched into (ajn, hjn) meanwhile; the caller
                    // swaps the roles of the two buffers, so nothing is copied
                    auto edge_step = [&](int i, float (&ajc)[TNLM], float (&hjc)[TNLM],
                                         float (&ajn)[TNLM], float (&hjn)[TNLM]) -> bool {
                        const int e = sl * 8 + i;
                        const int lr = w.row[e];
                        if (lr < 0) return false;
                        float R[PP::NP], dR[PP::NP];
#pragma unroll
                        for (int q = 0; q < PP::NP; ++q) {
                            float v2[2];
                            tc::tmem_ld2(tl + 16 * q + 2 * i, v2);
                            R[q] = v2[0];
                            dR[q] = v2[1];
                        }
                        if (i + 1 < 8) {
                            const int64_t jn = ((int64_t)w.col[e + 1] * TNLM) * TF + c;
#pragma unroll
                            for (int q = 0; q < TNLM; ++q) {
                                ajn[q] = __ldg(Alpha + jn + q * TF);
                                hjn[q] = __ldg(Hin + jn + q * TF);
                            }
                        }
                        if (lr != cur) {
                            if (cur >= 0) {
                                fold();
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
                                ak[q] = __ldg(Alpha + base + q * TF);
                                hk[q] = __ldg(Hin + base + q * TF);
                            }
#pragma unroll
                            for (int q = 0; q < 3; ++q) FK(q) = FC(q) = 0.f;
                            if (STRESS) {
#pragma unroll
                                for (int q = 0; q < 9; ++q) va[q] = 0.f;
                            }
                        }
                        tc::tmem_wait_ld();
                        float Y[TNLM];
                        {
                            const float4 y0 = *reinterpret_cast<const float4*>(&w.Y[e][0]);
                            const float4 y1 = *reinterpret_cast<const float4*>(&w.Y[e][4]);
                            Y[0] = 1.f;
                            Y[1] = y0.x; Y[2] = y0.y; Y[3] = y0.z; Y[4] = y0.w;
                            Y[5] = y1.x; Y[6] = y1.y; Y[7] = y1.z; Y[8] = y1.w;
                        }
                        const float hj0 = hjc[0], hk0 = hk[0];
                        float gr, gy[TNLM];
                        gy[0] = 0.f;
                        {
                            // Y-weighted sums of the sender's (j) and receiver's (k) alpha
                            float sj1 = 0.f, sk1 = 0.f, sj2 = 0.f, sk2 = 0.f;
#pragma unroll
                            for (int m = 0; m < 3; ++m) {
                                sj1 = fmaf(ajc[1 + m], Y[1 + m], sj1);
                                sk1 = fmaf(ak[1 + m], Y[1 + m], sk1);
                            }
#pragma unroll
                            for (int m = 0; m < 5; ++m) {
                                sj2 = fmaf(ajc[4 + m], Y[4 + m], sj2);
                                sk2 = fmaf(ak[4 + m], Y[4 + m], sk2);
                            }
                            {   // dE/dh_k as the sender of the reverse edge (i <- k)
                                gacc[0] = fmaf(R[0], ajc[0], gacc[0]);
                                gacc[0] = fmaf(-R[PP::sla(1)], sj1, gacc[0]);
                                gacc[0] = fmaf(R[PP::sla(2)], sj2, gacc[0]);
#pragma unroll
                                for (int m = 0; m < 3; ++m) gacc[1 + m] = fmaf(R[PP::slb(1)], ajc[1 + m], gacc[1 + m]);
#pragma unroll
                                for (int m = 0; m < 5; ++m) gacc[4 + m] = fmaf(R[PP::slb(2)], ajc[4 + m], gacc[4 + m]);
                            }
                            // this channel's share of dE_pair/dd: radial part along u (both
                            // directions' dE/dR contracted with dR/dr) and the angular part
                            // through dE/dY; the l = 1 term of the reverse edge changes sign
                            // (grouped by the receiver's and the sender's h0)
                            gr = hj0 * fmaf(ak[0], dR[0], fmaf(sk1, dR[PP::sla(1)], sk2 * dR[PP::sla(2)]));
                            gr = fmaf(hk0, fmaf(ajc[0], dR[0], fmaf(-sj1, dR[PP::sla(1)], sj2 * dR[PP::sla(2)])),
                                      gr);
                            {
                                float g1b = 0.f, g2b = 0.f;
#pragma unroll
                                for (int m = 0; m < 3; ++m)
                                    g1b = fmaf(ak[1 + m], hjc[1 + m], fmaf(ajc[1 + m], hk[1 + m], g1b));
#pragma unroll
                                for (int m = 0; m < 5; ++m)
                                    g2b = fmaf(ak[4 + m], hjc[4 + m], fmaf(ajc[4 + m], hk[4 + m], g2b));
                                gr = fmaf(g1b, dR[PP::slb(1)], gr);
                                gr = fmaf(g2b, dR[PP::slb(2)], gr);
                            }
                            {   // (with the harmonics' factors, see sph_grad_prescaled)
                                const float r1 = kS3 * R[PP::sla(1)], r2 = kS15 * R[PP::sla(2)];
                                const float a1 = r1 * hj0, b1 = r1 * hk0;
                                const float a2 = r2 * hj0, b2 = r2 * hk0;
#pragma unroll
                                for (int m = 0; m < 3; ++m) gy[1 + m] = fmaf(ak[1 + m], a1, -ajc[1 + m] * b1);
#pragma unroll
                                for (int m = 0; m < 5; ++m) gy[4 + m] = fmaf(ak[4 + m], a2, ajc[4 + m] * b2);
                            }
                        }
                        const float4 ue = *reinterpret_cast<const float4*>(&w.u[e][0]);
                        const float u[3] = {ue.x, ue.y, ue.z};
                        const float ir = ue.w;
                        float v[3];
                        sph_grad_prescaled(u, Y[3], gy, v);
                        const float vu = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
                        if (STRESS) {
                            // the force share is accumulated exactly as without the
                            // stress (same operations), gq only feeds the virial
                            const float t = fmaf(-ir, vu, gr);
                            float gq[3];
#pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                fs[q] = fmaf(t, u[q], fmaf(ir, v[q], fs[q]));
                                gq[q] = fmaf(t, u[q], ir * v[q]);
                            }
                            const float r = 1.f / ir;
#pragma unroll
                            for (int p = 0; p < 3; ++p)
#pragma unroll
                                for (int q = 0; q < 3; ++q) va[3 * p + q] = fmaf(gq[p], u[q] * r, va[3 * p + q]);
                        } else {   // gr u + (v - (v . u) u) / r, regrouped
                            const float t = fmaf(-ir, vu, gr);
#pragma unroll
                            for (int q = 0; q < 3; ++q) fs[q] = fmaf(t, u[q], fmaf(ir, v[q], fs[q]));
                        }
                        return true;
                    };
#pragma unroll 1
                    for (int i = 0; i < 8; i += 2) {
                        if (!edge_step(i, ajc, hjc, ajn, hjn)) break;
                        if (!edge_step(i + 1, ajn, hjn, ajc, hjc)) break;
                    }
                    fold();
                    tc::fence_before_sync();
                    wg_sync(g);
                    if (lt == 0 && sl + 1 < SCB / 8) {
                        tc::fence_after_sync();
#pragma unroll
                        for (int q = 0; q < PP::NP; ++q)
                            mma_k64<16>(tb + 16 * q, s.t.W3[q], w.B + (sl + 1) * 16 * 64);
                        tc::mma_commit(&w.mbar);
                    }
                }
            }
            wb = we;
        }
        if (!alive) break;
        if (cur >= 0) {
            flush(cur, true);
            next = cur + 1;
        }
        for (int q = next; q < nrows; ++q) flush(q, false);
        wg_sync(g);
        // the four warps' pairs of a row, summed in FP64 in a fixed order
        auto sum4 = [](const float2 (&p)[4][3], int q) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) v += (double)p[k][q].x + (double)p[k][q].y;
            return v;
        };
        if (lt < nrows * 3) {
            const int lr = lt / 3, q = lt % 3;
            a.frc[(r0 + lr) * 3 + q] += sum4(w.fpart[lr], q);
        }
        if (STRESS && lt < nrows * 9) {
            const int lr = lt / 9, q = lt % 9;
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) v += (double)w.vpart[lr][k][q].x + (double)w.vpart[lr][k][q].y;
            a.vir[(int64_t)q * a.vir_stride + r0 + lr] += v;
        }
        wg_sync(g);
    }
    tc_teardown(s, phase, err, tid);
}

// ------------------------------------------ layer-0 adjoint by hidden unit --
//
// At layer 0 the senders' features are species embeddings (h0_j = Emb[s_j],
// no l >= 1 inputs), so every channel sum of the adjoint factors through the
// radial MLP's last layer.  With R_q = W3_q a2 (W3_q the 128 x 64 block of
// radial path q) and the tangent dR_q/dr = W3_q da2,
//   sum_c R_q[c] Emb[s][c] alpha_k[c, lm] = sum_h a2[h] V_k[s][lm][h],
//   V_k[s][lm][h] = sum_c W3_q(l)[c][h] Emb[s][c] alpha_k[c, lm]
// (q(0) = R0, q(1) = R_1a, q(2) = R_2a), and the same with da2.  V is formed
// once per atom by k_v_first (FP32 on the CUDA cores, from the BF16 weight
// values the forward multiplies by), and the edge kernel's epilogue then runs
// over the 64 hidden units of an edge instead of its 128 channels, with no
// third MMA: for edge e = (k <- j), hidden unit h,
//   D_0 = Vk_0 + Vj_0,  D_1m = Vk_1m - Vj_1m,  D_2m = Vk_2m + Vj_2m
//   (Vk = V_k[s_j][.][h], Vj = V_j[s_k][.][h]: the edge's two directions,
//   Y_lm(-u) = (-1)^l Y_lm(u)),
//   dE/dr share = da2[h] (D_0 + sum_lm Y_lm D_lm),
//   dE/dY_lm share = a2[h] D_lm,
// and the pair-gradient share t u + v / r is formed and summed over the
// receiver row exactly as in the channel-wise kernel, the hidden units
// taking the place of the channels in the per-row sums.

constexpr int VTA = 16;           // atoms per tile of k_v_first
constexpr int VTH = 256;          // its threads: 16 hidden-unit quads x 16 atoms
constexpr int VCB = 16;           // channels summed in FP32 before the compensated addition
constexpr int VXS = TNLM * 128 + 4;   // floats per atom row of the staged alpha (padded)
struct alignas(16) VSmem {
    float W[3][128][kH];          // W3 blocks of paths R0, R1a, R2a (FP32 of the BF16 values) x Emb[s]
    float X[VTA][VXS];            // alpha of the tile's atoms, [atom][lm][c]
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(smem_dst)),
                 "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// V[a][s][lm][h] for atoms a < nrows (the rows with a nonzero adjoint).  The
// CTA keeps the three weight blocks, scaled by the species' embedding, in
// shared memory and loops over tiles of VTA atoms; a thread owns four hidden
// units of one atom for all nine (l, m) rows (36 sums), so that each
// shared-memory load feeds four or twelve multiply-adds.
__global__ void __launch_bounds__(VTH, 1)
    k_v_first(int64_t nrows, const float* __restrict__ alpha, const float* __restrict__ emb,
              int S, const __nv_bfloat16* __restrict__ W3b, float* __restrict__ V) {
    extern __shared__ float4 vsm_raw[];
    VSmem& s = *reinterpret_cast<VSmem*>(vsm_raw);
    const int tid = threadIdx.x;
    const int h4 = tid & 15, ta = tid >> 4;
    const int64_t ntiles = (nrows + VTA - 1) / VTA;
    for (int sp = 0; sp < S; ++sp) {
        __syncthreads();   // the previous species' weights consumed
        // W3_q[c][h] Emb[s][c]: rounded alike in every partition, so the
        // only partition-dependent roundings of V are those of its sum
        for (int q = tid; q < 3 * 128 * kH; q += VTH) {
            const int p = q / (128 * kH), r = q % (128 * kH);
            const int blk = p == 0 ? 0 : 2 * p - 1;
            (&s.W[0][0][0])[q] =
                __bfloat162float(W3b[(size_t)blk * 128 * kH + r]) * __ldg(&emb[sp * 128 + r / kH]);
        }
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int64_t a0 = tile * VTA;
            __syncthreads();   // weights ready; the previous X consumed
            // the tile's alpha rows, 16 bytes per asynchronous copy, all in flight at once
            for (int q = tid; q < VTA * (TNLM * 128 / 4); q += VTH) {
                const int a = q / (TNLM * 32), off = (q % (TNLM * 32)) * 4;
                const int64_t atom = a0 + a;
                if (atom < nrows)
                    cp_async16(&s.X[a][off], alpha + atom * (TNLM * 128) + off);
                else
                    *reinterpret_cast<float4*>(&s.X[a][off]) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            cp_async_wait_all();
            __syncthreads();
            // the channel sum in blocks of VCB (packed FP32 multiply-adds, two
            // hidden units per instruction, each rounded as a scalar FMA), the
            // block sums added into an unevaluated pair hi + lo by two-sum: a
            // per-partition adjoint's V stays within a few roundings of its
            // exact value, so that partition sums of V agree with the whole
            // system's
            float hi[TNLM][4], lo[TNLM][4];
#pragma unroll
            for (int i = 0; i < TNLM; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) hi[i][k] = lo[i][k] = 0.f;
#pragma unroll 1
            for (int cb = 0; cb < 128; cb += VCB) {
                float2 acc[TNLM][2];
#pragma unroll
                for (int i = 0; i < TNLM; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
#pragma unroll 2
                for (int c = cb; c < cb + VCB; ++c) {
                    float4 wv[3];
#pragma unroll
                    for (int p = 0; p < 3; ++p) wv[p] = *reinterpret_cast<const float4*>(&s.W[p][c][4 * h4]);
#pragma unroll
                    for (int i = 0; i < TNLM; ++i) {
                        const float4 w4 = wv[i == 0 ? 0 : (i < 4 ? 1 : 2)];
                        const float x = s.X[ta][i * 128 + c];
                        const float2 xx = make_float2(x, x);
                        acc[i][0] = __ffma2_rn(xx, make_float2(w4.x, w4.y), acc[i][0]);
                        acc[i][1] = __ffma2_rn(xx, make_float2(w4.z, w4.w), acc[i][1]);
                    }
                }
#pragma unroll
                for (int i = 0; i < TNLM; ++i) {
                    const float blk[4] = {acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float sum = __fadd_rn(hi[i][k], blk[k]);
                        const float bb = __fsub_rn(sum, hi[i][k]);
                        const float err = __fadd_rn(__fsub_rn(hi[i][k], __fsub_rn(sum, bb)),
                                                    __fsub_rn(blk[k], bb));
                        hi[i][k] = sum;
                        lo[i][k] = __fadd_rn(lo[i][k], err);
                    }
                }
            }
            const int64_t atom = a0 + ta;
            if (atom < nrows) {
#pragma unroll
                for (int i = 0; i < TNLM; ++i)
                    *reinterpret_cast<float4*>(&V[((atom * S + sp) * TNLM + i) * kH + 4 * h4]) =
                        make_float4(__fadd_rn(hi[i][0], lo[i][0]), __fadd_rn(hi[i][1], lo[i][1]),
                                    __fadd_rn(hi[i][2], lo[i][2]), __fadd_rn(hi[i][3], lo[i][3]));
            }
        }
    }
}

// The layer-0 hidden-unit adjoint: weight tiles W1 and W2 only.
struct alignas(1024) Tiles0 {
    static constexpr int NPATH = 0;
    __nv_bfloat16 W2[64 * 64];
    __nv_bfloat16 W1[64 * 64];
};

template <bool STRESS>
struct alignas(1024) WgState0 {
    __nv_bfloat16 B[128 * 64];       // basis rows, then the a1 and a2 tiles (row 2 e: edge e, 2 e + 1: its r-tangent)
    float Y[SCB][TNLM - 1];          // Y_lm for lm = 1..8
    float u[SCB][4];                 // unit vector, 1 / r
    int row[SCB], col[SCB], sj[SCB];  // receiver row (-1: past the end), sender, sender species
    int klist[KWIN];
    int kwarp[4];
    int spk[RPG_B];                  // species of the group's rows
    float2 fpart[RPG_B][4][3];
    float2 vpart[RPG_B][4][STRESS ? 9 : 1];
    int64_t rp[RPG_B + 1];
    int64_t next_grp;
    uint64_t mbar;
    int abort;
};

// Seven warpgroups at 72 registers (the few spilled bytes cost less than the
// extra warps gain: 4 % over six at 80), four with the stress (virial partials).
template <bool STRESS>
struct Bwd0Cfg {
    static constexpr int NWG = STRESS ? 4 : 7;
    static constexpr int NTH = 128 * NWG;
    static constexpr int COLS = 64;   // D0 and D1 (128 rows x 64 hidden units)
};
template <class WG, int N>
struct SmemT0 {
    Tiles0 t;
    WG wg[N];
    uint32_t taddr;
};
template <bool STRESS>
using SmemB0 = SmemT0<WgState0<STRESS>, Bwd0Cfg<STRESS>::NWG>;
static_assert(smem_fits<SmemB0<false>>() && smem_fits<SmemB0<true>>(),
              "shared memory of the layer-0 hidden-unit adjoint");
static_assert(Bwd0Cfg<false>::NWG * Bwd0Cfg<false>::COLS <= TM_COLS, "tensor memory");

// Edges of a super-chunk: the warpgroup's first half (threads 0..63, one
// hidden unit each) takes edges 0..31 in order, the second half edges 32..63,
// each with its own receiver-row state; a row's force is the sum of the four
// warps' shares (a warp's share of a row it did not meet stays zero).
template <bool STRESS>
__global__ void __launch_bounds__((Bwd0Cfg<STRESS>::NTH), 1)
    k_edge_bwd0_tc(EdgeArgs a, LayerW wl, int64_t n_groups, int* err) {
    using Cfg = Bwd0Cfg<STRESS>;
    extern __shared__ unsigned char smem_raw[];
    auto& s = smem_as<SmemB0<STRESS>>(smem_raw);
    const int tid = threadIdx.x, g = tid >> 7, lt = tid & 127, warp = tid >> 5, lane = tid & 31;
    const int half = lt >> 6, hu = lt & 63;   // edge half and hidden unit of this thread
    auto& w = s.wg[g];
    const float* __restrict__ Vf = a.vfirst;
    const int S = a.n_species;
    tc_setup<Cfg::NTH>(s, wl, 0, true, tid);
    const uint32_t tb = s.taddr + Cfg::COLS * g;
    const uint32_t tl = tb + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t phase = 0;
    bool alive = true;
    const unsigned char* Bb = reinterpret_cast<const unsigned char*>(w.B);

    for (int64_t grp = (int64_t)blockIdx.x * Cfg::NWG + g; grp < n_groups && alive;
         grp = next_group<Cfg::NWG>(w, a, g, lt)) {
        const int64_t r0 = grp * RPG_B;
        const int nrows = (int)min((int64_t)RPG_B, a.n - r0);
        if (lt <= nrows) w.rp[lt] = a.row_ptr[r0 + lt];
        if (lt < nrows) w.spk[lt] = a.species[r0 + lt];
        for (int q = lt; q < RPG_B * 12; q += 128) (&w.fpart[0][0][0])[q] = make_float2(0.f, 0.f);
        if (STRESS)
            for (int q = lt; q < RPG_B * 36; q += 128)
                (&w.vpart[0][0][0])[q] = make_float2(0.f, 0.f);
        wg_sync(g);
        const int64_t e_beg = w.rp[0], e_end = w.rp[nrows];
        // this thread's share of the row force, each edge's share added into
        // a compensated sum (fk, fc): a hidden unit's share of an edge is a
        // sum over all channels, larger than a channel's share, so it is not
        // first summed over several edges in plain FP32
        float fk[3] = {0.f, 0.f, 0.f}, fc[3] = {0.f, 0.f, 0.f};
        auto kadd = [&](int q, float gq) {
            const float y = gq - fc[q];
            const float t = fk[q] + y;
            fc[q] = (t - fk[q]) - y;
            fk[q] = t;
        };
        float va[STRESS ? 9 : 1];
#pragma unroll
        for (int q = 0; q < (STRESS ? 9 : 1); ++q) va[q] = 0.f;
        auto flush = [&](int lr) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {   // this thread's share is fk - fc
                float hi = fk[q], lo = -fc[q];
                warp_sum_pair(hi, lo);
                if (lane == 0) w.fpart[lr][warp & 3][q] = make_float2(hi, lo);
            }
            if (STRESS) {
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    float hi = va[q], lo = 0.f;
                    warp_sum_pair(hi, lo);
                    if (lane == 0) w.vpart[lr][warp & 3][q] = make_float2(hi, lo);
                }
            }
        };
        int cur = -1;
        int sk = 0;                  // species of the current row
        float vk[TNLM];              // V_k[s_j] of the current row (S = 1: loaded once per row)
#pragma unroll
        for (int q = 0; q < TNLM; ++q) vk[q] = 0.f;
        const bool compact = a.n_recv > 0 && r0 + nrows > a.n_recv;
        for (int64_t wb = e_beg; wb < e_end && alive;) {
            const int64_t we = compact ? min(wb + (int64_t)KWIN, e_end) : e_end;
            int64_t nk = we - wb;
            if (compact) {
                int keep[4], cnt = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t e = wb + 4 * lt + q;
                    keep[q] = 0;
                    if (e < we) {
                        const int lr = find_row_t(w.rp, nrows, e);
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
                if (lane == 31) w.kwarp[warp & 3] = inc;
                wg_sync(g);
                int off = inc - cnt;
                for (int q = 0; q < (warp & 3); ++q) off += w.kwarp[q];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (keep[q]) w.klist[off++] = 4 * lt + q;
                nk = w.kwarp[0] + w.kwarp[1] + w.kwarp[2] + w.kwarp[3];
                wg_sync(g);
            }
            for (int64_t kc = 0; kc < nk && alive; kc += SCB) {
                if (lt < SCB) {
                    float eps[kNB], deps[kNB], Y[TNLM], u4[4];
                    int col;
                    const int64_t v = kc + lt;
                    const int64_t e = v < nk ? wb + (compact ? (int64_t)w.klist[v] : v) : e_end;
                    const int lr = edge_geometry<true>(a, w.rp, e, e_end, r0, nrows, eps, deps,
                                                       Y, u4, col);
                    w.row[lt] = lr;
                    w.col[lt] = col;
                    w.sj[lt] = lr >= 0 ? a.species[col] : 0;
#pragma unroll
                    for (int q = 1; q < TNLM; ++q) w.Y[lt][q - 1] = Y[q];
#pragma unroll
                    for (int q = 0; q < 4; ++q) w.u[lt][q] = u4[q];
                    st_basis_row(w.B, 2 * lt, eps);
                    st_basis_row(w.B, 2 * lt + 1, deps);
                }
                tc::fence_proxy_async();
                tc::fence_before_sync();
                wg_sync(g);
                if (lt == 0) {   // MMA0: z1 = eps . W1^T, dz1 = (d eps/dr) . W1^T
                    tc::fence_after_sync();
                    mma_k32(tb, w.B, s.t.W1);
                    tc::mma_commit(&w.mbar);
                }
                if (!wg_wait(w, phase, g)) { alive = false; break; }
#pragma unroll
                for (int h = 0; h < 4; ++h) {   // value rows: silu(z1); tangent rows: silu'(z1) dz1
                    float z[16];
                    tc::tmem_ld16(tl + 16 * h, z);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float zv = __shfl_sync(0xffffffffu, z[q], lane & ~1);
                        const float sg = sigmoid_fast(zv);
                        z[q] = (lane & 1) ? sg * fmaf(zv, 1.f - sg, 1.f) * z[q] : zv * sg;
                    }
                    st_row_chunk(w.B, lt, 2 * h, z);
                    st_row_chunk(w.B, lt, 2 * h + 1, z + 8);
                }
                tc::fence_proxy_async();
                tc::fence_before_sync();
                wg_sync(g);
                if (lt == 0) {
                    tc::fence_after_sync();
                    mma_k64<64>(tb, w.B, s.t.W2);
                    tc::mma_commit(&w.mbar);
                }
                if (!wg_wait(w, phase, g)) { alive = false; break; }
#pragma unroll
                for (int h = 0; h < 4; ++h) {   // value rows: silu(z2); tangent rows: silu'(z2) dz2
                    float z[16];
                    tc::tmem_ld16(tl + 16 * h, z);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float zv = __shfl_sync(0xffffffffu, z[q], lane & ~1);
                        const float sg = sigmoid_fast(zv);
                        z[q] = (lane & 1) ? sg * fmaf(zv, 1.f - sg, 1.f) * z[q] : zv * sg;
                    }
                    st_row_chunk(w.B, lt, 2 * h, z);
                    st_row_chunk(w.B, lt, 2 * h + 1, z + 8);
                }
                tc::fence_before_sync();
                wg_sync(g);   // the a2 / da2 rows are complete (read below by hidden unit)
                // this half's edges; V_j of the first is requested at once, each
                // next one's while the current edge computes
                const int e0 = 32 * half;
                float vjc[TNLM], vjn[TNLM];
                auto vj_ptr = [&](int e) -> const float* {
                    const int lr = w.row[e];
                    const int spk = w.spk[lr < 0 ? 0 : lr];
                    return Vf + (((int64_t)w.col[e] * S + spk) * TNLM) * kH + hu;
                };
                {
                    const float* p = vj_ptr(e0);
#pragma unroll
                    for (int q = 0; q < TNLM; ++q) vjc[q] = __ldg(p + q * kH);
                }
                // k = e mod 4 (a literal at each call): rows 2 e and 2 e + 1 of
                // the swizzled tile then have constant XOR patterns 2 k, 2 k + 1
                const int c8 = hu >> 3, lo2 = (hu & 7) * 2;
                auto edge_step = [&](int e, int k, float (&vj)[TNLM], float (&vjnext)[TNLM]) -> bool {
                    const int lr = w.row[e];
                    if (lr < 0) return false;
                    if (e + 1 < e0 + 32) {
                        const float* p = vj_ptr(e + 1);
#pragma unroll
                        for (int q = 0; q < TNLM; ++q) vjnext[q] = __ldg(p + q * kH);
                    }
                    const int sj = w.sj[e];
                    if (lr != cur) {
                        if (cur >= 0) flush(cur);
                        cur = lr;
                        sk = w.spk[lr];
#pragma unroll
                        for (int q = 0; q < 3; ++q) fk[q] = fc[q] = 0.f;
                        if (STRESS) {
#pragma unroll
                            for (int q = 0; q < 9; ++q) va[q] = 0.f;
                        }
                        if (S == 1) {
                            const float* p = Vf + ((int64_t)(r0 + lr) * TNLM) * kH + hu;
#pragma unroll
                            for (int q = 0; q < TNLM; ++q) vk[q] = __ldg(p + q * kH);
                        }
                    }
                    if (S != 1) {
                        const float* p = Vf + (((int64_t)(r0 + lr) * S + sj) * TNLM) * kH + hu;
#pragma unroll
                        for (int q = 0; q < TNLM; ++q) vk[q] = __ldg(p + q * kH);
                    }
                    const unsigned char* brow = Bb + e * 256 + lo2;
                    const float a2 = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(
                        brow + (((c8 ^ (2 * k)) & 7) << 4)));
                    const float da2 = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(
                        brow + 128 + (((c8 ^ (2 * k + 1)) & 7) << 4)));
                    float Y[TNLM];
                    {
                        const float4 y0 = *reinterpret_cast<const float4*>(&w.Y[e][0]);
                        const float4 y1 = *reinterpret_cast<const float4*>(&w.Y[e][4]);
                        Y[0] = 1.f;
                        Y[1] = y0.x; Y[2] = y0.y; Y[3] = y0.z; Y[4] = y0.w;
                        Y[5] = y1.x; Y[6] = y1.y; Y[7] = y1.z; Y[8] = y1.w;
                    }
                    // both directions of the edge (Y_lm(-u) = (-1)^l Y_lm(u))
                    float D[TNLM];
                    D[0] = vk[0] + vj[0];
#pragma unroll
                    for (int m = 1; m < 4; ++m) D[m] = vk[m] - vj[m];
#pragma unroll
                    for (int m = 4; m < 9; ++m) D[m] = vk[m] + vj[m];
                    float wsum = D[0];
#pragma unroll
                    for (int m = 1; m < 9; ++m) wsum = fmaf(Y[m], D[m], wsum);
                    const float gr = da2 * wsum;
                    // dE/dY shares with the harmonics' factors (see sph_grad_prescaled)
                    const float c1 = kS3 * a2, c2 = kS15 * a2;
                    float gy[TNLM];
                    gy[0] = 0.f;
#pragma unroll
                    for (int m = 1; m < 4; ++m) gy[m] = c1 * D[m];
#pragma unroll
                    for (int m = 4; m < 9; ++m) gy[m] = c2 * D[m];
                    const float4 ue = *reinterpret_cast<const float4*>(&w.u[e][0]);
                    const float u[3] = {ue.x, ue.y, ue.z};
                    const float ir = ue.w;
                    float v[3];
                    sph_grad_prescaled(u, Y[3], gy, v);
                    const float vu = v[0] * u[0] + v[1] * u[1] + v[2] * u[2];
                    const float t = fmaf(-ir, vu, gr);
                    float gq[3];   // this hidden unit's share of dE_pair/dd
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        gq[q] = fmaf(t, u[q], ir * v[q]);
                        kadd(q, gq[q]);
                    }
                    if (STRESS) {
                        const float r = 1.f / ir;
#pragma unroll
                        for (int p = 0; p < 3; ++p)
#pragma unroll
                            for (int q = 0; q < 3; ++q) va[3 * p + q] = fmaf(gq[p], u[q] * r, va[3 * p + q]);
                    }
                    return true;
                };
#pragma unroll 1
                for (int i = 0; i < 32; i += 4) {
                    if (!edge_step(e0 + i, 0, vjc, vjn)) break;
                    if (!edge_step(e0 + i + 1, 1, vjn, vjc)) break;
                    if (!edge_step(e0 + i + 2, 2, vjc, vjn)) break;
                    if (!edge_step(e0 + i + 3, 3, vjn, vjc)) break;
                }
                wg_sync(g);   // the B tile and edge records are rewritten by the next chunk
            }
            wb = we;
        }
        if (!alive) break;
        if (cur >= 0) flush(cur);
        wg_sync(g);
        auto sum4 = [](const float2 (&p)[4][3], int q) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) v += (double)p[k][q].x + (double)p[k][q].y;
            return v;
        };
        if (lt < nrows * 3) {
            const int lr = lt / 3, q = lt % 3;
            a.frc[(r0 + lr) * 3 + q] += sum4(w.fpart[lr], q);
        }
        if (STRESS && lt < nrows * 9) {
            const int lr = lt / 9, q = lt % 9;
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) v += (double)w.vpart[lr][k][q].x + (double)w.vpart[lr][k][q].y;
            a.vir[(int64_t)q * a.vir_stride + r0 + lr] += v;
        }
        wg_sync(g);
    }
    tc_teardown(s, phase, err, tid);
}

// ------------------------------------------ layer-0 forward by hidden unit --
//
// The same factorisation as the layer-0 adjoint above, in the forward
// direction: with h0_j = Emb[s_j] and R_q = W3_q a2,
//   A_k[c, lm] = N_avg^-1 sum_e R_q(l)(e)[c] Emb[s_j][c] Y_lm(e)
//             = N_avg^-1 sum_s Emb[s][c] sum_h W3_q(l)[c][h] G_k[s][lm][h],
//   G_k[s][lm][h] = sum_{e in row k, s_j = s} a2_e[h] Y_lm(e).
// k_edge_fwd0_tc runs the geometry and the first two radial layers of each
// edge and sums G per receiver row (thread = hidden unit and half of the
// (l, m) rows, no third MMA, no per-channel work); k_a_first_tc then forms A
// from G on the tensor cores, 16 atoms per MMA, with G split into three
// BF16 parts so that the product keeps FP32 accuracy.

constexpr int SMAX0 = 3;          // species handled by the hidden-unit layer 0

template <int S>
struct alignas(1024) WgStateF0 {
    __nv_bfloat16 B[128 * 64];       // basis rows, then the a1 and a2 tiles (row = edge)
    float Y[SCF][TNLM - 1];          // Y_lm for lm = 1..8
    int row[SCF], sj[SCF];           // receiver row (-1: past the end), sender species
    int64_t rp[RPG + 1];
    int64_t next_grp;
    uint64_t mbar;
    int abort;
};
// Eight warpgroups at 64 registers (no spills; 8 % faster than six).
template <int S>
struct F0Cfg {
    static constexpr int NWG = 8;
    static constexpr int NTH = 128 * NWG;
    static constexpr int COLS = 64;   // D0 and D1 (128 edges x 64 hidden units)
};
template <int S>
using SmemF0 = SmemT0<WgStateF0<S>, F0Cfg<S>::NWG>;
static_assert(smem_fits<SmemF0<1>>() && smem_fits<SmemF0<SMAX0>>(),
              "shared memory of the layer-0 hidden-unit forward");

// G of every row of the pass (zero for a row without edges).  Thread lt of a
// warpgroup owns hidden unit lt & 63 and the (l, m) rows 0..4 (lt < 64) or
// 5..8, and runs through all edges of a super-chunk in order, so each row's
// sum is formed by one thread in edge order (the same in every partition).
template <int S>
__global__ void __launch_bounds__((F0Cfg<S>::NTH), 1)
    k_edge_fwd0_tc(EdgeArgs a, LayerW wl, int64_t n_groups, int* err) {
    using Cfg = F0Cfg<S>;
    extern __shared__ unsigned char smem_raw[];
    auto& s = smem_as<SmemF0<S>>(smem_raw);
    const int tid = threadIdx.x, g = tid >> 7, lt = tid & 127, warp = tid >> 5;
    const int hu = lt & 63, grp = lt >> 6;
    const int lm0 = grp ? 5 : 0;
    constexpr int NL = 5;              // (l, m) rows per thread (4 used by the second half)
    auto& w = s.wg[g];
    float* __restrict__ Gout = a.vfirst;
    tc_setup<Cfg::NTH>(s, wl, 0, true, tid);
    const uint32_t tb = s.taddr + Cfg::COLS * g;
    const uint32_t tl = tb + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t phase = 0;
    bool alive = true;
    const unsigned char* Bb = reinterpret_cast<const unsigned char*>(w.B);
    const int nlm = grp ? 4 : 5;

    for (int64_t gi = (int64_t)blockIdx.x * Cfg::NWG + g; gi < n_groups && alive;
         gi = next_group<Cfg::NWG>(w, a, g, lt)) {
        const int64_t r0 = gi * RPG_F;
        const int nrows = (int)min((int64_t)RPG_F, a.n - r0);
        if (lt <= nrows) w.rp[lt] = a.row_ptr[r0 + lt];
        wg_sync(g);
        const int64_t e_beg = w.rp[0], e_end = w.rp[nrows];
        float acc[S][NL];
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
            for (int i = 0; i < NL; ++i) acc[q][i] = 0.f;
        int cur = -1, next = 0;
        auto write_row = [&](int lr, bool zero) {
            float* __restrict__ o = Gout + ((r0 + lr) * S * TNLM + lm0) * kH + hu;
#pragma unroll
            for (int q = 0; q < S; ++q)
#pragma unroll
                for (int i = 0; i < NL; ++i)
                    if (i < nlm) o[(q * TNLM + i) * kH] = zero ? 0.f : acc[q][i];
        };
        for (int64_t sc = e_beg; sc < e_end && alive; sc += SCF) {
            {   // geometry of edge lt; its radial basis -> tile row lt
                float eps[kNB], deps[kNB], Y[TNLM], u4[4];
                int col;
                const int lr = edge_geometry<false>(a, w.rp, sc + lt, e_end, r0, nrows, eps, deps,
                                                    Y, u4, col);
                w.row[lt] = lr;
                w.sj[lt] = (S > 1 && lr >= 0) ? a.species[col] : 0;
#pragma unroll
                for (int q = 1; q < TNLM; ++q) w.Y[lt][q - 1] = Y[q];
                st_basis_row(w.B, lt, eps);
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            wg_sync(g);
            if (lt == 0) {   // MMA0: z1 = eps . W1^T
                tc::fence_after_sync();
                mma_k32(tb, w.B, s.t.W1);
                tc::mma_commit(&w.mbar);
            }
            if (!wg_wait(w, phase, g)) { alive = false; break; }
#pragma unroll
            for (int h = 0; h < 4; ++h) {   // a1 = silu(z1): lane lt holds tile row lt
                float z[16];
                tc::tmem_ld16(tl + 16 * h, z);
                tc::tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) z[q] = z[q] * sigmoid_fast(z[q]);
                st_row_chunk(w.B, lt, 2 * h, z);
                st_row_chunk(w.B, lt, 2 * h + 1, z + 8);
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            wg_sync(g);
            if (lt == 0) {
                tc::fence_after_sync();
                mma_k64<64>(tb, w.B, s.t.W2);
                tc::mma_commit(&w.mbar);
            }
            if (!wg_wait(w, phase, g)) { alive = false; break; }
#pragma unroll
            for (int h = 0; h < 4; ++h) {   // a2 = silu(z2)
                float z[16];
                tc::tmem_ld16(tl + 16 * h, z);
                tc::tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) z[q] = z[q] * sigmoid_fast(z[q]);
                st_row_chunk(w.B, lt, 2 * h, z);
                st_row_chunk(w.B, lt, 2 * h + 1, z + 8);
            }
            tc::fence_before_sync();
            wg_sync(g);   // the a2 rows are complete (read below by hidden unit)
            // the chunk's edges in order, eight per step so that each edge's
            // swizzled a2 column offset is a constant XOR pattern; the two
            // halves of the warpgroup (warp-uniform) run their own loop, with
            // their (l, m) rows fixed at compile time
            auto run = [&](auto half) {
                constexpr int HALF = decltype(half)::value;
                const int c8 = hu >> 3, lo2 = (hu & 7) * 2;
                bool done = false;
#pragma unroll 1
                for (int e8 = 0; e8 < SCF && !done; e8 += 8) {
#pragma unroll
                    for (int k = 0; k < 8; ++k) {
                        const int e = e8 + k;
                        const int lr = w.row[e];
                        if (lr < 0) { done = true; break; }
                        if (lr != cur) {
                            if (cur >= 0) {
                                write_row(cur, false);
                                next = cur + 1;
                            }
                            for (int q = next; q < lr; ++q) write_row(q, true);
                            next = lr;
                            cur = lr;
#pragma unroll
                            for (int q = 0; q < S; ++q)
#pragma unroll
                                for (int i = 0; i < NL; ++i) acc[q][i] = 0.f;
                        }
                        const float a2 = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(
                            Bb + e * 128 + (((c8 ^ k) & 7) << 4) + lo2));
                        const float4 yv = *reinterpret_cast<const float4*>(&w.Y[e][HALF ? 4 : 0]);
                        // this half's (l, m) rows: Y_0 = 1, Y_1..Y_4 or Y_5..Y_8
                        const float y[NL] = {HALF ? yv.x : 1.f, HALF ? yv.y : yv.x,
                                             HALF ? yv.z : yv.y, HALF ? yv.w : yv.z,
                                             HALF ? 0.f : yv.w};
                        const int sp = S > 1 ? w.sj[e] : 0;
#pragma unroll
                        for (int q = 0; q < S; ++q) {
                            if (S == 1 || q == sp) {
#pragma unroll
                                for (int i = 0; i < NL - HALF; ++i) acc[q][i] = fmaf(a2, y[i], acc[q][i]);
                            }
                        }
                    }
                }
            };
            if (grp)
                run(std::integral_constant<int, 1>{});
            else
                run(std::integral_constant<int, 0>{});
            wg_sync(g);   // the tile and edge records are rewritten by the next chunk
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

// A of 16 atoms per tile.  G_s (per species, (l, m) and hidden unit) is
// split into three BF16 parts; the operand rows of one species are ordered
// ((l, m), part, atom), so each radial path's rows are contiguous and one MMA
// chain per path (N = 3 x 16 x the path's (l, m) count: 48, 144, 240)
// computes W3_q . G^T for all of them.  The epilogue sums the three parts'
// columns, weights them by Emb[s][c] and sums the species:
//   A[atom][lm][c] = N_avg^-1 sum_s Emb[s][c] sum_part D_s[lm][part][c][atom].
// The next tile's G is loaded into registers while the MMAs run.
constexpr int AF_NT = 16;         // atoms per tile
constexpr int AF_NTH = 512;       // threads: 16 atoms x 32 in the load phase
constexpr int AF_COLS = TNLM * 3 * AF_NT;   // tensor-memory columns of one species (432)
template <int S>
struct alignas(1024) AfSmem {
    __nv_bfloat16 W3[3][128 * 64];              // paths R0, R1a, R2a (swizzled images)
    __nv_bfloat16 X[S][TNLM][3][AF_NT * 64];    // G parts: species, (l, m), part
    uint64_t mbar;
    uint32_t taddr;
    int abort;
};
template <int S>
constexpr bool af_fits() { return sizeof(AfSmem<S>) + 1024 <= 232448; }
static_assert(af_fits<1>() && af_fits<SMAX0>(), "shared memory of k_a_first_tc");
static_assert(AF_COLS <= TM_COLS, "tensor memory of k_a_first_tc");

// D[tmem, 128 x N] = A(128 x 64 tile) . B(N x 64, N consecutive tile rows)^T,
// four K = 16 steps.
template <int N>
__device__ __forceinline__ void mma_k64_n(uint32_t d, const __nv_bfloat16* A,
                                          const __nv_bfloat16* B) {
    const uint64_t ad = tc::desc_sw128(tc::smem_u32(A));
    const uint64_t bd = tc::desc_sw128(tc::smem_u32(B));
    constexpr uint32_t idesc = tc::idesc_bf16(128, N);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) tc::mma_bf16(d, ad + 2 * kk, bd + 2 * kk, idesc, kk > 0 ? 1u : 0u);
}

template <int S>
__global__ void __launch_bounds__(AF_NTH, 1)
    k_a_first_tc(int64_t n, const float* __restrict__ G, const float* __restrict__ emb,
                 const __nv_bfloat16* __restrict__ W3sw, float inv_navg,
                 float* __restrict__ Aout, int64_t n_tiles, int* err) {
    extern __shared__ unsigned char smem_raw[];
    auto& s = smem_as<AfSmem<S>>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ia = tid >> 5, q = tid & 31;            // load phase: atom, float4 slot
    const int lq = warp & 3, ag = warp >> 2;          // epilogue: lane quarter, atom group
    const int c = 32 * lq + lane;
    constexpr int NV = (S * TNLM * 16 + 31) / 32;     // float4 slots of G per thread
    for (int p = 0; p < 3; ++p) {
        const int blk = p == 0 ? 0 : 2 * p - 1;
        const uint4* src = reinterpret_cast<const uint4*>(W3sw + (size_t)blk * 128 * 64);
        uint4* dst = reinterpret_cast<uint4*>(s.W3[p]);
        for (int k = tid; k < 128 * 64 * 2 / 16; k += AF_NTH) dst[k] = __ldg(&src[k]);
    }
    if (tid == 0) {
        tc::mbar_init(&s.mbar, 1);
        s.abort = 0;
    }
    if (warp == 0) tc::tmem_alloc<TM_COLS>(&s.taddr);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    float es[S];
#pragma unroll
    for (int k = 0; k < S; ++k) es[k] = __ldg(&emb[k * 128 + c]);
    float4 gv[NV];
    auto load = [&](int64_t tile) {   // this thread's slots r = q + 32 v of atom ia
        const int64_t atom = tile * AF_NT + ia;
        const bool ok = tile < n_tiles && atom < n;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int r = q + 32 * v;
            gv[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok && r < S * TNLM * 16)
                gv[v] = __ldg(reinterpret_cast<const float4*>(G + (atom * S * TNLM) * kH) + r);
        }
    };
    uint32_t phase = 0;
    int64_t tile = blockIdx.x;
    load(tile);
    for (; tile < n_tiles; tile += gridDim.x) {
        // this tile's G (in registers) in three BF16 parts, each the rounding
        // of what the previous parts leave, into the swizzled operand rows
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int r = q + 32 * v;
            if (r >= S * TNLM * 16) break;
            const int sp = r / (TNLM * 16), lm = (r / 16) % TNLM, h4 = r & 15;
            float rr[4] = {gv[v].x, gv[v].y, gv[v].z, gv[v].w};
            const uint32_t off = ia * 128 + ((((h4 >> 1) ^ (ia & 7)) & 7) << 4) + ((h4 & 1) << 3);
#pragma unroll
            for (int part = 0; part < 3; ++part) {
                const __nv_bfloat162 lo = __floats2bfloat162_rn(rr[0], rr[1]);
                const __nv_bfloat162 hi = __floats2bfloat162_rn(rr[2], rr[3]);
                rr[0] -= __low2float(lo);
                rr[1] -= __high2float(lo);
                rr[2] -= __low2float(hi);
                rr[3] -= __high2float(hi);
                uint2 u;
                u.x = *reinterpret_cast<const uint32_t*>(&lo);
                u.y = *reinterpret_cast<const uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(reinterpret_cast<unsigned char*>(s.X[sp][lm][part]) + off) = u;
            }
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        float o[TNLM][4];
#pragma unroll
        for (int lm = 0; lm < TNLM; ++lm)
#pragma unroll
            for (int r = 0; r < 4; ++r) o[lm][r] = 0.f;
        for (int sp = 0; sp < S; ++sp) {
            if (tid == 0) {   // one chain per radial path: rows ((l, m), part, atom)
                tc::fence_after_sync();
                mma_k64_n<3 * AF_NT * 1>(s.taddr, s.W3[0], s.X[sp][0][0]);
                mma_k64_n<3 * AF_NT * 3>(s.taddr + 3 * AF_NT * 1, s.W3[1], s.X[sp][1][0]);
                mma_k64_n<3 * AF_NT * 5>(s.taddr + 3 * AF_NT * 4, s.W3[2], s.X[sp][4][0]);
                tc::mma_commit(&s.mbar);
            }
            if (sp == 0) load(tile + gridDim.x);   // the next tile's G, meanwhile
            if (tc::mbar_wait(&s.mbar, phase))
                phase ^= 1u;
            else
                s.abort = 1;
            __syncthreads();
            tc::fence_after_sync();
            if (s.abort) break;
            const uint32_t tcol = s.taddr + ((uint32_t)(32 * lq) << 16) + 4 * ag;
#pragma unroll
            for (int lm = 0; lm < TNLM; ++lm) {
                float d0[4], d1[4], d2[4];
                tc::tmem_ld4(tcol + AF_NT * (3 * lm + 0), d0);
                tc::tmem_ld4(tcol + AF_NT * (3 * lm + 1), d1);
                tc::tmem_ld4(tcol + AF_NT * (3 * lm + 2), d2);
                tc::tmem_wait_ld();
#pragma unroll
                for (int r = 0; r < 4; ++r) o[lm][r] = fmaf(es[sp], d0[r] + d1[r] + d2[r], o[lm][r]);
            }
            tc::fence_before_sync();
            __syncthreads();   // tensor memory is rewritten by the next species or tile
        }
        if (s.abort) break;
        const int64_t i0 = tile * AF_NT + 4 * ag;
#pragma unroll
        for (int lm = 0; lm < TNLM; ++lm)
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (i0 + r < n) Aout[((i0 + r) * TNLM + lm) * 128 + c] = o[lm][r] * inv_navg;
    }
    if (s.abort) {
        tc::mbar_wait(&s.mbar, phase, 20000000LL);
        if (tid == 0) atomicOr(err, kErrTimeout);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc<TM_COLS>(s.taddr);
}

template <class S, int N, class K>
int launch_tc(K kernel, const EdgeArgs& a, int rpg, int num_sms, cudaStream_t st) {
    const int64_t groups = (a.n + rpg - 1) / rpg;
    const size_t smem = sizeof(S) + 1024;
    MP_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    int64_t grid = (int64_t)num_sms;   // one CTA (one 512-column TMEM allocation) per SM
    const int64_t need = (groups + N - 1) / N;
    if (grid > need) grid = need;
    MP_CUDA_TRY(cudaMemsetAsync(a.sched, 0, sizeof(int), st));
    kernel<<<(unsigned)grid, 128 * N, smem, st>>>(a, *a.w, groups, a.err);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

namespace {

// Every position coordinate as an unevaluated FP32 pair hi + lo (hi = the
// FP32 rounding of x, lo = the rounding of the remainder: about 48
// significant bits, more than the edge vector needs).
__global__ void k_split_positions(int64_t n, const double* __restrict__ x,
                                  float4* __restrict__ hi, float4* __restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float h[3], l[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double v = x[3 * i + a];
        h[a] = (float)v;
        l[a] = (float)(v - (double)h[a]);
    }
    hi[i] = make_float4(h[0], h[1], h[2], 0.f);
    lo[i] = make_float4(l[0], l[1], l[2], 0.f);
}

// One component of x_j - x_i + n L (n in {-1, 0, 1}) from the FP32 pairs, in
// FP32 only: the difference of the high parts and the addition of the high
// part of n L are exact by Knuth's two-sum (s + e = a + b), the low parts and
// the errors are then summed, and the result is rounded once.
__device__ __forceinline__ float image_diff_pair(float hj, float lj, float hi, float li, int n,
                                                 float Lh, float Ll) {
    float s = __fsub_rn(hj, hi);
    float bb = __fsub_rn(s, hj);
    float err = __fadd_rn(__fsub_rn(hj, __fsub_rn(s, bb)), __fsub_rn(-hi, bb));
    float low = __fsub_rn(lj, li);
    if (n != 0) {
        const float b = n > 0 ? Lh : -Lh;
        const float s2 = __fadd_rn(s, b);
        const float bb2 = __fsub_rn(s2, s);
        err = __fadd_rn(err, __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bb2)), __fsub_rn(b, bb2)));
        low = __fadd_rn(low, n > 0 ? Ll : -Ll);
        s = s2;
    }
    return __fadd_rn(s, __fadd_rn(err, low));
}

// Warp per row: (u, r) of each of the row's edges, in CSR order.  The edge
// vector is formed in FP32 from the positions' FP32 pairs (FP64 runs at a
// small fraction of the FP32 rate on this GPU); it agrees with the FP64
// formula of edge_vector to within one FP32 rounding.
__global__ void k_edge_geometry(int64_t n, const int64_t* __restrict__ row_ptr,
                                const int32_t* __restrict__ col, const int8_t* __restrict__ shift,
                                const float4* __restrict__ hi, const float4* __restrict__ lo,
                                float Lh0, float Lh1, float Lh2, float Ll0, float Ll1, float Ll2,
                                float4* __restrict__ geo) {
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const float4 hi_i = hi[i], lo_i = lo[i];
    for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
        const int j = col[e];
        const int code = shift[e];
        const float4 hj = hi[j], lj = lo[j];
        float d[3], u[3];
        d[0] = image_diff_pair(hj.x, lj.x, hi_i.x, lo_i.x, code / 9 - 1, Lh0, Ll0);
        d[1] = image_diff_pair(hj.y, lj.y, hi_i.y, lo_i.y, (code / 3) % 3 - 1, Lh1, Ll1);
        d[2] = image_diff_pair(hj.z, lj.z, hi_i.z, lo_i.z, code % 3 - 1, Lh2, Ll2);
        const float r = edge_unit(d, u);
        geo[e] = make_float4(u[0], u[1], u[2], r);
    }
}

}  // namespace

int launch_edge_geometry(int64_t n, const int64_t* row_ptr, const int32_t* col,
                         const int8_t* shift, const double* x, const EdgeConst& k, float4* geo,
                         float4* split, cudaStream_t st) {
    if (n <= 0) return MP_OK;
    float4* hi = split;
    float4* lo = split + n;
    k_split_positions<<<grid_for(n, 256), 256, 0, st>>>(n, x, hi, lo);
    note_launch();
    float Lh[3], Ll[3];
    for (int a = 0; a < 3; ++a) {
        Lh[a] = (float)k.L[a];
        Ll[a] = (float)(k.L[a] - (double)Lh[a]);
    }
    const int wpb = 8;
    k_edge_geometry<<<(unsigned)((n + wpb - 1) / wpb), 32 * wpb, 0, st>>>(
        n, row_ptr, col, shift, hi, lo, Lh[0], Lh[1], Lh[2], Ll[0], Ll[1], Ll[2], geo);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int launch_edge_fwd_bf16(const Model& m, const EdgeArgs& a, cudaStream_t st, int num_sms) {
    if (!(m.d.F == TF && m.d.lmax == TLMAX) || !a.w->W3sw || !a.err || !a.sched || !a.geo)
        return MP_ERR_UNSUPPORTED;
    if (a.n == 0) return MP_OK;
    if (a.first && a.vfirst && a.species && a.emb && a.n_species >= 1 && a.n_species <= SMAX0) {
        // layer 0 by hidden unit: G per row (scratch a.vfirst), then A from G
        int rc = MP_OK;
        switch (a.n_species) {
            case 1: rc = launch_tc<SmemF0<1>, F0Cfg<1>::NWG>(k_edge_fwd0_tc<1>, a, RPG_F, num_sms, st); break;
            case 2: rc = launch_tc<SmemF0<2>, F0Cfg<2>::NWG>(k_edge_fwd0_tc<2>, a, RPG_F, num_sms, st); break;
            default: rc = launch_tc<SmemF0<3>, F0Cfg<3>::NWG>(k_edge_fwd0_tc<3>, a, RPG_F, num_sms, st); break;
        }
        if (rc != MP_OK) return rc;
        const int64_t tiles = (a.n + AF_NT - 1) / AF_NT;
        const int grid = (int)(tiles < num_sms ? tiles : num_sms);
        auto run = [&](auto kernel, size_t smem) -> int {
            MP_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            kernel<<<grid, AF_NTH, smem, st>>>(a.n, a.vfirst, a.emb, a.w->W3sw, a.k.inv_navg,
                                               a.Aout, tiles, a.err);
            note_launch();
            MP_CUDA_TRY(cudaGetLastError());
            return MP_OK;
        };
        switch (a.n_species) {
            case 1: return run(k_a_first_tc<1>, sizeof(AfSmem<1>) + 1024);
            case 2: return run(k_a_first_tc<2>, sizeof(AfSmem<2>) + 1024);
            default: return run(k_a_first_tc<3>, sizeof(AfSmem<3>) + 1024);
        }
    }
    return a.first
               ? launch_tc<SmemF<true>, FwdCfg<true>::NWG>(k_edge_fwd_tc<true>, a, RPG_F, num_sms, st)
               : launch_tc<SmemF<false>, FwdCfg<false>::NWG>(k_edge_fwd_tc<false>, a, RPG_F,
                                                            num_sms, st);
}

int launch_edge_bwd_bf16(const Model& m, const EdgeArgs& a, cudaStream_t st, int num_sms) {
    if (!(m.d.F == TF && m.d.lmax == TLMAX) || !a.w->W3sw || !a.err || !a.sched || !a.geo)
        return MP_ERR_UNSUPPORTED;
    if (a.n == 0) return MP_OK;
    if (a.first && a.vfirst && a.species && a.emb && a.n_species >= 1) {
        // layer 0 by hidden unit: V for the rows with a nonzero adjoint, zero
        // for the rest, then the edge pass
        const int64_t nv = a.n_recv > 0 ? a.n_recv : a.n;
        const size_t per_atom = (size_t)a.n_species * TNLM * kH;
        if (nv < a.n)
            MP_CUDA_TRY(cudaMemsetAsync(a.vfirst + (size_t)nv * per_atom, 0,
                                        sizeof(float) * (size_t)(a.n - nv) * per_atom, st));
        if (nv > 0) {
            const size_t vsm = sizeof(VSmem);
            MP_CUDA_TRY(cudaFuncSetAttribute(k_v_first, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)vsm));
            const int64_t tiles = (nv + VTA - 1) / VTA;
            const int grid = (int)(tiles < num_sms ? tiles : num_sms);
            k_v_first<<<grid, VTH, vsm, st>>>(nv, a.Alpha, a.emb, a.n_species, a.w->W3b, a.vfirst);
            note_launch();
            MP_CUDA_TRY(cudaGetLastError());
        }
        return a.vir ? launch_tc<SmemB0<true>, Bwd0Cfg<true>::NWG>(k_edge_bwd0_tc<true>, a, RPG_B,
                                                                     num_sms, st)
                     : launch_tc<SmemB0<false>, Bwd0Cfg<false>::NWG>(k_edge_bwd0_tc<false>, a,
                                                                       RPG_B, num_sms, st);
    }
    // layer 0 runs only by hidden unit (above), which needs the scratch
    if (a.first) return MP_ERR_UNSUPPORTED;
    return a.vir ? launch_tc<SmemB<true>, BwdCfg<true>::NWG>(k_edge_bwd_tc<true>, a, RPG_B,
                                                             num_sms, st)
                 : launch_tc<SmemB<false>, BwdCfg<false>::NWG>(k_edge_bwd_tc<false>, a, RPG_B,
                                                               num_sms, st);
}

}  // namespace mp

// Multilevel k-way graph partitioner for Stage 1 on heterogeneous systems
// (Methods, "Graph Partitioning": for nanoparticles on supports a METIS-like
// multilevel partitioner replaces the spatial grid, giving balanced, compact
// subgraphs at near-linear cost; Supplementary S1, Figs. S1-S2).
//
// The atom graph (unit vertex and edge weights) is
//  1. coarsened level by level on the GPU: a heavy-edge matching (each
//     unmatched vertex proposes to the unmatched neighbour across its
//     heaviest edge; ties are broken by a hash of the pair, so an edge has
//     the same priority from both ends and mutual proposals exist in every
//     round; a pair whose weight would exceed a cap stays unmatched), then
//     contraction (vertex weights added; the merged neighbour lists sorted
//     per coarse vertex, self loops dropped, parallel edges merged with their
//     weights added);
//  2. split on the host at the coarsest level by recursive bisection, each
//     bisection grown greedily from a pseudo-peripheral start vertex (the
//     vertex with the largest gain joins next), the best of several starts
//     by cut;
//  3. projected back level by level with k-way boundary refinement on the
//     GPU at every level: each vertex proposes its best move to a
//     neighbouring part; a proposal survives only if it still gains when
//     every neighbour that outranks it (larger gain, then smaller index)
//     makes its own move; a receiving part admits moves, best gain buckets
//     first, only while it stays under the weight bound (1 + imbalance) W/k.
//     A part above the bound first sheds its cheapest boundary vertices.
// All arithmetic is on integers in an order-independent way, so the result
// depends only on the graph and the seed.
#include <algorithm>
#include <cmath>
#include <queue>
#include <vector>

#include "common.cuh"

namespace mp {

namespace {

constexpr int kMaxParts = 64;       // bound of the API (bucket tables are per part)
constexpr int kBuckets = 64;        // gain buckets per part
constexpr int kNbrParts = 8;        // distinct neighbouring parts tracked per vertex
constexpr int kMatchRounds = 8;
constexpr int kRefineRounds = 12;
constexpr int kContractThreads = 128;
constexpr int kMaxSortKeys = 16384; // per coarse vertex (128 KB of shared memory)

// splitmix64 (Steele, Lea and Flood), used as an integer hash.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ int vweight(const int32_t* vw, int u) { return vw ? vw[u] : 1; }
__device__ __forceinline__ int eweight(const int32_t* ew, int64_t e) { return ew ? ew[e] : 1; }

// ---- coarsening ----------------------------------------------------------

__global__ void k_propose(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                          const int32_t* __restrict__ ew, const int32_t* __restrict__ vw, int n,
                          const int32_t* __restrict__ match, int cap, uint64_t salt,
                          int32_t* __restrict__ prop) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    if (match[u] >= 0) {
        prop[u] = -1;
        return;
    }
    const int wu = vweight(vw, u);
    int best = -1;
    uint64_t bkey = 0, bpair = 0;
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        const int v = col[e];
        if (v == u || match[v] >= 0 || wu + vweight(vw, v) > cap) continue;
        const uint64_t pair = ((uint64_t)(uint32_t)min(u, v) << 32) | (uint32_t)max(u, v);
        const uint64_t key =
            ((uint64_t)(uint32_t)eweight(ew, e) << 32) | (mix64(salt ^ pair) >> 32);
        if (best < 0 || key > bkey || (key == bkey && pair > bpair)) {
            best = v;
            bkey = key;
            bpair = pair;
        }
    }
    prop[u] = best;
}

__global__ void k_accept(int n, const int32_t* __restrict__ prop, int32_t* __restrict__ match) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n || match[u] >= 0) return;
    const int v = prop[u];
    if (v >= 0 && prop[v] == u) match[u] = v;
}

// Leader of a pair = its smaller vertex; an unmatched vertex leads itself.
__global__ void k_leader_flag(int n, const int32_t* __restrict__ match, int32_t* __restrict__ flag) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int m = match[u];
    flag[u] = (m < 0 || u < m) ? 1 : 0;
}

__global__ void k_cmap(int n, const int32_t* __restrict__ match, const int32_t* __restrict__ pre,
                       int32_t* __restrict__ cmap, int32_t* __restrict__ lead) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int m = match[u];
    const int l = (m < 0 || u < m) ? u : m;
    cmap[u] = pre[l];
    if (l == u) lead[pre[u]] = u;
}

// Coarse vertex c: weight and the length of its members' joint edge list.
__global__ void k_cinfo(int nc, const int32_t* __restrict__ lead, const int32_t* __restrict__ match,
                        const int64_t* __restrict__ rp, const int32_t* __restrict__ vw,
                        int32_t* __restrict__ cvw, int32_t* __restrict__ dsz,
                        int* __restrict__ dmax) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int u = lead[c], v = match[u];
    int d = (int)(rp[u + 1] - rp[u]);
    int w = vweight(vw, u);
    if (v >= 0) {
        d += (int)(rp[v + 1] - rp[v]);
        w += vweight(vw, v);
    }
    dsz[c] = d;
    cvw[c] = w;
    atomicMax(dmax, d);
}

// One block per coarse vertex: keys (coarse neighbour << 32 | edge weight)
// of both members' edges, self loops replaced by the sentinel, bitonic sort
// in shared memory, then runs of equal neighbours summed in order.
__global__ void __launch_bounds__(kContractThreads) k_contract(
    const int32_t* __restrict__ lead, const int32_t* __restrict__ match,
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const int32_t* __restrict__ ew,
    const int32_t* __restrict__ cmap, const int64_t* __restrict__ off, int32_t* __restrict__ scol,
    int32_t* __restrict__ sw, int32_t* __restrict__ ucnt) {
    extern __shared__ uint64_t keys[];
    const int c = blockIdx.x;
    const int u = lead[c], v = match[u];
    const int64_t du = rp[u + 1] - rp[u];
    const int D = (int)(off[c + 1] - off[c]);
    int P = 1;
    while (P < D) P <<= 1;
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
        uint64_t k = ~0ull;
        if (q < D) {
            const int64_t e = q < du ? rp[u] + q : rp[v] + (q - du);
            const int t = cmap[col[e]];
            if (t != c) k = ((uint64_t)(uint32_t)t << 32) | (uint32_t)eweight(ew, e);
        }
        keys[q] = k;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = keys[i], b = keys[ixj];
                    if ((a > b) == ((i & k) == 0)) {
                        keys[i] = b;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    if (threadIdx.x == 0) {
        const int64_t base = off[c];
        int cnt = 0, q = 0;
        while (q < P && keys[q] != ~0ull) {
            const uint32_t t = (uint32_t)(keys[q] >> 32);
            uint32_t w = 0;
            while (q < P && keys[q] != ~0ull && (uint32_t)(keys[q] >> 32) == t) {
                w += (uint32_t)keys[q];
                ++q;
            }
            scol[base + cnt] = (int32_t)t;
            sw[base + cnt] = (int32_t)w;
            ++cnt;
        }
        ucnt[c] = cnt;
    }
}

__global__ void k_compact(int nc, const int64_t* __restrict__ off, const int32_t* __restrict__ ucnt,
                          const int64_t* __restrict__ crp, const int32_t* __restrict__ scol,
                          const int32_t* __restrict__ sw, int32_t* __restrict__ ccol,
                          int32_t* __restrict__ cew) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (int)(t >> 5), lane = (int)(t & 31);
    if (c >= nc) return;
    const int64_t src = off[c], dst = crp[c];
    for (int q = lane; q < ucnt[c]; q += 32) {
        ccol[dst + q] = scol[src + q];
        cew[dst + q] = sw[src + q];
    }
}

// ---- refinement ------------------------------------------------------------

__device__ __forceinline__ int gain_bucket(int g) {
    if (g > 0) return 32 + min(30, 31 - __clz(g));
    if (g == 0) return 31;
    return 30 - min(30, 31 - __clz(-g));
}

// Connectivity of u to its own part and its best admissible other part
// (room for u's weight; ties to the smaller part id).
__device__ __forceinline__ void best_move(const int64_t* __restrict__ rp,
                                          const int32_t* __restrict__ col,
                                          const int32_t* __restrict__ ew,
                                          const int32_t* __restrict__ part,
                                          const int64_t* __restrict__ room, int u, int own, int wu,
                                          int& c_own, int& q_best, int& c_best) {
    int pid[kNbrParts], pc[kNbrParts], np = 0;
    c_own = 0;
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        const int q = part[col[e]];
        const int w = eweight(ew, e);
        if (q == own) {
            c_own += w;
            continue;
        }
        int k = 0;
        while (k < np && pid[k] != q) ++k;
        if (k < np) {
            pc[k] += w;
        } else if (np < kNbrParts) {
            pid[np] = q;
            pc[np] = w;
            ++np;
        }
    }
    q_best = -1;
    c_best = 0;
    for (int k = 0; k < np; ++k) {
        if (room[pid[k]] < wu) continue;
        if (q_best < 0 || pc[k] > c_best || (pc[k] == c_best && pid[k] < q_best)) {
            q_best = pid[k];
            c_best = pc[k];
        }
    }
}

// mode 0 (refine): positive-gain moves.  mode 1 (balance): the best move of
// every boundary vertex of a part above the bound, whatever its gain.
__global__ void k_select(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const int32_t* __restrict__ ew, const int32_t* __restrict__ vw, int n,
                         const int32_t* __restrict__ part, const int64_t* __restrict__ room,
                         const int64_t* __restrict__ over, int mode, int32_t* __restrict__ dest,
                         int32_t* __restrict__ gain) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int own = part[u];
    int q = -1, g = 0;
    if (mode == 0 || over[own] > 0) {
        int c_own, c_best;
        best_move(rp, col, ew, part, room, u, own, vweight(vw, u), c_own, q, c_best);
        g = c_best - c_own;
        if (q >= 0 && mode == 0 && g <= 0) q = -1;
    }
    dest[u] = q;
    gain[u] = g;
}

// A proposal survives if it still gains when every neighbour that outranks
// it (larger gain, then smaller index) has made its own proposed move.
__global__ void k_afterburn(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ ew, int n, const int32_t* __restrict__ part,
                            const int32_t* __restrict__ dest, const int32_t* __restrict__ gain,
                            int32_t* __restrict__ dest2, int32_t* __restrict__ gain2) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int q = dest[u];
    if (q < 0) {
        dest2[u] = -1;
        gain2[u] = 0;
        return;
    }
    const int own = part[u], gu = gain[u];
    int c_own = 0, c_q = 0;
    for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
        const int v = col[e];
        int pv = part[v];
        const int dv = dest[v];
        if (dv >= 0 && (gain[v] > gu || (gain[v] == gu && v < u))) pv = dv;
        const int w = eweight(ew, e);
        if (pv == own) c_own += w;
        else if (pv == q) c_q += w;
    }
    const int g = c_q - c_own;
    dest2[u] = g > 0 ? q : -1;
    gain2[u] = g;
}

__global__ void k_hist(int n, const int32_t* __restrict__ vw, const int32_t* __restrict__ part,
                       const int32_t* __restrict__ dest, const int32_t* __restrict__ gain,
                       unsigned long long* __restrict__ hin, unsigned long long* __restrict__ hout) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int q = dest[u];
    if (q < 0) return;
    const int b = gain_bucket(gain[u]);
    const unsigned long long w = (unsigned long long)vweight(vw, u);
    atomicAdd(&hin[q * kBuckets + b], w);
    atomicAdd(&hout[part[u] * kBuckets + b], w);
}

// Thresholds: part q admits buckets >= tin[q] (the best buckets that fit in
// its room); a part above the bound releases buckets >= tout[p] (the best
// buckets that cover its excess).
__global__ void k_thresh(int k, const unsigned long long* __restrict__ hin,
                         const unsigned long long* __restrict__ hout,
                         const int64_t* __restrict__ room, const int64_t* __restrict__ over,
                         int32_t* __restrict__ tin, int32_t* __restrict__ tout) {
    const int q = threadIdx.x;
    if (q >= k) return;
    int64_t cum = 0;
    int t = 0;
    for (int b = kBuckets - 1; b >= 0; --b) {
        const int64_t h = (int64_t)hin[q * kBuckets + b];
        if (cum + h > room[q]) {
            t = b + 1;
            break;
        }
        cum += h;
    }
    tin[q] = t;
    t = 0;
    cum = 0;
    if (over[q] > 0) {
        for (int b = kBuckets - 1; b >= 0; --b) {
            cum += (int64_t)hout[q * kBuckets + b];
            if (cum >= over[q]) {
                t = b;
                break;
            }
        }
    }
    tout[q] = t;
}

__global__ void k_apply(int n, int mode, const int32_t* __restrict__ dest,
                        const int32_t* __restrict__ gain, const int32_t* __restrict__ tin,
                        const int32_t* __restrict__ tout, int32_t* __restrict__ part,
                        unsigned long long* __restrict__ moved) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int q = dest[u];
    if (q < 0) return;
    const int b = gain_bucket(gain[u]);
    if (b < tin[q] || (mode == 1 && b < tout[part[u]])) return;
    part[u] = q;
    atomicAdd(moved, 1ull);
}

__global__ void k_part_weight(int n, const int32_t* __restrict__ vw,
                              const int32_t* __restrict__ part, unsigned long long* __restrict__ pw) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    atomicAdd(&pw[part[u]], (unsigned long long)vweight(vw, u));
}

__global__ void k_room(int k, const unsigned long long* __restrict__ pw, int64_t maxw,
                       int64_t* __restrict__ room, int64_t* __restrict__ over) {
    const int q = threadIdx.x;
    if (q >= k) return;
    const int64_t w = (int64_t)pw[q];
    room[q] = maxw - w;
    over[q] = w - maxw;
}

__global__ void k_project(int n, const int32_t* __restrict__ cmap,
                          const int32_t* __restrict__ coarse, int32_t* __restrict__ fine) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    fine[u] = coarse[cmap[u]];
}

__global__ void k_cut(const int64_t* __restrict__ rp, const int32_t* __restrict__ col, int n,
                      const int32_t* __restrict__ part, unsigned long long* __restrict__ cut) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long c = 0;
    if (u < n) {
        const int pu = part[u];
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) c += part[col[e]] != pu;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cut, c);
}

__global__ void k_scatter_out(int n, const int32_t* __restrict__ perm,
                              const int32_t* __restrict__ part, int32_t* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    out[perm[s]] = part[s];
}

// ---- host: recursive bisection of the coarsest graph ----------------------

struct HostGraph {
    int n = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> col, ew, vw;
};

// Last vertex reached by a breadth-first search from s inside the subset
// (loc >= 0): a pseudo-peripheral start for growing a region.
int bfs_last(const HostGraph& G, const std::vector<int32_t>& loc, int s, std::vector<int>& seen,
             int stamp) {
    std::vector<int> queue{s};
    seen[s] = stamp;
    size_t h = 0;
    int last = s;
    while (h < queue.size()) {
        const int u = queue[h++];
        last = u;
        for (int64_t e = G.rp[u]; e < G.rp[u + 1]; ++e) {
            const int v = G.col[e];
            if (loc[v] < 0 || seen[v] == stamp) continue;
            seen[v] = stamp;
            queue.push_back(v);
        }
    }
    return last;
}

void bisect(const HostGraph& G, const std::vector<int32_t>& verts, int k, int part0, uint64_t seed,
            int depth, std::vector<int32_t>& loc, std::vector<int>& seen, int& stamp,
            std::vector<int32_t>& part) {
    if (verts.empty()) return;
    if (k == 1) {
        for (int v : verts) part[v] = part0;
        return;
    }
    const int nv = (int)verts.size();
    for (int i = 0; i < nv; ++i) loc[verts[i]] = i;
    int64_t W = 0;
    for (int v : verts) W += G.vw[v];
    const int kA = k / 2;
    const int64_t tA = W * kA / k;
    std::vector<int64_t> gain(nv);
    std::vector<char> inA(nv), bestA;
    int64_t best_cut = -1;
    const int trials = 8;
    for (int t = 0; t < trials; ++t) {
        const int s0 = verts[mix64(seed ^ ((uint64_t)depth << 32) ^ (uint64_t)(part0 << 8) ^ t) % nv];
        const int start = bfs_last(G, loc, s0, seen, ++stamp);
        std::fill(inA.begin(), inA.end(), 0);
        for (int i = 0; i < nv; ++i) {
            const int u = verts[i];
            int64_t g = 0;
            for (int64_t e = G.rp[u]; e < G.rp[u + 1]; ++e)
                if (loc[G.col[e]] >= 0) g -= G.ew[e];
            gain[i] = g;
        }
        std::priority_queue<std::pair<int64_t, int>> heap;
        heap.push({gain[loc[start]], loc[start]});
        int64_t wA = 0;
        int next_free = 0;
        while (wA < tA) {
            if (heap.empty()) {   // region exhausted (disconnected subset): restart
                while (next_free < nv && inA[next_free]) ++next_free;
                if (next_free == nv) break;
                heap.push({gain[next_free], next_free});
            }
            const auto top = heap.top();
            heap.pop();
            const int i = top.second;
            if (inA[i] || top.first != gain[i]) continue;
            const int u = verts[i];
            if (wA + G.vw[u] > tA && wA + G.vw[u] - tA > tA - wA) break;
            inA[i] = 1;
            wA += G.vw[u];
            for (int64_t e = G.rp[u]; e < G.rp[u + 1]; ++e) {
                const int j = loc[G.col[e]];
                if (j < 0 || inA[j]) continue;
                gain[j] += 2 * (int64_t)G.ew[e];
                heap.push({gain[j], j});
            }
        }
        int64_t cut = 0;
        for (int i = 0; i < nv; ++i) {
            if (!inA[i]) continue;
            const int u = verts[i];
            for (int64_t e = G.rp[u]; e < G.rp[u + 1]; ++e) {
                const int j = loc[G.col[e]];
                if (j >= 0 && !inA[j]) cut += G.ew[e];
            }
        }
        if (best_cut < 0 || cut < best_cut) {
            best_cut = cut;
            bestA = inA;
        }
    }
    std::vector<int32_t> A, B;
    for (int i = 0; i < nv; ++i) (bestA[i] ? A : B).push_back(verts[i]);
    for (int v : verts) loc[v] = -1;
    bisect(G, A, kA, part0, seed, depth + 1, loc, seen, stamp, part);
    bisect(G, B, k - kA, part0 + kA, seed, depth + 1, loc, seen, stamp, part);
}

struct Level {
    int n = 0;
    int64_t m = 0;
    const int64_t* rp = nullptr;
    const int32_t* col = nullptr;
    const int32_t* ew = nullptr;   // nullptr = unit weights
    const int32_t* vw = nullptr;   // nullptr = unit weights
    DevBuf brp, bcol, bew, bvw;    // storage of coarse levels
    DevBuf cmap;                   // this level -> next coarser
    DevBuf part;
    void release() {
        DevBuf* all[] = {&brp, &bcol, &bew, &bvw, &cmap, &part};
        for (DevBuf* b : all) b->release();
    }
};

// Owns the level stack; capacity is reserved up front so references to
// levels stay valid while coarser ones are appended.
struct LevelStack {
    std::vector<Level> lv;
    explicit LevelStack(size_t cap) { lv.reserve(cap); }
    LevelStack(const LevelStack&) = delete;
    LevelStack& operator=(const LevelStack&) = delete;
    ~LevelStack() {
        for (Level& L : lv) L.release();
    }
};

}  // namespace

int graph_partition(mp_ctx* ctx, const Graph& g, int k, double imbalance, uint64_t seed,
                    int32_t* d_out, int64_t* cut_out) {
    if (k < 1 || k > kMaxParts || !(imbalance >= 0.0) || !d_out || g.n < k || g.n > INT32_MAX)
        return MP_ERR_ARG;
    cudaStream_t st = ctx->stream;
    const int n0 = (int)g.n;
    if (k == 1) {   // one part: every atom in part 0, nothing cut
        MP_CUDA_TRY(cudaMemsetAsync(d_out, 0, sizeof(int32_t) * n0, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        if (cut_out) *cut_out = 0;
        return MP_OK;
    }
    const int64_t W = n0;
    int64_t maxw = (int64_t)std::floor((1.0 + imbalance) * (double)W / k);
    maxw = std::max<int64_t>(maxw, (W + k - 1) / k);
    const int coarsen_to = std::max(1024, 128 * k);
    const int cap = std::max(2, (int)(1.5 * (double)W / coarsen_to));

    constexpr int kMaxLevels = 40;
    LevelStack stack(kMaxLevels + 1);
    std::vector<Level>& lv = stack.lv;
    lv.emplace_back();
    lv[0].n = n0;
    lv[0].m = g.n_edges;
    lv[0].rp = g.row_ptr.as<int64_t>();
    lv[0].col = g.col.as<int32_t>();

    // scratch sized for level 0
    DevBuf bmatch, bprop, bflag, bpre, blead, bdsz, boff, bucnt, bscol, bsw, bsmall;
    DevBuf bdest, bgain, bdest2, bgain2;
    BufGuard guard{&bmatch, &bprop, &bflag, &bpre, &blead, &bdsz, &boff, &bucnt, &bscol, &bsw,
                   &bsmall, &bdest, &bgain, &bdest2, &bgain2};
    MP_TRY(bmatch.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(bprop.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(bflag.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(bpre.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(blead.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(bdsz.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(boff.reserve(sizeof(int64_t) * (n0 + 1)));
    MP_TRY(bucnt.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(bscol.reserve(sizeof(int32_t) * (g.n_edges + 1)));
    MP_TRY(bsw.reserve(sizeof(int32_t) * (g.n_edges + 1)));
    // small: dmax, counters, histograms, thresholds, room/over
    const size_t small_bytes = 64 + sizeof(unsigned long long) * (2 * kMaxParts * kBuckets + kMaxParts + 4) +
                               sizeof(int64_t) * 2 * kMaxParts + sizeof(int32_t) * 2 * kMaxParts;
    MP_TRY(bsmall.reserve(small_bytes));
    int* d_dmax = bsmall.as<int>();
    unsigned long long* d_cnt = reinterpret_cast<unsigned long long*>(bsmall.as<char>() + 64);
    unsigned long long* d_hin = d_cnt + 4;
    unsigned long long* d_hout = d_hin + kMaxParts * kBuckets;
    unsigned long long* d_pw = d_hout + kMaxParts * kBuckets;
    int64_t* d_room = reinterpret_cast<int64_t*>(d_pw + kMaxParts);
    int64_t* d_over = d_room + kMaxParts;
    int32_t* d_tin = reinterpret_cast<int32_t*>(d_over + kMaxParts);
    int32_t* d_tout = d_tin + kMaxParts;
    int32_t* match = bmatch.as<int32_t>();
    int32_t* prop = bprop.as<int32_t>();

    // 1. coarsening
    while (lv.back().n > coarsen_to && (int)lv.size() < kMaxLevels) {
        Level& f = lv.back();
        const int n = f.n;
        MP_CUDA_TRY(cudaMemsetAsync(match, 0xFF, sizeof(int32_t) * n, st));
        for (int r = 0; r < kMatchRounds; ++r) {
            const uint64_t salt = mix64(seed ^ ((uint64_t)lv.size() << 40) ^ (uint64_t)r);
            k_propose<<<grid_for(n, 256), 256, 0, st>>>(f.rp, f.col, f.ew, f.vw, n, match, cap,
                                                        salt, prop);
            note_launch();
            k_accept<<<grid_for(n, 256), 256, 0, st>>>(n, prop, match);
            note_launch();
        }
        k_leader_flag<<<grid_for(n, 256), 256, 0, st>>>(n, match, bflag.as<int32_t>());
        note_launch();
        MP_TRY(exclusive_scan_i32(bflag.as<int32_t>(), bpre.as<int32_t>(), n, ctx->ws.tmp, st));
        int nc = 0;
        MP_CUDA_TRY(cudaMemcpyAsync(&nc, bpre.as<int32_t>() + n, sizeof(int), cudaMemcpyDeviceToHost,
                                    st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        if (nc == n) break;   // nothing matched
        MP_TRY(f.cmap.reserve(sizeof(int32_t) * (n + 1)));
        k_cmap<<<grid_for(n, 256), 256, 0, st>>>(n, match, bpre.as<int32_t>(), f.cmap.as<int32_t>(),
                                                 blead.as<int32_t>());
        note_launch();
        lv.emplace_back();   // no reallocation: capacity reserved, f stays valid
        Level& c = lv.back();
        c.n = nc;
        MP_TRY(c.bvw.reserve(sizeof(int32_t) * (nc + 1)));
        MP_CUDA_TRY(cudaMemsetAsync(d_dmax, 0, sizeof(int), st));
        k_cinfo<<<grid_for(nc, 256), 256, 0, st>>>(nc, blead.as<int32_t>(), match, f.rp, f.vw,
                                                   c.bvw.as<int32_t>(), bdsz.as<int32_t>(), d_dmax);
        note_launch();
        MP_TRY(exclusive_scan_i64(bdsz.as<int32_t>(), boff.as<int64_t>(), nc, ctx->ws.tmp, st));
        int dmax = 0;
        MP_CUDA_TRY(cudaMemcpyAsync(&dmax, d_dmax, sizeof(int), cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        if (dmax > kMaxSortKeys) return MP_ERR_UNSUPPORTED;
        int P = 1;
        while (P < dmax) P <<= 1;
        const int smem = (int)sizeof(uint64_t) * P;
        MP_CUDA_TRY(cudaFuncSetAttribute(k_contract, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         std::max(smem, 48 * 1024)));
        k_contract<<<nc, kContractThreads, smem, st>>>(blead.as<int32_t>(), match, f.rp, f.col,
                                                       f.ew, f.cmap.as<int32_t>(),
                                                       boff.as<int64_t>(), bscol.as<int32_t>(),
                                                       bsw.as<int32_t>(), bucnt.as<int32_t>());
        note_launch();
        MP_TRY(c.brp.reserve(sizeof(int64_t) * (nc + 1)));
        MP_TRY(exclusive_scan_i64(bucnt.as<int32_t>(), c.brp.as<int64_t>(), nc, ctx->ws.tmp, st));
        MP_CUDA_TRY(cudaMemcpyAsync(&c.m, c.brp.as<int64_t>() + nc, sizeof(int64_t),
                                    cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        MP_TRY(c.bcol.reserve(sizeof(int32_t) * (c.m + 1)));
        MP_TRY(c.bew.reserve(sizeof(int32_t) * (c.m + 1)));
        k_compact<<<grid_for((int64_t)nc * 32, 256), 256, 0, st>>>(
            nc, boff.as<int64_t>(), bucnt.as<int32_t>(), c.brp.as<int64_t>(), bscol.as<int32_t>(),
            bsw.as<int32_t>(), c.bcol.as<int32_t>(), c.bew.as<int32_t>());
        note_launch();
        c.rp = c.brp.as<int64_t>();
        c.col = c.bcol.as<int32_t>();
        c.ew = c.bew.as<int32_t>();
        c.vw = c.bvw.as<int32_t>();
        if ((double)nc > 0.95 * (double)n) break;   // matching has stalled (isolated or capped vertices)
    }

    // 2. initial partition of the coarsest graph on the host
    {
        Level& c = lv.back();
        HostGraph G;
        G.n = c.n;
        G.rp.resize(c.n + 1);
        G.col.resize(c.m);
        G.ew.assign(c.m, 1);
        G.vw.assign(c.n, 1);
        MP_CUDA_TRY(cudaMemcpyAsync(G.rp.data(), c.rp, sizeof(int64_t) * (c.n + 1),
                                    cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaMemcpyAsync(G.col.data(), c.col, sizeof(int32_t) * c.m,
                                    cudaMemcpyDeviceToHost, st));
        if (c.ew)
            MP_CUDA_TRY(cudaMemcpyAsync(G.ew.data(), c.ew, sizeof(int32_t) * c.m,
                                        cudaMemcpyDeviceToHost, st));
        if (c.vw)
            MP_CUDA_TRY(cudaMemcpyAsync(G.vw.data(), c.vw, sizeof(int32_t) * c.n,
                                        cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        std::vector<int32_t> verts(c.n), loc(c.n, -1), part(c.n, 0);
        std::vector<int> seen(c.n, 0);
        int stamp = 0;
        for (int i = 0; i < c.n; ++i) verts[i] = i;
        bisect(G, verts, k, 0, seed, 0, loc, seen, stamp, part);
        MP_TRY(c.part.reserve(sizeof(int32_t) * (c.n + 1)));
        MP_CUDA_TRY(cudaMemcpyAsync(c.part.as<int32_t>(), part.data(), sizeof(int32_t) * c.n,
                                    cudaMemcpyHostToDevice, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));   // host vector goes out of scope
    }

    // 3. refinement, coarsest to finest
    MP_TRY(bdest.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(bgain.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(bdest2.reserve(sizeof(int32_t) * (n0 + 1)));
    MP_TRY(bgain2.reserve(sizeof(int32_t) * (n0 + 1)));
    auto weights = [&](const Level& L) -> int {
        MP_CUDA_TRY(cudaMemsetAsync(d_pw, 0, sizeof(unsigned long long) * k, st));
        k_part_weight<<<grid_for(L.n, 256), 256, 0, st>>>(L.n, L.vw, L.part.as<int32_t>(), d_pw);
        note_launch();
        k_room<<<1, kMaxParts, 0, st>>>(k, d_pw, maxw, d_room, d_over);
        note_launch();
        return MP_OK;
    };
    auto refine = [&](Level& L) -> int {
        MP_TRY(weights(L));
        std::vector<int64_t> h_over(k);
        MP_CUDA_TRY(cudaMemcpyAsync(h_over.data(), d_over, sizeof(int64_t) * k,
                                    cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        int balance_rounds = 0;
        for (int r = 0; r < kRefineRounds; ++r) {
            const bool unbalanced = *std::max_element(h_over.begin(), h_over.end()) > 0;
            const int mode = unbalanced && balance_rounds < kRefineRounds / 2 ? 1 : 0;
            balance_rounds += mode;
            int32_t *dest = bdest.as<int32_t>(), *gain = bgain.as<int32_t>();
            k_select<<<grid_for(L.n, 256), 256, 0, st>>>(L.rp, L.col, L.ew, L.vw, L.n,
                                                         L.part.as<int32_t>(), d_room, d_over, mode,
                                                         dest, gain);
            note_launch();
            if (mode == 0) {
                k_afterburn<<<grid_for(L.n, 256), 256, 0, st>>>(L.rp, L.col, L.ew, L.n,
                                                                L.part.as<int32_t>(), dest, gain,
                                                                bdest2.as<int32_t>(),
                                                                bgain2.as<int32_t>());
                note_launch();
                dest = bdest2.as<int32_t>();
                gain = bgain2.as<int32_t>();
            }
            MP_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) *
                                                      (4 + 2 * kMaxParts * kBuckets), st));
            k_hist<<<grid_for(L.n, 256), 256, 0, st>>>(L.n, L.vw, L.part.as<int32_t>(), dest, gain,
                                                       d_hin, d_hout);
            note_launch();
            k_thresh<<<1, kMaxParts, 0, st>>>(k, d_hin, d_hout, d_room, d_over, d_tin, d_tout);
            note_launch();
            k_apply<<<grid_for(L.n, 256), 256, 0, st>>>(L.n, mode, dest, gain, d_tin, d_tout,
                                                        L.part.as<int32_t>(), d_cnt);
            note_launch();
            MP_TRY(weights(L));
            unsigned long long moved = 0;
            MP_CUDA_TRY(cudaMemcpyAsync(&moved, d_cnt, sizeof(moved), cudaMemcpyDeviceToHost, st));
            MP_CUDA_TRY(cudaMemcpyAsync(h_over.data(), d_over, sizeof(int64_t) * k,
                                        cudaMemcpyDeviceToHost, st));
            MP_CUDA_TRY(cudaStreamSynchronize(st));
            if (moved == 0 && mode == 0) break;
        }
        return MP_OK;
    };
    MP_TRY(refine(lv.back()));
    for (int l = (int)lv.size() - 2; l >= 0; --l) {
        Level& f = lv[l];
        MP_TRY(f.part.reserve(sizeof(int32_t) * (f.n + 1)));
        k_project<<<grid_for(f.n, 256), 256, 0, st>>>(f.n, f.cmap.as<int32_t>(),
                                                      lv[l + 1].part.as<int32_t>(),
                                                      f.part.as<int32_t>());
        note_launch();
        MP_TRY(refine(f));
    }
    // Exact balance on the atom graph: if a part is still above the bound,
    // its vertices with the best admissible moves (largest gain, then
    // smallest index) move on the host, exactly as many as the excess, to
    // parts with room; vertices without a neighbouring part that has room
    // move, in index order, to the part with the most room.  Total room is
    // at least the total excess, so this ends balanced.
    {
        Level& L = lv[0];
        MP_TRY(weights(L));
        std::vector<int64_t> h_over(k);
        MP_CUDA_TRY(cudaMemcpyAsync(h_over.data(), d_over, sizeof(int64_t) * k,
                                    cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        if (*std::max_element(h_over.begin(), h_over.end()) > 0) {
            int32_t* dest = bdest.as<int32_t>();
            int32_t* gain = bgain.as<int32_t>();
            k_select<<<grid_for(L.n, 256), 256, 0, st>>>(L.rp, L.col, L.ew, L.vw, L.n,
                                                         L.part.as<int32_t>(), d_room, d_over, 1,
                                                         dest, gain);
            note_launch();
            std::vector<int32_t> h_part(L.n), h_dest(L.n), h_gain(L.n);
            MP_CUDA_TRY(cudaMemcpyAsync(h_part.data(), L.part.as<int32_t>(),
                                        sizeof(int32_t) * L.n, cudaMemcpyDeviceToHost, st));
            MP_CUDA_TRY(cudaMemcpyAsync(h_dest.data(), dest, sizeof(int32_t) * L.n,
                                        cudaMemcpyDeviceToHost, st));
            MP_CUDA_TRY(cudaMemcpyAsync(h_gain.data(), gain, sizeof(int32_t) * L.n,
                                        cudaMemcpyDeviceToHost, st));
            MP_CUDA_TRY(cudaStreamSynchronize(st));
            std::vector<int64_t> room(k);
            for (int q = 0; q < k; ++q) room[q] = -h_over[q];   // unit vertex weights at level 0
            std::vector<std::pair<int64_t, int>> cand;          // (-gain, vertex)
            for (int u = 0; u < L.n; ++u)
                if (h_over[h_part[u]] > 0 && h_dest[u] >= 0) cand.push_back({-(int64_t)h_gain[u], u});
            std::sort(cand.begin(), cand.end());
            for (const auto& cu : cand) {
                const int u = cu.second, p = h_part[u], q = h_dest[u];
                if (h_over[p] <= 0 || room[q] <= 0) continue;
                h_part[u] = q;
                --h_over[p];
                ++h_over[q];
                --room[q];
                ++room[p];
            }
            for (int u = 0; u < L.n; ++u) {
                const int p = h_part[u];
                if (h_over[p] <= 0) continue;
                const int q = (int)(std::max_element(room.begin(), room.end()) - room.begin());
                if (room[q] <= 0 || q == p) break;   // cannot happen: total room >= excess
                h_part[u] = q;
                --h_over[p];
                ++h_over[q];
                --room[q];
                ++room[p];
            }
            MP_CUDA_TRY(cudaMemcpyAsync(L.part.as<int32_t>(), h_part.data(),
                                        sizeof(int32_t) * L.n, cudaMemcpyHostToDevice, st));
            MP_CUDA_TRY(cudaStreamSynchronize(st));   // the host copy goes out of scope
        }
    }
    const int32_t* part0 = lv[0].part.as<int32_t>();
    k_scatter_out<<<grid_for(n0, 256), 256, 0, st>>>(n0, g.perm.as<int32_t>(), part0, d_out);
    note_launch();
    MP_CUDA_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st));
    k_cut<<<grid_for(n0, 256), 256, 0, st>>>(lv[0].rp, lv[0].col, n0, part0, d_cnt);
    note_launch();
    unsigned long long cut2 = 0;
    MP_CUDA_TRY(cudaMemcpyAsync(&cut2, d_cnt, sizeof(cut2), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));   // local buffers are freed on return
    if (cut_out) *cut_out = (int64_t)(cut2 / 2);
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace mp

// Host entry to the coarsest-level step alone: recursive greedy bisection
// of a small graph given as host CSR arrays (no device work).
extern "C" int mp_partition_host_bisect(int n, const int64_t* row_ptr, const int32_t* col,
                                        const int32_t* edge_w, const int32_t* vertex_w,
                                        int n_parts, uint64_t seed, int32_t* part_out) {
    using namespace mp;
    if (n < 0 || n_parts < 1 || (n > 0 && (!row_ptr || !part_out)) ||
        (row_ptr && row_ptr[0] != 0))
        return MP_ERR_ARG;
    if (n == 0) return MP_OK;
    const int64_t m = row_ptr[n];
    if (m < 0 || (m > 0 && !col)) return MP_ERR_ARG;
    // row offsets never decrease, so every row lies inside col[0..m)
    for (int i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return MP_ERR_ARG;
    HostGraph G;
    G.n = n;
    G.rp.assign(row_ptr, row_ptr + n + 1);
    G.col.assign(col, col + m);
    for (int64_t e = 0; e < m; ++e)
        if (G.col[e] < 0 || G.col[e] >= n) return MP_ERR_ARG;
    G.ew = edge_w ? std::vector<int32_t>(edge_w, edge_w + m) : std::vector<int32_t>(m, 1);
    G.vw = vertex_w ? std::vector<int32_t>(vertex_w, vertex_w + n) : std::vector<int32_t>(n, 1);
    for (int32_t v : G.ew)
        if (v < 0) return MP_ERR_ARG;
    for (int32_t v : G.vw)
        if (v < 0) return MP_ERR_ARG;
    std::vector<int32_t> verts(n), loc(n, -1), part(n, 0);
    std::vector<int> seen(n, 0);
    int stamp = 0;
    for (int i = 0; i < n; ++i) verts[i] = i;
    bisect(G, verts, n_parts, 0, seed, 0, loc, seen, stamp, part);
    std::copy(part.begin(), part.end(), part_out);
    return MP_OK;
}

// Spatial-grid partitions with ghost halos and local CSR extraction.
//
// Stage 1 (Methods, "Graph Partitioning"): P uniform bins of the scaled z
// coordinate, root bin = min(floor(x_w,z / L_z * P), P - 1), or the roots a
// caller-given assignment names (a graph partitioner's output).
// Stage 2: every root keeps its K-hop neighbourhood, either by K BFS
// expansions over the global CSR (MP_HALO_BFS) or by the geometric slab
// halo of width K r_c (MP_HALO_GEOM, a superset: each hop is shorter than
// r_c).  The extended set keeps ascending cell order, so each local row holds
// the global row's edges in the same order, filtered to senders in the set.
// Local atoms are ordered by hop class (roots, then atoms within r_c of the
// slab or one hop of a root, ...), each class in Morton order of the cells,
// so the rows a layer needs form a prefix of the local numbering.
#include <algorithm>
#include <utility>
#include <vector>

#include "common.cuh"

namespace mp {

namespace {

__device__ __forceinline__ int root_bin(double z, double L, int P) {
    double f = __ddiv_rn(z, L);
    int b = (int)floor(__dmul_rn(f, (double)P));
    return b < P - 1 ? b : P - 1;
}

// Rows of the extended set: n_ext = cnt[0] + ... + cnt[K] (on the device);
// the grid covers all n atoms and rows l >= n_ext get degree 0.
__device__ __forceinline__ int64_t ext_rows(const int32_t* cnt, int K) {
    int64_t t = 0;
    for (int m = 0; m <= K; ++m) t += cnt[m];
    return t;
}

// Hop class of local row l: rows are placed class by class.
__device__ __forceinline__ int local_class(const int32_t* cnt, int K, int64_t l) {
    int64_t t = 0;
    for (int m = 0; m <= K; ++m) {
        t += cnt[m];
        if (l < t) return m;
    }
    return K + 1;
}

// Local degree of every row, and per class m the number of local edges whose
// two ends are both of class m (esame[m], accumulated).  A warp takes one
// extended row at a time (grid-stride) and reads its global edges 32 at a
// time, so the col and g2l loads of a step are one contiguous segment;
// rows l >= n_ext get degree 0.  The same-class counts are summed per block
// in shared memory (rows come class by class, so a block meets few classes)
// and added to esame once per class and block.
__global__ void __launch_bounds__(256) k_local_deg(
    const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const int32_t* __restrict__ gid, const int32_t* __restrict__ g2l, int64_t n,
    const int32_t* __restrict__ cnt, int K, int32_t* __restrict__ deg,
    unsigned long long* __restrict__ esame) {
    extern __shared__ unsigned long long s_same[];   // K + 1 counters
    for (int m = threadIdx.x; m <= K; m += blockDim.x) s_same[m] = 0ull;
    __syncthreads();
    const int64_t n_ext = ext_rows(cnt, K);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < n_ext;
         l += nwarps) {
        const int m = local_class(cnt, K, l);
        const int s = gid[l];
        const int64_t e1 = row_ptr[s + 1];
        int c = 0, same = 0;
        for (int64_t e = row_ptr[s] + lane; e < e1; e += 32) {
            const int t = g2l[col[e]];
            if (t >= 0) {
                ++c;
                same += local_class(cnt, K, t) == m;
            }
        }
        c = __reduce_add_sync(0xffffffffu, (unsigned)c);
        same = __reduce_add_sync(0xffffffffu, (unsigned)same);
        if (lane == 0) {
            deg[l] = c;
            if (same) atomicAdd(&s_same[m], (unsigned long long)same);
        }
    }
    for (int64_t l = n_ext + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (int64_t)gridDim.x * blockDim.x)
        deg[l] = 0;
    __syncthreads();
    for (int m = threadIdx.x; m <= K; m += blockDim.x)
        if (s_same[m]) atomicAdd(&esame[m], s_same[m]);
}

// The local CSR: each extended row keeps its global edges, in order, whose
// sender is in the extended set (col mapped to the local index).  A warp per
// row (grid-stride), 32 edges per step, compacted by a ballot.
__global__ void __launch_bounds__(256) k_local_fill(
    const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
    const int8_t* __restrict__ shift, const int32_t* __restrict__ gid,
    const int32_t* __restrict__ g2l, const int32_t* __restrict__ cnt, int K,
    const int64_t* __restrict__ lrow, int32_t* __restrict__ lcol, int8_t* __restrict__ lshift) {
    const int64_t n_ext = ext_rows(cnt, K);
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; l < n_ext;
         l += nwarps) {
        const int s = gid[l];
        const int64_t e0 = row_ptr[s], e1 = row_ptr[s + 1];
        int64_t o = lrow[l];
        for (int64_t eb = e0; eb < e1; eb += 32) {
            const int64_t e = eb + lane;
            int t = -1;
            if (e < e1) t = g2l[col[e]];
            const unsigned keep = __ballot_sync(0xffffffffu, t >= 0);
            if (t >= 0) {
                const int64_t q = o + __popc(keep & below);
                lcol[q] = t;
                lshift[q] = shift[e];
            }
            o += __popc(keep);
        }
    }
}

// Hop class of every atom for partition p: 0 = root, m = 1..K = halo atom
// whose z-distance to the slab is below m r_c + s_m and not below
// (m-1) r_c + s_{m-1}, K + 1 = outside the extended set.  s_K = 1e-6 (the
// halo width rule) and s_m = 1e-6 m / K below it: a neighbour of a class-m
// atom is closer than (m+1) r_c + s_m, so it has class <= m + 1 with a
// margin of 1e-6 / K over rounding, and any atom h hops from a root has
// class <= h.
// The slab bounds and class thresholds of partition p, formed on the host
// with the same FP64 operations the definition above gives (lo = L p / P,
// hi = L (p + 1) / P, thr[m - 1] = m r_c + s_m), so that each atom costs one
// division (its root bin) instead of one per threshold.
constexpr int kGeomThr = 16;
struct ClassGeom {
    double lo, hi;
    double thr[kGeomThr];   // m = 1..min(K, kGeomThr); larger m formed in the kernel
};

__global__ void k_class_geom(const double* __restrict__ xs, int64_t n, double Lz, int P, int p,
                             double rc, int K, ClassGeom cg, int32_t* __restrict__ cls) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double z = xs[3 * s + 2];
    if (root_bin(z, Lz, P) == p) {
        cls[s] = 0;
        return;
    }
    const double lo = cg.lo, hi = cg.hi;
    const bool below = z < lo;
    const double d_lo = below ? __dsub_rn(lo, z) : __dsub_rn(__dadd_rn(lo, Lz), z);
    const double d_hi = below ? __dsub_rn(__dadd_rn(z, Lz), hi) : __dsub_rn(z, hi);
    const double dist = d_lo < d_hi ? d_lo : d_hi;
    int c = K + 1;
    for (int m = 1; m <= K; ++m) {
        double thr;
        if (m <= kGeomThr) {
            thr = cg.thr[m - 1];
        } else {
            const double slack =
                m == K ? 1e-6 : __ddiv_rn(__dmul_rn(1e-6, (double)m), (double)K);
            thr = __dadd_rn(__dmul_rn((double)m, rc), slack);
        }
        if (dist < thr) { c = m; break; }
    }
    cls[s] = c;
}

__global__ void k_class_root(const double* __restrict__ xs, int64_t n, double Lz, int P, int p,
                             int K, int32_t* __restrict__ cls) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    cls[s] = root_bin(xs[3 * s + 2], Lz, P) == p ? 0 : K + 1;
}

// Roots from a caller-given assignment (Stage 1 by any partitioner):
// assign[perm[s]] is the partition of sorted atom s.
__global__ void k_class_assign(const int32_t* __restrict__ assign, const int32_t* __restrict__ perm,
                               int64_t n, int p, int K, int32_t* __restrict__ cls) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    cls[s] = assign[perm[s]] == p ? 0 : K + 1;
}

// Number of assignment entries outside [0, P).
__global__ void k_check_assign(const int32_t* __restrict__ assign, int64_t n, int P,
                               unsigned long long* __restrict__ bad) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t a = assign[i];
    if (a < 0 || a >= P) atomicAdd(bad, 1ull);
}

// BFS level h: an atom outside the set joins at level h if a neighbour has a
// level below h (pull form over the symmetric edge set, double-buffered).
__global__ void k_class_hop(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            int64_t n, int h, int K, const int32_t* __restrict__ cur,
                            int32_t* __restrict__ nxt) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int c = cur[s];
    if (c > K) {
        for (int64_t e = row_ptr[s]; e < row_ptr[s + 1]; ++e)
            if (cur[col[e]] < h) { c = h; break; }
    }
    nxt[s] = c;
}

// Atom order used for placement: cells in Morton order of their grid
// coordinates, the atoms of a cell in sorted order.  bperm[pos] = atom.
__global__ void k_cell_sizes(const int32_t* __restrict__ cell_start,
                             const int32_t* __restrict__ corder, int ncell,
                             int32_t* __restrict__ sz) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncell) return;
    const int c = corder[k];
    sz[k] = cell_start[c + 1] - cell_start[c];
}

__global__ void k_bperm(const int32_t* __restrict__ cell_start, const int32_t* __restrict__ corder,
                        const int32_t* __restrict__ boff, int ncell, int32_t* __restrict__ bperm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ncell) return;
    const int c = corder[k];
    const int s0 = cell_start[c], cnt = cell_start[c + 1] - s0, o = boff[k];
    for (int q = 0; q < cnt; ++q) bperm[o + q] = s0 + q;
}

__global__ void k_flag_class(const int32_t* __restrict__ cls, const int32_t* __restrict__ bperm,
                             int64_t n, int m, int32_t* __restrict__ flag) {
    int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n) return;
    flag[pos] = cls[bperm[pos]] == m ? 1 : 0;
}

// Place the atoms of class m after those of classes < m, in placement order.
// pre = exclusive scan of the class-m flags (pre[n] = their count); the
// counts of earlier classes are in cnt[0..m-1], and cnt[m] is recorded here.
__global__ void k_place_class(const int32_t* __restrict__ cls, const int32_t* __restrict__ bperm,
                              const int32_t* __restrict__ pre, int64_t n, int m,
                              int32_t* __restrict__ cnt, int32_t* __restrict__ gid,
                              uint8_t* __restrict__ lroot, int32_t* __restrict__ g2l) {
    int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n) return;
    if (pos == 0) cnt[m] = pre[n];
    const int s = bperm[pos];
    if (cls[s] != m) return;
    int base = 0;
    for (int q = 0; q < m; ++q) base += cnt[q];
    const int l = base + pre[pos];
    gid[l] = s;
    lroot[l] = m == 0 ? 1 : 0;
    g2l[s] = l;
}

// Per-partition sizes for the host: n_le[m] (rows of classes <= m), e_le[m]
// (their edges), m = 0..K.
__global__ void k_plan_stats(const int32_t* __restrict__ cnt, int K,
                             const int64_t* __restrict__ lrow, int64_t* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t t = 0;
    for (int m = 0; m <= K; ++m) {
        t += cnt[m];
        out[m] = t;
        out[K + 1 + m] = lrow[t];
    }
}

__global__ void k_plan_export(const int32_t* __restrict__ gid, const uint8_t* __restrict__ root,
                              const int32_t* __restrict__ perm, int64_t n_ext,
                              int32_t* __restrict__ out_gid, uint8_t* __restrict__ out_root) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_ext) return;
    out_gid[l] = perm[gid[l]];
    out_root[l] = root[l];
}

// Cells of an nc[0] x nc[1] x nc[2] grid (id = (z nc1 + y) nc0 + x) sorted by
// the Morton code of (x, y, z): bit b of x, y, z lands at bits 3b, 3b+1, 3b+2.
std::vector<int32_t> morton_cell_order(const int nc[3]) {
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    std::vector<std::pair<uint64_t, int32_t>> key(ncell);
    for (int z = 0; z < nc[2]; ++z)
        for (int y = 0; y < nc[1]; ++y)
            for (int x = 0; x < nc[0]; ++x) {
                uint64_t k = 0;
                for (int b = 0; b < 21; ++b)
                    k |= (((uint64_t)(x >> b) & 1u) << (3 * b)) |
                         (((uint64_t)(y >> b) & 1u) << (3 * b + 1)) |
                         (((uint64_t)(z >> b) & 1u) << (3 * b + 2));
                const int32_t id = (z * nc[1] + y) * nc[0] + x;
                key[id] = {k, id};
            }
    std::sort(key.begin(), key.end());
    std::vector<int32_t> order(ncell);
    for (int64_t q = 0; q < ncell; ++q) order[q] = key[q].second;
    return order;
}

}  // namespace

int build_plan(mp_ctx* ctx, const Graph& g, int n_parts, int k_hops, int mode, Plan& plan,
               double* halo_factor, const int32_t* d_assign) {
    if (n_parts < 1 || k_hops < 0 || (mode != MP_HALO_GEOM && mode != MP_HALO_BFS))
        return MP_ERR_ARG;
    // an arbitrary root set has no slab to measure a geometric halo from
    if (d_assign && mode != MP_HALO_BFS) return MP_ERR_ARG;
    cudaStream_t st = ctx->stream;
    const int64_t n = g.n;
    const int K = k_hops;
    plan.n_parts = n_parts;
    plan.k_hops = k_hops;
    plan.mode = mode;
    plan.n = n;
    // a plan rebuilt with fewer partitions frees the buffers of the extra ones
    for (size_t q = (size_t)n_parts; q < plan.parts.size(); ++q) {
        Part& X = plan.parts[q];
        DevBuf* bufs[] = {&X.gid, &X.is_root, &X.row_ptr, &X.col, &X.shift};
        for (DevBuf* b : bufs) b->release();
    }
    plan.parts.resize(n_parts);
    Workspace& ws = ctx->ws;
    TimerScope ts(ctx, MP_TIMER_PARTITION, 0, n);
    // scratch: cls[n], cls2[n], flag[n], pre[n+1], g2l[n], bperm[n]
    DevBuf& scratch = ws.pscr;
    MP_TRY(scratch.reserve(sizeof(int32_t) * (6 * n + 4) + 64));
    int32_t* cls = scratch.as<int32_t>();
    int32_t* cls2 = cls + n;
    int32_t* flag = cls2 + n;
    int32_t* pre = flag + n;
    int32_t* g2l = pre + n + 1;
    int32_t* bperm = g2l + n + 1;
    // Placement order: Morton order of cells (cached per grid), so that the
    // rows in flight together in the edge kernels are a compact region and
    // their senders' features fit in L2 better than a z-slowest sweep's.
    const int ncell = g.nc[0] * g.nc[1] * g.nc[2];
    if (ctx->corder_nc[0] != g.nc[0] || ctx->corder_nc[1] != g.nc[1] ||
        ctx->corder_nc[2] != g.nc[2]) {
        const std::vector<int32_t> order = morton_cell_order(g.nc);
        MP_TRY(ws.corder.reserve(sizeof(int32_t) * (3 * (size_t)ncell + 4)));
        MP_CUDA_TRY(cudaMemcpyAsync(ws.corder.as<int32_t>(), order.data(),
                                    sizeof(int32_t) * ncell, cudaMemcpyHostToDevice, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        for (int a = 0; a < 3; ++a) ctx->corder_nc[a] = g.nc[a];
    }
    {
        const int32_t* corder = ws.corder.as<int32_t>();
        int32_t* csz = ws.corder.as<int32_t>() + ncell;
        int32_t* coff = csz + ncell + 1;
        k_cell_sizes<<<grid_for(ncell, 256), 256, 0, st>>>(g.cell_start.as<int32_t>(), corder,
                                                             ncell, csz);
        note_launch();
        MP_TRY(exclusive_scan_i32(csz, coff, ncell, ws.tmp, st));
        k_bperm<<<grid_for(ncell, 128), 128, 0, st>>>(g.cell_start.as<int32_t>(), corder, coff,
                                                       ncell, bperm);
        note_launch();
    }
    const double* xs = g.xs.as<double>();
    const double Lz = g.box[2];
    // geometric halo widths in units of the graph's list cutoff (r_c + skin
    // for a skin list: every hop of the current r_c graph is an edge of it)
    const double rc = g.r_list > 0.0 ? g.r_list : ctx->model.d.r_cut;
    // No host synchronisation until every partition is built: class counts
    // stay on the device, buffers are sized by their upper bounds (n rows;
    // a partition's edges are a subset of the graph's), and the sizes come
    // back in one copy at the end.
    DevBuf& stats = ws.pstats;
    const int ns = 3 * (K + 1);   // n_le, e_le, e_same per class
    // per partition: ns sizes; then one slot for the count of invalid
    // assignment entries; then the class counts
    MP_TRY(stats.reserve(sizeof(int64_t) * (n_parts * ns + 1) +
                         sizeof(int32_t) * n_parts * (K + 1)));
    int64_t* d_stats = stats.as<int64_t>();
    int64_t* d_bad = d_stats + (size_t)n_parts * ns;
    int32_t* d_cnt = reinterpret_cast<int32_t*>(d_bad + 1);
    MP_CUDA_TRY(cudaMemsetAsync(d_stats, 0, sizeof(int64_t) * ((size_t)n_parts * ns + 1), st));
    if (d_assign) {
        k_check_assign<<<grid_for(n, 256), 256, 0, st>>>(
            d_assign, n, n_parts, reinterpret_cast<unsigned long long*>(d_bad));
        note_launch();
    }
    for (int p = 0; p < n_parts; ++p) {
        Part& P = plan.parts[p];
        int32_t* cnt = d_cnt + (size_t)p * (K + 1);
        int32_t* cur = cls;
        if (mode == MP_HALO_GEOM) {
            ClassGeom cg;
            cg.lo = Lz * (double)p / (double)n_parts;
            cg.hi = Lz * (double)(p + 1) / (double)n_parts;
            for (int m = 1; m <= K && m <= kGeomThr; ++m) {
                const double slack = m == K ? 1e-6 : 1e-6 * (double)m / (double)K;
                cg.thr[m - 1] = (double)m * rc + slack;
            }
            k_class_geom<<<grid_for(n, 256), 256, 0, st>>>(xs, n, Lz, n_parts, p, rc, K, cg,
                                                           cls);
            note_launch();
        } else {
            if (d_assign)
                k_class_assign<<<grid_for(n, 256), 256, 0, st>>>(d_assign, g.perm.as<int32_t>(),
                                                                 n, p, K, cls);
            else
                k_class_root<<<grid_for(n, 256), 256, 0, st>>>(xs, n, Lz, n_parts, p, K, cls);
            note_launch();
            int32_t* other = cls2;
            for (int h = 1; h <= K; ++h) {
                k_class_hop<<<grid_for(n, 256), 256, 0, st>>>(g.row_ptr.as<int64_t>(),
                                                              g.col.as<int32_t>(), n, h, K, cur, other);
                note_launch();
                int32_t* t = cur;
                cur = other;
                other = t;
            }
        }
        // stable placement class by class
        MP_CUDA_TRY(cudaMemsetAsync(g2l, 0xFF, sizeof(int32_t) * n, st));
        MP_TRY(P.gid.reserve(sizeof(int32_t) * (n + 1)));
        MP_TRY(P.is_root.reserve(n + 16));
        MP_TRY(P.row_ptr.reserve(sizeof(int64_t) * (n + 1)));
        MP_TRY(P.col.reserve(sizeof(int32_t) * (g.n_edges + 1)));
        MP_TRY(P.shift.reserve(g.n_edges + 16));
        for (int m = 0; m <= K; ++m) {
            k_flag_class<<<grid_for(n, 256), 256, 0, st>>>(cur, bperm, n, m, flag);
            note_launch();
            MP_TRY(exclusive_scan_i32(flag, pre, n, ws.tmp, st));
            k_place_class<<<grid_for(n, 256), 256, 0, st>>>(cur, bperm, pre, n, m, cnt,
                                                            P.gid.as<int32_t>(),
                                                            P.is_root.as<uint8_t>(), g2l);
            note_launch();
        }
        // a warp per extended row, grid-stride (the row count is on the device)
        const int row_blocks = 8 * (ctx->num_sms > 0 ? ctx->num_sms : 152);
        k_local_deg<<<row_blocks, 256, sizeof(unsigned long long) * (K + 1), st>>>(
            g.row_ptr.as<int64_t>(), g.col.as<int32_t>(), P.gid.as<int32_t>(), g2l, n, cnt, K, flag,
            reinterpret_cast<unsigned long long*>(d_stats + (size_t)p * ns + 2 * (K + 1)));
        note_launch();
        MP_TRY(exclusive_scan_i64(flag, P.row_ptr.as<int64_t>(), n, ws.tmp, st));
        k_local_fill<<<row_blocks, 256, 0, st>>>(
            g.row_ptr.as<int64_t>(), g.col.as<int32_t>(), g.shift.as<int8_t>(),
            P.gid.as<int32_t>(), g2l, cnt, K, P.row_ptr.as<int64_t>(), P.col.as<int32_t>(),
            P.shift.as<int8_t>());
        note_launch();
        k_plan_stats<<<1, 32, 0, st>>>(cnt, K, P.row_ptr.as<int64_t>(), d_stats + (size_t)p * ns);
        note_launch();
    }
    std::vector<int64_t> h_stats((size_t)n_parts * ns + 1);
    MP_CUDA_TRY(cudaMemcpyAsync(h_stats.data(), d_stats, sizeof(int64_t) * h_stats.size(),
                                cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_stats[(size_t)n_parts * ns] != 0) return MP_ERR_ARG;   // assignment outside [0, P)
    int64_t halo_total = 0;
    for (int p = 0; p < n_parts; ++p) {
        Part& P = plan.parts[p];
        const int64_t* h = h_stats.data() + (size_t)p * ns;
        P.n_le.assign(h, h + K + 1);
        P.e_le.assign(h + K + 1, h + 2 * (K + 1));
        P.e_same.assign(h + 2 * (K + 1), h + 3 * (K + 1));
        P.n_root = P.n_le[0];
        P.n_ext = P.n_le[K];
        P.n_edges = P.e_le[K];
        halo_total += P.n_ext - P.n_root;
    }
    MP_CUDA_TRY(cudaGetLastError());
    if (halo_factor) *halo_factor = (double)halo_total / (double)n;
    return MP_OK;
}

int export_plan(const Plan& plan, const Graph& g, int p, cudaStream_t st, int32_t* gid,
                uint8_t* root) {
    const Part& P = plan.parts[p];
    k_plan_export<<<grid_for(P.n_ext, 256), 256, 0, st>>>(P.gid.as<int32_t>(),
                                                          P.is_root.as<uint8_t>(),
                                                          g.perm.as<int32_t>(), P.n_ext, gid, root); note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace mp

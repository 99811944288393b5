// Spatial-grid partitions with ghost halos and local CSR extraction.
//
// Stage 1 (Methods, "Graph Partitioning"): P uniform bins of the scaled z
// coordinate, root bin = min(floor(x_w,z / L_z * P), P - 1).
// Stage 2: every root keeps its K-hop neighbourhood, either by K BFS
// expansions over the global CSR (MP_HALO_BFS) or by the geometric slab
// halo of width K r_c (MP_HALO_GEOM, a superset: each hop is shorter than
// r_c).  The extended set keeps ascending cell order, so each local row holds
// the global row's edges in the same order, filtered to senders in the set.
#include "common.cuh"

namespace mp {

namespace {

__device__ __forceinline__ int root_bin(double z, double L, int P) {
    double f = __ddiv_rn(z, L);
    int b = (int)floor(__dmul_rn(f, (double)P));
    return b < P - 1 ? b : P - 1;
}

__global__ void k_flags_geom(const double* __restrict__ xs, int64_t n, double Lz, int P, int p,
                             double width, int32_t* __restrict__ flag, uint8_t* __restrict__ root) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double z = xs[3 * s + 2];
    bool r = root_bin(z, Lz, P) == p;
    double lo = __ddiv_rn(__dmul_rn(Lz, (double)p), (double)P);
    double hi = __ddiv_rn(__dmul_rn(Lz, (double)(p + 1)), (double)P);
    bool below = z < lo;
    double d_lo = below ? __dsub_rn(lo, z) : __dsub_rn(__dadd_rn(lo, Lz), z);
    double d_hi = below ? __dsub_rn(__dadd_rn(z, Lz), hi) : __dsub_rn(z, hi);
    double dist = d_lo < d_hi ? d_lo : d_hi;
    flag[s] = (r || dist < width) ? 1 : 0;
    root[s] = r ? 1 : 0;
}

__global__ void k_flags_root(const double* __restrict__ xs, int64_t n, double Lz, int P, int p,
                             int32_t* __restrict__ flag, uint8_t* __restrict__ root) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    bool r = root_bin(xs[3 * s + 2], Lz, P) == p;
    flag[s] = r ? 1 : 0;
    root[s] = r ? 1 : 0;
}

// One BFS hop over the symmetric edge set (pull form).
__global__ void k_bfs_hop(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                          int64_t n, const int32_t* __restrict__ cur, int32_t* __restrict__ nxt) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int v = cur[s];
    if (!v) {
        for (int64_t e = row_ptr[s]; e < row_ptr[s + 1]; ++e)
            if (cur[col[e]]) { v = 1; break; }
    }
    nxt[s] = v;
}

__global__ void k_compact(const int32_t* __restrict__ flag, const int32_t* __restrict__ pre,
                          const uint8_t* __restrict__ root, int64_t n, int32_t* __restrict__ gid,
                          uint8_t* __restrict__ lroot, int32_t* __restrict__ g2l) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    if (flag[s]) {
        int l = pre[s];
        gid[l] = (int32_t)s;
        lroot[l] = root[s];
        g2l[s] = l;
    } else {
        g2l[s] = -1;
    }
}

__global__ void k_local_deg(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ gid, const int32_t* __restrict__ g2l,
                            int64_t n_ext, int32_t* __restrict__ deg) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_ext) return;
    int s = gid[l];
    int c = 0;
    for (int64_t e = row_ptr[s]; e < row_ptr[s + 1]; ++e) c += g2l[col[e]] >= 0;
    deg[l] = c;
}

__global__ void k_local_fill(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                             const int8_t* __restrict__ shift, const int32_t* __restrict__ gid,
                             const int32_t* __restrict__ g2l, int64_t n_ext,
                             const int64_t* __restrict__ lrow, int32_t* __restrict__ lcol,
                             int8_t* __restrict__ lshift) {
    int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_ext) return;
    int s = gid[l];
    int64_t o = lrow[l];
    for (int64_t e = row_ptr[s]; e < row_ptr[s + 1]; ++e) {
        int t = g2l[col[e]];
        if (t >= 0) {
            lcol[o] = t;
            lshift[o] = shift[e];
            ++o;
        }
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

}  // namespace

int build_plan(mp_ctx* ctx, const Graph& g, int n_parts, int k_hops, int mode, Plan& plan,
               double* halo_factor) {
    if (n_parts < 1 || k_hops < 0 || (mode != MP_HALO_GEOM && mode != MP_HALO_BFS))
        return MP_ERR_ARG;
    cudaStream_t st = ctx->stream;
    const int64_t n = g.n;
    plan.n_parts = n_parts;
    plan.k_hops = k_hops;
    plan.mode = mode;
    plan.n = n;
    plan.parts.resize(n_parts);
    Workspace& ws = ctx->ws;
    TimerScope ts(ctx, MP_TIMER_PARTITION, 0, n);
    // scratch: flag[n], flag2[n], pre[n+1], g2l[n], root[n] bytes
    DevBuf& scratch = ws.pscr;
    MP_TRY(scratch.reserve(sizeof(int32_t) * (4 * n + 2) + n + 64));
    int32_t* flag = scratch.as<int32_t>();
    int32_t* flag2 = flag + n;
    int32_t* pre = flag2 + n;
    int32_t* g2l = pre + n + 1;
    uint8_t* root = reinterpret_cast<uint8_t*>(g2l + n + 1);
    const double* xs = g.xs.as<double>();
    const double Lz = g.box[2];
    // same operation order as the reference definition: (K * r_c) + 1e-6
    volatile double kw = (double)k_hops * ctx->model.d.r_cut;
    const double width = kw + 1e-6;
    int64_t halo_total = 0;
    int rc = MP_OK;
    for (int p = 0; p < n_parts && rc == MP_OK; ++p) {
        Part& P = plan.parts[p];
        int32_t* cur = flag;
        if (mode == MP_HALO_GEOM) {
            k_flags_geom<<<grid_for(n, 256), 256, 0, st>>>(xs, n, Lz, n_parts, p, width, flag, root); note_launch();
        } else {
            k_flags_root<<<grid_for(n, 256), 256, 0, st>>>(xs, n, Lz, n_parts, p, flag, root); note_launch();
            int32_t* other = flag2;
            for (int h = 0; h < k_hops; ++h) {
                k_bfs_hop<<<grid_for(n, 256), 256, 0, st>>>(g.row_ptr.as<int64_t>(),
                                                            g.col.as<int32_t>(), n, cur, other); note_launch();
                int32_t* t = cur;
                cur = other;
                other = t;
            }
        }
        rc = exclusive_scan_i32(cur, pre, n, ws.tmp, st);
        if (rc) break;
        int32_t n_ext32 = 0;
        if (cudaMemcpyAsync(&n_ext32, pre + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st) ||
            cudaStreamSynchronize(st)) { rc = MP_ERR_CUDA; break; }
        P.n_ext = n_ext32;
        if ((rc = P.gid.reserve(sizeof(int32_t) * (P.n_ext + 1)))) break;
        if ((rc = P.is_root.reserve(P.n_ext + 16))) break;
        if ((rc = P.row_ptr.reserve(sizeof(int64_t) * (P.n_ext + 1)))) break;
        k_compact<<<grid_for(n, 256), 256, 0, st>>>(cur, pre, root, n, P.gid.as<int32_t>(),
                                                    P.is_root.as<uint8_t>(), g2l); note_launch();
        int32_t* ldeg = cur == flag ? flag2 : flag;   // free flag buffer
        k_local_deg<<<grid_for(P.n_ext, 256), 256, 0, st>>>(
            g.row_ptr.as<int64_t>(), g.col.as<int32_t>(), P.gid.as<int32_t>(), g2l, P.n_ext, ldeg); note_launch();
        rc = exclusive_scan_i64(ldeg, P.row_ptr.as<int64_t>(), P.n_ext, ws.tmp, st);
        if (rc) break;
        int64_t ne = 0;
        int32_t nroot = 0;
        if (cudaMemcpyAsync(&ne, P.row_ptr.as<int64_t>() + P.n_ext, sizeof(int64_t),
                            cudaMemcpyDeviceToHost, st) ||
            cudaStreamSynchronize(st)) { rc = MP_ERR_CUDA; break; }
        P.n_edges = ne;
        if ((rc = P.col.reserve(sizeof(int32_t) * (ne + 1)))) break;
        if ((rc = P.shift.reserve(ne + 16))) break;
        k_local_fill<<<grid_for(P.n_ext, 256), 256, 0, st>>>(
            g.row_ptr.as<int64_t>(), g.col.as<int32_t>(), g.shift.as<int8_t>(),
            P.gid.as<int32_t>(), g2l, P.n_ext, P.row_ptr.as<int64_t>(), P.col.as<int32_t>(),
            P.shift.as<int8_t>()); note_launch();
        // root count: roots are flagged in `root` (uint8) -> count with a scan of flags
        k_flags_root<<<grid_for(n, 256), 256, 0, st>>>(xs, n, Lz, n_parts, p, ldeg, root); note_launch();
        rc = exclusive_scan_i32(ldeg, pre, n, ws.tmp, st);
        if (rc) break;
        if (cudaMemcpyAsync(&nroot, pre + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st) ||
            cudaStreamSynchronize(st)) { rc = MP_ERR_CUDA; break; }
        P.n_root = nroot;
        halo_total += P.n_ext - P.n_root;
    }
    if (rc) return rc;
    if (cudaGetLastError() != cudaSuccess) return MP_ERR_CUDA;
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

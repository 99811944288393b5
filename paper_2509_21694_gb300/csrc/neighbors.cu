// Periodic cell-list neighbour search emitting a receiver-sorted CSR.
//
// Edge (i <- j, n): i != j and |x_w[j] - x_w[i] + n L| < r_c, with the
// canonical wrap x_w = x - L floor(x / L) and n = -rint((x_w[j] - x_w[i]) / L)
// per axis, decided in FP64 (the atom graph of the paper's message passing,
// Methods "Graph Partitioning").  A fast FP32 test settles every pair whose
// r^2 is farther than 5e-4 r_c^2 from r_c^2; pairs inside that band are
// decided by the exact FP64 formula (IEEE round-to-nearest, no contraction),
// so the edge set is bit-exact with an FP64 O(N^2) search.
//
// Atoms are re-ordered by cell (x fastest, z slowest) with a deterministic
// counting sort; within a cell they keep increasing caller id.  Each row is
// emitted by one warp scanning the stencil cells in increasing cell order,
// so senders come out in increasing sorted id without a per-row sort.  The
// default search runs one block per cell with the stencil's atoms staged in
// shared memory; a warp-per-receiver search reading them from global memory
// is the fallback for stencils too large to stage.
#include "common.cuh"

namespace mp {

namespace {

constexpr int kErrOverlap = 1;
constexpr int kErrCapacity = 2;    // a cell's stencil holds more than kCellCand atoms
constexpr int kErrNonFinite = 4;   // a position coordinate is NaN or infinite
constexpr int kCellCand = 2048;    // candidates a cell block stages in shared memory

__device__ __forceinline__ double wrap1(double x, double L) {
    double w = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    if (w >= L) w = __dsub_rn(w, L);
    return w;
}

__device__ __forceinline__ int cell_coord(double xw, double L, int nc) {
    int c = (int)(xw / L * (double)nc);
    return c < nc - 1 ? (c < 0 ? 0 : c) : nc - 1;
}

struct BoxP {
    double L[3];
    float Lf[3], invLf[3];
    int nc[3];
    double rc2;
    float rc2_lo, rc2_hi;
};

// A non-finite coordinate sets kErrNonFinite (the call then fails with
// MP_ERR_ARG); such an atom lands in cell 0 and every distance test with it
// is false, so nothing downstream indexes out of range before the check.
__global__ void k_wrap_bin(const double* __restrict__ pos, int64_t n, BoxP b,
                           double* __restrict__ xw, int32_t* __restrict__ cell,
                           int32_t* __restrict__ count, int* __restrict__ err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double x = pos[3 * i + a];
        if (!isfinite(x)) atomicOr(err, kErrNonFinite);
        double w = wrap1(x, b.L[a]);
        xw[3 * i + a] = w;
        c[a] = cell_coord(w, b.L[a], b.nc[a]);
    }
    int id = (c[2] * b.nc[1] + c[1]) * b.nc[0] + c[0];
    cell[i] = id;
    atomicAdd(&count[id], 1);
}

__global__ void k_place(const int32_t* __restrict__ cell, int64_t n,
                        const int32_t* __restrict__ start, int32_t* __restrict__ cursor,
                        int32_t* __restrict__ order) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = cell[i];
    int slot = start[c] + atomicAdd(&cursor[c], 1);
    order[slot] = (int32_t)i;
}

// Insertion sort of each cell's members by caller id: makes the order
// independent of the atomic placement above.
__global__ void k_sort_cells(const int32_t* __restrict__ start, int ncell,
                             int32_t* __restrict__ order) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int b = start[c], e = start[c + 1];
    for (int k = b + 1; k < e; ++k) {
        int v = order[k];
        int m = k - 1;
        while (m >= b && order[m] > v) {
            order[m + 1] = order[m];
            --m;
        }
        order[m + 1] = v;
    }
}

__global__ void k_gather_sorted(const int32_t* __restrict__ order, int64_t n,
                                const double* __restrict__ xw, int32_t* __restrict__ inv,
                                double* __restrict__ xs, float4* __restrict__ xsf) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    int i = order[s];
    inv[i] = (int32_t)s;
    double x = xw[3 * (int64_t)i], y = xw[3 * (int64_t)i + 1], z = xw[3 * (int64_t)i + 2];
    xs[3 * s] = x;
    xs[3 * s + 1] = y;
    xs[3 * s + 2] = z;
    xsf[s] = make_float4((float)x, (float)y, (float)z, 0.f);
}

// Stencil coordinates along one axis in increasing order: {c-1, c, c+1} mod
// nc when nc >= 3, else every cell of the axis.
__device__ __forceinline__ int stencil(int c, int nc, int* out) {
    if (nc >= 3) {
        int a = c == 0 ? nc - 1 : c - 1, m = c, p = c == nc - 1 ? 0 : c + 1;
        // sort three values
        int v0 = a, v1 = m, v2 = p, t;
        if (v0 > v1) { t = v0; v0 = v1; v1 = t; }
        if (v1 > v2) { t = v1; v1 = v2; v2 = t; }
        if (v0 > v1) { t = v0; v0 = v1; v1 = t; }
        out[0] = v0; out[1] = v1; out[2] = v2;
        return 3;
    }
    for (int k = 0; k < nc; ++k) out[k] = k;
    return nc;
}

// Exact FP64 decision for one pair (the definition).
__device__ __forceinline__ bool exact_pair(const double* xi, const double* xj, const BoxP& b,
                                           int* code, double* r2o) {
    double d[3];
    int n[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double dx = __dsub_rn(xj[a], xi[a]);
        double nn = -rint(__ddiv_rn(dx, b.L[a]));
        d[a] = __dadd_rn(dx, __dmul_rn(nn, b.L[a]));
        n[a] = (int)nn;
    }
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                          __dmul_rn(d[2], d[2]));
    *code = (n[0] + 1) * 9 + (n[1] + 1) * 3 + (n[2] + 1);
    *r2o = r2;
    return r2 < b.rc2;
}

template <bool FILL>
__global__ void k_neighbors(const float4* __restrict__ xsf, const double* __restrict__ xs,
                            int64_t n, BoxP b, const int32_t* __restrict__ start,
                            int32_t* __restrict__ deg, const int64_t* __restrict__ row_ptr,
                            int32_t* __restrict__ col, int8_t* __restrict__ shift,
                            int* __restrict__ err) {
    int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (s >= n) return;
    float4 pi = xsf[s];
    double xi[3] = {xs[3 * s], xs[3 * s + 1], xs[3 * s + 2]};
    int cs[3][3], ns[3];
    for (int a = 0; a < 3; ++a) ns[a] = stencil(cell_coord(xi[a], b.L[a], b.nc[a]), b.nc[a], cs[a]);
    int64_t out = FILL ? row_ptr[s] : 0;
    int count = 0;
    for (int iz = 0; iz < ns[2]; ++iz)
        for (int iy = 0; iy < ns[1]; ++iy)
            for (int ix = 0; ix < ns[0]; ++ix) {
                int cell = (cs[2][iz] * b.nc[1] + cs[1][iy]) * b.nc[0] + cs[0][ix];
                int cb = start[cell], ce = start[cell + 1];
                for (int kb = cb; kb < ce; kb += 32) {
                    int k = kb + lane;
                    bool keep = false;
                    int code = 13;
                    if (k < ce && k != s) {
                        float4 pj = xsf[k];
                        float d0 = pj.x - pi.x, d1 = pj.y - pi.y, d2 = pj.z - pi.z;
                        float n0 = -rintf(d0 * b.invLf[0]), n1 = -rintf(d1 * b.invLf[1]),
                              n2 = -rintf(d2 * b.invLf[2]);
                        d0 = fmaf(n0, b.Lf[0], d0);
                        d1 = fmaf(n1, b.Lf[1], d1);
                        d2 = fmaf(n2, b.Lf[2], d2);
                        float r2f = d0 * d0 + d1 * d1 + d2 * d2;
                        if (r2f < b.rc2_lo) {
                            keep = true;
                            code = ((int)n0 + 1) * 9 + ((int)n1 + 1) * 3 + ((int)n2 + 1);
                            if (r2f < 1e-6f) atomicOr(err, kErrOverlap);
                        } else if (r2f <= b.rc2_hi) {
                            double xj[3] = {xs[3 * (int64_t)k], xs[3 * (int64_t)k + 1],
                                            xs[3 * (int64_t)k + 2]};
                            double r2;
                            keep = exact_pair(xi, xj, b, &code, &r2);
                        }
                    }
                    unsigned m = __ballot_sync(0xffffffffu, keep);
                    if (FILL && keep) {
                        int64_t e = out + count + __popc(m & ((1u << lane) - 1u));
                        col[e] = k;
                        shift[e] = (int8_t)code;
                    }
                    count += __popc(m);
                }
            }
    if (!FILL && lane == 0) deg[s] = count;
}

// The same search with one block per cell: the cell's stencil atoms (the 27
// cells, or all cells of an axis shorter than 3, in increasing cell order)
// are staged once in shared memory, then each warp takes one of the cell's
// receivers and scans them 32 at a time.  Candidate order, arithmetic and
// therefore the CSR are identical to k_neighbors.  A cell whose stencil
// exceeds kCellCand atoms sets kErrCapacity (the caller then falls back to
// k_neighbors).
template <bool FILL>
__global__ void __launch_bounds__(256) k_neighbors_cell(
    const float4* __restrict__ xsf, const double* __restrict__ xs, BoxP b,
    const int32_t* __restrict__ start, int32_t* __restrict__ deg,
    const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col, int8_t* __restrict__ shift,
    int* __restrict__ err) {
    __shared__ float4 cpos[kCellCand];
    __shared__ int32_t cidx[kCellCand];
    __shared__ int rbeg[27], roff[28], s_nr;
    const int cell = blockIdx.x;
    const int sb = start[cell], se = start[cell + 1];
    if (sb == se) return;
    if (threadIdx.x == 0) {
        const int cx = cell % b.nc[0], cy = (cell / b.nc[0]) % b.nc[1],
                  cz = cell / (b.nc[0] * b.nc[1]);
        int cs[3][3], ns[3];
        ns[0] = stencil(cx, b.nc[0], cs[0]);
        ns[1] = stencil(cy, b.nc[1], cs[1]);
        ns[2] = stencil(cz, b.nc[2], cs[2]);
        int nr = 0, tot = 0;
        for (int iz = 0; iz < ns[2]; ++iz)
            for (int iy = 0; iy < ns[1]; ++iy)
                for (int ix = 0; ix < ns[0]; ++ix) {
                    const int c = (cs[2][iz] * b.nc[1] + cs[1][iy]) * b.nc[0] + cs[0][ix];
                    rbeg[nr] = start[c];
                    roff[nr] = tot;
                    tot += start[c + 1] - start[c];
                    ++nr;
                }
        roff[nr] = tot;
        s_nr = nr;
    }
    __syncthreads();
    const int nr = s_nr, tot = roff[nr];
    if (tot > kCellCand) {
        if (threadIdx.x == 0) atomicOr(err, kErrCapacity);
        return;
    }
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        int r = 0;
        while (q >= roff[r + 1]) ++r;
        const int k = rbeg[r] + (q - roff[r]);
        cpos[q] = xsf[k];
        cidx[q] = k;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int s = sb + warp; s < se; s += nw) {
        const float4 pi = xsf[s];
        const double xi[3] = {xs[3 * (int64_t)s], xs[3 * (int64_t)s + 1], xs[3 * (int64_t)s + 2]};
        const int64_t out = FILL ? row_ptr[s] : 0;
        int count = 0;
        for (int kb = 0; kb < tot; kb += 32) {
            const int q = kb + lane;
            bool keep = false;
            int code = 13, k = -1;
            if (q < tot) {
                k = cidx[q];
                if (k != s) {
                    const float4 pj = cpos[q];
                    float d0 = pj.x - pi.x, d1 = pj.y - pi.y, d2 = pj.z - pi.z;
                    float n0 = -rintf(d0 * b.invLf[0]), n1 = -rintf(d1 * b.invLf[1]),
                          n2 = -rintf(d2 * b.invLf[2]);
                    d0 = fmaf(n0, b.Lf[0], d0);
                    d1 = fmaf(n1, b.Lf[1], d1);
                    d2 = fmaf(n2, b.Lf[2], d2);
                    float r2f = d0 * d0 + d1 * d1 + d2 * d2;
                    if (r2f < b.rc2_lo) {
                        keep = true;
                        code = ((int)n0 + 1) * 9 + ((int)n1 + 1) * 3 + ((int)n2 + 1);
                        if (r2f < 1e-6f) atomicOr(err, kErrOverlap);
                    } else if (r2f <= b.rc2_hi) {
                        double xj[3] = {xs[3 * (int64_t)k], xs[3 * (int64_t)k + 1],
                                        xs[3 * (int64_t)k + 2]};
                        double r2;
                        keep = exact_pair(xi, xj, b, &code, &r2);
                    }
                }
            }
            unsigned m = __ballot_sync(0xffffffffu, keep);
            if (FILL && keep) {
                int64_t e = out + count + __popc(m & ((1u << lane) - 1u));
                col[e] = k;
                shift[e] = (int8_t)code;
            }
            count += __popc(m);
        }
        if (!FILL && lane == 0) deg[s] = count;
    }
}

__global__ void k_export(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                         const int8_t* __restrict__ shift, const int32_t* __restrict__ perm,
                         int64_t n, int32_t* __restrict__ recv, int32_t* __restrict__ send,
                         int8_t* __restrict__ sh) {
    int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (s >= n) return;
    int me = perm[s];
    for (int64_t e = row_ptr[s] + lane; e < row_ptr[s + 1]; e += 32) {
        recv[e] = me;
        send[e] = perm[col[e]];
        sh[e] = shift[e];
    }
}

}  // namespace

int build_graph(mp_ctx* ctx, const double* d_pos, int64_t n, const double box[3], Graph& g,
                double r_list) {
    // the list cutoff: r_c, or r_c + skin for a list reused while atoms move
    const double rc = r_list > 0.0 ? r_list : ctx->model.d.r_cut;
    g.r_list = rc;
    cudaStream_t st = ctx->stream;
    if (n <= 0 || !d_pos) return MP_ERR_ARG;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0)) return MP_ERR_ARG;
        if (box[a] < 2.0 * rc) return MP_ERR_BOX_TOO_SMALL;
    }
    BoxP b;
    for (int a = 0; a < 3; ++a) {
        b.L[a] = box[a];
        b.Lf[a] = (float)box[a];
        b.invLf[a] = (float)(1.0 / box[a]);
        int nc = (int)floor(box[a] / (rc + 1e-6));
        b.nc[a] = nc < 1 ? 1 : nc;
        g.box[a] = box[a];
        g.nc[a] = b.nc[a];
    }
    b.rc2 = rc * rc;
    b.rc2_lo = (float)(b.rc2 * (1.0 - 5e-4));
    b.rc2_hi = (float)(b.rc2 * (1.0 + 5e-4));
    g.n = n;
    int64_t ncell = (int64_t)b.nc[0] * b.nc[1] * b.nc[2];

    Workspace& ws = ctx->ws;
    TimerScope ts(ctx, MP_TIMER_NEIGHBORS, 0, n);
    MP_TRY(g.perm.reserve(sizeof(int32_t) * n));
    MP_TRY(g.inv.reserve(sizeof(int32_t) * n));
    MP_TRY(g.xs.reserve(sizeof(double) * 3 * n + sizeof(float4) * n + 64));
    MP_TRY(g.cell_start.reserve(sizeof(int32_t) * (ncell + 1)));
    MP_TRY(g.row_ptr.reserve(sizeof(int64_t) * (n + 1)));
    // scratch: xw [3n] double, cell [n], count/cursor [ncell], deg [n]
    size_t scr = sizeof(double) * 3 * n + sizeof(int32_t) * (2 * n + 2 * ncell + 2);
    MP_TRY(g.scratch.reserve(scr));
    MP_TRY(ws.err.reserve(64));
    double* xw = g.scratch.as<double>();
    int32_t* cell = reinterpret_cast<int32_t*>(xw + 3 * n);
    int32_t* count = cell + n;
    int32_t* cursor = count + ncell + 1;
    int32_t* deg = cursor + ncell + 1;
    double* xs = g.xs.as<double>();
    float4* xsf = reinterpret_cast<float4*>(
        (reinterpret_cast<uintptr_t>(xs + 3 * n) + 15) & ~uintptr_t(15));
    int* err = ws.err.as<int>();

    MP_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int32_t) * (2 * ncell + 2), st));
    MP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    k_wrap_bin<<<grid_for(n, 256), 256, 0, st>>>(d_pos, n, b, xw, cell, count, err); note_launch();
    MP_TRY(exclusive_scan_i32(count, g.cell_start.as<int32_t>(), ncell, ws.tmp, st));
    k_place<<<grid_for(n, 256), 256, 0, st>>>(cell, n, g.cell_start.as<int32_t>(), cursor,
                                              g.perm.as<int32_t>()); note_launch();
    k_sort_cells<<<grid_for(ncell, 128), 128, 0, st>>>(g.cell_start.as<int32_t>(), (int)ncell,
                                                       g.perm.as<int32_t>()); note_launch();
    k_gather_sorted<<<grid_for(n, 256), 256, 0, st>>>(g.perm.as<int32_t>(), n, xw,
                                                      g.inv.as<int32_t>(), xs, xsf); note_launch();
    int warps_per_block = 8;
    int nb = grid_for(n, warps_per_block);
    // degrees with the cell-block search; a stencil too large for its shared
    // memory switches both passes to the warp-per-receiver search
    k_neighbors_cell<false><<<(unsigned)ncell, 256, 0, st>>>(
        xsf, xs, b, g.cell_start.as<int32_t>(), deg, nullptr, nullptr, nullptr, err); note_launch();
    int herr = 0;
    MP_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr & kErrNonFinite) return MP_ERR_ARG;
    const bool by_cell = !(herr & kErrCapacity);
    if (!by_cell) {
        MP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
        k_neighbors<false><<<nb, 32 * warps_per_block, 0, st>>>(
            xsf, xs, n, b, g.cell_start.as<int32_t>(), deg, nullptr, nullptr, nullptr, err); note_launch();
    }
    MP_TRY(exclusive_scan_i64(deg, g.row_ptr.as<int64_t>(), n, ws.tmp, st));
    int64_t ne = 0;
    MP_CUDA_TRY(cudaMemcpyAsync(&ne, g.row_ptr.as<int64_t>() + n, sizeof(int64_t),
                                cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr & kErrOverlap) return MP_ERR_OVERLAP;
    g.n_edges = ne;
    MP_TRY(g.col.reserve(sizeof(int32_t) * (ne + 1)));
    MP_TRY(g.shift.reserve(ne + 16));
    if (by_cell)
        k_neighbors_cell<true><<<(unsigned)ncell, 256, 0, st>>>(
            xsf, xs, b, g.cell_start.as<int32_t>(), nullptr, g.row_ptr.as<int64_t>(),
            g.col.as<int32_t>(), g.shift.as<int8_t>(), err);
    else
        k_neighbors<true><<<nb, 32 * warps_per_block, 0, st>>>(
            xsf, xs, n, b, g.cell_start.as<int32_t>(), nullptr, g.row_ptr.as<int64_t>(),
            g.col.as<int32_t>(), g.shift.as<int8_t>(), err);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int export_graph(const Graph& g, cudaStream_t st, int32_t* recv, int32_t* send, int8_t* sh) {
    int wpb = 8;
    k_export<<<grid_for(g.n, wpb), 32 * wpb, 0, st>>>(g.row_ptr.as<int64_t>(),
                                                      g.col.as<int32_t>(), g.shift.as<int8_t>(),
                                                      g.perm.as<int32_t>(), g.n, recv, send, sh); note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace mp

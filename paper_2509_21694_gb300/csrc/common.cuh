// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <vector>

#include "mpip.h"

namespace mp {

constexpr int kH = 64;        // radial MLP hidden width
constexpr int kNB = 8;        // Bessel functions
constexpr int kHeadH = 32;    // correction-head hidden width
constexpr double kKappa = 9.648533212e-3;   // eV/(A amu) -> A/fs^2

#define MP_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return MP_ERR_CUDA;          \
    } while (0)

#define MP_TRY(expr)                                        \
    do {                                                    \
        int _rc = (expr);                                   \
        if (_rc != MP_OK) return _rc;                       \
    } while (0)

// Grow-only device buffer.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int reserve(size_t nbytes);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Releases function-local buffers when the scope ends, early error returns
// included (DevBuf itself does not own its memory past release()).
struct BufGuard {
    std::vector<DevBuf*> bufs;
    BufGuard(std::initializer_list<DevBuf*> b) : bufs(b) {}
    BufGuard(const BufGuard&) = delete;
    BufGuard& operator=(const BufGuard&) = delete;
    ~BufGuard() {
        for (DevBuf* b : bufs) b->release();
    }
};

// Device copies of one layer's weights.  *T arrays are transposed
// ([in][out]) so that a thread owning an output channel reads coalesced.
struct LayerW {
    float* W1;     // [H][NB]
    float* W2;     // [H][H]   (out, in)
    float* W2T;    // [H][H]   (in, out)
    float* W3;     // [P][H]
    float* W3T;    // [H][P]
    float* W0;     // [F][F]  (out, in)
    float* W0T;
    float* U[2];   // U1, U2 (out, in)
    float* UT[2];
    float* b;      // [F]
    float* V[2];   // V1, V2 (out, in)
    float* VT[2];
    // BF16 operand copies for the tensor-core path
    __nv_bfloat16* W2b;    // [H][H]   (out, in), K-major
    __nv_bfloat16* W3b;    // [P][H]   K-major
    __nv_bfloat16* W3Tb;   // [H][P]   (backward operand, K = P)
    __nv_bfloat16* W2Tb;   // [H][H]   (in, out)
    // Tensor-core operand images, already laid out as K-major tiles with the
    // 128-byte swizzle (rows of 64 BF16): W2 padded to 128 rows with zeros,
    // W3 as (1 + 2 lmax) tiles of 128 rows (one per radial path).
    __nv_bfloat16* W2sw;
    __nv_bfloat16* W3sw;
    // Node-update operand images (F = 128): five 128 x 128 matrices, each two
    // K-blocks of 64 in the same swizzled layout.  NswF = [W0, U1, U2, V1, V2]
    // (out, in); NswB = their transposes (in, out) for the adjoint.
    __nv_bfloat16* NswF;
    __nv_bfloat16* NswB;
};

struct Model {
    mp_model_desc d;
    int P = 0;      // radial outputs F (1 + 2 lmax)
    int NLM = 0;    // (lmax + 1)^2
    float* emb = nullptr;      // [S][F]
    float* e0 = nullptr;       // [S]
    float* w_out = nullptr;    // [F]
    float* head = nullptr;     // W1[Hh][F], b1[Hh], W2[Hh], b2[1] contiguous
    std::vector<LayerW> layers;
    DevBuf store;              // owns every array above
};

// Neighbour graph in cell order.  perm[s] = caller id of sorted atom s.
struct Graph {
    int64_t n = 0, n_edges = 0;
    double r_list = 0.0;   // the cutoff the edges were selected with (r_c, or r_c + skin)
    double box[3];
    int nc[3];
    DevBuf perm, inv, xs, cell_start, row_ptr, col, shift, scratch;
};

struct Part {
    int64_t n_ext = 0, n_root = 0, n_edges = 0;
    std::vector<int64_t> n_le;   // atoms of hop class <= m, m = 0..K (prefix sizes)
    std::vector<int64_t> e_le;   // edges of the rows of those prefixes
    std::vector<int64_t> e_same; // edges of class-m rows whose sender is also class m
    DevBuf gid;       // int32 [n_ext]  sorted-global ids
    DevBuf is_root;   // uint8 [n_ext]
    DevBuf row_ptr;   // int64 [n_ext + 1]
    DevBuf col;       // int32 [n_edges]  local ids
    DevBuf shift;     // int8  [n_edges]
};

struct Plan {
    int n_parts = 0, k_hops = 0, mode = 0;
    int64_t n = 0;
    std::vector<Part> parts;
};

// Views of one sub-system (whole graph or one partition) for the evaluator.
struct SubSys {
    int64_t n, n_edges;
    const int64_t* row_ptr;
    const int32_t* col;
    const int8_t* shift;
    const int32_t* gid;       // local -> sorted-global id, nullptr = identity
    const uint8_t* is_root;   // nullptr = all roots
    std::vector<int64_t> n_le; // prefix sizes of hop classes 0..K (empty = all n)
    std::vector<int64_t> e_le; // their edge counts
    std::vector<int64_t> e_same; // per class m: edges with both ends in class m (empty = none)
};

struct Workspace {
    DevBuf xl, sp, H, A, S, G0, G1, alpha, floc, eatom, esum, fsum, ebuf,
        err, tmp, xw, perm_pos, pscr, pstats, red, headbuf, adam, sched, vir,
        corder,   // partition placement: cells in Morton order [ncell], sizes, offsets
        geo,      // tensor-core edge kernels: per edge (u_x, u_y, u_z, r) of a sub-system
        vfirst;   // BF16 layer 0 by hidden unit: per atom, species and (l, m), G (forward) or V (adjoint)
    void release_all() {
        DevBuf* all[] = {&xl, &sp, &H, &A, &S, &G0, &G1, &alpha, &floc, &eatom, &esum, &fsum,
                         &ebuf, &err, &tmp, &xw, &perm_pos, &pscr, &pstats, &red, &headbuf,
                         &adam, &sched, &vir, &corder, &geo, &vfirst};
        for (DevBuf* b : all) b->release();
    }
};

// Graph, plan and ledger buffers of mp_md_step, kept by the context so that
// consecutive calls reuse their device memory.
struct MdState {
    Graph g;
    Plan plan;
    DevBuf led, scal, ke, red, xref, disp;   // xref: positions at the last list build
    // the skin list kept between calls and what it was built for
    bool list_valid = false;
    int64_t list_n = 0;
    double list_r = 0.0, list_box[3] = {0, 0, 0};
    int list_parts = 0, list_mode = 0, list_hops = 0;
    void release_all() {
        DevBuf* all[] = {&g.perm, &g.inv, &g.xs, &g.cell_start, &g.row_ptr, &g.col, &g.shift,
                         &g.scratch, &led, &scal, &ke, &red, &xref, &disp};
        for (DevBuf* b : all) b->release();
        list_valid = false;
        for (Part& P : plan.parts) {
            P.gid.release(); P.is_root.release(); P.row_ptr.release(); P.col.release();
            P.shift.release();
        }
    }
};

}  // namespace mp

namespace mp {
// CUDA-event timing of kernel classes (diagnostics).
struct TimerRec {
    int id;
    cudaEvent_t a, b;
    int64_t edges, atoms;
};
struct Timing {
    bool on = false;
    std::vector<TimerRec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[MP_TIMER_COUNT] = {0};
    int64_t launches[MP_TIMER_COUNT] = {0}, edges[MP_TIMER_COUNT] = {0},
            atoms[MP_TIMER_COUNT] = {0};
};
}  // namespace mp

struct mp_ctx {
    mp::Model model;
    mp::Timing timing;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    mp::Workspace ws;
    mp::MdState md;
    int* h_err = nullptr;      // pinned host word for error read-back
    int corder_nc[3] = {0, 0, 0};   // cell grid the cached Morton order belongs to
};

struct mp_graph {
    mp::Graph g;
    mp_ctx* ctx;
};

struct mp_plan {
    mp::Plan p;
    mp_ctx* ctx;
    const mp_graph* graph;     // the graph the plan was built from (not owned)
};

namespace mp {

// neighbors.cu
int build_graph(mp_ctx* ctx, const double* d_pos, int64_t n, const double box[3], Graph& g,
                double r_list = 0.0);
// partition.cu
int build_plan(mp_ctx* ctx, const Graph& g, int n_parts, int k_hops, int mode, Plan& plan,
               double* halo_factor, const int32_t* d_assign = nullptr);
// gpart.cu
int graph_partition(mp_ctx* ctx, const Graph& g, int k, double imbalance, uint64_t seed,
                    int32_t* d_out, int64_t* cut_out);
// evaluate.cu
int evaluate(mp_ctx* ctx, const double* d_pos, const int32_t* d_species, const Graph& g,
             const Plan* plan, int n_layers, int precision, int use_head, double* d_energy,
             float* d_forces, double* d_e_atom, double* d_stress = nullptr, int part_begin = 0,
             int part_end = -1, double* d_forces64 = nullptr, bool wrap_pos = true);
// diagnostics.cu
int layer_stats(mp_ctx* ctx, const double* d_pos, const int32_t* d_species, const Graph& g, int K,
                int precision, double* h_mfs, double* h_cka);
// head.cu
int64_t head_param_count(const Model& m);
int head_loss_grad(mp_ctx* ctx, const double* d_pos, const int32_t* d_species, const Graph& g,
                   int K, int precision, const double* d_e_ref, const float* d_f_ref,
                   double lambda, double* d_loss, double* d_grad);
int head_adam(mp_ctx* ctx, const double* d_grad, double lr, double beta1, double beta2,
              double eps, int64_t step);
// scan.cu
int exclusive_scan_i64(const int32_t* in, int64_t* out, int64_t n, DevBuf& tmp, cudaStream_t s);
int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, DevBuf& tmp, cudaStream_t s);
// md.cu
int md_run(mp_ctx* ctx, double* d_pos, double* d_vel, float* d_forces, const double* d_mass,
           const int32_t* d_species, int64_t n, const double box[3], double dt, int n_steps,
           const mp_md_opts* o, double* h_ledger);
int verlet_first_half(mp_ctx* ctx, double* d_pos, double* d_vel, const double* d_forces64,
                      const double* d_mass, int64_t n, const double box[3], double dt);
int verlet_second_half(mp_ctx* ctx, double* d_vel, const double* d_forces64,
                       const double* d_mass, int64_t n, double dt, double* d_ke);

inline int grid_for(int64_t n, int block) { return (int)((n + block - 1) / block); }

// RAII scope recording start/stop events of one kernel class when timing
// is enabled on the context.
struct TimerScope {
    mp_ctx* ctx;
    int idx = -1;
    TimerScope(mp_ctx* c, int id, int64_t edges, int64_t atoms);
    ~TimerScope();
};

// Process-wide count of kernel launches issued by this library.
void note_launch();
int64_t launch_count();

}  // namespace mp

/*
 * mpip.h - C ABI of the GB300 (sm_103a) library for energy-and-force
 * evaluation of a depth-pruned message-passing interatomic potential on a
 * periodic system split into spatial partitions with ghost halos.
 *
 * Paper: "Scalable Foundation Interatomic Potentials via Message-Passing
 * Pruning and Graph Partitioning" (arXiv 2509.21694).
 *   - depth pruning: keep the first K of the backbone's message-passing
 *     layers and read the energy from layer K (Methods, "Message Passing
 *     Depth Pruning");
 *   - partitioning: spatial-grid root sets (Stage 1) extended by a K-hop
 *     neighbourhood (Stage 2), processed one after another on one GPU
 *     (Methods, "Graph Partitioning"; Results, Table 2 single-GPU columns);
 *   - output integration: E is the sum of root energies, F the sum over
 *     partitions of the gradients of root energies (Methods, "Global Output
 *     Integration").
 * The paper leaves the network equations open; the network computed here
 * is fixed in the oracle's model module header and in the design notes.
 *
 * Conventions (all calls):
 *   - Units: Angstrom, eV, amu, fs.
 *   - Pointers named d_* are DEVICE pointers owned by the caller; h_* and
 *     plain pointers are HOST pointers.  The library never frees caller
 *     memory.  Opaque objects (mp_ctx, mp_graph, mp_plan) are owned by the
 *     library and released with their *_free / mp_destroy call.
 *   - Every call enqueues work on the context's CUDA stream and returns
 *     without synchronising, except where a call documents a host read-back.
 *   - Return value: MP_OK (0) or a negative MP_ERR_* code; nothing is thrown
 *     across the ABI and no kernel traps.  mp_strerror() names a code.
 *   - Atom arrays are in the caller's atom order.  Internally atoms are
 *     re-ordered by spatial cell; the re-ordering is invisible at the ABI.
 *   - Box: orthorhombic, periodic in x, y and z, every edge >= 2 r_c.
 */
#ifndef MPIP_H
#define MPIP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MP_OK                  0
#define MP_ERR_ARG            -1  /* bad argument (null, size, mode)           */
#define MP_ERR_BOX_TOO_SMALL  -2  /* some box edge < 2 r_c                      */
#define MP_ERR_OVERLAP        -3  /* two atoms closer than 1e-3 Angstrom        */
#define MP_ERR_CAPACITY       -4  /* internal buffer too small (retried inside) */
#define MP_ERR_CUDA           -5  /* a CUDA runtime call failed                 */
#define MP_ERR_NOT_FINITE     -6  /* NaN or Inf in energy or forces             */
#define MP_ERR_NOMEM          -7  /* device allocation failed                   */
#define MP_ERR_UNSUPPORTED    -8  /* model shape not compiled in (F, lmax, ...) */
#define MP_ERR_TIMEOUT        -9  /* a bounded wait ran out                     */
#define MP_ERR_TOO_LARGE     -10  /* size beyond a fixed, documented maximum    */

/* ---- precision and partition modes --------------------------------------- */
#define MP_FP32  0   /* every contraction in FP32 on CUDA cores               */
#define MP_BF16  1   /* radial-MLP and node GEMM operands in BF16 on tcgen05
                        tensor cores, FP32 accumulation; geometry, messages,
                        features and forces stay FP32.  At layer 0 (inputs =
                        species embeddings) the last radial layer's product
                        is applied to per-row or per-atom sums over hidden
                        units instead of to every edge: the same sums in
                        another order, with the BF16 weight values        */
#define MP_HALO_GEOM 0   /* halo = atoms within K r_c (z) of the slab         */
#define MP_HALO_BFS  1   /* halo = atoms within K edges of a root (Stage 2)   */

typedef struct mp_ctx   mp_ctx;
typedef struct mp_graph mp_graph;
typedef struct mp_plan  mp_plan;

/* Model hyper-parameters.  Compiled shapes: F in {64, 128}, lmax in {1, 2},
 * H = 64, n_basis = 8, head_hidden = 32. */
typedef struct {
    int32_t n_species;      /* S, species indices are 0..S-1                */
    int32_t F;              /* channels per (l, m) block                    */
    int32_t lmax;           /* highest spherical-harmonic degree            */
    int32_t n_layers_full;  /* L_full: layers with weights                  */
    int32_t H;              /* radial MLP hidden width                      */
    int32_t n_basis;        /* Bessel functions                             */
    int32_t p_env;          /* envelope exponent p                          */
    int32_t head_hidden;    /* correction-head hidden width                 */
    double  r_cut;          /* cutoff radius r_c                            */
    double  n_avg;          /* message normaliser (constant)                */
    double  rep_eps;        /* pair repulsion strength (0 = off)            */
    double  rep_sigma;      /* pair repulsion length                        */
} mp_model_desc;

/* Number of doubles in the packed weight vector for desc (see mp_create). */
int mp_weights_count(const mp_model_desc* desc, int64_t* n_out);

/* Create a context bound to cuda_stream (a cudaStream_t; NULL = legacy
 * default stream) on the current device.  weights: host array of
 * mp_weights_count() doubles, copied (converted to FP32 and BF16 device
 * copies) before return.  Packing order, every tensor row-major, "out = W in":
 *   emb[S][F], e0[S], w_out[F],
 *   head_W1[Hh][F], head_b1[Hh], head_W2[Hh], head_b2[1],
 *   then per layer t = 0..L_full-1:
 *     W1[H][n_basis], W2[H][H], W3[P][H] (P = F(1+2 lmax), rows ordered
 *     R0, R1a, R1b, R2a, R2b, F rows each), W0[F][F], U1[F][F], U2[F][F]
 *     (lmax = 2 only), b[F], V1[F][F], V2[F][F] (lmax = 2 only).
 * Errors: MP_ERR_ARG, MP_ERR_UNSUPPORTED, MP_ERR_NOMEM, MP_ERR_CUDA. */
int mp_create(mp_ctx** ctx_out, const mp_model_desc* desc, const double* weights,
              int64_t n_weights, void* cuda_stream);
int mp_set_stream(mp_ctx* ctx, void* cuda_stream);
void mp_destroy(mp_ctx* ctx);

/* Replace the correction-head parameters (head_W1, head_b1, head_W2,
 * head_b2 packed as in mp_create) from a HOST array. */
int mp_set_head(mp_ctx* ctx, const double* head_params, int64_t n);

/* ---- neighbour list (periodic cell list) ---------------------------------
 * Builds the directed edge set of the atom graph: (i <- j, image shift n)
 * with i != j and |r_j - r_i + n L| < r_c, decided in FP64 with the
 * canonical wrap x_w = x - L floor(x / L) and the minimum image
 * n = -rint((x_w[j] - x_w[i]) / L) per axis (the graph the paper's message
 * passing and its K-hop neighbourhoods run on, Methods "Graph
 * Partitioning").  The result is bit-exact with an FP64 O(N^2) search.
 *   d_pos  [n][3] double, caller's order, any (unwrapped) coordinates.
 *   box    host double[3], edge lengths.
 * The graph keeps its own wrapped copy of the positions, the cell order and
 * a receiver-sorted CSR.  Errors: MP_ERR_ARG (also when a coordinate is
 * NaN or infinite, checked on the device), MP_ERR_BOX_TOO_SMALL,
 * MP_ERR_NOMEM, MP_ERR_CUDA. */
int mp_build_neighbors(mp_ctx* ctx, const double* d_pos, int64_t n, const double box[3],
                       mp_graph** graph_out);
/* Host read-back (synchronises): atom and directed-edge counts. */
int mp_graph_info(const mp_graph* g, int64_t* n_atoms, int64_t* n_edges);
/* Edge list in the CALLER's atom ids: d_recv, d_send int32 [n_edges],
 * d_shift int8 [n_edges] with code (n_x+1)*9 + (n_y+1)*3 + (n_z+1).  Order:
 * grouped by receiver in cell order, senders ascending in cell order. */
int mp_graph_export(const mp_graph* g, int32_t* d_recv, int32_t* d_send, int8_t* d_shift);
void mp_graph_free(mp_graph* g);

/* ---- partition (Stage 1 + Stage 2) ----------------------------------------
 * Root sets: P uniform bins of the scaled z coordinate, bin =
 * min(floor(x_w,z / L_z * P), P - 1) (Stage 1, spatial grid).  Halo:
 * MP_HALO_BFS = atoms within k_hops edges of a root (Stage 2);
 * MP_HALO_GEOM = atoms whose periodic z-distance to the slab
 * [L_z p / P, L_z (p+1) / P) is below k_hops r_c + 1e-6 (a superset).  Each
 * partition keeps the edges with both ends in its extended set.
 *   halo_factor_out  host, may be NULL: H = sum_p #halo_p / N (Supplementary
 *                    S1's halo growth factor).
 * Errors: MP_ERR_ARG, MP_ERR_NOMEM, MP_ERR_CUDA. */
int mp_partition(mp_ctx* ctx, const mp_graph* g, int n_parts, int k_hops, int mode,
                 mp_plan** plan_out, double* halo_factor_out);
/* Partitions whose roots a caller gives (Stage 1 by any partitioner, e.g.
 * mp_graph_partition for heterogeneous geometries), halos by k_hops BFS
 * expansions over the graph (Stage 2).  The partitioned result is exact for
 * any assignment: every root keeps its k_hops-hop neighbourhood.
 *   d_part  [n] int32 device, caller's atom order: partition of each atom,
 *           in 0..n_parts-1 (checked on the device; an entry outside the
 *           range makes the call return MP_ERR_ARG).  Not kept by the plan.
 *   halo_factor_out  as for mp_partition.
 * Plans export and evaluate like those of mp_partition (hop classes are BFS
 * levels).  Synchronises once.  Errors: MP_ERR_ARG, MP_ERR_NOMEM,
 * MP_ERR_CUDA. */
int mp_partition_assign(mp_ctx* ctx, const mp_graph* g, const int32_t* d_part, int n_parts,
                        int k_hops, mp_plan** plan_out, double* halo_factor_out);

/* Multilevel k-way graph partitioner (Methods, "Graph Partitioning": a
 * METIS-like partitioner for nanoparticles on supports and other
 * heterogeneous geometries, where uniform bins give unbalanced or
 * fragmented subgraphs; Supplementary S1 compares its halo growth factor
 * with the spatial grid's).  Heuristically minimises the number of cut
 * edges; every part's atom count is guaranteed <= max(ceil(N / n_parts),
 * floor((1 + imbalance) N / n_parts)).  Coarsening (heavy-edge matching and
 * contraction) and k-way boundary refinement run on the GPU; the coarsest
 * graph (at most max(1024, 128 n_parts) vertices unless matching stalls) is
 * split on the host by recursive greedy bisection, and a residual excess
 * on the atom graph is moved on the host, exactly.  The result is a
 * function of the graph and the seed only.
 *   n_parts       1..64, <= N.   imbalance  >= 0 (e.g. 0.03).
 *   d_part        [n] int32 device, written, caller's atom order.
 *   edge_cut_out  host, may be NULL: number of cut (undirected) edges.
 * Allocates and frees its own scratch; synchronises the stream several
 * times.  Errors: MP_ERR_ARG, MP_ERR_NOMEM, MP_ERR_CUDA, MP_ERR_UNSUPPORTED
 * (a coarse vertex with more than 16384 edge entries to merge). */
int mp_graph_partition(mp_ctx* ctx, const mp_graph* g, int n_parts, double imbalance,
                       uint64_t seed, int32_t* d_part, int64_t* edge_cut_out);

/* The coarsest-level step of mp_graph_partition on its own, on the host:
 * recursive greedy bisection of a graph given as HOST CSR arrays (each
 * bisection grows a region from a pseudo-peripheral vertex, adding the
 * vertex with the largest gain, until it holds its share of the vertex
 * weight; the best of 8 starts by cut).  No device work; for callers that
 * hold small host graphs, and for tests of this step.
 *   row_ptr [n+1] int64 (row_ptr[0] = 0, non-decreasing), col [row_ptr[n]]
 *   int32 in 0..n-1 (a symmetric graph), edge_w / vertex_w int32 >= 0 or
 *   NULL (= 1).
 *   part_out [n] int32, written: 0..n_parts-1.
 * Errors: MP_ERR_ARG (also for a decreasing row_ptr, a column outside
 * 0..n-1 or a negative weight; nothing is read past the arrays' ends). */
int mp_partition_host_bisect(int n, const int64_t* row_ptr, const int32_t* col,
                             const int32_t* edge_w, const int32_t* vertex_w, int n_parts,
                             uint64_t seed, int32_t* part_out);

/* Host read-back: sizes of partition p. */
int mp_plan_info(const mp_plan* plan, int p, int64_t* n_ext, int64_t* n_root, int64_t* n_edges);
/* Extended set of partition p in caller ids and a root flag per entry:
 * d_gid int32 [n_ext], d_is_root uint8 [n_ext].  Order: by hop class
 * (roots first, then halo atoms nearer than r_c + s_1, 2 r_c + s_2, ...,
 * with s_K = 1e-6 and s_m = 1e-6 m / K; for MP_HALO_BFS the BFS level),
 * within a class the cells in Morton order of their grid coordinates.  Layer t of a K-layer evaluation
 * computes only the classes <= K-1-t it needs. */
int mp_plan_export(const mp_plan* plan, int p, int32_t* d_gid, uint8_t* d_is_root);
void mp_plan_free(mp_plan* plan);

/* ---- energy and forces ----------------------------------------------------
 * Evaluates the first n_layers layers (the pruned model when n_layers <
 * L_full) and F = -dE/dr by a hand-written adjoint, either on the whole
 * graph (plan == NULL) or partition by partition with the adjoint seeded on
 * roots only and the results summed (Methods, "Global Output Integration").
 *   d_pos      [n][3] double, the positions g was built from.
 *   d_species  [n] int32 in 0..S-1 (checked on the device: an index outside
 *              the range is treated as 0 and the call returns MP_ERR_ARG).
 *   precision  MP_FP32 or MP_BF16.   use_head: add the correction head.
 *   d_energy   [1] double, written (FP64 sum of per-atom energies).
 *   d_forces   [n][3] float, written.
 *   d_e_atom   [n] double per-atom energies, or NULL.
 * Synchronises the stream once at the end (to read the device error word).
 * Errors: MP_ERR_ARG, MP_ERR_UNSUPPORTED, MP_ERR_NOMEM, MP_ERR_CUDA,
 * MP_ERR_TIMEOUT (a tensor-core kernel's bounded wait ran out). */
int mp_energy_forces(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                     const mp_graph* g, const mp_plan* plan, int n_layers, int precision,
                     int use_head, double* d_energy, float* d_forces, double* d_e_atom);

/* As mp_energy_forces, plus the stress of the potential energy (Methods,
 * "Global Output Integration": stress is assembled from the partitions like
 * the forces).
 *   d_stress  [3][3] double (device, row-major), written:
 *             sigma = (1/V) dE/d(eps), the derivative of E under the
 *             homogeneous strain r -> (I + eps) r of positions and box, in
 *             eV/A^3; V = box volume.  Computed as the virial
 *             1/(2V) sum over rows and their edges of g_e (x) d_e, with g_e
 *             the pair gradient the adjoint adds to the row's force and d_e
 *             the edge vector (each pair is visited from both ends).
 * Errors: as mp_energy_forces; MP_ERR_ARG if d_stress is NULL. */
int mp_energy_forces_stress(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                            const mp_graph* g, const mp_plan* plan, int n_layers, int precision,
                            int use_head, double* d_energy, float* d_forces, double* d_e_atom,
                            double* d_stress);

/* ---- multi-GPU partition distribution --------------------------------------
 * Partitions are independent during inference (Introduction, Fig. 1c;
 * Methods, "Global Output Integration": E = sum of root energies, F = sum
 * over partitions of the root-energy gradients), so several processes, one
 * per GPU, can each evaluate a contiguous range of one plan's partitions and
 * sum their outputs.  This call evaluates partitions part_begin ..
 * part_end - 1 of plan only and returns that range's shares in FP64:
 *   d_energy    [1] double, written: sum of the range's root energies.
 *   d_forces64  [n][3] double, written (caller order): sum over the range's
 *               partitions of the gradients of their root energies (zero for
 *               atoms in none of the range's extended sets).
 *   d_e_atom    [n] double or NULL: the range's root energies, 0 elsewhere.
 * Summing d_energy and d_forces64 over ranges that cover 0 .. n_parts - 1
 * (an all-reduce across ranks) gives mp_energy_forces' energy and its forces
 * before their FP32 rounding, up to the order of the FP64 additions.
 * Errors: as mp_energy_forces; MP_ERR_ARG for a missing plan or a range
 * outside 0 .. n_parts. */
int mp_energy_forces_parts(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                           const mp_graph* g, const mp_plan* plan, int part_begin, int part_end,
                           int n_layers, int precision, int use_head, double* d_energy,
                           double* d_forces64, double* d_e_atom);

/* ---- layer diagnostics ---------------------------------------------------
 * Methods, "Mean Feature Shift and Linear CKA": for the scalar features h0
 * (N x F) after each layer t = 0..n_layers of one unpartitioned evaluation
 * (t = 0: the embedding), centred H~ = H - (1/N) 1 1^T H:
 *   h_mfs[t] = (1/N) || H~(t+1) - H~(t) ||_F
 *   h_cka[t] = || H~(t)^T H~(t+1) ||_F^2
 *              / (|| H~(t)^T H~(t) ||_F || H~(t+1)^T H~(t+1) ||_F)
 * for t = 0..n_layers-1 (host arrays of n_layers doubles).  Sums in FP64, in
 * a fixed order.  The CKA is NaN when a layer's centred features vanish
 * (e.g. the embedding of a one-species system).  Synchronises the stream.
 * Errors: MP_ERR_ARG (n_layers < 1 or above L_full), MP_ERR_UNSUPPORTED
 * (F not a multiple of 32), those of mp_energy_forces. */
int mp_layer_stats(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                   const mp_graph* g, int n_layers, int precision, double* h_mfs,
                   double* h_cka);

/* ---- molecular dynamics ------------------------------------------------ */
typedef struct {
    int32_t n_layers;       /* K                                             */
    int32_t precision;      /* MP_FP32 / MP_BF16                             */
    int32_t n_parts;        /* partitions (1 = unpartitioned)                */
    int32_t k_hops;         /* halo depth in hops / in units of r_c; <= 0 =  */
                            /* n_layers (the depth exactness needs)          */
    int32_t halo_mode;      /* MP_HALO_GEOM / MP_HALO_BFS                    */
    int32_t use_head;       /* add the correction head                       */
    int32_t forces_valid;   /* d_forces already holds F(d_pos)               */
    int32_t check_every;    /* read the error word every n steps (0 = end)   */
    int32_t thermostat;     /* MP_NVE or MP_LANGEVIN                         */
    int32_t reserved;       /* 0                                             */
    double temperature;     /* K (Langevin)                                  */
    double friction;        /* gamma, 1/fs (Langevin)                        */
    uint64_t seed;          /* noise seed (Langevin)                         */
    int64_t step0;          /* global index of the first step (Langevin      */
                            /* noise counters; continue a run with step0 +=  */
                            /* n_steps)                                      */
    const int32_t* d_part;  /* NULL = z slabs; else [n] int32 device roots   */
                            /* per atom (caller order, as for                */
                            /* mp_partition_assign), halos by BFS            */
    double skin;            /* Verlet skin, Angstrom; 0 = neighbours and     */
                            /* partitions rebuilt after every position       */
                            /* update.  > 0: built with r_c + skin (halos in */
                            /* units of r_c + skin) and reused, also across  */
                            /* calls, until an atom has moved more than      */
                            /* skin / 2 since the build (not with d_part)    */
    int64_t* h_builds;      /* host, may be NULL: neighbour-list builds done */
                            /* by this call                                  */
} mp_md_opts;
#define MP_NVE      0
#define MP_LANGEVIN 1

/* n_steps MD steps with a = kappa F / m, kappa = 9.648533212e-3
 * Angstrom/fs^2 per eV/(Angstrom amu), rebuilding neighbours, partitions and
 * forces after every position update (with a skin: neighbours and
 * partitions only when some atom has moved more than skin / 2 since their
 * build; the result is the same, because the list holds every pair within
 * r_c until then and its pairs beyond r_c add exact zeros: R(r >= r_c) = 0).
 * MP_NVE: velocity Verlet (v += dt/2 a; r += dt v, wrapped; F; v += dt/2 a).
 * MP_LANGEVIN: BAOAB (Leimkuhler and Matthews): v += dt/2 a; r += dt/2 v;
 *   v = c1 v + c2 sqrt(kB T kappa / m) xi with c1 = exp(-gamma dt),
 *   c2 = sqrt(1 - c1^2); r += dt/2 v, wrapped; F; v += dt/2 a.  xi is the
 *   standard normal number k = ((step0 + s) N + i) 3 + a of a counter-based
 *   generator: u(j) = (splitmix64(seed ^ (0x106 << 40) ^ j) >> 11) 2^-53,
 *   xi = sqrt(-2 ln(1 - u(2k))) cos(2 pi u(2k + 1)) (atom i in the caller's
 *   order, step s of this call, axis a).  The paper's MD runs use a Langevin
 *   thermostat (Results, Table 2 conditions).
 *   d_pos, d_vel  [n][3] double, updated in place (positions are wrapped
 *                 into the box after every step, or with a skin at every
 *                 list build only: in between they continue unwrapped, so
 *                 they may lie outside the box by less than skin / 2).
 *   d_forces      [n][3] float: forces at the final positions on return.
 *   d_mass        [n] double amu.   dt_fs: time step.
 *   h_ledger      host double [n_steps][3] = (PE, KE, PE + KE) after each
 *                 step, or NULL.  Copied back at the end (synchronises).
 * Errors: as mp_build_neighbors / mp_energy_forces, MP_ERR_NOT_FINITE. */
int mp_md_step(mp_ctx* ctx, double* d_pos, double* d_vel, float* d_forces,
               const double* d_mass, const int32_t* d_species, int64_t n,
               const double box[3], double dt_fs, int n_steps, const mp_md_opts* opts,
               double* h_ledger);

/* The two halves of a velocity-Verlet step, for callers that assemble the
 * forces themselves (the multi-GPU path: FP64 force sums all-reduced across
 * ranks).  Every force is rounded to FP32 first, as mp_md_step rounds its
 * FP64 force sums, so both paths integrate the same numbers.
 * first half:  v += dt/2 kappa F / m;  r += dt v, wrapped into the box.
 * second half: v += dt/2 kappa F / m;  d_ke [1] double, written:
 *              sum_i m_i |v_i|^2 / (2 kappa) (fixed-order FP64 sum).
 *   d_forces64 [n][3] double, caller order.  Async on the context stream.
 * Errors: MP_ERR_ARG, MP_ERR_NOMEM, MP_ERR_CUDA. */
int mp_verlet_first_half(mp_ctx* ctx, double* d_pos, double* d_vel, const double* d_forces64,
                         const double* d_mass, int64_t n, const double box[3], double dt_fs);
int mp_verlet_second_half(mp_ctx* ctx, double* d_vel, const double* d_forces64,
                          const double* d_mass, int64_t n, double dt_fs, double* d_ke);

/* ---- correction head: training -------------------------------------------
 * The learned part: a per-atom head E_i^head = w2 . silu(W1 h0_i^(K) + b1)
 * + b2 on the pruned model's final scalar features, trained on energies and
 * forces of a reference model (the full-depth network) with the backbone
 * frozen.  Loss of one snapshot of N atoms:
 *   L = ((E - E_ref) / N)^2 + lambda / (3N) sum_k |F_k - F_ref,k|^2,
 * E and F the student's (backbone + head).  The gradient's force term needs
 * the tangent of h0^(K) along F - F_ref, computed by a forward-mode pass of
 * the backbone on the GPU.  Head parameters live in the context (packed as
 * in mp_create: W1[Hh][F], b1[Hh], w2[Hh], b2), count Hh F + 2 Hh + 1. */
int mp_head_count(const mp_ctx* ctx, int64_t* n_out);
/* Loss (and gradient, when d_grad != NULL) for one snapshot, whole graph.
 *   d_e_ref  [1] double device; d_f_ref [n][3] float device (caller order).
 *   d_loss   [1] double device, written; d_grad [mp_head_count] double
 *            device, written.   n_layers = K >= 1. */
int mp_head_loss_grad(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                      const mp_graph* g, int n_layers, int precision, const double* d_e_ref,
                      const float* d_f_ref, double lambda_f, double* d_loss, double* d_grad);
/* One Adam step on the context's head parameters with gradient d_grad;
 * step = 1 resets the moment estimates. */
int mp_head_adam_step(mp_ctx* ctx, const double* d_grad, double lr, double beta1, double beta2,
                      double eps, int64_t step);
/* Host copy of the current head parameters (synchronises). */
int mp_head_get(mp_ctx* ctx, double* h_params, int64_t n);

/* ---- diagnostics ---------------------------------------------------------
 * Per-context CUDA-event timing of kernel classes, on the context stream.
 * The paper has no counterpart; these calls let a caller measure the
 * library's kernels inside its own timed region. */
#define MP_TIMER_NEIGHBORS   0   /* wrap, bin, cell sort, CSR count + fill     */
#define MP_TIMER_PARTITION   1   /* root/halo flags, compaction, local CSR;
                                    also the per-edge geometry pass of the
                                    BF16 tensor-core edge kernels             */
#define MP_TIMER_EDGE_FWD    2   /* edge forward (basis, radial MLP, messages), */
                                 /* layers >= 1                                 */
#define MP_TIMER_EDGE_BWD    3   /* edge adjoint (forces, sender gradients),    */
                                 /* layers >= 1                                 */
#define MP_TIMER_NODE_FWD    4   /* node update                                 */
#define MP_TIMER_NODE_BWD    5   /* node adjoint                                */
#define MP_TIMER_EDGE_FWD_L0 6   /* edge forward of layer 0 (l >= 1 inputs zero) */
#define MP_TIMER_EDGE_BWD_L0 7   /* edge adjoint of layer 0                     */
#define MP_TIMER_NODE_FWD_L0 8   /* node update of layer 0 (timer 4: the others) */
#define MP_TIMER_NODE_BWD_L0 9   /* node adjoint of layer 0 (timer 5: the others) */
#define MP_TIMER_COUNT       10
/* enable != 0 starts recording and clears the accumulators; 0 stops. */
int mp_timing_enable(mp_ctx* ctx, int enable);
/* Synchronises the stream, then fills host arrays of MP_TIMER_COUNT
 * entries: total milliseconds, launches, edges and atoms processed. */
int mp_timing_read(mp_ctx* ctx, double* ms, int64_t* launches, int64_t* edges, int64_t* atoms);

/* Diagnostics: number of CUDA kernels this library has launched in this
 * process so far (host counter, no synchronisation).  The paper has no
 * counterpart; it lets a caller attribute GPU work to the library. */
int mp_kernel_launches(int64_t* count);

/* Self-test of the bounded waits (failure detection).  The tensor-core
 * kernels wait for their MMAs on an mbarrier with a wait that gives up after
 * a number of SM clock cycles; on a timeout they set a bit in the context's
 * device error word, drain with a second bounded wait, free their tensor
 * memory and return, and the call reports MP_ERR_TIMEOUT.  This call runs
 * the same sequence in a one-CTA kernel that holds 32 tensor-memory columns
 * and waits on an mbarrier that nothing arrives at (arrive = 0; arrive != 0
 * arrives once first, so the wait succeeds), with no MMA issued.  The paper
 * has no counterpart.
 *   max_cycles  the wait's limit in SM clock cycles, 1 .. 4e9.
 * Synchronises the context stream.  Returns MP_OK (the wait succeeded) or
 * MP_ERR_TIMEOUT (it ran out); the context stays usable either way.
 * Errors: MP_ERR_ARG, MP_ERR_NOMEM, MP_ERR_CUDA. */
int mp_wait_selftest(mp_ctx* ctx, int64_t max_cycles, int arrive);

/* ---- energy sum without device allocation ---------------------------------
 * Some callers cannot allocate device memory at the moment they need a
 * result: an MD engine that reserves all of its GPU memory in a pool at
 * start-up and forbids cudaMalloc/cudaFree during a run (they synchronise
 * the device and fragment the pool), or code running where an allocation
 * failure cannot be handled.  This call sums per-atom energies in FP64 with
 * the same fixed block-tree reduction that mp_energy_forces uses for its
 * d_energy, applied to the array as given, but keeps its block partial sums
 * in a fixed array compiled into the library instead of allocating scratch.
 * The result is deterministic, yet not bitwise equal to d_energy:
 * mp_energy_forces reduces the energies in its internal cell-sorted order,
 * while d_e_atom is in the caller's atom order, so the operands are added
 * in a different order.  The paper has no counterpart; it is a service for
 * such callers.
 *   d_e_atom   [n] double, device (e.g. the d_e_atom output of
 *              mp_energy_forces).
 *   d_energy   [1] double, device, written.
 *   cuda_stream  stream to run on (NULL = legacy default stream).
 * Limits and behaviour:
 *   - n <= MP_NOALLOC_MAX_ATOMS, else MP_ERR_TOO_LARGE and nothing runs.
 *   - Allocates nothing (no cudaMalloc, cudaFree or allocating library
 *     routine).  The fixed array (MP_NOALLOC_MAX_PARTIALS doubles, 128 KB)
 *     exists on every GPU that loads the library until the process exits.
 *   - The first call on a device looks up that array's device address
 *     (with the device current) and caches it; make that first call before
 *     any stream capture.
 *   - All calls on a GPU share that GPU's array, which keeps the last call's
 *     partial sums: calls that overlap on one GPU (for example on two
 *     streams) race and must be ordered by the caller.  Every partial is
 *     rewritten before it is read, so nothing needs clearing between calls.
 * Errors: MP_ERR_ARG (null pointer, n < 0), MP_ERR_TOO_LARGE, MP_ERR_CUDA. */
#define MP_NOALLOC_MAX_PARTIALS 16384
#define MP_NOALLOC_MAX_ATOMS    (MP_NOALLOC_MAX_PARTIALS * 2048LL)
int mp_energy_sum_noalloc(const double* d_e_atom, int64_t n, double* d_energy, void* cuda_stream);

const char* mp_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* MPIP_H */

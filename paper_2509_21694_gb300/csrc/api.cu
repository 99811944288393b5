// C ABI entry points: argument checks, context / weights / object lifetime.
#include <cmath>
#include <cstring>
#include <atomic>
#include <new>

#include "kernels.h"

namespace mp {

static std::atomic<int64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

static cudaEvent_t take_event(Timing& t) {
    if (!t.pool.empty()) {
        cudaEvent_t e = t.pool.back();
        t.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

TimerScope::TimerScope(mp_ctx* c, int id, int64_t edges, int64_t atoms) : ctx(c) {
    if (!ctx->timing.on) return;
    TimerRec r{id, take_event(ctx->timing), take_event(ctx->timing), edges, atoms};
    cudaEventRecord(r.a, ctx->stream);
    idx = (int)ctx->timing.recs.size();
    ctx->timing.recs.push_back(r);
}

TimerScope::~TimerScope() {
    if (idx >= 0) cudaEventRecord(ctx->timing.recs[idx].b, ctx->stream);
}

static void timing_collect(mp_ctx* ctx) {
    Timing& t = ctx->timing;
    for (TimerRec& r : t.recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            t.ms[r.id] += ms;
            t.launches[r.id] += 1;
            t.edges[r.id] += r.edges;
            t.atoms[r.id] += r.atoms;
        }
        t.pool.push_back(r.a);
        t.pool.push_back(r.b);
    }
    t.recs.clear();
}

int export_graph(const Graph& g, cudaStream_t st, int32_t* recv, int32_t* send, int8_t* sh);
int export_plan(const Plan& plan, const Graph& g, int p, cudaStream_t st, int32_t* gid,
                uint8_t* root);

namespace {

bool shape_supported(const mp_model_desc& d) {
    return d.H == kH && d.n_basis == kNB && d.head_hidden == kHeadH && d.p_env >= 2 &&
           d.n_species >= 1 && d.n_layers_full >= 0 && d.r_cut > 0 && d.n_avg > 0 &&
           ((d.F == 128 && d.lmax == 2) || (d.F == 64 && d.lmax == 1));
}

int64_t weights_count(const mp_model_desc& d) {
    const int64_t S = d.n_species, F = d.F, H = d.H, NB = d.n_basis, Hh = d.head_hidden;
    const int64_t P = F * (1 + 2 * d.lmax);
    const int64_t per = H * NB + H * H + P * H + F * F + d.lmax * F * F + F + d.lmax * F * F;
    return S * F + S + F + Hh * F + Hh + Hh + 1 + (int64_t)d.n_layers_full * per;
}

// Host-side layout of every device array of a model, in floats then bf16.
struct HostModel {
    std::vector<float> f;
    std::vector<__nv_bfloat16> h;
};

void transpose(const float* src, int rows, int cols, float* dst) {
    for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) dst[(size_t)c * rows + r] = src[(size_t)r * cols + c];
}

}  // namespace

static int upload_model(Model& m, const double* w) {
    const mp_model_desc& d = m.d;
    const int S = d.n_species, F = d.F, H = d.H, NB = d.n_basis, Hh = d.head_hidden;
    const int P = m.P, L = d.n_layers_full, lm = d.lmax;
    // float offsets
    size_t nf = 0, nh = 0;
    auto takef = [&](size_t k) { size_t o = nf; nf += (k + 31) / 32 * 32; return o; };
    auto takeh = [&](size_t k) { size_t o = nh; nh += (k + 63) / 64 * 64; return o; };
    size_t o_emb = takef((size_t)S * F), o_e0 = takef(S), o_wout = takef(F),
           o_head = takef((size_t)Hh * F + 2 * Hh + 1);
    struct LO { size_t W1, W2, W2T, W3, W3T, W0, W0T, U[2], UT[2], b, V[2], VT[2]; size_t W2b, W3b, W3Tb, W2Tb, W2sw, W3sw, NswF, NswB; };
    const bool tc_shape = (F == 128 && lm == 2 && H == 64);
    std::vector<LO> lo(L);
    for (int t = 0; t < L; ++t) {
        lo[t].W1 = takef((size_t)H * NB);
        lo[t].W2 = takef((size_t)H * H);
        lo[t].W2T = takef((size_t)H * H);
        lo[t].W3 = takef((size_t)P * H);
        lo[t].W3T = takef((size_t)P * H);
        lo[t].W0 = takef((size_t)F * F);
        lo[t].W0T = takef((size_t)F * F);
        for (int l = 0; l < 2; ++l) {
            lo[t].U[l] = l < lm ? takef((size_t)F * F) : 0;
            lo[t].UT[l] = l < lm ? takef((size_t)F * F) : 0;
            lo[t].V[l] = l < lm ? takef((size_t)F * F) : 0;
            lo[t].VT[l] = l < lm ? takef((size_t)F * F) : 0;
        }
        lo[t].b = takef(F);
        lo[t].W2b = takeh((size_t)H * H);
        lo[t].W3b = takeh((size_t)P * H);
        lo[t].W3Tb = takeh((size_t)P * H);
        lo[t].W2Tb = takeh((size_t)H * H);
        lo[t].W2sw = tc_shape ? takeh((size_t)128 * H) : 0;
        lo[t].W3sw = tc_shape ? takeh((size_t)P * H) : 0;
        lo[t].NswF = tc_shape ? takeh((size_t)5 * F * F) : 0;
        lo[t].NswB = tc_shape ? takeh((size_t)5 * F * F) : 0;
    }
    std::vector<float> hf(nf, 0.f);
    std::vector<__nv_bfloat16> hh(nh > 0 ? nh : 1);
    const double* p = w;
    auto rd = [&](size_t off, size_t k) {
        for (size_t q = 0; q < k; ++q) hf[off + q] = (float)p[q];
        p += k;
    };
    rd(o_emb, (size_t)S * F);
    rd(o_e0, S);
    rd(o_wout, F);
    rd(o_head, (size_t)Hh * F + 2 * Hh + 1);
    for (int t = 0; t < L; ++t) {
        rd(lo[t].W1, (size_t)H * NB);
        rd(lo[t].W2, (size_t)H * H);
        rd(lo[t].W3, (size_t)P * H);
        rd(lo[t].W0, (size_t)F * F);
        for (int l = 0; l < lm; ++l) rd(lo[t].U[l], (size_t)F * F);
        rd(lo[t].b, F);
        for (int l = 0; l < lm; ++l) rd(lo[t].V[l], (size_t)F * F);
        transpose(&hf[lo[t].W2], H, H, &hf[lo[t].W2T]);
        transpose(&hf[lo[t].W3], P, H, &hf[lo[t].W3T]);
        transpose(&hf[lo[t].W0], F, F, &hf[lo[t].W0T]);
        for (int l = 0; l < lm; ++l) {
            transpose(&hf[lo[t].U[l]], F, F, &hf[lo[t].UT[l]]);
            transpose(&hf[lo[t].V[l]], F, F, &hf[lo[t].VT[l]]);
        }
        for (size_t q = 0; q < (size_t)H * H; ++q) {
            hh[lo[t].W2b + q] = __float2bfloat16_rn(hf[lo[t].W2 + q]);
            hh[lo[t].W2Tb + q] = __float2bfloat16_rn(hf[lo[t].W2T + q]);
        }
        for (size_t q = 0; q < (size_t)P * H; ++q) {
            hh[lo[t].W3b + q] = __float2bfloat16_rn(hf[lo[t].W3 + q]);
            hh[lo[t].W3Tb + q] = __float2bfloat16_rn(hf[lo[t].W3T + q]);
        }
        if (tc_shape) {
            // swizzled images: element (row, k) at byte sw128_off(row, k) of its tile
            auto put = [&](size_t base, int row, int k, float v) {
                const int byte = row * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + (k & 7) * 2;
                hh[base + byte / 2] = __float2bfloat16_rn(v);
            };
            for (size_t q = 0; q < (size_t)128 * H; ++q) hh[lo[t].W2sw + q] = __float2bfloat16_rn(0.f);
            for (int r = 0; r < H; ++r)
                for (int k = 0; k < H; ++k) put(lo[t].W2sw, r, k, hf[lo[t].W2 + (size_t)r * H + k]);
            for (int tile = 0; tile < P / 128; ++tile)
                for (int r = 0; r < 128; ++r)
                    for (int k = 0; k < H; ++k)
                        put(lo[t].W3sw + (size_t)tile * 128 * H, r, k,
                            hf[lo[t].W3 + (size_t)(tile * 128 + r) * H + k]);
            // node matrices: K-block kb of matrix g at (2 g + kb) * 128 * 64
            const size_t mats[5] = {lo[t].W0, lo[t].U[0], lo[t].U[1], lo[t].V[0], lo[t].V[1]};
            for (int g = 0; g < 5; ++g)
                for (int r = 0; r < F; ++r)
                    for (int k = 0; k < F; ++k) {
                        const size_t blk = (size_t)(2 * g + k / 64) * 128 * 64;
                        put(lo[t].NswF + blk, r, k % 64, hf[mats[g] + (size_t)r * F + k]);
                        put(lo[t].NswB + blk, r, k % 64, hf[mats[g] + (size_t)k * F + r]);
                    }
        }
    }
    const size_t fbytes = nf * sizeof(float), hbytes = hh.size() * sizeof(__nv_bfloat16);
    MP_TRY(m.store.reserve(fbytes + hbytes + 256));
    float* base = m.store.as<float>();
    __nv_bfloat16* hbase = reinterpret_cast<__nv_bfloat16*>(
        (reinterpret_cast<uintptr_t>(base + nf) + 255) & ~uintptr_t(255));
    MP_CUDA_TRY(cudaMemcpy(base, hf.data(), fbytes, cudaMemcpyHostToDevice));
    MP_CUDA_TRY(cudaMemcpy(hbase, hh.data(), hbytes, cudaMemcpyHostToDevice));
    m.emb = base + o_emb;
    m.e0 = base + o_e0;
    m.w_out = base + o_wout;
    m.head = base + o_head;
    m.layers.resize(L);
    for (int t = 0; t < L; ++t) {
        LayerW& q = m.layers[t];
        q.W1 = base + lo[t].W1;
        q.W2 = base + lo[t].W2;
        q.W2T = base + lo[t].W2T;
        q.W3 = base + lo[t].W3;
        q.W3T = base + lo[t].W3T;
        q.W0 = base + lo[t].W0;
        q.W0T = base + lo[t].W0T;
        for (int l = 0; l < 2; ++l) {
            q.U[l] = l < lm ? base + lo[t].U[l] : nullptr;
            q.UT[l] = l < lm ? base + lo[t].UT[l] : nullptr;
            q.V[l] = l < lm ? base + lo[t].V[l] : nullptr;
            q.VT[l] = l < lm ? base + lo[t].VT[l] : nullptr;
        }
        q.b = base + lo[t].b;
        q.W2b = hbase + lo[t].W2b;
        q.W3b = hbase + lo[t].W3b;
        q.W3Tb = hbase + lo[t].W3Tb;
        q.W2Tb = hbase + lo[t].W2Tb;
        q.W2sw = tc_shape ? hbase + lo[t].W2sw : nullptr;
        q.W3sw = tc_shape ? hbase + lo[t].W3sw : nullptr;
        q.NswF = tc_shape ? hbase + lo[t].NswF : nullptr;
        q.NswB = tc_shape ? hbase + lo[t].NswB : nullptr;
    }
    return MP_OK;
}

}  // namespace mp

using namespace mp;

extern "C" {

int mp_weights_count(const mp_model_desc* desc, int64_t* n_out) {
    if (!desc || !n_out) return MP_ERR_ARG;
    *n_out = weights_count(*desc);
    return MP_OK;
}

int mp_create(mp_ctx** ctx_out, const mp_model_desc* desc, const double* weights,
              int64_t n_weights, void* cuda_stream) {
    if (!ctx_out || !desc || !weights) return MP_ERR_ARG;
    *ctx_out = nullptr;
    if (!shape_supported(*desc)) return MP_ERR_UNSUPPORTED;
    if (n_weights != weights_count(*desc)) return MP_ERR_ARG;
    for (int64_t q = 0; q < n_weights; ++q)
        if (!std::isfinite(weights[q])) return MP_ERR_ARG;
    mp_ctx* c = new (std::nothrow) mp_ctx();
    if (!c) return MP_ERR_NOMEM;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess) {
        delete c;
        return MP_ERR_CUDA;
    }
    c->model.d = *desc;
    c->model.P = desc->F * (1 + 2 * desc->lmax);
    c->model.NLM = (desc->lmax + 1) * (desc->lmax + 1);
    int rc = upload_model(c->model, weights);
    if (rc != MP_OK) {
        mp_destroy(c);
        return rc;
    }
    *ctx_out = c;
    return MP_OK;
}

int mp_set_stream(mp_ctx* ctx, void* cuda_stream) {
    if (!ctx) return MP_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return MP_OK;
}

int mp_set_head(mp_ctx* ctx, const double* head_params, int64_t n) {
    if (!ctx || !head_params) return MP_ERR_ARG;
    const int64_t want = (int64_t)ctx->model.d.head_hidden * ctx->model.d.F +
                         2 * ctx->model.d.head_hidden + 1;
    if (n != want) return MP_ERR_ARG;
    std::vector<float> h(n);
    for (int64_t q = 0; q < n; ++q) h[q] = (float)head_params[q];
    MP_CUDA_TRY(cudaMemcpyAsync(ctx->model.head, h.data(), sizeof(float) * n,
                                cudaMemcpyHostToDevice, ctx->stream));
    MP_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return MP_OK;
}

void mp_destroy(mp_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    ctx->model.store.release();
    ctx->ws.release_all();
    ctx->md.release_all();
    timing_collect(ctx);
    for (cudaEvent_t e : ctx->timing.pool) cudaEventDestroy(e);
    delete ctx;
}

int mp_build_neighbors(mp_ctx* ctx, const double* d_pos, int64_t n, const double box[3],
                       mp_graph** graph_out) {
    if (!ctx || !d_pos || !box || !graph_out || n <= 0 || n > INT32_MAX) return MP_ERR_ARG;
    *graph_out = nullptr;
    mp_graph* g = new (std::nothrow) mp_graph();
    if (!g) return MP_ERR_NOMEM;
    g->ctx = ctx;
    int rc = build_graph(ctx, d_pos, n, box, g->g);
    if (rc != MP_OK) {
        mp_graph_free(g);
        return rc;
    }
    *graph_out = g;
    return MP_OK;
}

int mp_graph_info(const mp_graph* g, int64_t* n_atoms, int64_t* n_edges) {
    if (!g) return MP_ERR_ARG;
    if (n_atoms) *n_atoms = g->g.n;
    if (n_edges) *n_edges = g->g.n_edges;
    return MP_OK;
}

int mp_graph_export(const mp_graph* g, int32_t* d_recv, int32_t* d_send, int8_t* d_shift) {
    if (!g || !d_recv || !d_send || !d_shift) return MP_ERR_ARG;
    return export_graph(g->g, g->ctx->stream, d_recv, d_send, d_shift);
}

void mp_graph_free(mp_graph* g) {
    if (!g) return;
    cudaStreamSynchronize(g->ctx->stream);
    Graph& q = g->g;
    DevBuf* bufs[] = {&q.perm, &q.inv, &q.xs, &q.cell_start, &q.row_ptr, &q.col, &q.shift,
                      &q.scratch};
    for (DevBuf* b : bufs) b->release();
    delete g;
}

int mp_partition(mp_ctx* ctx, const mp_graph* g, int n_parts, int k_hops, int mode,
                 mp_plan** plan_out, double* halo_factor_out) {
    if (!ctx || !g || !plan_out) return MP_ERR_ARG;
    *plan_out = nullptr;
    mp_plan* p = new (std::nothrow) mp_plan();
    if (!p) return MP_ERR_NOMEM;
    p->ctx = ctx;
    p->graph = g;
    int rc = build_plan(ctx, g->g, n_parts, k_hops, mode, p->p, halo_factor_out);
    if (rc != MP_OK) {
        mp_plan_free(p);
        return rc;
    }
    *plan_out = p;
    return MP_OK;
}

int mp_partition_assign(mp_ctx* ctx, const mp_graph* g, const int32_t* d_part, int n_parts,
                        int k_hops, mp_plan** plan_out, double* halo_factor_out) {
    if (!ctx || !g || !d_part || !plan_out) return MP_ERR_ARG;
    *plan_out = nullptr;
    mp_plan* p = new (std::nothrow) mp_plan();
    if (!p) return MP_ERR_NOMEM;
    p->ctx = ctx;
    p->graph = g;
    int rc = build_plan(ctx, g->g, n_parts, k_hops, MP_HALO_BFS, p->p, halo_factor_out, d_part);
    if (rc != MP_OK) {
        mp_plan_free(p);
        return rc;
    }
    *plan_out = p;
    return MP_OK;
}

int mp_graph_partition(mp_ctx* ctx, const mp_graph* g, int n_parts, double imbalance,
                       uint64_t seed, int32_t* d_part, int64_t* edge_cut_out) {
    if (!ctx || !g || !d_part) return MP_ERR_ARG;
    return graph_partition(ctx, g->g, n_parts, imbalance, seed, d_part, edge_cut_out);
}

int mp_plan_info(const mp_plan* plan, int p, int64_t* n_ext, int64_t* n_root, int64_t* n_edges) {
    if (!plan || p < 0 || p >= plan->p.n_parts) return MP_ERR_ARG;
    const Part& P = plan->p.parts[p];
    if (n_ext) *n_ext = P.n_ext;
    if (n_root) *n_root = P.n_root;
    if (n_edges) *n_edges = P.n_edges;
    return MP_OK;
}

int mp_plan_export(const mp_plan* plan, int p, int32_t* d_gid, uint8_t* d_is_root) {
    if (!plan || p < 0 || p >= plan->p.n_parts || !d_gid || !d_is_root) return MP_ERR_ARG;
    return export_plan(plan->p, plan->graph->g, p, plan->ctx->stream, d_gid, d_is_root);
}

void mp_plan_free(mp_plan* plan) {
    if (!plan) return;
    cudaStreamSynchronize(plan->ctx->stream);
    for (Part& P : plan->p.parts) {
        P.gid.release();
        P.is_root.release();
        P.row_ptr.release();
        P.col.release();
        P.shift.release();
    }
    delete plan;
}

int mp_energy_forces(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                     const mp_graph* g, const mp_plan* plan, int n_layers, int precision,
                     int use_head, double* d_energy, float* d_forces, double* d_e_atom) {
    if (!ctx || !g) return MP_ERR_ARG;
    if (plan && plan->ctx != ctx) return MP_ERR_ARG;
    return evaluate(ctx, d_pos, d_species, g->g, plan ? &plan->p : nullptr, n_layers, precision,
                    use_head, d_energy, d_forces, d_e_atom);
}

int mp_energy_forces_stress(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                            const mp_graph* g, const mp_plan* plan, int n_layers, int precision,
                            int use_head, double* d_energy, float* d_forces, double* d_e_atom,
                            double* d_stress) {
    if (!ctx || !g || !d_stress) return MP_ERR_ARG;
    if (plan && plan->ctx != ctx) return MP_ERR_ARG;
    return evaluate(ctx, d_pos, d_species, g->g, plan ? &plan->p : nullptr, n_layers, precision,
                    use_head, d_energy, d_forces, d_e_atom, d_stress);
}

int mp_energy_forces_parts(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                           const mp_graph* g, const mp_plan* plan, int part_begin, int part_end,
                           int n_layers, int precision, int use_head, double* d_energy,
                           double* d_forces64, double* d_e_atom) {
    if (!ctx || !g || !plan || plan->ctx != ctx || !d_forces64) return MP_ERR_ARG;
    if (part_begin < 0 || part_begin > part_end || part_end > (int)plan->p.parts.size())
        return MP_ERR_ARG;
    return evaluate(ctx, d_pos, d_species, g->g, &plan->p, n_layers, precision, use_head,
                    d_energy, nullptr, d_e_atom, nullptr, part_begin, part_end, d_forces64);
}

int mp_verlet_first_half(mp_ctx* ctx, double* d_pos, double* d_vel, const double* d_forces64,
                         const double* d_mass, int64_t n, const double box[3], double dt_fs) {
    if (!ctx || !box || !(dt_fs > 0)) return MP_ERR_ARG;
    return verlet_first_half(ctx, d_pos, d_vel, d_forces64, d_mass, n, box, dt_fs);
}

int mp_verlet_second_half(mp_ctx* ctx, double* d_vel, const double* d_forces64,
                          const double* d_mass, int64_t n, double dt_fs, double* d_ke) {
    if (!ctx || !(dt_fs > 0)) return MP_ERR_ARG;
    return verlet_second_half(ctx, d_vel, d_forces64, d_mass, n, dt_fs, d_ke);
}

int mp_md_step(mp_ctx* ctx, double* d_pos, double* d_vel, float* d_forces, const double* d_mass,
               const int32_t* d_species, int64_t n, const double box[3], double dt_fs,
               int n_steps, const mp_md_opts* opts, double* h_ledger) {
    if (!ctx || !box || !(dt_fs > 0)) return MP_ERR_ARG;
    return md_run(ctx, d_pos, d_vel, d_forces, d_mass, d_species, n, box, dt_fs, n_steps, opts,
                  h_ledger);
}

int mp_head_count(const mp_ctx* ctx, int64_t* n_out) {
    if (!ctx || !n_out) return MP_ERR_ARG;
    *n_out = head_param_count(ctx->model);
    return MP_OK;
}

int mp_head_loss_grad(mp_ctx* ctx, const double* d_pos, const int32_t* d_species,
                      const mp_graph* g, int n_layers, int precision, const double* d_e_ref,
                      const float* d_f_ref, double lambda_f, double* d_loss, double* d_grad) {
    if (!ctx || !g || !(lambda_f >= 0)) return MP_ERR_ARG;
    return head_loss_grad(ctx, d_pos, d_species, g->g, n_layers, precision, d_e_ref, d_f_ref,
                          lambda_f, d_loss, d_grad);
}

int mp_head_adam_step(mp_ctx* ctx, const double* d_grad, double lr, double beta1, double beta2,
                      double eps, int64_t step) {
    if (!ctx) return MP_ERR_ARG;
    return head_adam(ctx, d_grad, lr, beta1, beta2, eps, step);
}

int mp_head_get(mp_ctx* ctx, double* h_params, int64_t n) {
    if (!ctx || !h_params || n != head_param_count(ctx->model)) return MP_ERR_ARG;
    std::vector<float> h(n);
    MP_CUDA_TRY(cudaMemcpyAsync(h.data(), ctx->model.head, sizeof(float) * n,
                                cudaMemcpyDeviceToHost, ctx->stream));
    MP_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    for (int64_t q = 0; q < n; ++q) h_params[q] = h[q];
    return MP_OK;
}

int mp_timing_enable(mp_ctx* ctx, int enable) {
    if (!ctx) return MP_ERR_ARG;
    timing_collect(ctx);
    Timing& t = ctx->timing;
    for (int q = 0; q < MP_TIMER_COUNT; ++q) {
        t.ms[q] = 0;
        t.launches[q] = t.edges[q] = t.atoms[q] = 0;
    }
    t.on = enable != 0;
    return MP_OK;
}

int mp_timing_read(mp_ctx* ctx, double* ms, int64_t* launches, int64_t* edges, int64_t* atoms) {
    if (!ctx) return MP_ERR_ARG;
    timing_collect(ctx);
    const Timing& t = ctx->timing;
    for (int q = 0; q < MP_TIMER_COUNT; ++q) {
        if (ms) ms[q] = t.ms[q];
        if (launches) launches[q] = t.launches[q];
        if (edges) edges[q] = t.edges[q];
        if (atoms) atoms[q] = t.atoms[q];
    }
    return MP_OK;
}

int mp_kernel_launches(int64_t* count) {
    if (!count) return MP_ERR_ARG;
    *count = launch_count();
    return MP_OK;
}

const char* mp_strerror(int code) {
    switch (code) {
        case MP_OK: return "ok";
        case MP_ERR_ARG: return "invalid argument";
        case MP_ERR_BOX_TOO_SMALL: return "box edge shorter than 2 r_c";
        case MP_ERR_OVERLAP: return "two atoms closer than 1e-3 Angstrom";
        case MP_ERR_CAPACITY: return "internal capacity exceeded";
        case MP_ERR_CUDA: return "CUDA runtime error";
        case MP_ERR_NOT_FINITE: return "non-finite energy or forces";
        case MP_ERR_NOMEM: return "device allocation failed";
        case MP_ERR_UNSUPPORTED: return "model shape not compiled in";
        case MP_ERR_TIMEOUT: return "bounded wait timed out";
        case MP_ERR_TOO_LARGE: return "size exceeds the fixed maximum of this call";
        default: return "unknown error";
    }
}

}  // extern "C"

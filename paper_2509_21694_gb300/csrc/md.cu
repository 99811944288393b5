// Velocity-Verlet NVE driver (FP64 positions, velocities and energy ledger).
//
//   v += dt/2 kappa F / m;  x += dt v (wrapped);  rebuild neighbours and
//   partitions;  F = F(x);  v += dt/2 kappa F / m;  KE = sum m v^2 / (2 kappa)
#include <cmath>

#include "kernels.h"

namespace mp {

int reduce_sum(const double* v, int64_t n, double* out, DevBuf& tmp, cudaStream_t st);

namespace {

__global__ void k_kick_drift(int64_t n, double* __restrict__ x, double* __restrict__ v,
                             const float* __restrict__ f, const double* __restrict__ m, double dt,
                             double L0, double L1, double L2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = 0.5 * dt * kKappa / m[i];
    const double L[3] = {L0, L1, L2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double vv = v[3 * i + a] + c * (double)f[3 * i + a];
        v[3 * i + a] = vv;
        double xx = __dadd_rn(x[3 * i + a], __dmul_rn(dt, vv));
        xx = __dsub_rn(xx, __dmul_rn(L[a], floor(__ddiv_rn(xx, L[a]))));
        if (xx >= L[a]) xx = __dsub_rn(xx, L[a]);
        x[3 * i + a] = xx;
    }
}

__global__ void k_kick_ke(int64_t n, double* __restrict__ v, const float* __restrict__ f,
                          const double* __restrict__ m, double dt, double* __restrict__ ke) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = 0.5 * dt * kKappa / m[i];
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double vv = v[3 * i + a] + c * (double)f[3 * i + a];
        v[3 * i + a] = vv;
        s += vv * vv;
    }
    ke[i] = 0.5 * m[i] * s / kKappa;
}

__global__ void k_ledger(const double* __restrict__ pe, const double* __restrict__ ke,
                         double* __restrict__ row) {
    row[0] = *pe;
    row[1] = *ke;
    row[2] = *pe + *ke;
}

}  // namespace

int md_run(mp_ctx* ctx, double* d_pos, double* d_vel, float* d_forces, const double* d_mass,
           const int32_t* d_species, int64_t n, const double box[3], double dt, int n_steps,
           const mp_md_opts* o, double* h_ledger) {
    if (!o || n <= 0 || n_steps < 0 || !d_pos || !d_vel || !d_forces || !d_mass || !d_species)
        return MP_ERR_ARG;
    cudaStream_t st = ctx->stream;
    DevBuf led, scal, ke, red;
    MP_TRY(led.reserve(sizeof(double) * 3 * (n_steps > 0 ? n_steps : 1)));
    MP_TRY(scal.reserve(sizeof(double) * 4));
    MP_TRY(ke.reserve(sizeof(double) * n));
    double* pe = scal.as<double>();
    double* kes = pe + 1;
    Graph g;
    Plan plan;
    int rc = MP_OK;
    auto forces = [&]() -> int {
        MP_TRY(build_graph(ctx, d_pos, n, box, g));
        const Plan* pp = nullptr;
        if (o->n_parts > 1) {
            // the halo must reach K hops for the partitioned result to be exact
            const int hops = o->k_hops > 0 ? o->k_hops : o->n_layers;
            MP_TRY(build_plan(ctx, g, o->n_parts, hops, o->halo_mode, plan, nullptr));
            pp = &plan;
        }
        return evaluate(ctx, d_pos, d_species, g, pp, o->n_layers, o->precision, o->use_head, pe,
                        d_forces, nullptr);
    };
    if (!o->forces_valid) rc = forces();
    for (int s = 0; s < n_steps && rc == MP_OK; ++s) {
        k_kick_drift<<<grid_for(n, 256), 256, 0, st>>>(n, d_pos, d_vel, d_forces, d_mass, dt,
                                                       box[0], box[1], box[2]); note_launch();
        rc = forces();
        if (rc) break;
        k_kick_ke<<<grid_for(n, 256), 256, 0, st>>>(n, d_vel, d_forces, d_mass, dt,
                                                    ke.as<double>()); note_launch();
        rc = reduce_sum(ke.as<double>(), n, kes, red, st);
        if (rc) break;
        k_ledger<<<1, 1, 0, st>>>(pe, kes, led.as<double>() + 3 * s); note_launch();
        if (o->check_every > 0 && (s + 1) % o->check_every == 0) {
            double e = 0;
            if (cudaMemcpyAsync(&e, pe, sizeof(double), cudaMemcpyDeviceToHost, st) ||
                cudaStreamSynchronize(st)) { rc = MP_ERR_CUDA; break; }
            if (!std::isfinite(e)) { rc = MP_ERR_NOT_FINITE; break; }
        }
    }
    if (rc == MP_OK && n_steps > 0) {
        double last[3];
        if (cudaMemcpyAsync(last, led.as<double>() + 3 * (n_steps - 1), sizeof(last),
                            cudaMemcpyDeviceToHost, st) ||
            cudaStreamSynchronize(st))
            rc = MP_ERR_CUDA;
        else if (!std::isfinite(last[2]))
            rc = MP_ERR_NOT_FINITE;
        if (rc == MP_OK && h_ledger) {
            if (cudaMemcpyAsync(h_ledger, led.as<double>(), sizeof(double) * 3 * n_steps,
                                cudaMemcpyDeviceToHost, st) ||
                cudaStreamSynchronize(st))
                rc = MP_ERR_CUDA;
        }
    }
    cudaStreamSynchronize(st);
    led.release();
    scal.release();
    ke.release();
    red.release();
    g.perm.release(); g.inv.release(); g.xs.release(); g.cell_start.release();
    g.row_ptr.release(); g.col.release(); g.shift.release(); g.scratch.release();
    for (Part& P : plan.parts) {
        P.gid.release(); P.is_root.release(); P.row_ptr.release(); P.col.release();
        P.shift.release();
    }
    return rc;
}

}  // namespace mp

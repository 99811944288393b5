// MD driver (FP64 positions, velocities and energy ledger).
//
// NVE, velocity Verlet:
//   v += dt/2 kappa F / m;  x += dt v (wrapped);  rebuild neighbours and
//   partitions;  F = F(x);  v += dt/2 kappa F / m;  KE = sum m v^2 / (2 kappa)
// Langevin, BAOAB (Leimkuhler and Matthews 2013):
//   v += dt/2 kappa F / m;  x += dt/2 v;  v = c1 v + c2 sqrt(kB T kappa / m) xi;
//   x += dt/2 v (wrapped);  F = F(x);  v += dt/2 kappa F / m
//   with c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2) and xi standard normals
//   from a counter-based generator: splitmix64 (Steele, Lea and Flood) of
//   seed ^ (stream << 40) ^ counter, 53-bit uniforms, Box-Muller.
// Skin (opts.skin > 0): the neighbour list is built with r_c + skin and the
// plan's halos in units of r_c + skin, and both are reused until some atom
// has moved more than skin / 2 since the build (checked after every drift):
// until then every pair within r_c is in the list, and the list's extra
// pairs beyond r_c add exact zeros.  Positions are wrapped into the box only
// at a build, so the list's image shifts stay valid in between.
#include <cmath>
#include <cstring>

#include "kernels.h"

namespace mp {

int reduce_sum(const double* v, int64_t n, double* out, DevBuf& tmp, cudaStream_t st);

namespace {

__device__ __forceinline__ double wrap_into(double x, double L) {
    double w = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
    if (w >= L) w = __dsub_rn(w, L);
    return w;
}

__global__ void k_kick_drift(int64_t n, double* __restrict__ x, double* __restrict__ v,
                             const float* __restrict__ f, const double* __restrict__ m, double dt,
                             double L0, double L1, double L2, int wrap) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = 0.5 * dt * kKappa / m[i];
    const double L[3] = {L0, L1, L2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double vv = v[3 * i + a] + c * (double)f[3 * i + a];
        v[3 * i + a] = vv;
        double xx = __dadd_rn(x[3 * i + a], __dmul_rn(dt, vv));
        if (wrap) xx = wrap_into(xx, L[a]);
        x[3 * i + a] = xx;
    }
}

// Positions wrapped into the box in place (before a skin list is built).
__global__ void k_wrap_positions(int64_t n, double* __restrict__ x, double L0, double L1,
                                 double L2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double L[3] = {L0, L1, L2};
#pragma unroll
    for (int a = 0; a < 3; ++a) x[3 * i + a] = wrap_into(x[3 * i + a], L[a]);
}

// Largest squared displacement since the list build: a block maximum, then
// one atomicMax on the bit pattern (non-negative doubles order as integers).
__global__ void k_max_disp2(int64_t n, const double* __restrict__ x,
                            const double* __restrict__ xref, unsigned long long* __restrict__ out) {
    __shared__ double sm[256];
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double d2 = 0.0;
    if (i < n) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double d = x[3 * i + a] - xref[3 * i + a];
            d2 += d * d;
        }
        if (!(d2 == d2)) d2 = 1e300;   // NaN: force a rebuild, which reports it
    }
    sm[threadIdx.x] = d2;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sm[0]));
}

// Counter-based standard normal number k of the Langevin stream.
constexpr uint64_t kStreamLangevin = 0x106;

__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform_dev(uint64_t seed, uint64_t j) {
    const uint64_t key = seed ^ (kStreamLangevin << 40) ^ j;
    return (double)(splitmix64_dev(key) >> 11) * 0x1.0p-53;
}

__device__ __forceinline__ double normal_dev(uint64_t seed, uint64_t k) {
    const double u1 = 1.0 - uniform_dev(seed, 2 * k);     // (0, 1]
    const double u2 = uniform_dev(seed, 2 * k + 1);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
}

// B, A, O and A of a BAOAB step (the closing B follows the force update).
__global__ void k_baoab(int64_t n, double* __restrict__ x, double* __restrict__ v,
                        const float* __restrict__ f, const double* __restrict__ m, double dt,
                        double L0, double L1, double L2, double c1, double c2, double kt_kappa,
                        uint64_t seed, uint64_t k0, int wrap) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = 0.5 * dt * kKappa / m[i];
    const double sig = sqrt(kt_kappa / m[i]);
    const double L[3] = {L0, L1, L2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double vv = v[3 * i + a] + c * (double)f[3 * i + a];
        double xx = x[3 * i + a] + 0.5 * dt * vv;
        vv = c1 * vv + c2 * sig * normal_dev(seed, k0 + 3 * (uint64_t)i + a);
        xx = xx + 0.5 * dt * vv;
        if (wrap) xx = wrap_into(xx, L[a]);
        v[3 * i + a] = vv;
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

// The two Verlet halves for callers that assemble the forces themselves
// (FP64 sums of partial forces): each force is rounded to FP32 first, as the
// single-process step rounds its FP64 force sums, so both paths integrate the
// same numbers.
__global__ void k_kick_drift64(int64_t n, double* __restrict__ x, double* __restrict__ v,
                               const double* __restrict__ f, const double* __restrict__ m,
                               double dt, double L0, double L1, double L2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = 0.5 * dt * kKappa / m[i];
    const double L[3] = {L0, L1, L2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double vv = v[3 * i + a] + c * (double)(float)f[3 * i + a];
        v[3 * i + a] = vv;
        double xx = __dadd_rn(x[3 * i + a], __dmul_rn(dt, vv));
        xx = __dsub_rn(xx, __dmul_rn(L[a], floor(__ddiv_rn(xx, L[a]))));
        if (xx >= L[a]) xx = __dsub_rn(xx, L[a]);
        x[3 * i + a] = xx;
    }
}

__global__ void k_kick_ke64(int64_t n, double* __restrict__ v, const double* __restrict__ f,
                            const double* __restrict__ m, double dt, double* __restrict__ ke) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c = 0.5 * dt * kKappa / m[i];
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double vv = v[3 * i + a] + c * (double)(float)f[3 * i + a];
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

int verlet_first_half(mp_ctx* ctx, double* d_pos, double* d_vel, const double* d_forces64,
                      const double* d_mass, int64_t n, const double box[3], double dt) {
    if (n <= 0 || !d_pos || !d_vel || !d_forces64 || !d_mass) return MP_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0)) return MP_ERR_ARG;
    k_kick_drift64<<<grid_for(n, 256), 256, 0, ctx->stream>>>(n, d_pos, d_vel, d_forces64, d_mass,
                                                              dt, box[0], box[1], box[2]);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int verlet_second_half(mp_ctx* ctx, double* d_vel, const double* d_forces64,
                       const double* d_mass, int64_t n, double dt, double* d_ke) {
    if (n <= 0 || !d_vel || !d_forces64 || !d_mass || !d_ke) return MP_ERR_ARG;
    cudaStream_t st = ctx->stream;
    MdState& md = ctx->md;
    MP_TRY(md.ke.reserve(sizeof(double) * n));
    k_kick_ke64<<<grid_for(n, 256), 256, 0, st>>>(n, d_vel, d_forces64, d_mass, dt,
                                                  md.ke.as<double>());
    note_launch();
    MP_TRY(reduce_sum(md.ke.as<double>(), n, d_ke, md.red, st));
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

int md_run(mp_ctx* ctx, double* d_pos, double* d_vel, float* d_forces, const double* d_mass,
           const int32_t* d_species, int64_t n, const double box[3], double dt, int n_steps,
           const mp_md_opts* o, double* h_ledger) {
    if (!o || n <= 0 || n_steps < 0 || !d_pos || !d_vel || !d_forces || !d_mass || !d_species)
        return MP_ERR_ARG;
    if (o->thermostat != MP_NVE && o->thermostat != MP_LANGEVIN) return MP_ERR_ARG;
    if (o->thermostat == MP_LANGEVIN && !(o->temperature >= 0.0 && o->friction >= 0.0))
        return MP_ERR_ARG;
    if (!(o->skin >= 0.0 && o->skin < 1e3)) return MP_ERR_ARG;
    cudaStream_t st = ctx->stream;
    MdState& md = ctx->md;
    DevBuf &led = md.led, &scal = md.scal, &ke = md.ke, &red = md.red;
    MP_TRY(led.reserve(sizeof(double) * 3 * (n_steps > 0 ? n_steps : 1)));
    MP_TRY(scal.reserve(sizeof(double) * 4));
    MP_TRY(ke.reserve(sizeof(double) * n));
    double* pe = scal.as<double>();
    double* kes = pe + 1;
    Graph& g = md.g;
    Plan& plan = md.plan;
    int rc = MP_OK;
    const double c1 = exp(-o->friction * dt), c2 = sqrt(1.0 - c1 * c1);
    const double kt_kappa = 8.617333262e-5 * o->temperature * kKappa;   // kB T kappa
    const bool skin = o->skin > 0.0;
    const double r_list = skin ? ctx->model.d.r_cut + o->skin : 0.0;
    const double half2 = 0.25 * o->skin * o->skin;
    int64_t builds = 0;
    if (skin) {
        MP_TRY(md.xref.reserve(sizeof(double) * 3 * n));
        MP_TRY(md.disp.reserve(64));
    }
    // a skin list from an earlier call is reused only if it belongs to this
    // system size, box, cutoff and partitioning (and, checked below, no atom
    // has moved more than skin / 2 since it was built)
    bool list_ok = skin && md.list_valid && md.list_n == n && md.list_r == r_list &&
                   md.list_box[0] == box[0] && md.list_box[1] == box[1] &&
                   md.list_box[2] == box[2] && md.list_parts == o->n_parts &&
                   md.list_mode == (o->d_part ? MP_HALO_BFS : o->halo_mode) &&
                   md.list_hops == (o->k_hops > 0 ? o->k_hops : o->n_layers) && !o->d_part;
    auto moved_too_far = [&](bool& far) -> int {
        unsigned long long* dm = md.disp.as<unsigned long long>();
        MP_CUDA_TRY(cudaMemsetAsync(dm, 0, sizeof(unsigned long long), st));
        k_max_disp2<<<grid_for(n, 256), 256, 0, st>>>(n, d_pos, md.xref.as<double>(), dm);
        note_launch();
        unsigned long long h = 0;
        MP_CUDA_TRY(cudaMemcpyAsync(&h, dm, sizeof(h), cudaMemcpyDeviceToHost, st));
        MP_CUDA_TRY(cudaStreamSynchronize(st));
        double d2;
        memcpy(&d2, &h, sizeof(d2));
        far = !(d2 <= half2);
        return MP_OK;
    };
    auto forces = [&]() -> int {
        bool build = !list_ok;
        if (!build) MP_TRY(moved_too_far(build));
        const int hops = o->k_hops > 0 ? o->k_hops : o->n_layers;
        if (build) {
            if (skin) {
                k_wrap_positions<<<grid_for(n, 256), 256, 0, st>>>(n, d_pos, box[0], box[1],
                                                                   box[2]);
                note_launch();
            }
            list_ok = false;
            md.list_valid = false;
            MP_TRY(build_graph(ctx, d_pos, n, box, g, r_list));
            if (o->n_parts > 1)   // the halo must reach K hops for the result to be exact
                MP_TRY(build_plan(ctx, g, o->n_parts, hops, o->d_part ? MP_HALO_BFS : o->halo_mode,
                                  plan, nullptr, o->d_part));
            ++builds;
            if (skin) {
                MP_CUDA_TRY(cudaMemcpyAsync(md.xref.as<double>(), d_pos, sizeof(double) * 3 * n,
                                            cudaMemcpyDeviceToDevice, st));
                list_ok = !o->d_part;
                md.list_valid = list_ok;
                md.list_n = n;
                md.list_r = r_list;
                for (int a = 0; a < 3; ++a) md.list_box[a] = box[a];
                md.list_parts = o->n_parts;
                md.list_mode = o->d_part ? MP_HALO_BFS : o->halo_mode;
                md.list_hops = hops;
            }
        }
        return evaluate(ctx, d_pos, d_species, g, o->n_parts > 1 ? &plan : nullptr, o->n_layers,
                        o->precision, o->use_head, pe, d_forces, nullptr, nullptr, 0, -1, nullptr,
                        !skin);
    };
    if (!skin) md.list_valid = false;
    if (!o->forces_valid) rc = forces();
    for (int s = 0; s < n_steps && rc == MP_OK; ++s) {
        if (o->thermostat == MP_LANGEVIN)
            k_baoab<<<grid_for(n, 256), 256, 0, st>>>(
                n, d_pos, d_vel, d_forces, d_mass, dt, box[0], box[1], box[2], c1, c2, kt_kappa,
                o->seed, (uint64_t)(o->step0 + s) * 3 * (uint64_t)n, skin ? 0 : 1);
        else
            k_kick_drift<<<grid_for(n, 256), 256, 0, st>>>(n, d_pos, d_vel, d_forces, d_mass, dt,
                                                           box[0], box[1], box[2], skin ? 0 : 1);
        note_launch();
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
    if (o->h_builds) *o->h_builds = builds;
    if (rc != MP_OK) md.list_valid = false;
    return rc;   // graph, plan and ledger buffers stay with the context for the next call
}

}  // namespace mp

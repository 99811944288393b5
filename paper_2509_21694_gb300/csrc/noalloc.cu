// Energy sum that allocates no device memory (mp_energy_sum_noalloc).
//
// Same reduction as the one behind mp_energy_forces' d_energy: blocks of 256
// threads each sum 2048 consecutive values in a fixed order, then one block
// sums the block partials in a fixed order.  The partials live in a
// file-scope __device__ array instead of allocated scratch.  In host code
// the array's name is only a host-side stand-in, so its device address is
// looked up once per device with cudaGetSymbolAddress and passed to the
// kernels.
#include <mutex>

#include "common.cuh"

namespace mp {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
static_assert(MP_NOALLOC_MAX_ATOMS == (long long)MP_NOALLOC_MAX_PARTIALS * kThreads * kItems,
              "header limit must match the reduction geometry");

static __device__ __align__(256) double g_noalloc_partials[MP_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
double* g_addr[kMaxDevices] = {nullptr};

__global__ void k_noalloc_partial(const double* __restrict__ v, int64_t n,
                                  double* __restrict__ part) {
    __shared__ double sm[kThreads];
    const int64_t base = (int64_t)blockIdx.x * kThreads * kItems;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int64_t idx = base + (int64_t)q * kThreads + threadIdx.x;
        if (idx < n) acc += v[idx];
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}

__global__ void k_noalloc_final(const double* __restrict__ part, int64_t m,
                                double* __restrict__ out) {
    __shared__ double sm[kThreads];
    double acc = 0.0;
    for (int64_t idx = threadIdx.x; idx < m; idx += kThreads) acc += part[idx];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sm[0];
}

// Device address of the partials array on the current device (looked up on
// the first call per device, then cached).
int partials_address(double** out) {
    int dev = 0;
    MP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return MP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
            cudaGetLastError();
            return MP_ERR_CUDA;
        }
        g_addr[dev] = static_cast<double*>(p);
    }
    *out = g_addr[dev];
    return MP_OK;
}

}  // namespace

}  // namespace mp

extern "C" int mp_energy_sum_noalloc(const double* d_e_atom, int64_t n, double* d_energy,
                                     void* cuda_stream) {
    using namespace mp;
    if (!d_energy || n < 0 || (n > 0 && !d_e_atom)) return MP_ERR_ARG;
    if (n > (int64_t)MP_NOALLOC_MAX_ATOMS) return MP_ERR_TOO_LARGE;
    double* part = nullptr;
    MP_TRY(partials_address(&part));
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int64_t per = (int64_t)kThreads * kItems;
    const int64_t blocks = (n + per - 1) / per;
    if (blocks > 0) {
        k_noalloc_partial<<<(unsigned)blocks, kThreads, 0, st>>>(d_e_atom, n, part);
        note_launch();
    }
    k_noalloc_final<<<1, kThreads, 0, st>>>(part, blocks, d_energy);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

// Deterministic device-wide exclusive prefix sums (three passes: tile sums,
// scan of tile sums, tile re-scan with offsets).
#include "common.cuh"

namespace mp {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kItems = 4;
constexpr int kTile = kScanThreads * kItems;

template <class Out>
__device__ Out block_exclusive_scan(Out v, Out* smem, Out* total) {
    // Warp-shuffle scan, then a scan of the 32 warp totals.
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Out x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Out y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[warp] = x;
    __syncthreads();
    if (warp == 0) {
        Out w = (lane < (int)(blockDim.x >> 5)) ? smem[lane] : Out(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            Out y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        smem[lane] = w;
    }
    __syncthreads();
    Out warp_prefix = warp ? smem[warp - 1] : Out(0);
    *total = smem[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

template <class Out>
__global__ void k_tile_sums(const int32_t* __restrict__ in, int64_t n, Out* __restrict__ sums) {
    __shared__ Out sm[32];
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    Out s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k)
        if (base + k < n) s += (Out)in[base + k];
    Out total;
    block_exclusive_scan<Out>(s, sm, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <class Out>
__global__ void k_scan_small(Out* __restrict__ v, int64_t m) {
    // One block: each thread scans a contiguous run, then runs are offset.
    __shared__ Out sm[32];
    int64_t per = (m + blockDim.x - 1) / blockDim.x;
    int64_t b = (int64_t)threadIdx.x * per, e = b + per < m ? b + per : m;
    Out s = 0;
    for (int64_t i = b; i < e; ++i) s += v[i];
    Out total;
    Out off = block_exclusive_scan<Out>(s, sm, &total);
    for (int64_t i = b; i < e; ++i) {
        Out t = v[i];
        v[i] = off;
        off += t;
    }
}

template <class Out>
__global__ void k_tile_scan(const int32_t* __restrict__ in, int64_t n,
                            const Out* __restrict__ offs, Out* __restrict__ out) {
    __shared__ Out sm[32];
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    Out vals[kItems];
    Out s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        vals[k] = (base + k < n) ? (Out)in[base + k] : Out(0);
        s += vals[k];
    }
    Out total;
    Out pre = block_exclusive_scan<Out>(s, sm, &total) + offs[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (base + k < n) out[base + k] = pre;
        pre += vals[k];
    }
    // the element one past the end receives the grand total
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = pre;
}

template <class Out>
int scan_impl(const int32_t* in, Out* out, int64_t n, DevBuf& tmp, cudaStream_t s) {
    if (n == 0) {
        MP_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(Out), s));
        return MP_OK;
    }
    int64_t tiles = (n + kTile - 1) / kTile;
    MP_TRY(tmp.reserve(sizeof(Out) * (size_t)tiles));
    Out* sums = tmp.as<Out>();
    k_tile_sums<Out><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums); note_launch();
    k_scan_small<Out><<<1, kScanThreads, 0, s>>>(sums, tiles); note_launch();
    k_tile_scan<Out><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums, out); note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    return MP_OK;
}

}  // namespace

// out[0..n] = exclusive prefix sums of in[0..n-1]; out[n] = total.
int exclusive_scan_i64(const int32_t* in, int64_t* out, int64_t n, DevBuf& tmp, cudaStream_t s) {
    return scan_impl<long long>(in, reinterpret_cast<long long*>(out), n, tmp, s);
}

int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, DevBuf& tmp, cudaStream_t s) {
    return scan_impl<int>(in, out, n, tmp, s);
}

int DevBuf::reserve(size_t nbytes) {
    if (nbytes <= bytes && p) return MP_OK;
    // a buffer that has to grow gets 1/8 of headroom, so sizes that drift
    // from one MD step to the next (edge counts) do not reallocate each time
    const bool grow = p != nullptr;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    size_t want = nbytes < 256 ? 256 : nbytes;
    if (grow) want += want / 8;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        return MP_ERR_NOMEM;
    }
    bytes = want;
    return MP_OK;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

}  // namespace mp

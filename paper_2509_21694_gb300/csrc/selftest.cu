// Self-test of the bounded-wait path of the tensor-core kernels
// (mp_wait_selftest).
//
// The tensor-core kernels wait for their MMAs on an mbarrier with a wait that
// gives up after a number of SM clock cycles; a warpgroup whose wait ran out
// sets a bit in the context's device error word, gives its in-flight work a
// second bounded wait, frees the CTA's tensor memory and returns, and the
// host turns the bit into MP_ERR_TIMEOUT.  A timeout cannot be provoked in
// those kernels without breaking them, so this kernel takes the same steps
// on its own: one CTA allocates tensor-memory columns, initialises an
// mbarrier with one expected arrival and (unless asked to arrive) lets
// nothing arrive, waits with the caller's cycle limit, and on a timeout
// drains with the same limit, sets the bit, frees the columns and returns.
// No MMA is issued, so nothing is in flight when it gives up.
#include "kernels.h"
#include "tc.cuh"

namespace mp {

namespace {

constexpr int kErrSelfTimeout = 16;   // error-word bit of this self-test
constexpr int kSelfCols = 32;         // tensor-memory columns held during the wait

__global__ void __launch_bounds__(128, 1) k_wait_selftest(long long max_cycles, int arrive,
                                                          int* __restrict__ err) {
    __shared__ uint64_t mbar;
    __shared__ uint32_t taddr;
    __shared__ int timed_out;
    const int tid = threadIdx.x;
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        timed_out = 0;
    }
    if ((tid >> 5) == 0) tc::tmem_alloc<kSelfCols>(&taddr);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (arrive && tid == 0) {
        uint64_t state;
        asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];"
                     : "=l"(state) : "r"(tc::smem_u32(&mbar)) : "memory");
    }
    // every thread waits for phase 0, as the kernels' warpgroups do
    if (!tc::mbar_wait(&mbar, 0, max_cycles)) timed_out = 1;
    __syncthreads();
    if (timed_out) {
        tc::mbar_wait(&mbar, 0, max_cycles);   // the drain: bounded as well
        if (tid == 0) atomicOr(err, kErrSelfTimeout);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if ((tid >> 5) == 0) tc::tmem_dealloc<kSelfCols>(taddr);
}

}  // namespace

int wait_selftest(mp_ctx* ctx, int64_t max_cycles, int arrive) {
    cudaStream_t st = ctx->stream;
    MP_TRY(ctx->ws.err.reserve(64));
    int* err = ctx->ws.err.as<int>();
    MP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    k_wait_selftest<<<1, 128, 0, st>>>((long long)max_cycles, arrive ? 1 : 0, err);
    note_launch();
    MP_CUDA_TRY(cudaGetLastError());
    int herr = 0;
    MP_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MP_CUDA_TRY(cudaStreamSynchronize(st));
    return (herr & kErrSelfTimeout) ? MP_ERR_TIMEOUT : MP_OK;
}

}  // namespace mp

extern "C" int mp_wait_selftest(mp_ctx* ctx, int64_t max_cycles, int arrive) {
    if (!ctx || max_cycles < 1 || max_cycles > 4000000000LL) return MP_ERR_ARG;
    return mp::wait_selftest(ctx, max_cycles, arrive);
}

// Self-check of the failure-detection path shared by the tcgen05 / TMA kernels: one 32-thread
// block takes TMEM, waits on an mbarrier with the same bounded wait (tc::mbar_wait) the
// pipelines use, then frees TMEM and returns.  With `arrive` the block arrives on the barrier
// first and the wait succeeds; without it nothing ever arrives, the wait gives up after
// `limit_ns` and records tc::ERR_WAIT_CHECK in the parameter set's error flag, which
// hefx_stream_check reports as HEFX_ETIMEOUT.  Nothing else is in flight when the wait gives
// up, so the kernel ends cleanly and the context stays usable.
#include "hefx_internal.h"
#include "tc_common.cuh"

namespace hefx {
namespace {

__global__ void __launch_bounds__(32, 1) wait_check_kernel(uint32_t* err, uint64_t limit_ns, int arrive) {
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_slot;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    tc::tmem_alloc(&tmem_slot, 32);  // warp-wide; the waiting pipeline role holds TMEM like this
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (threadIdx.x == 0) {
        if (arrive) tc::mbar_arrive(&bar);
        tc::mbar_wait(&bar, 0, err, tc::ERR_WAIT_CHECK, limit_ns);
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 32);
}

}  // namespace

cudaError_t launch_wait_check(uint32_t* err, uint64_t limit_ns, int arrive, cudaStream_t s) {
    wait_check_kernel<<<1, 32, 0, s>>>(err, limit_ns, arrive);
    return cudaGetLastError();
}

}  // namespace hefx

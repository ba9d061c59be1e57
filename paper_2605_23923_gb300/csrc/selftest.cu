// Self-test of the device-side bounded waits that every multi-CTA kernel of
// this library relies on (no counterpart in the paper): one small kernel waits
// on something that never happens -- a counter that nothing increments, or an
// mbarrier phase that nothing arrives on -- with the same helpers the kernels
// use.  After about a second the wait gives up, latches the plan's error word
// and the kernel returns normally, so the context stays usable and the host
// reads SU2_ERR_TIMEOUT from su2_sync_status.
#include <cuda_runtime.h>

#include "common.cuh"
#include "su2_internal.h"

namespace su2 {

__global__ void bounded_wait_selftest(const unsigned* never, int* err, int kind) {
    __shared__ uint64_t bar;
    if (kind == 1) {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            mbar_fence_init();
        }
        __syncthreads();
        if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, err);    // phase 0 never completes
    } else if (threadIdx.x == 0) {
        wait_counter_bounded(never, 1u, err);                      // *never stays 0
    }
}

cudaError_t launch_bounded_wait_selftest(const unsigned* never, int* err, int kind, cudaStream_t st) {
    bounded_wait_selftest<<<1, 32, 0, st>>>(never, err, kind);
    return cudaGetLastError();
}

}  // namespace su2

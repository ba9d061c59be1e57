// Allocation-free forward transform: su2_forward with the stage-1 planes held
// in a fixed-size scratch array that lives in this library's device image
// instead of a caller-provided workspace.
//
// Who needs this: callers that cannot allocate device memory when they run a
// transform -- code that has no device allocator at hand (a plain C host
// program that only receives device pointers from elsewhere), code that runs
// under a fixed memory budget where every cudaMalloc must happen up front, or
// steady-state loops that must not touch the allocator.  They still create
// the plan beforehand (su2_plan allocates its small tables once) and pass the
// grid and coefficient buffers; the planes go to the array below.
//
// The array occupies SU2_NOALLOC_SCRATCH_BYTES on every GPU that loads this
// library, for the lifetime of the process.  Host code cannot use the array's
// name as a device address, so the device address is looked up with
// cudaGetSymbolAddress, with the device current, and cached per device.  The
// lookup is done by su2_plan (noalloc_prepare), not by the entry point: under
// CUDA's lazy module loading it is what loads this file's module, array
// included, onto the device, and plan creation allocates its tables anyway.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/su2fft.h"
#include "su2_internal.h"

static __device__ __align__(256) unsigned char su2_noalloc_scratch[SU2_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::atomic<void*> g_scratch_ptr[kMaxDevices];

}  // namespace

namespace su2 {
cudaError_t noalloc_prepare(int device) {
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    if (g_scratch_ptr[device].load(std::memory_order_acquire)) return cudaSuccess;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, su2_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_scratch_ptr[device].store(p, std::memory_order_release);
    return cudaSuccess;
}
}  // namespace su2

extern "C" su2_status su2_forward_noalloc(su2_plan_t plan, const void* grid, void* coeffs, void* cuda_stream) {
    if (!plan || !grid || !coeffs) return SU2_ERR_INVALID_ARG;
    size_t need = 0;
    su2_status s = su2_workspace_size(plan, &need);
    if (s != SU2_OK) return s;
    if (need > (size_t)SU2_NOALLOC_SCRATCH_BYTES) return SU2_ERR_WORKSPACE;
    const int plan_dev = su2::plan_device(plan);     // su2_forward runs on the plan's device
    if (plan_dev < 0 || plan_dev >= kMaxDevices) return SU2_ERR_CUDA;
    void* ptr = g_scratch_ptr[plan_dev].load(std::memory_order_acquire);
    if (!ptr) return SU2_ERR_CUDA;                   // su2_plan looked it up on this device
    // launch by launch even for SU2_FLAG_CUDA_GRAPH plans: recording and
    // instantiating a graph would allocate
    return (su2_status)su2::forward_direct(plan, grid, coeffs, ptr, cuda_stream);
}

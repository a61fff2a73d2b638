// tct_noalloc.cu -- tct_build_evaluate for callers that cannot allocate.
//
// Some callers have no way to obtain device memory at the point where they
// want a tomogram: code that runs under a pre-reserved memory budget where
// cudaMalloc is forbidden after start-up (a robot's real-time control loop),
// a plug-in whose host application owns the only allocator, or an
// environment whose allocation calls are intercepted and refused.  For them
// this entry point takes its scratch from a fixed array compiled into the
// library instead of a caller-provided workspace.  The caller still passes
// the points and every output buffer.
//
// The array below is TCT_NOALLOC_SCRATCH_BYTES per device; a GPU keeps it
// from the moment the library's code for it is loaded there until the
// process exits.  Its device address is looked up once per device (with
// that device current) by the first call on the device, so that first call
// should be made before any stream capture begins.  All calls share the one
// array and it keeps whatever the last call left in it; the build clears
// every part it relies on being zero before use.  Calls whose work overlaps
// on the GPU (other streams, other host threads) race on the array and must
// be serialised by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "tct_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[TCT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices];

// Device address of the scratch array on the current device.  In host code
// the array's name only stands for the symbol; the address the kernels need
// comes from cudaGetSymbolAddress, asked once per device.
int scratch_on_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TCT_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return TCT_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return TCT_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TCT_OK;
}

}  // namespace

extern "C" int tct_build_evaluate_noalloc(const float *d_xyz, int64_t n, int32_t stride,
                                          const tct_grid *grid, const tct_params *params,
                                          float *d_ground, float *d_ceil, float *d_cost,
                                          uint8_t *d_mask, uint8_t *d_keep, tct_stats *d_stats,
                                          tct_stream stream) {
    // an invalid grid reports 0 here and is rejected by tct_build_evaluate
    if (tct_workspace_bytes(grid, n, params) > (size_t)TCT_NOALLOC_SCRATCH_BYTES)
        return TCT_ERR_WORKSPACE_TOO_SMALL;
    void *scratch = nullptr;
    const int rc = scratch_on_current_device(&scratch);
    if (rc != TCT_OK) return rc;
    return tct_build_evaluate(d_xyz, n, stride, grid, params, scratch,
                              (size_t)TCT_NOALLOC_SCRATCH_BYTES, d_ground, d_ceil, d_cost, d_mask,
                              d_keep, d_stats, stream);
}

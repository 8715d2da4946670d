// mot_fastsum_static: the kernel matrix-vector product for callers that cannot allocate GPU memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: plug-ins of a host
// application that owns all device memory through its own pool (they get no allocator and no
// spare buffer to lend), and real-time loops where an allocation could block or fail at the
// wrong moment.  For them this entry point keeps its scratch in one file-scope __device__
// array that is created when the library's device code is loaded on a GPU and lives until the
// process exits (every GPU that loads the library holds MOT_STATIC_SCRATCH_BYTES of it).
//
// Set-up: the first call on each device (with that device current) looks up the array's
// device address with cudaGetSymbolAddress, checks the return code and caches it per device;
// make that first call before any stream capture.  The host-side name of the array is only a
// stand-in and is never passed to a kernel.  All calls share the array and it keeps the
// previous call's contents; the fast summation clears everything that must start at zero
// (grids, bin counts) on the stream before use.  Calls whose work overlaps on the GPU
// (different streams or threads, same device) race on the array and must be serialised by the
// caller.  Like mot_fastsum, a call ends by reading a few scalars back on its stream and
// synchronising that stream.
#include <mutex>

#include "motfft.h"
#include <cuda_runtime.h>

namespace {

__device__ __align__(256) unsigned char g_mot_static_scratch[MOT_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

int scratch_for_current_device(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MOT_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_ptr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_mot_static_scratch);
        if (e != cudaSuccess || p == nullptr) return MOT_ECUDA;
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return MOT_OK;
}

}  // namespace

extern "C" int mot_fastsum_static(int d, double eta, const float* x_src, int64_t n_src, const float* x_tgt,
                                  int64_t n_tgt, const float* alpha, int nrhs, float* beta,
                                  const mot_options* opt, double* scale_out, void* stream) {
    size_t need = 0;
    int rc = mot_fastsum_workspace_bytes(d, n_src, n_tgt, nrhs, opt, &need);
    if (rc != MOT_OK) return rc;
    if (need > (size_t)MOT_STATIC_SCRATCH_BYTES) return MOT_ENOMEM;   // request exceeds the static scratch
    void* ws = nullptr;
    rc = scratch_for_current_device(&ws);
    if (rc != MOT_OK) return rc;
    return mot_fastsum(d, eta, x_src, n_src, x_tgt, n_tgt, alpha, nrhs, beta, opt, ws,
                       (size_t)MOT_STATIC_SCRATCH_BYTES, scale_out, stream);
}

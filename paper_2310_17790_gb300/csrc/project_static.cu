// nsf_project_static: the network inversion of nsf_project with its scratch
// memory in a fixed file-scope device array instead of a caller workspace.
//
// Some callers cannot allocate device memory when they need the inversion:
// a host application whose memory manager owns every device allocation and
// forbids outside ones, a real-time loop that must never enter the CUDA
// allocator, or a plugin that has no place to keep a workspace alive between
// calls.  This entry point lets them run it anyway: the caller still passes
// the inputs and outputs, and the scratch lives in `g_project_scratch`, which
// every GPU that loads the library holds until the process exits.
#include <mutex>

#include <cuda_runtime.h>

#include "nsf.h"

namespace {

// Fixed scratch for nsf_project_static (NSF_PROJECT_STATIC_BYTES bytes).
static __device__ __align__(256) unsigned char g_project_scratch[NSF_PROJECT_STATIC_BYTES];

// Device address of the array, looked up once per device.  In host code the
// symbol itself is only a host-side stand-in, never a device pointer.
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

nsf_status scratch_for_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return NSF_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_project_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return NSF_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return NSF_OK;
}

}  // namespace

extern "C" nsf_status nsf_project_static(const nsf_fields *fields, const float *d_X_S,
                                         const float *d_x_target, int n_S, double *d_z_inout,
                                         const nsf_gn_opts *opts, double *d_z_iter,
                                         float *d_residual, int *d_status, void *stream) {
    if (!fields || n_S < 1) return NSF_ERR_INVALID_ARG;
    if (n_S > NSF_PROJECT_STATIC_MAX_S) return NSF_ERR_WORKSPACE;
    size_t need = 0;
    nsf_status st = nsf_project_workspace_size(fields, n_S, &need);
    if (st != NSF_OK) return st;
    if (need > (size_t)NSF_PROJECT_STATIC_BYTES) return NSF_ERR_WORKSPACE;
    void *ws = nullptr;
    st = scratch_for_current_device(&ws);
    if (st != NSF_OK) return st;
    // The array keeps the previous call's contents: start from zeros, as a
    // fresh workspace would.
    if (cudaMemsetAsync(ws, 0, need, static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return NSF_ERR_CUDA;
    return nsf_project(fields, d_X_S, d_x_target, n_S, d_z_inout, opts, d_z_iter, d_residual, ws,
                       need, d_status, stream);
}

// rast_mesh_fwd_static: the forward rasterizer for callers that cannot
// allocate device memory.
//
// Some callers have no way to hand this library a workspace: code running
// where cudaMalloc is forbidden or unavailable (a host framework that owns
// every allocation and exposes none to plugins, a real-time loop that must
// not allocate after start-up, or an environment whose allocator is not
// reachable from the calling thread).  For them this entry point runs the
// same forward as rast_mesh_fwd on a workspace that lives in a fixed-size
// device array inside this library, so the caller passes only inputs and
// outputs.  It never calls cudaMalloc, cudaFree or any allocating routine.
#include <cuda_runtime.h>

#include <mutex>

#include "meshrast.h"

// The shared scratch: every GPU that loads the library holds these bytes
// until the process exits.
static __device__ __align__(256) unsigned char g_static_workspace[MESHRAST_STATIC_WORKSPACE_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void *g_ws_ptr[kMaxDevices];
std::mutex g_ws_mutex;

// The array's name in host code is only a host-side stand-in; its device
// address is looked up with the device current, on the first call on that
// device, and kept.  A failed lookup is not kept: the next call tries again.
cudaError_t device_workspace(void **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_ws_mutex);
    if (g_ws_ptr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_workspace);
        if (e != cudaSuccess) return e;
        g_ws_ptr[dev] = p;
    }
    *ptr = g_ws_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" MESHRAST_API int rast_mesh_fwd_static(const rast_params *p, const float *verts, int64_t V,
                                                 const int64_t *faces, int64_t F, const int64_t *first_face,
                                                 const int64_t *num_faces, const float *cams, int64_t *pix_to_face,
                                                 float *zbuf, float *bary, float *dists, void *stream) {
    const size_t need = rast_workspace_bytes(p, V, F);
    if (need == 0) return MESHRAST_ERR_INVALID_ARG;
    if (need > (size_t)MESHRAST_STATIC_WORKSPACE_BYTES) return MESHRAST_ERR_STATIC_TOO_LARGE;
    void *ws = nullptr;
    if (device_workspace(&ws) != cudaSuccess || ws == nullptr) return MESHRAST_ERR_CUDA;
    // rast_mesh_fwd clears the status word and the bin counters it relies on
    // at the start of every call, so what an earlier call left behind in the
    // shared array does not matter.
    return rast_mesh_fwd(p, verts, V, faces, F, first_face, num_faces, cams, pix_to_face, zbuf, bary, dists,
                         ws, (size_t)MESHRAST_STATIC_WORKSPACE_BYTES, stream);
}

// The status word sits at the start of the array, as in any workspace.
extern "C" MESHRAST_API int rast_query_static_status(uint32_t *status, void *stream) {
    if (!status) return MESHRAST_ERR_INVALID_ARG;
    void *ws = nullptr;
    if (device_workspace(&ws) != cudaSuccess || ws == nullptr) return MESHRAST_ERR_CUDA;
    return rast_query_status(ws, status, stream);
}

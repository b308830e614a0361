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
cudaError_t g_ws_err[kMaxDevices];
std::once_flag g_ws_once[kMaxDevices];

// The array's name in host code is only a host-side stand-in; its device
// address is looked up once per device, with that device current.
cudaError_t device_workspace(void **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(g_ws_once[dev], [dev]() {
        void *p = nullptr;
        g_ws_err[dev] = cudaGetSymbolAddress(&p, g_static_workspace);
        g_ws_ptr[dev] = (g_ws_err[dev] == cudaSuccess) ? p : nullptr;
    });
    *ptr = g_ws_ptr[dev];
    return g_ws_err[dev];
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

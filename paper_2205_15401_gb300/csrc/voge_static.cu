// voge_static.cu -- forward render without a caller-provided workspace.
//
// Some callers cannot allocate device memory at the point where they render:
// a real-time loop whose device memory budget is fixed up front and must not
// grow, or a host program that links only this library and owns no
// allocator.  For them voge_render_fwd_static() uses a workspace that lives
// in the library itself: a file-scope device array of
// VOGE_STATIC_WORKSPACE_BYTES that every GPU loading the library holds until
// the process exits.  Nothing here calls cudaMalloc, cudaFree or any
// allocating routine.
#include "../../include/voge.h"

namespace {

static __device__ __align__(256) unsigned char g_static_workspace[VOGE_STATIC_WORKSPACE_BYTES];

// Device address of the array in the current device's context.  The
// host-side symbol is only a stand-in and must never reach a kernel.  The
// address is looked up on every call (the lookup allocates nothing): a
// context that was torn down and created again (cudaDeviceReset) loads the
// module anew, and the array may then sit at another address.
int static_workspace(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_workspace) != cudaSuccess || !p) return VOGE_ERR_CUDA;
    *out = p;
    return VOGE_OK;
}

}  // namespace

extern "C" int voge_render_fwd_static(const voge_camera* cams, const voge_params* p, const float* means,
                                      const float* inv_cov, const float* attr, float* image, float* weights,
                                      int32_t* index, voge_stream_t stream) {
    const size_t need = voge_workspace_bytes(cams, p);
    if (need == 0) return VOGE_ERR_ARG;
    if (need > (size_t)VOGE_STATIC_WORKSPACE_BYTES) return VOGE_ERR_WORKSPACE;
    void* ws = nullptr;
    const int rc = static_workspace(&ws);
    if (rc != VOGE_OK) return rc;
    // voge_render_fwd clears every part of the workspace that must start at
    // zero (the tile counters) before it uses it.
    return voge_render_fwd(cams, p, means, inv_cov, attr, image, weights, index, ws, VOGE_STATIC_WORKSPACE_BYTES,
                           stream);
}

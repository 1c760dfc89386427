// Render forward for callers that cannot allocate device memory.
//
// vpgs_render_fwd carves its scratch space from a workspace the caller
// allocates.  Some callers cannot allocate: a plugin handed only a stream and
// the tensors it must read and write; a process whose memory pool reserved
// the GPU's memory up front and forbids further cudaMalloc calls.  For them,
// vpgs_render_fwd_noalloc takes its scratch from a fixed array that is
// compiled into this library and lives as long as the library is loaded.
#include <mutex>

#include "../../include/vpgs.h"

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)VPGS_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

}  // namespace

extern "C" vpgs_status vpgs_render_fwd_noalloc(const vpgs_gaussians *g, const vpgs_camera *cam,
                                               const double *T_cw, int32_t n_views,
                                               const vpgs_render_opts *opts, const vpgs_images *out,
                                               int32_t *status_out, vpgs_stream stream) {
    if (!g || !cam || !opts || n_views <= 0) return VPGS_ERR_INVALID_ARG;
    // the smallest workspace this render can use (room for one tile instance)
    const size_t need = vpgs_render_workspace_bytes(g->n, n_views, cam, opts, 1);
    if (need == 0) return VPGS_ERR_INVALID_ARG;
    if (need > kNoallocScratchBytes) return VPGS_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return VPGS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return VPGS_ERR_UNSUPPORTED;
    void *ws = nullptr;
    {
        // The host name of the array is not a device address: ask the runtime
        // once per device, with that device current.
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
                return VPGS_ERR_CUDA;
            g_noalloc_addr[dev] = p;
        }
        ws = g_noalloc_addr[dev];
    }
    const vpgs_status st = vpgs_render_fwd(ws, kNoallocScratchBytes, g, cam, T_cw, n_views, opts, out, stream);
    if (st != VPGS_OK || status_out == nullptr) return st;
    // the device status word sits at offset 0 of the render workspace
    if (cudaMemcpyAsync(status_out, ws, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                        reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess)
        return VPGS_ERR_CUDA;
    return VPGS_OK;
}

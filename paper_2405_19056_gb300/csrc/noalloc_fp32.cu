// glassnet_render_fp32_static: the FP32 plain render with its scratch in a
// fixed device array, so the call allocates no device memory.
//
// glassnet_render grows a model-owned workspace with cudaMalloc the first time
// it meets a larger frame (and synchronises the device to do it), and
// glassnet_render_ws needs a workspace the caller has allocated.  Neither works
// for a caller that cannot allocate device memory when it renders: for
// example a program whose device memory is all handed out up front by its own
// pooling allocator, or a frame loop that must never block in the allocator.
// This entry point takes its scratch from a file-scope array that every GPU
// which loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "internal.h"

namespace {

// Scratch of the plain path (layer intermediates U, V, pool, R, Y1, Y2, Q).
constexpr size_t kStaticScratchBytes = 48ull << 20;  // 48 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_plain_scratch[kStaticScratchBytes];

std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

namespace gn {
int set_error(int code, const char* msg);  // defined in glassnet_api.cu
}

extern "C" int glassnet_render_fp32_static(const gn_model* m, const gn_latent* lat,
                                           const float* gbuf, const float* tbuf,
                                           const uint8_t* layer_count, int K, int h, int w,
                                           float* out, cudaStream_t stream) {
  if (!m) return gn::set_error(GN_EINVAL, "model is NULL");
  if (m->precision != GN_FP32_PLAIN)
    return gn::set_error(GN_EINVAL, "glassnet_render_fp32_static needs a GN_FP32_PLAIN model");
  if (K < 0 || K > gn::kMaxK || h < 1 || w < 1)
    return gn::set_error(GN_EINVAL, "bad frame size");
  const size_t need = gn::plain_workspace_bytes(m->H, K, h * w);
  if (need > kStaticScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof(buf),
             "frame %d x %d with K = %d needs %zu bytes of scratch; the static scratch holds "
             "%zu bytes (48 MiB)",
             h, w, K, need, kStaticScratchBytes);
    return gn::set_error(GN_EINVAL, buf);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gn::set_error(GN_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return gn::set_error(GN_EUNSUPPORTED, "device index too large");
  void* scratch = nullptr;
  {
    // First call on a device: look up the device address of the array (host
    // code cannot use the array's name as a device pointer).
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
      e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_plain_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        return gn::set_error(GN_ECUDA, cudaGetErrorString(e));
      }
    }
    scratch = g_scratch_addr[dev];
  }
  return glassnet_render_ws(m, lat, gbuf, tbuf, layer_count, K, h, w, out, scratch,
                            kStaticScratchBytes, stream);
}

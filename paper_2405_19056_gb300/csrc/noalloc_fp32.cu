// glassnet_render_fp32_static: the FP32 plain render with its scratch in a
// fixed device array, so the call allocates no device memory.
//
// glassnet_render grows a model-owned workspace with cudaMalloc the first time
// it meets a larger frame (and synchronises the device to do it), and
// glassnet_render_ws needs a workspace the caller has allocated.  Neither works
// for a caller that cannot allocate device memory when it renders: for
// example a program whose device memory is all handed out up front by its own
// pooling allocator, or a frame loop that must never block in the allocator.
// This entry point takes its scratch from a file-scope array, which a GPU
// maps when the first GN_FP32_PLAIN model is loaded on it and holds until the
// process exits.
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

// Set-up, run by glassnet_load_weights for every GN_FP32_PLAIN model with the
// model's device current: looks up the device address of the array (host
// code cannot use the array's name as a device pointer).  The lookup also
// loads this file's module on the device, which maps the 48 MiB, so the
// render call below never does.  Every load refreshes the address (a model
// loaded after cudaDeviceReset sees the new one).
cudaError_t setup_static_scratch(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_plain_scratch);
  std::lock_guard<std::mutex> lock(g_mutex);
  g_scratch_addr[dev] = e == cudaSuccess ? p : nullptr;
  return e;
}
}  // namespace gn

extern "C" int glassnet_render_fp32_static(const gn_model* m, const gn_latent* lat,
                                           const float* gbuf, const float* tbuf,
                                           const uint8_t* layer_count, int K, int h, int w,
                                           float* out, cudaStream_t stream) {
  if (!m) return gn::set_error(GN_EINVAL, "model is NULL");
  if (m->precision != GN_FP32_PLAIN)
    return gn::set_error(GN_EINVAL, "glassnet_render_fp32_static needs a GN_FP32_PLAIN model");
  if (K < 0 || K > gn::kMaxK || h < 1 || w < 1)
    return gn::set_error(GN_EINVAL, "bad frame size");
  // the pixel count in 64 bits: a frame far beyond the scratch must not
  // overflow before it is rejected
  const long long P = static_cast<long long>(h) * w;
  const size_t need = P > (1ll << 30) ? ~size_t(0) : gn::plain_workspace_bytes(m->H, K, static_cast<int>(P));
  if (need > kStaticScratchBytes) {
    char buf[200];
    snprintf(buf, sizeof(buf),
             "frame %d x %d with K = %d needs more than the %zu bytes (48 MiB) that the static "
             "scratch holds",
             h, w, K, kStaticScratchBytes);
    return gn::set_error(GN_EINVAL, buf);
  }
  void* scratch = nullptr;
  if (m->device >= 0 && m->device < kMaxDevices) {
    std::lock_guard<std::mutex> lock(g_mutex);
    scratch = g_scratch_addr[m->device];
  }
  if (!scratch) return gn::set_error(GN_ECUDA, "the static scratch was not set up on the model's device");
  return glassnet_render_ws(m, lat, gbuf, tbuf, layer_count, K, h, w, out, scratch,
                            kStaticScratchBytes, stream);
}

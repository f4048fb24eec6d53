// Internal declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/glassnet.h"

namespace gn {

constexpr int kScene = 32;     // scene-parameter vector
constexpr int kTC = 12;        // transparency-layer channels
constexpr int kGC = 14;        // opaque G-buffer channels
constexpr int kOut = 3;        // RGB
constexpr int kMaxK = 8;       // layer slots per pixel
constexpr int kTile = 128;     // pixels per fused tile (tcgen05 M)

// Fused tile plan: one entry per tile row, pixel | count << 28 (pixel indices
// stay below 2^28 because 12 max(K, 1) P < 2^31), or kPlanEmpty for a row past
// the frame's last pixel.
constexpr uint32_t kPlanEmpty = 0xffffffffu;
// The plan workspace starts with a 256-byte header holding the dynamic tile
// counter; the entries follow.
constexpr size_t kPlanHeader = 256;
constexpr uint32_t kPlanPixelMask = 0x0fffffffu;

// Sticky device error bits (model error word).
constexpr uint32_t kErrCount = 1u;    // layer count above K
constexpr uint32_t kErrRange = 2u;    // exact set-sum left its fixed-point range
constexpr uint32_t kErrTimeout = 4u;  // a device wait gave up

// Linear layers in blob order.
enum Layer { LF1 = 0, LF2, LPHI1, LPHI2, LRHO, LB1, LB2, LR1, LR2, kLayers };

// Offsets (in floats) of each W and b inside the concat-form f32 weights.
struct WeightIndex {
  int H = 0, Z = 0;
  size_t w[kLayers] = {}, b[kLayers] = {};
  int out[kLayers] = {}, in[kLayers] = {};
  size_t total = 0;
  void build(int H_, int Z_);
};

// Packed operand image of the fused kernels: B operands (weights, [N][K]) in
// the K-major no-swizzle core-matrix layout [K/8][N][8] bf16, then the f32
// biases that are added in epilogues.  The same bytes are copied verbatim
// into each CTA's shared memory.
//   phi1 [16][H]    K = 12 channels, 2 folded-bias columns (per scene), 2 zero
//   phi2 [H][H]     rho [2H][H]  (K = [max ; mean])
//   B1   [16+H][H]  K = 14 channels, 2 folded-bias columns, then r (H)
//   B2, R1 [H][H]   R2 [H][16]   (N = 3 outputs + 13 zero rows)
//   phi2b [16][H]   phi2's bias as a K = 16 operand: k = 0 / 1 hold the bias
//                   split into a high and a low BF16 part, k >= 2 zero; the
//                   GEMM multiplies it by a constant [1, 1, 0, ...] A column
//   bias f32: phi2[H], rho[H], B2[H], R1[H], R2[16]
template <int H>
struct FusedLayout {
  static constexpr int KT = 16;
  static constexpr int KB1 = 16 + H;
  static constexpr int NR2 = 16;
  static constexpr uint32_t phi1 = 0;
  static constexpr uint32_t phi2 = phi1 + KT * H * 2;
  static constexpr uint32_t rho = phi2 + H * H * 2;
  static constexpr uint32_t b1 = rho + 2 * H * H * 2;
  static constexpr uint32_t b2 = b1 + KB1 * H * 2;
  static constexpr uint32_t r1 = b2 + H * H * 2;
  static constexpr uint32_t r2 = r1 + H * H * 2;
  static constexpr uint32_t phi2b = r2 + H * NR2 * 2;
  static constexpr uint32_t bias = phi2b + 16 * H * 2;
  static constexpr uint32_t bias_phi2 = bias;
  static constexpr uint32_t bias_rho = bias + H * 4;
  static constexpr uint32_t bias_b2 = bias + 2 * H * 4;
  static constexpr uint32_t bias_r1 = bias + 3 * H * 4;
  static constexpr uint32_t bias_r2 = bias + 4 * H * 4;
  static constexpr uint32_t bytes = bias + (4 * H + 16) * 4;
  // Shared memory beyond the weights, each a [2][128][8] bf16 A operand
  // (K = 16 for 128 rows): two layer operands of phi1, the constant
  // [1, 1, 0, ...] operand that multiplies phi2b, and the G-buffer block
  // [g0..g13, 1, 1] of B1.
  static constexpr uint32_t at0 = (bytes + 127) / 128 * 128;
  static constexpr uint32_t at1 = at0 + 4096;
  static constexpr uint32_t aone = at1 + 4096;
  static constexpr uint32_t ag = aone + 4096;
  static constexpr uint32_t smem_bytes = ag + 4096;
};

// One frame as the fused kernel sees it.
struct FusedFrame {
  const float* gbuf;
  const float* tbuf;
  const uint8_t* counts;
  float* out;
  const float* fold;  // c_phi [H] then c_B [H]
  int K;
  int P;      // pixels
  int tile0;  // first global tile index of this frame
  int win0;   // first global plan window of this frame (set by the launcher)
};

constexpr int kMaxBatch = 64;

struct FusedParams {
  FusedFrame f[kMaxBatch];
  int nframes;
  int total_tiles;
  int total_windows;    // set by the launcher
  uint32_t* err;
  uint32_t* plan;       // total_tiles * kTile entries (device)
  uint32_t* next_tile;  // dynamic tile counter (device), zeroed by the plan kernel
};

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_encode(const float* w32, const WeightIndex& wi, const float* scene_dev,
                          float* latent_dev, cudaStream_t s);
// Plan kernel, then the fused kernel.
cudaError_t launch_fused_bf16(int H, const void* wimg, const FusedParams& p, cudaStream_t s);
// Kernel attributes the fused launch needs; call once outside stream capture.
cudaError_t prepare_fused_bf16(int H);
size_t fused_plan_bytes(long long tiles);
size_t plain_workspace_bytes(int H, int K, int P);
cudaError_t launch_plain_fp32(const float* w32, const WeightIndex& wi, const float* latent,
                              const float* gbuf, const float* tbuf, const uint8_t* counts, int K,
                              int P, float* out, void* ws, uint32_t* err, cudaStream_t s);
int device_sm_count();

}  // namespace gn

struct gn_model {
  int H = 0, Z = 0, precision = 0, device = 0;
  gn::WeightIndex wi;
  float* w32 = nullptr;     // concat-form f32 weights (device)
  void* fused = nullptr;    // packed operand image (device)
  size_t fused_bytes = 0;
  uint32_t* err = nullptr;  // sticky error word (device)
  void* ws = nullptr;       // FP32 plain workspace (device), grown on demand
  size_t ws_bytes = 0;
  void* stage = nullptr;    // glassnet_render_host staging (device)
  size_t stage_bytes = 0;
  void* plan = nullptr;     // fused tile plan of glassnet_render / _batch (device)
  size_t plan_bytes = 0;
};

namespace gn {
// Validates a batch and fills the frame table (no plan binding); sets the
// thread's error message on failure.
int build_batch(const gn_model* m, const gn_frame* frames, int n, FusedParams* out);
// Points the params at a plan workspace of fused_plan_bytes(p.total_tiles) bytes.
void bind_plan(FusedParams& p, void* ws);
// Sets the calling thread's glassnet_last_error message; returns `code`.
int set_error(int code, const char* msg);
}  // namespace gn

struct gn_latent {
  int H = 0, Z = 0;
  // device: sigma [Z], c_phi [H], c_B [H], scene [32]
  float* d = nullptr;
  float* scene() const { return d + Z + 2 * H; }
  float* fold() const { return d + Z; }
};

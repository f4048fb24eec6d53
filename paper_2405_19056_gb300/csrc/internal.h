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
constexpr uint32_t kErrSaturated = 8u;  // an FP8 input beyond its calibrated range (clamped)
// Kernels named by the second error word after a timeout (report_timeout).
enum : uint32_t { kKernelFusedBf16 = 1, kKernelFusedFp8 = 2, kKernelCompact = 3, kKernelConvR3 = 4 };

// Linear layers in blob order.
enum Layer { LF1 = 0, LF2, LPHI1, LPHI2, LRHO, LB1, LB2, LR1, LR2, kLayers };

// Positional encoding of the inputs (Sec. 3.4): an input of n channels
// enters as n (1 + 2L) values, the blocks [x ; sin(2^0 pi x) ; cos(2^0 pi x) ;
// ... ; sin(2^(L-1) pi x) ; cos(2^(L-1) pi x)].  Band t of an input is block t.
constexpr int kMaxPeFreqs = 10;       // any precision's limit
constexpr int kMaxPeFreqsFused = 4;   // the fused BF16 and FP8 kernels

// Offsets (in floats) of each W and b inside the concat-form f32 weights.
struct WeightIndex {
  int H = 0, Z = 0, L = 0;  // L: positional-encoding frequencies (0: none)
  int RK = 1;               // kernel size of R's first layer (1, or 3 over the frame)
  size_t w[kLayers] = {}, b[kLayers] = {};
  int out[kLayers] = {}, in[kLayers] = {};
  size_t total = 0;
  int bands() const { return 1 + 2 * L; }
  int tc_enc() const { return kTC * bands(); }     // encoded layer channels (phi1's first block)
  int gc_enc() const { return kGC * bands(); }     // encoded G-buffer channels (B1's first block)
  int sc_enc() const { return kScene * bands(); }  // encoded scene vector (F1's input)
  void build(int H_, int Z_, int L_ = 0, int RK_ = 1);
};

#ifdef __CUDACC__
// Band t of the encoding of x: x (t = 0), sin(2^f pi x) (t = 2f + 1) or
// cos(2^f pi x) (t = 2f + 2).  The scaling by 2^f is exact; sinpif / cospif
// reduce the argument exactly.
__device__ __forceinline__ float pe_band_value(float x, int t) {
  if (t == 0) return x;
  const float y = ldexpf(x, (t - 1) >> 1);
  return (t & 1) ? sinpif(y) : cospif(y);
}
#endif

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
//
// With positional encoding (PE) every band of phi1's input and of B1's
// G-buffer block takes 16 K columns (12 or 14 values, then zeros),
// for up to kMaxPeFreqsFused frequencies: band 0 keeps the layout above
// (constant-one columns at k = 12, 13 of phi1 and k = 14, 15 of B1), band t
// sits at k = 16 t, and B1's r block starts after the last band.  The
// operands are sized for the largest L; a model with fewer frequencies uses
// the first 1 + 2L bands.  At H = 128 the per-pixel weights stream (below).
template <int H, bool PE = false>
struct FusedLayout {
  static constexpr int kBands = PE ? 1 + 2 * kMaxPeFreqsFused : 1;
  static constexpr int KT = 16 * kBands;
  static constexpr int KG = 16 * kBands;
  static constexpr int KB1 = KG + H;
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
  // Shared memory beyond the weights, each a [K/8][128][8] bf16 A operand
  // for 128 rows: two layer operands of phi1 (K = KT), the constant
  // [1, 1, 0, ...] operand that multiplies phi2b (K = 16), and the G-buffer
  // block [g0..g13, 1, 1] of B1 (K = KG).
  static constexpr uint32_t at0 = (bytes + 127) / 128 * 128;
  static constexpr uint32_t at1 = at0 + KT * 256;
  static constexpr uint32_t aone = at1 + KT * 256;
  static constexpr uint32_t ag = aone + 4096;
  static constexpr uint32_t smem_bytes = ag + KG * 256;
  static_assert(smem_bytes <= 232448, "operands exceed the 227 KB of shared memory per CTA");
  static constexpr bool kStream = false;
};

// Doubled widths with positional encoding: the encoded operands and weights
// (phi1 and B1's G-buffer block at K = 16 (1 + 2 kMaxPeFreqsFused)) do not
// fit beside every weight, so the per-pixel weights stream from device
// memory (through L2) into a ring of two 16 KB shared-memory stages, one
// chunk of K = 64 rows at a time, while phi1, phi2, phi2b, the biases and
// band 0 of B1 (which carries the folded per-scene bias) stay resident.
// The image starts with the resident block, copied verbatim at offset 0:
//   phi1 [KT][H] | phi2 [H][H] | B1 band 0 [16][H] | phi2b [16][H] | bias f32
// then the chunks, each a contiguous [64/8][N][8] (or smaller) block:
//   rho      4 chunks (K = [max ; mean], 64 rows each)
//   B1 bands 2 chunks (bands 1-4 and 5-8 of the G-buffer block, 16 K each;
//            a model with fewer frequencies copies the bands it uses)
//   B1 r     2 chunks    B2  2 chunks    R1  2 chunks    R2  1 chunk [H][16]
template <>
struct FusedLayout<128, true> {
  static constexpr int H = 128;
  static constexpr int kBands = 1 + 2 * kMaxPeFreqsFused;
  static constexpr int KT = 16 * kBands;
  static constexpr int KG = 16 * kBands;
  static constexpr int NR2 = 16;
  static constexpr uint32_t kChunk = 64 * H * 2;  // one ring stage: K = 64 rows of an N = H operand
  // resident block (smem offset = image offset)
  static constexpr uint32_t phi1 = 0;
  static constexpr uint32_t phi2 = phi1 + KT * H * 2;
  static constexpr uint32_t b1 = phi2 + H * H * 2;  // band 0 of B1's G-buffer block only
  static constexpr uint32_t phi2b = b1 + 16 * H * 2;
  static constexpr uint32_t bias = phi2b + 16 * H * 2;
  static constexpr uint32_t bias_phi2 = bias;
  static constexpr uint32_t bias_rho = bias + H * 4;
  static constexpr uint32_t bias_b2 = bias + 2 * H * 4;
  static constexpr uint32_t bias_r1 = bias + 3 * H * 4;
  static constexpr uint32_t bias_r2 = bias + 4 * H * 4;
  static constexpr uint32_t bytes = bias + (4 * H + 16) * 4;  // resident bytes
  // chunks in the image
  static constexpr uint32_t img_rho = (bytes + 127) / 128 * 128;
  static constexpr uint32_t img_b1g = img_rho + 4 * kChunk;
  static constexpr uint32_t img_b1r = img_b1g + 2 * kChunk;
  static constexpr uint32_t img_b2 = img_b1r + 2 * kChunk;
  static constexpr uint32_t img_r1 = img_b2 + 2 * kChunk;
  static constexpr uint32_t img_r2 = img_r1 + 2 * kChunk;
  static constexpr uint32_t img_bytes = img_r2 + H * NR2 * 2;
  // shared memory beyond the resident block: the ring, then the A operands
  // as in the general layout
  static constexpr uint32_t ring0 = (bytes + 127) / 128 * 128;
  static constexpr uint32_t ring1 = ring0 + kChunk;
  static constexpr uint32_t at0 = ring1 + kChunk;
  static constexpr uint32_t at1 = at0 + KT * 256;
  static constexpr uint32_t aone = at1 + KT * 256;
  static constexpr uint32_t ag = aone + 4096;
  static constexpr uint32_t smem_bytes = ag + KG * 256;
  static_assert(smem_bytes + 1024 <= 232448, "operands exceed the 227 KB of shared memory per CTA");
  static constexpr bool kStream = true;
};

// Packed operand image of the FP8 fused kernel (E4M3 operands, FP32
// accumulate), copied verbatim into shared memory.  E4M3 matrices use the
// same K-major core matrices of 8 rows x 16 bytes, i.e. [K/16][N][16] bytes;
// one MMA consumes K = 32.
//   phi1  [32][H]     K = 12 channels + 20 zero
//   phi1b [16][H]     BF16: the per-scene bias c_phi in accumulator units,
//                     split hi / lo in rows k = 0 / 1 (written per frame)
//   phi2  [H][H]      rho [2H][H]
//   b1    [32+H][H]   K = 14 channels + 18 zero, then r (H)
//   b1b   [16][H]     BF16: per-scene c_B in accumulator units (per frame)
//   b2, r1 [H][H]     r2 [H][16]  (N = 3 outputs + 13 zero rows)
//   FP32 constants (indices in floats from `cst`): per output column a
//   dequantisation scale (accumulator -> next layer's quantised input, or
//   real units where the result is not re-quantised) and a bias; u_phi1 and
//   u_b1 turn c_phi / c_B into accumulator units; then three scalars: 1/s_r
//   (the scale of B1's r input, or of tau in the sum form), 1/s_pool and s_y2
//   (B2's output in real units, for the neural buffer of a 3x3 R); then the
//   per-channel input scales 1/s_t[c] (12, padded to 16) and 1/s_g[c] (14,
//   padded to 16).  The first layers' weight columns carry the per-channel
//   scales (W[n][c] s[c] is quantised), so an input code is x[c] / s[c]
//   and the accumulator stays in the weight scale's units.
//   A operands: at0, at1, ag ([2][128][16] bytes each, K block 1 zero) and
//   the constant BF16 [1, 1, 0, ...] operand of the bias MMAs.
// With positional encoding (PE, up to kMaxPeFreqsFused frequencies) phi1's
// input and B1's G-buffer block are K = 128 wide: the bands of the 12 (14)
// channels band-major, code k = 12 t + c (14 t + c) for band t, zeros after
// the last band (108 and 126 codes at L = 4); band 0 carries the channels'
// calibrated scales, the sine and cosine bands the fixed code scale
// kFp8BandCode; B1's r block starts at k = 128.  at0, at1 and ag are then
// [8][128][16] bytes each.
template <int H, bool PE = false>
struct FusedLayoutF8 {
  static constexpr int KT = PE ? 128 : 32;  // phi1's K (E4M3 codes)
  static constexpr int KG = PE ? 128 : 32;  // B1's G-buffer block
  static constexpr uint32_t phi1 = 0;
  static constexpr uint32_t phi1b = phi1 + KT * H;
  static constexpr uint32_t phi2 = phi1b + 16 * H * 2;
  static constexpr uint32_t rho = phi2 + H * H;
  static constexpr uint32_t b1 = rho + 2 * H * H;
  static constexpr uint32_t b1b = b1 + (KG + H) * H;
  static constexpr uint32_t b2 = b1b + 16 * H * 2;
  static constexpr uint32_t r1 = b2 + H * H;
  static constexpr uint32_t r2 = r1 + H * H;
  static constexpr uint32_t cst = r2 + H * 16;
  enum : int {
    S_PHI1 = 0, S_PHI2 = H, B_PHI2 = 2 * H, S_RHO = 3 * H, B_RHO = 4 * H, S_B1 = 5 * H,
    S_B2 = 6 * H, B_B2 = 7 * H, S_R1 = 8 * H, B_R1 = 9 * H, U_PHI1 = 10 * H, U_B1 = 11 * H,
    S_R2 = 12 * H, B_R2 = 12 * H + 16, INV_S_R = 12 * H + 32, INV_S_POOL, S_Y2,
    INV_S_TCH = 12 * H + 36, INV_S_GCH = 12 * H + 52, N_CST = 12 * H + 68
  };
  static constexpr uint32_t bytes = cst + N_CST * 4;
  static constexpr uint32_t at0 = (bytes + 127) / 128 * 128;
  static constexpr uint32_t at1 = at0 + 128 * KT;
  static constexpr uint32_t ag = at1 + 128 * KT;
  static constexpr uint32_t aone = ag + 128 * KG;
  static constexpr uint32_t smem_bytes = aone + 4096;
  static_assert(bytes % 16 == 0, "bulk copy size must be a multiple of 16 bytes");
  static_assert(smem_bytes + 2048 <= 232448, "operands exceed the shared memory per CTA");
};
// Code scale of the sine and cosine bands in the FP8 kernel: a band value
// v in [-1, 1] enters as the E4M3 code v * 256 (at most 256 of 448).
constexpr float kFp8BandCode = 256.0f;

// Activation scales of the FP8 path (static): the real value of an E4M3 code
// x is x * s.  Order: the 12 transparency-layer channels (phi1's input, per
// channel), the 14 G-buffer channels (B1's, per channel), then per tensor U
// (phi2), pool (rho), r (B1's r block), y (B2), y2 (R1), q (R2).
constexpr int kFp8Acts = 32;
enum : int { FP8_T0 = 0, FP8_G0 = 12, FP8_U = 26, FP8_POOL, FP8_R, FP8_Y, FP8_Y2, FP8_Q };
// Headroom of the calibrated ranges: scale = headroom |max| / 448.  The input
// channels take 8 (direct lighting is log-normal: a frame of more pixels than
// the calibration frame reaches further into its tail), the hidden
// activations 4.  E4M3 keeps the same relative step over its normal range, so
// headroom costs precision only below 2^-6 s.
constexpr float kFp8InputHeadroom = 8.0f;
constexpr float kFp8HiddenHeadroom = 4.0f;

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
  // 3x3 R: the neural buffer the fused kernel writes, BF16 [h][H/8][w][8],
  // and the frame width.
  uint16_t* phi;
  int w;
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
  // Tail of the schedule (set by the launcher): the last frame's last
  // tail_n full windows of win_tiles tiles start at tile tail0, its partial
  // window (tail_part tiles) follows them.
  int win_tiles;
  int tail0, tail_n, tail_part;
  // Streaming launches (accumulate / resolve): the plan keeps pixel order
  // (identity), a frame's counts may be NULL (every pixel has K layers), and
  // the pool state lives in device planes of P values each.
  int plan_identity;
  // Pool state, tile-major: per 128-pixel tile of the frame a block of
  // H/2 + H planes of 128 words (running max as bf16 pairs, then the
  // fixed-point sums as f32 bits, start 2^11), so a tile's state is one
  // contiguous block and a warp's access to a plane is coalesced.
  uint32_t* pool_st;
  uint8_t* pool_cnt;  // [P] layers accumulated
  int pool_fresh;     // the pool is empty: its state is the start value, not read
  // Pooling of Eq. 5: 0 = [max ; mean] then rho, 1 = the sum tau fed to B1
  // directly (frame and resolve launches; accumulation is the same for both).
  int pool_sum;
  // Positional-encoding frequencies of the inputs (0: none; the PE kernel
  // variant serves 1 .. kMaxPeFreqsFused).
  int pe_freqs;
  // Test hook of the BF16 kernel's timeout path (0 in every render): the MMA
  // warp waits this long on a barrier that nothing arrives on, then every
  // warp leaves and the error word gets the timeout bit.
  uint64_t stall_ns;
};

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_encode(const float* w32, const WeightIndex& wi, const float* scene_dev,
                          float* latent_dev, cudaStream_t s);
// Plan kernel, then the fused kernel.
// mode: 0 a whole frame, 1 accumulate one streamed layer into the pool state,
// 2 resolve the pool state (see fused_bf16.cu).
cudaError_t launch_fused_bf16(int H, const void* wimg, const FusedParams& p, cudaStream_t s,
                              int mode = 0);
// Kernel attributes the fused launch needs; call once outside stream capture.
cudaError_t prepare_fused_bf16(int H);
size_t fused_plan_bytes(long long tiles);
// Numbers the plan windows of `p` (win0, total_windows) and launches the
// tile-plan kernel that the fused kernels read.
cudaError_t launch_plan(FusedParams& p, cudaStream_t s);
size_t plain_workspace_bytes(int H, int K, int P);
// pool_sum: Eq. 5's sum form (tau = sum of the valid layers' phi outputs, no
// rho) instead of [max ; mean] then rho.
// w: frame width (the 3x3 R1 reads neighbouring pixels; P = h w).
cudaError_t launch_plain_fp32(const float* w32, const WeightIndex& wi, const float* latent,
                              const float* gbuf, const float* tbuf, const uint8_t* counts, int K,
                              int P, float* out, void* ws, uint32_t* err, cudaStream_t s,
                              int pool_sum, int w);
int device_sm_count();
// Looks up (and so maps) the static scratch of glassnet_render_fp32_static on
// device `dev`, which must be current (noalloc_fp32.cu).
cudaError_t setup_static_scratch(int dev);
// 3x3 R (conv_r3.cu): R1 as a 3x3 kernel over the neural buffer phi
// (BF16 [h][H/8][w][8]) the fused kernel wrote, then R2 and the sigmoid.
// The image holds the 9 taps' [H/8][H][8] BF16 weights (tap = (dy + 1) 3 +
// dx + 1), R2 as [H/8][16][8] BF16, then b_R1 [H] and b_R2 [16] FP32.
size_t conv_r3_image_bytes(int H);
cudaError_t prepare_conv_r3(int H);
cudaError_t launch_conv_r3(int H, const void* img, const uint16_t* phi, float* out, int h, int w,
                           uint32_t* err, cudaStream_t s);
// FP8 fused path (fused_fp8.cu): plan kernel, then the fused E4M3 kernel.
cudaError_t launch_fused_fp8(int H, const void* wimg, const FusedParams& p, cudaStream_t s);
cudaError_t prepare_fused_fp8(int H);
// Compacted ragged-layer kernel (fused_compact.cu, BF16, H = 64, whole frames,
// no encoding, 1x1 R): plan kernel (identity order), then the fused kernel.
cudaError_t launch_fused_compact(const void* wimg, const FusedParams& p, cudaStream_t s);
cudaError_t prepare_fused_compact();
// Per-layer |activation| maxima of an FP32 plain render held in `ws` (the
// workspace launch_plain_fp32 filled for the same frame), in the order of
// the FP8 activation scales, as FP32 bit patterns in amax[kFp8Acts].
cudaError_t launch_fp8_act_amax(const void* ws, const float* gbuf, const float* tbuf,
                                const uint8_t* counts, int H, int K, int P, uint32_t* amax,
                                cudaStream_t s);

}  // namespace gn

struct gn_model {
  int H = 0, Z = 0, precision = 0, device = 0;
  int pooling = GN_POOL_MAX_MEAN;  // gn_pooling (the frequency count is wi.L)
  gn::WeightIndex wi;
  float* w32 = nullptr;     // concat-form f32 weights (device)
  void* fused = nullptr;    // packed operand image (device)
  size_t fused_bytes = 0;
  void* conv = nullptr;     // 3x3 R image of the BF16 path (device)
  uint32_t* err = nullptr;  // sticky error word (device)
  void* ws = nullptr;       // FP32 plain workspace (device), grown on demand
  size_t ws_bytes = 0;
  void* stage = nullptr;    // glassnet_render_host staging (device)
  size_t stage_bytes = 0;
  void* plan = nullptr;     // fused tile plan of glassnet_render / _batch (device)
  size_t plan_bytes = 0;
  float* host_w = nullptr;  // FP8 models: concat-form f32 weights kept for packing
  bool fp8_ready = false;   // FP8 models: calibrated and packed
  float fp8_act[gn::kFp8Acts] = {};  // FP8 activation scales (real value of a code = code * s)
  uint64_t stall_ns = 0;    // test hook: the next fused BF16 launch stalls (glassnet_debug_stall_next_render)
  int schedule = GN_SCHEDULE_SORTED;  // gn_schedule of the fused BF16 frame renders
};

namespace gn {
// Validates a batch and fills the frame table (no plan binding); sets the
// thread's error message on failure.
int build_batch(const gn_model* m, const gn_frame* frames, int n, FusedParams* out);
// Launches the fused path of the model's precision (plan + fused kernel), or
// sets its kernel attributes (once, outside stream capture).
cudaError_t launch_fused(const gn_model* m, const FusedParams& p, cudaStream_t s);
cudaError_t prepare_fused(const gn_model* m);
// Points the params at a plan workspace of fused_plan_bytes(p.total_tiles) bytes.
void bind_plan(FusedParams& p, void* ws);
// Workspace of a launch of the model's form: the plan (256-byte rounded),
// then, for a 3x3 R, each frame's neural buffer; binding sets both.
size_t batch_ws_bytes(const gn_model* m, const FusedParams& p);
void bind_batch_ws(const gn_model* m, FusedParams& p, void* ws);
// The fused launch and, for a 3x3 R, each frame's 3x3 kernel.
cudaError_t launch_render(const gn_model* m, const FusedParams& p, cudaStream_t s);
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

// Tile plan of the fused kernels (count-sorting windows, Eq. 5's per-pixel
// layer sets) and the launch bookkeeping shared by the BF16 and FP8 kernels.
#include "fused_common.cuh"

namespace gn {
namespace {
using namespace fused;

// ------------------------------------------------------------- tile plan
#ifndef GN_WIN_TILES
#define GN_WIN_TILES 4
#endif
constexpr int kWinTiles = GN_WIN_TILES;  // tiles per count-sorting window
constexpr int kPlanWarps = 4;                         // windows per plan CTA
constexpr int kPlanPer = kWinTiles * kTile / 32;        // pixels per lane
constexpr int kClasses = kMaxK + 1;                     // counts 0..8
static_assert(kPlanPer <= 32, "window too large for one warp");

// One warp per window of up to kWinTiles tiles of one frame (lane l holds
// pixels l * kPlanPer ..).  Every pixel of the window gets the entry
// pixel | count << 28 at its sorted position: counts in descending order,
// pixel index ascending within a count.  Rows past the frame's last pixel get
// kPlanEmpty.  Counts above K are clamped to K and set the count error bit.
// The fused kernel is launched as a programmatic dependent of this grid, so
// it may start (and load its weights) before this grid ends; it waits on the
// grid dependency before it reads the plan.
__global__ void __launch_bounds__(kPlanWarps * 32) plan_kernel(const __grid_constant__ FusedParams prm) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int win = blockIdx.x * kPlanWarps + (threadIdx.x >> 5);
  if (win == 0 && lane == 0) *prm.next_tile = 0u;
  if (win >= prm.total_windows) return;
  int fi = 0;
  while (fi + 1 < prm.nframes && win >= prm.f[fi + 1].win0) ++fi;
  const FusedFrame& F = prm.f[fi];
  const int lw = win - F.win0;
  const int tiles_f = (F.P + kTile - 1) / kTile;
  const int rows = min(kWinTiles, tiles_f - lw * kWinTiles) * kTile;  // rows of this window
  const int p0 = lw * kWinTiles * kTile + lane * kPlanPer;            // lane's first pixel
  uint32_t* out = prm.plan + static_cast<size_t>(F.tile0 + lw * kWinTiles) * kTile;

  int c[kPlanPer];
  int pre[kClasses];
#pragma unroll
  for (int b = 0; b < kClasses; ++b) pre[b] = 0;
  bool over = false;
#pragma unroll
  for (int i = 0; i < kPlanPer; ++i) {
    int v = -1;
    if (p0 + i < F.P) {
      v = F.counts[p0 + i];
      if (v > F.K) {
        over = true;
        v = F.K;
      }
    }
    c[i] = v;
#pragma unroll
    for (int b = 0; b < kClasses; ++b) pre[b] += v == b ? 1 : 0;
  }
  if (over) atomicOr(prm.err, kErrCount);
  // exclusive prefix of every class over the lanes; classes 8, 7, ..., 0 are
  // laid out one after the other
  int base = 0;
#pragma unroll
  for (int b = kClasses - 1; b >= 0; --b) {
    int x = pre[b];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    const int total = __shfl_sync(0xffffffffu, x, 31);
    pre[b] = base + x - pre[b];
    base += total;
  }
#pragma unroll
  for (int i = 0; i < kPlanPer; ++i) {
    const uint32_t p = static_cast<uint32_t>(p0 + i);
#pragma unroll
    for (int b = 0; b < kClasses; ++b) {
      if (c[i] == b) {
        out[pre[b]] = p | (static_cast<uint32_t>(b) << 28);
        ++pre[b];
      }
    }
  }
  for (int r = base + lane; r < rows; r += 32) out[r] = kPlanEmpty;
}

int g_sm_count = 0;

}  // namespace

int device_sm_count() {
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (g_sm_count <= 0) g_sm_count = 1;
  }
  return g_sm_count;
}

size_t fused_plan_bytes(long long tiles) {
  return kPlanHeader + static_cast<size_t>(tiles) * kTile * sizeof(uint32_t);
}

cudaError_t launch_plan(FusedParams& p, cudaStream_t s) {
  int wins = 0;
  for (int i = 0; i < p.nframes; ++i) {
    p.f[i].win0 = wins;
    const int t = (p.f[i].P + kTile - 1) / kTile;
    wins += (t + kWinTiles - 1) / kWinTiles;
  }
  p.total_windows = wins;
  plan_kernel<<<(p.total_windows + kPlanWarps - 1) / kPlanWarps, kPlanWarps * 32, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace gn

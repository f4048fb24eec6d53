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
#ifndef GN_TAIL_WINDOWS
#define GN_TAIL_WINDOWS 64
#endif
constexpr int kTailWindows = GN_TAIL_WINDOWS;  // windows scheduled rank-major at the end
constexpr int kPlanWarps = 4;                         // windows per plan CTA
constexpr int kPlanPer = kWinTiles * kTile / 32;        // pixels per lane
static_assert(kPlanPer % 16 == 0 && kPlanPer <= 32, "a lane holds 16 or 32 pixels");
static_assert(kWinTiles * kTile < 4096, "per-class positions must fit 12 bits");

// Per-class counters packed 12 bits per count class: classes 0..4 in `lo`,
// 5..8 in `hi` (a window holds < 4096 pixels, so no field overflows).
struct Classes {
  uint64_t lo = 0, hi = 0;
  __device__ __forceinline__ uint64_t& word(int c) { return c < 5 ? lo : hi; }
  __device__ __forceinline__ static int shift(int c) { return 12 * (c < 5 ? c : c - 5); }
  __device__ __forceinline__ int get(int c) const {
    return static_cast<int>(((c < 5 ? lo : hi) >> shift(c)) & 0xfffu);
  }
  __device__ __forceinline__ void add(int c, uint64_t n) { word(c) += n << shift(c); }
};

// One warp per window of up to kWinTiles tiles of one frame (lane l holds
// pixels l * kPlanPer ..).  Every pixel of the window gets the entry
// pixel | count << 28 at its sorted position: counts in descending order,
// pixel index ascending within a count (a warp prefix over per-lane class
// counts).  Rows past the frame's last pixel get kPlanEmpty.  Counts above K
// are clamped to K and set the count error bit.  The fused kernel is launched
// as a programmatic dependent of this grid, so it may start (and load its
// weights) before this grid ends; it waits on the grid dependency before it
// reads the plan.
__global__ void __launch_bounds__(kPlanWarps * 32) plan_kernel(const __grid_constant__ FusedParams prm) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31;
  const int win = blockIdx.x * kPlanWarps + (threadIdx.x >> 5);
  if (win == 0 && lane == 0) *prm.next_tile = 0u;
  if (win >= prm.total_windows) return;
  int fi = 0;
  while (fi + 1 < prm.nframes && win >= prm.f[fi + 1].win0) ++fi;
  const int P = prm.f[fi].P, K = prm.f[fi].K;
  const uint8_t* counts = prm.f[fi].counts;
  const int lw = win - prm.f[fi].win0;
  const int tiles_f = (P + kTile - 1) / kTile;
  const int rows = min(kWinTiles, tiles_f - lw * kWinTiles) * kTile;  // rows of this window
  const int p0 = lw * kWinTiles * kTile + lane * kPlanPer;            // lane's first pixel
  uint32_t* out = prm.plan + static_cast<size_t>(prm.f[fi].tile0 + lw * kWinTiles) * kTile;

  // the lane's counts, one byte each (0 past the frame; presence is p < P;
  // no count array: every pixel has K layers)
  uint32_t cw[kPlanPer / 4];
  if (counts == nullptr) {
#pragma unroll
    for (int j = 0; j < kPlanPer / 4; ++j) cw[j] = static_cast<uint32_t>(K) * 0x01010101u;
  } else if ((reinterpret_cast<uintptr_t>(counts + p0) & 15u) == 0 && p0 + kPlanPer <= P) {
#pragma unroll
    for (int j = 0; j < kPlanPer / 16; ++j) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(counts + p0) + j);
      cw[4 * j] = v.x;
      cw[4 * j + 1] = v.y;
      cw[4 * j + 2] = v.z;
      cw[4 * j + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < kPlanPer / 4; ++j) {
      uint32_t w = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int p = p0 + 4 * j + i;
        w |= static_cast<uint32_t>(p < P ? counts[p] : 0u) << (8 * i);
      }
      cw[j] = w;
    }
  }
  Classes own;
  bool over = false;
#pragma unroll
  for (int i = 0; i < kPlanPer; ++i) {
    if (p0 + i >= P) continue;
    int c = static_cast<int>((cw[i / 4] >> (8 * (i % 4))) & 0xffu);
    if (c > K) {
      over = true;
      c = K;
      cw[i / 4] = (cw[i / 4] & ~(0xffu << (8 * (i % 4)))) | (static_cast<uint32_t>(c) << (8 * (i % 4)));
    }
    own.add(c, 1);
  }
  if (over) atomicOr(prm.err, kErrCount);
  if (prm.plan_identity) {
    // pixel order: row r of the window holds its r-th pixel
#pragma unroll
    for (int i = 0; i < kPlanPer; ++i) {
      const int r = lane * kPlanPer + i;
      if (r >= rows) continue;
      const int c = static_cast<int>((cw[i / 4] >> (8 * (i % 4))) & 0xffu);
      out[r] = p0 + i < P ? static_cast<uint32_t>(p0 + i) | (static_cast<uint32_t>(c) << 28)
                          : kPlanEmpty;
    }
    return;
  }
  // exclusive prefix of the packed counters over the lanes, and the totals
  Classes pre = own;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t ylo = __shfl_up_sync(0xffffffffu, pre.lo, d);
    const uint64_t yhi = __shfl_up_sync(0xffffffffu, pre.hi, d);
    if (lane >= d) {
      pre.lo += ylo;
      pre.hi += yhi;
    }
  }
  Classes tot;
  tot.lo = __shfl_sync(0xffffffffu, pre.lo, 31);
  tot.hi = __shfl_sync(0xffffffffu, pre.hi, 31);
  pre.lo -= own.lo;
  pre.hi -= own.hi;
  // class c starts after every pixel of a larger count
  Classes pos;
  int base = 0;
#pragma unroll
  for (int c = kMaxK; c >= 0; --c) {
    pos.add(c, static_cast<uint64_t>(base));
    base += tot.get(c);
  }
  pos.lo += pre.lo;
  pos.hi += pre.hi;
#pragma unroll
  for (int i = 0; i < kPlanPer; ++i) {
    if (p0 + i >= P) continue;
    const int c = static_cast<int>((cw[i / 4] >> (8 * (i % 4))) & 0xffu);
    out[pos.get(c)] = static_cast<uint32_t>(p0 + i) | (static_cast<uint32_t>(c) << 28);
    pos.add(c, 1);
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
  // schedule tail: the last frame's last full windows (see schedule_tile)
  const FusedFrame& lf = p.f[p.nframes - 1];
  const int tf = (lf.P + kTile - 1) / kTile;
  const int wf = tf / kWinTiles;
  p.win_tiles = kWinTiles;
  p.tail_n = wf < kTailWindows ? wf : kTailWindows;
  p.tail_part = tf % kWinTiles;
  p.tail0 = lf.tile0 + (wf - p.tail_n) * kWinTiles;
  plan_kernel<<<(p.total_windows + kPlanWarps - 1) / kPlanWarps, kPlanWarps * 32, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace gn

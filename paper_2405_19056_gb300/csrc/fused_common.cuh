// Device-side pieces shared by the fused kernels (BF16 and FP8): warp roles,
// mbarrier slots, the pooling arithmetic helpers, bounded waits, the frame
// lookup and the loader's shared bookkeeping.
#pragma once
#include <cuda_bf16.h>

#include "internal.h"
#include "tc_ptx.cuh"

namespace gn {
namespace fused {
// Epilogue warps per TMEM lane quadrant (each serves H / kEW accumulator
// columns of 32 pixel rows), then the MMA warp, then the two loader warps.
#ifndef GN_FUSED_EW
#define GN_FUSED_EW 2
#endif
constexpr int kEW = GN_FUSED_EW;
constexpr int kEpiWarps = 4 * kEW;
constexpr int kMmaWarp = 4 * kEW;
constexpr int kLoadWarp0 = 4 * kEW + 1;
constexpr int kLoadWarps = 2;      // loader warps of the FP8 kernel and the plain BF16 one
constexpr int kMaxLoadWarps = 4;   // the BF16 kernel with positional encoding
constexpr int kThreadsF = (4 * kEW + 3) * 32;
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s per device-side wait
constexpr float kSumBase = 2048.0f;          // 2^11: quantum 2^-12 in [2^11, 2^12)
constexpr float kSumLimit = 4096.0f;
constexpr float kHalfQuantum = 1.0f / 8192.0f;

// mbarrier slots.
enum : int {
  B_W = 0,       // weights copied (transaction count)
  B_IN = 1,      // + (n & 1): an A operand in TMEM written (epilogue warps arrive)
  B_DP = 3,      // per-pixel layer accumulator ready (commit)
  B_DR2 = 4,     // R2 accumulator ready (commit)
  B_AG_F = 5,    // B1's G-buffer operand written (loaders)
  B_AG_E = 6,    // B1's G-buffer operand consumed (commit)
  B_D1 = 7,      // + buffer (3): phi1 accumulator ready (commit)
  B_D2 = 10,     // + buffer (3): phi2 accumulator ready (commit)
  B_BE = 13,     // + buffer (3): phi2 accumulator read (epilogue warps arrive)
  B_AT_F = 16,   // + buffer (2): layer operand written (loaders)
  B_AT_E = 18,   // + buffer (2): layer operand consumed (commit)
  B_TILE = 20,   // + tile parity: tile index and slot count published (loaders)
  B_SCHED = 22,  // + tile parity: tile index taken (loader warp 0)
  B_COUNT = 24
};


// Position in the rotating sequence of layer slots: buffer b = g mod 3 and
// use u = g / 3 (the phase parity of the buffer's barriers is u & 1).
struct SlotPos {
  uint32_t b = 0, u = 0;
  __device__ __forceinline__ void next() {
    if (++b == 3) {
      b = 0;
      ++u;
    }
  }
};

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  __nv_bfloat16 b = __float2bfloat16_rn(x);
  return *reinterpret_cast<uint16_t*>(&b);
}
__device__ __forceinline__ float bf16_value(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// (a0, a1) + (b0, b1), round to nearest even, two lanes per op.
__device__ __forceinline__ void fadd2_rn(float& r0, float& r1, float a0, float a1, float b0,
                                         float b1) {
  asm("{.reg .b64 p, q, r;\n\tmov.b64 p, {%2, %3};\n\tmov.b64 q, {%4, %5};\n\t"
      "add.rn.f32x2 r, p, q;\n\tmov.b64 {%0, %1}, r;}"
      : "=f"(r0), "=f"(r1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
// s0 += low bf16 of p, s1 += high bf16 of p, each rounded toward zero (the
// bf16 value is exact in FP32, so only the sum is rounded).
__device__ __forceinline__ void add_bf16x2_rz(float& s0, float& s1, uint32_t p) {
  asm("{.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
      "add.rz.f32.bf16 %0, lo, %0;\n\tadd.rz.f32.bf16 %1, hi, %1;}"
      : "+f"(s0), "+f"(s1)
      : "r"(p));
}
__device__ __forceinline__ uint32_t bmax2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("max.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                       uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

// Positional encoding (Sec. 3.4), shared by the BF16 and FP8 loaders: each
// input channel x enters as the bands
// [x ; sin(2^0 pi x) ; cos(2^0 pi x) ; ... ; cos(2^(L-1) pi x)].
// First band: x = n + r with n = rint(x) and r = x - n exact, |r| <= 1/2, so
// sin(pi x) = (-1)^n sin(pi r) and cos(pi x) = (-1)^n cos(pi r) with
// |pi r| <= pi/2, where the hardware sine and cosine (__sinf, __cosf) are
// accurate to about 2^-21 absolute.  Every next band follows from the
// double-angle identities sin 2a = 2 sin a cos a and cos 2a = 1 - 2 sin^2 a
// in FP32; each doubling at most quadruples the error, so band f is within
// about 4^f 2^-21 of the exact value (3e-5 at f = 3), far below the rounding
// of the operand it feeds (2^-9 relative in BF16, 2^-4 in E4M3).
__device__ __forceinline__ void sincospi_reduced(float x, float& sn, float& cs) {
  const float n = rintf(x);
  const float a = (x - n) * 3.14159265358979f;
  const float h = 0.5f * n;
  const float sign = rintf(h) == h ? 1.0f : -1.0f;  // (-1)^n, also for |n| >= 2^24 (even)
  sn = sign * __sinf(a);
  cs = sign * __cosf(a);
}
template <int N>
__device__ __forceinline__ void pe_first(const float (&x)[N], float (&sn)[N], float (&cs)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) sincospi_reduced(x[j], sn[j], cs[j]);
}
template <int N>
__device__ __forceinline__ void pe_double(float (&sn)[N], float (&cs)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float a = sn[j];
    sn[j] = 2.0f * a * cs[j];
    cs[j] = fmaf(-2.0f * a, a, 1.0f);
  }
}

// Bounded wait shared by a whole warp: every lane waits, then the warp agrees.
// On a timeout the CTA-wide abort flag is raised (to the shared-memory
// address of the barrier that gave up, bit 0 set so that it is never 0) and
// every later wait fails at once, so all warps reach the common exit.
// Polling loop of a wait whose first test failed.
__device__ __forceinline__ bool wait_poll_inl(uint32_t bar, uint32_t parity,
                                              volatile int* abort_flag, uint64_t limit_ns) {
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer_ns() - t0 > limit_ns) {
      *abort_flag = static_cast<int>(bar | 1u);
      return false;
    }
  }
}
// The same loop out of line: only the first test of each wait is on the hot
// path, so with many inlined waits the loop's code would otherwise sit in the
// instruction-cache lines of the hot loops.  Measured per frame (A/B in one
// call each): two CTAs of the base widths per SM 0.0906 against 0.0942 ms;
// the kernels whose loaders encode their inputs 0.2725 against 0.2848 ms at
// H = 128 and 0.1386 against 0.1404 at H = 64; the FP8 kernel 0.1327
// against 0.1372 ms.  In the unencoded H = 128 BF16 kernel the epilogue
// warps' waits stay inline (their 96 registers of pool state would cross
// the call: 0.1231 against 0.1153 ms with every wait out of line), and
// its MMA and loader warps' waits go out of line (0.1136 against 0.1150).
static __device__ __noinline__ bool wait_poll_ool(uint32_t bar, uint32_t parity,
                                                  volatile int* abort_flag, uint64_t limit_ns) {
  return wait_poll_inl(bar, parity, abort_flag, limit_ns);
}
template <bool kOutOfLine = false>
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t limit_ns = kWaitNs) {
  bool ok = mbar_try_wait(bar, parity);
  if (!ok)
    ok = kOutOfLine ? wait_poll_ool(bar, parity, abort_flag, limit_ns)
                    : wait_poll_inl(bar, parity, abort_flag, limit_ns);
  return __all_sync(0xffffffffu, ok);
}

// Exit path of a CTA whose waits gave up: called by the warp that issued the
// CTA's MMAs and its weight copy (completion on `bar_w`, phase 0), so that
// nothing of the CTA is in flight when its TMEM is freed and it leaves:
// waits (bounded) for the copy, then commits every MMA it issued to
// `bar_drain` and waits (bounded) for that.  MMAs and copies complete by
// themselves, so both waits end.
__device__ __forceinline__ void drain_async(uint32_t bar_w, uint32_t bar_drain) {
  mbar_wait(bar_w, 0, kWaitNs);
  mma_commit_e(bar_drain);
  __syncwarp();
  mbar_wait(bar_drain, 0, kWaitNs);
  __syncwarp();
}

// Exit-path report of a CTA whose wait gave up: the timeout bit of the error
// word, and in the second word (the first reporting CTA of an error epoch
// wins) the kernel, its launch mode and the mbarrier slot that gave up:
// 1 << 31 | kernel << 16 | mode << 8 | slot.  `abort_val` is the CTA's
// abort flag, `bar_base` the address of its barrier array.
__device__ __forceinline__ void report_timeout(uint32_t* err, int abort_val, uint32_t bar_base,
                                               uint32_t kernel, uint32_t mode) {
  const uint32_t a = static_cast<uint32_t>(abort_val) & ~1u;
  const uint32_t slot = a >= bar_base ? (a - bar_base) / 8u : 0xffu;
  atomicCAS(err + 1, 0u, 0x80000000u | (kernel << 16) | (mode << 8) | (slot & 0xffu));
  atomicOr(err, kErrTimeout);
}

// Frame that owns global tile `tile`.
__device__ __forceinline__ const FusedFrame& frame_of(const FusedParams& prm, int tile) {
  int fi = 0;
  while (fi + 1 < prm.nframes && tile >= prm.f[fi + 1].tile0) ++fi;
  return prm.f[fi];
}

// Schedule index (the value the dynamic tile counter handed out) -> tile.
// Tiles go out in plan order, so the tiles of a window, which gather from the
// same stretch of every plane, run at about the same time.  The last frame's
// last windows are the end of the grid: there the partial window goes first,
// then every window's largest tile, then every window's second tile and so
// on, so that the CTAs that finish last finish on the smallest tiles.
__device__ __forceinline__ int schedule_tile(const FusedParams& prm, uint32_t s) {
  const int si = static_cast<int>(s);
  if (si < prm.tail0 || si >= prm.total_tiles) return si;
  int j = si - prm.tail0;
  const int full = prm.tail_n * prm.win_tiles;
  if (j < prm.tail_part) return prm.tail0 + full + j;
  j -= prm.tail_part;
  return prm.tail0 + (j % prm.tail_n) * prm.win_tiles + j / prm.tail_n;
}

// ---------------------------------------------------------------- loader
// Slot count of the tile of each parity, per loader warp (max over its rows).
struct LoaderShared {
  // Frame of the tile of each index mod 4 (written by loader warp 0): output
  // planes, folded per-scene biases and pixel count.  Four deep, so that the
  // epilogue can still read them after the next tile has been published.
  float* out[4];
  const float* fold[4];
  int P[4];
  int ns[2][kMaxLoadWarps];
  int tile[2];
  uint8_t cnt[2][kTile];  // per tile parity: each row's layer count (0 for an empty row)
};

constexpr int kRowsPerLoadLane = kTile / (kLoadWarps * 32);  // 2

}  // namespace fused
}  // namespace gn

// R with a 3x3 first layer (Sec. 3.4: larger kernels ahead of the 1x1 end of
// R help with global effects) over the neural buffer y of a frame, then R2
// (1x1) and the sigmoid:
//   q(p)   = ReLU(b_R1 + sum over (dy, dx) in {-1, 0, 1}^2 of W_(dy,dx) y(p + (dy, dx)))
//   rgb(p) = sigmoid(W_R2 q(p) + b_R2)
// with y = 0 outside the frame.  y comes from the fused kernel as BF16 in
// the layout [h][H/8][w][8] (8-channel chunks of one image row contiguous).
//
// Tiles are 128 consecutive pixels of one image row (M = 128 = TMEM lanes).
// The 3x3 kernel is 9 taps x H/16 K steps of tcgen05 BF16 MMAs into one
// H-column FP32 accumulator.  The A operand of tap (dy, dx) is a shifted
// view of a shared-memory halo: halo row y + dy holds the columns x0 - 1 ..
// x0 + 128 as [H/8 chunks][130 columns][8 channels], 16 bytes per pixel and
// chunk, so 8 consecutive pixels of a chunk form one core matrix and the tap
// is the descriptor started dx + 1 columns into the row (leading byte offset
// 130 * 16 between chunks, stride byte offset 128 between groups of 8
// pixels).  Halo rows live in a ring of 4 slots: a CTA runs consecutive rows
// of one 128-column strip, so a tile loads one new row while its three are
// in use.  Each tap's weights (H x H BF16) stream from L2 through a 2-stage
// ring; R2's weights and the biases stay resident.
//
// Warps: 0-3 epilogue (TMEM lane quadrant = warp), 4 MMA, 5 loads.  For tile
// t the MMA warp runs the taps into accumulator D[t & 1]; the epilogue then
// finishes tile t - 1 (R2's result + bias, sigmoid, store) and turns D into
// q = ReLU(D + b_R1) as BF16 in TMEM (Q), which R2 (K = H, N = 16) reads
// after tile t + 1's taps.  Every wait gives up after 1 s (error bit, common
// exit), as in the fused kernel.
#include <cuda_bf16.h>

#include "fused_common.cuh"

namespace gn {
namespace {
using namespace fused;

template <int H>
struct ConvLayout {
  static constexpr uint32_t kCols = 130;                  // halo columns of a row
  static constexpr uint32_t kChunkBytes = kCols * 16;     // one 8-channel chunk of a halo row
  static constexpr uint32_t kRowBytes = (H / 8) * kChunkBytes;
  static constexpr int kSlots = 4;
  static constexpr uint32_t kTapBytes = H * H * 2;        // [H/8][H][8] bf16
  static constexpr uint32_t kR2Bytes = (H / 8) * 16 * 16;  // [H/8][16][8] bf16
  static constexpr uint32_t kTailBytes = kR2Bytes + (H + 16) * 4;  // R2, b_R1 [H], b_R2 [16]
  // shared memory
  static constexpr uint32_t rows = 0;
  static constexpr uint32_t taps = rows + kSlots * kRowBytes;
  static constexpr uint32_t r2 = taps + 2 * kTapBytes;
  static constexpr uint32_t bias = r2 + kR2Bytes;
  static constexpr uint32_t smem_bytes = r2 + kTailBytes;
  // device image: the 9 taps (t = (dy + 1) * 3 + dx + 1), then the tail
  static constexpr uint32_t img_tail = 9 * kTapBytes;
  static constexpr uint32_t img_bytes = img_tail + kTailBytes;
  // TMEM: accumulators D0, D1, then Q (H/2 columns of bf16 pairs), then R2's
  static constexpr uint32_t tD = 0, tQ = 2 * H, tD2 = 2 * H + H / 2;
  static constexpr uint32_t tcols = H == 128 ? 512 : 256;
  static_assert(smem_bytes <= 232448, "conv operands exceed shared memory");
  static_assert(kTailBytes % 16 == 0 && kTapBytes % 16 == 0, "bulk copies move 16-byte units");
};

struct ConvParams {
  const uint16_t* phi;  // [h][H/8][w][8] bf16
  float* out;           // [3][h][w]
  uint32_t* err;
  int h, w, strips, tiles;
};

enum : int {
  C_TAIL = 0,    // R2 + biases copied
  C_FULL = 1,    // + slot (4): halo row loaded
  C_FREE = 5,    // + slot (4): halo row no longer read (commit)
  C_WFULL = 9,   // + stage (2): tap weights loaded
  C_WEMPTY = 11, // + stage (2): tap weights consumed (commit)
  C_DFULL = 13,  // + buffer (2): accumulator ready (commit)
  C_DFREE = 15,  // + buffer (2): accumulator read (epilogue warps)
  C_QFULL = 17,  // Q written (epilogue warps)
  C_D2FULL = 18, // R2 accumulator ready (commit)
  C_COUNT = 19
};

constexpr int kConvEpi = 4, kConvMma = 4, kConvLoad = 5, kConvThreads = 6 * 32;

// Tile i (of T, strip-major): strip s = i / h, row y = i % h.  The loads of
// the halo rows are numbered in the order a CTA issues them; tile j of a CTA
// reads loads base .. base + 2 (rows y - 1, y, y + 1).  A tile that starts a
// strip (or the CTA's range) loads all three rows, the next tile of the same
// strip one.
struct TileSeq {
  int s = 0, y = 0, base = 0;
  bool fresh = true;  // this tile loads three rows
};
__device__ __forceinline__ TileSeq next_tile(const TileSeq& prev, int i, int h, bool first) {
  TileSeq t;
  t.s = i / h;
  t.y = i - t.s * h;
  t.fresh = first || t.y == 0;
  t.base = first ? 0 : prev.base + (t.fresh ? 3 : 1);
  return t;
}

template <int H>
__global__ void __launch_bounds__(kConvThreads, 1)
    conv_r3_kernel(const __grid_constant__ ConvParams prm, const uint8_t* __restrict__ img) {
  using L = ConvLayout<H>;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[C_COUNT];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar_base = smem_u32(&bars[0]);
  auto bar = [&](int i) { return bar_base + static_cast<uint32_t>(i) * 8u; };
  // this CTA's tiles: a contiguous range of the strip-major order
  const int G = gridDim.x;
  const int t0 = static_cast<int>(static_cast<long long>(prm.tiles) * blockIdx.x / G);
  const int t1 = static_cast<int>(static_cast<long long>(prm.tiles) * (blockIdx.x + 1) / G);
  const int n = t1 - t0;

  if (tid == 0) {
    mbar_init(bar(C_TAIL), 1);
    for (int i = 0; i < 4; ++i) {
      mbar_init(bar(C_FULL + i), 1);
      mbar_init(bar(C_FREE + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(C_WFULL + i), 1);
      mbar_init(bar(C_WEMPTY + i), 1);
      mbar_init(bar(C_DFULL + i), 1);
      mbar_init(bar(C_DFREE + i), kConvEpi);
    }
    mbar_init(bar(C_QFULL), kConvEpi);
    mbar_init(bar(C_D2FULL), 1);
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == kConvMma) {
    tmem_alloc(smem_u32(&s_tmem), L::tcols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = s_tmem;
  // the halo row slot of load l
  auto slot_addr = [&](int l) { return sbase + L::rows + static_cast<uint32_t>(l & 3) * L::kRowBytes; };

  if (warp == kConvLoad) {
    // ------------------------------------------------------------ loads
    if (lane == 0) {
      mbar_arrive_expect_tx(bar(C_TAIL), L::kTailBytes);
      bulk_g2s(sbase + L::r2, img + L::img_tail, L::kTailBytes, bar(C_TAIL));
    }
    __syncwarp();
    const int h = prm.h, w = prm.w;
    // halo row yy of strip s into the slot of load l
    auto load_row = [&](int l, int s, int yy) -> bool {
      if (l >= 4 && !warp_wait(bar(C_FREE + (l & 3)), ((l >> 2) - 1) & 1, &s_abort)) return false;
      const uint32_t dst = slot_addr(l);
      if (yy < 0 || yy >= h) {  // outside the frame: zeros
        for (uint32_t o = static_cast<uint32_t>(lane) * 16u; o < L::kRowBytes; o += 32u * 16u)
          sts128(dst + o, 0u, 0u, 0u, 0u);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(C_FULL + (l & 3)));
        return true;
      }
      const int x0 = s * 128;
      const int cs = x0 > 0 ? x0 - 1 : 0;                   // first frame column copied
      const int ce = x0 + 128 < w - 1 ? x0 + 128 : w - 1;  // last frame column copied
      const uint32_t off = static_cast<uint32_t>(cs - (x0 - 1)) * 16u;  // halo column of cs
      const uint32_t bytes = static_cast<uint32_t>(ce - cs + 1) * 16u;
      // zero padding: column -1 of the frame, and column w if the halo holds it
      if (lane < H / 8) {
        const uint32_t c = dst + static_cast<uint32_t>(lane) * L::kChunkBytes;
        if (x0 == 0) sts128(c, 0u, 0u, 0u, 0u);
        if (w - x0 + 1 <= 129) sts128(c + static_cast<uint32_t>(w - x0 + 1) * 16u, 0u, 0u, 0u, 0u);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive_expect_tx(bar(C_FULL + (l & 3)), (H / 8) * bytes);
      __syncwarp();
      if (lane < H / 8) {
        const uint16_t* src = prm.phi + ((static_cast<size_t>(yy) * (H / 8) + lane) * w + cs) * 8;
        bulk_g2s(dst + static_cast<uint32_t>(lane) * L::kChunkBytes + off, src, bytes,
                 bar(C_FULL + (l & 3)));
      }
      return true;
    };
    TileSeq ts;
    for (int j = 0; j < n; ++j) {
      ts = next_tile(ts, t0 + j, h, j == 0);
      if (ts.fresh) {
        if (!load_row(ts.base, ts.s, ts.y - 1) || !load_row(ts.base + 1, ts.s, ts.y) ||
            !load_row(ts.base + 2, ts.s, ts.y + 1))
          goto done;
      } else if (!load_row(ts.base + 2, ts.s, ts.y + 1)) {
        goto done;
      }
      for (int tap = 0; tap < 9; ++tap) {
        const int g = j * 9 + tap, st = g & 1;
        if (g >= 2 && !warp_wait(bar(C_WEMPTY + st), ((g >> 1) - 1) & 1, &s_abort)) goto done;
        if (lane == 0) {
          mbar_arrive_expect_tx(bar(C_WFULL + st), L::kTapBytes);
          bulk_g2s(sbase + L::taps + static_cast<uint32_t>(st) * L::kTapBytes,
                   img + static_cast<size_t>(tap) * L::kTapBytes, L::kTapBytes, bar(C_WFULL + st));
        }
        __syncwarp();
      }
    }
  } else if (warp == kConvMma) {
    // -------------------------------------------------------------- MMA
    constexpr uint32_t idH = make_idesc(128, H, kFmtBF16);
    constexpr uint32_t id16 = make_idesc(128, 16, kFmtBF16);
    const uint64_t dsc_r2 = make_sdesc(sbase + L::r2, 16 * 16, 128);
    auto r2 = [&](int j) -> bool {  // R2 of tile j: D2 = Q W_R2^T
      if (!warp_wait(bar(C_QFULL), j & 1, &s_abort)) return false;
      tc_fence_after();
#pragma unroll
      for (int kc = 0; kc < H / 16; ++kc)
        mma_f16_ts_e(tbase + L::tD2, tbase + L::tQ + kc * 8,
                     dsc_r2 + static_cast<uint64_t>(kc) * ((2 * 16 * 16) >> 4), id16, kc > 0 ? 1u : 0u);
      mma_commit_e(bar(C_D2FULL));
      __syncwarp();
      return true;
    };
    if (!warp_wait(bar(C_TAIL), 0, &s_abort)) goto done;
    TileSeq ts;
    for (int j = 0; j < n; ++j) {
      ts = next_tile(ts, t0 + j, prm.h, j == 0);
      for (int r = 0; r < 3; ++r) {
        const int l = ts.base + r;
        if (!warp_wait(bar(C_FULL + (l & 3)), (l >> 2) & 1, &s_abort)) goto done;
      }
      const int d = j & 1;
      if (j >= 2 && !warp_wait(bar(C_DFREE + d), ((j >> 1) - 1) & 1, &s_abort)) goto done;
      tc_fence_after();
      const uint32_t D = tbase + L::tD + static_cast<uint32_t>(d) * H;
      for (int tap = 0; tap < 9; ++tap) {
        const int g = j * 9 + tap, st = g & 1;
        if (!warp_wait(bar(C_WFULL + st), (g >> 1) & 1, &s_abort)) goto done;
        tc_fence_after();
        const int ky = tap / 3, kx = tap - ky * 3;
        const uint64_t a0 = make_sdesc(slot_addr(ts.base + ky) + static_cast<uint32_t>(kx) * 16u,
                                       L::kChunkBytes, 128);
        const uint64_t b0 = make_sdesc(sbase + L::taps + static_cast<uint32_t>(st) * L::kTapBytes,
                                       H * 16, 128);
#pragma unroll
        for (int kc = 0; kc < H / 16; ++kc)
          mma_f16_ss_e(D, a0 + static_cast<uint64_t>(kc) * ((2 * L::kChunkBytes) >> 4),
                       b0 + static_cast<uint64_t>(kc) * ((2 * H * 16) >> 4), idH,
                       (tap > 0 || kc > 0) ? 1u : 0u);
        mma_commit_e(bar(C_WEMPTY + st));
        __syncwarp();
      }
      mma_commit_e(bar(C_DFULL + d));
      // halo rows no later tile of this CTA reads
      const bool cont = j + 1 < n && (t0 + j + 1) % prm.h != 0;
      mma_commit_e(bar(C_FREE + (ts.base & 3)));
      if (!cont) {
        mma_commit_e(bar(C_FREE + ((ts.base + 1) & 3)));
        mma_commit_e(bar(C_FREE + ((ts.base + 2) & 3)));
      }
      __syncwarp();
      if (j >= 1 && !r2(j - 1)) goto done;
    }
    if (n > 0 && !r2(n - 1)) goto done;
  } else if (warp < kConvEpi) {
    // --------------------------------------------------------- epilogue
    const int row = warp * 32 + lane;
    const uint32_t tl = tbase + (static_cast<uint32_t>(warp * 32) << 16);
    const float* b_r1 = reinterpret_cast<const float*>(smem + L::bias);
    const float* b_r2 = b_r1 + H;
    if (!warp_wait(bar(C_TAIL), 0, &s_abort)) goto done;
    auto finish = [&](int j) -> bool {  // tile j's RGB from R2's accumulator
      if (!warp_wait(bar(C_D2FULL), j & 1, &s_abort)) return false;
      tc_fence_after();
      uint32_t r[4];
      tmem_ld4(tl + L::tD2, r);
      const int i = t0 + j, s = i / prm.h, y = i - s * prm.h;
      const int x = s * 128 + row;
      if (x < prm.w) {
        const size_t P = static_cast<size_t>(prm.h) * prm.w;
        float* o = prm.out + static_cast<size_t>(y) * prm.w + x;
#pragma unroll
        for (int c = 0; c < kOut; ++c) o[c * P] = 1.0f / (1.0f + expf(-(__uint_as_float(r[c]) + b_r2[c])));
      }
      return true;
    };
    for (int j = 0; j < n; ++j) {
      const int d = j & 1;
      if (!warp_wait(bar(C_DFULL + d), (j >> 1) & 1, &s_abort)) goto done;
      if (j >= 1 && !finish(j - 1)) goto done;  // R2(j - 1) has read Q: Q is free
      tc_fence_after();
      const uint32_t src = tl + L::tD + static_cast<uint32_t>(d) * H;
      uint32_t ra[16], rb[16];
      tmem_ld16_async(src, ra);
      tmem_wait_ld_tied(ra);
#pragma unroll
      for (int cb = 0; cb < H / 16; ++cb) {
        uint32_t(&cur)[16] = (cb & 1) ? rb : ra;
        uint32_t(&nxt)[16] = (cb & 1) ? ra : rb;
        if (cb + 1 < H / 16) tmem_ld16_async(src + (cb + 1) * 16, nxt);
        uint32_t u[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float v0, v1;
          fadd2_rn(v0, v1, __uint_as_float(cur[2 * i]), __uint_as_float(cur[2 * i + 1]),
                   b_r1[cb * 16 + 2 * i], b_r1[cb * 16 + 2 * i + 1]);
          u[i] = pack_bf16_relu(v0, v1);
        }
        tmem_st8(tl + L::tQ + cb * 8, u);
        if (cb + 1 < H / 16) tmem_wait_ld_tied(nxt);
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(bar(C_DFREE + d));
        mbar_arrive(bar(C_QFULL));
      }
    }
    if (n > 0 && !finish(n - 1)) goto done;
  }
done:
  if (s_abort && tid == 0) atomicOr(prm.err, kErrTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == kConvMma) {
    tc_fence_after();
    tmem_dealloc(tbase, L::tcols);
  }
}

template <int H>
cudaError_t prepare_conv_h() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(conv_r3_kernel<H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ConvLayout<H>::smem_bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

}  // namespace

size_t conv_r3_image_bytes(int H) {
  return H == 128 ? ConvLayout<128>::img_bytes : ConvLayout<64>::img_bytes;
}

cudaError_t prepare_conv_r3(int H) {
  return H == 128 ? prepare_conv_h<128>() : prepare_conv_h<64>();
}

cudaError_t launch_conv_r3(int H, const void* img, const uint16_t* phi, float* out, int h, int w,
                           uint32_t* err, cudaStream_t s) {
  if (h < 1 || w < 1) return cudaSuccess;
  ConvParams p;
  p.phi = phi;
  p.out = out;
  p.err = err;
  p.h = h;
  p.w = w;
  p.strips = (w + 127) / 128;
  p.tiles = p.strips * h;
  const int grid = p.tiles < device_sm_count() ? p.tiles : device_sm_count();
  cudaError_t e = prepare_conv_r3(H);
  if (e != cudaSuccess) return e;
  if (H == 128) {
    conv_r3_kernel<128><<<grid, kConvThreads, ConvLayout<128>::smem_bytes, s>>>(
        p, static_cast<const uint8_t*>(img));
  } else {
    conv_r3_kernel<64><<<grid, kConvThreads, ConvLayout<64>::smem_bytes, s>>>(
        p, static_cast<const uint8_t*>(img));
  }
  return cudaGetLastError();
}

}  // namespace gn

// R with a 3x3 first layer (Sec. 3.4: larger kernels ahead of the 1x1 end of
// R help with global effects) over the neural buffer y of a frame, then R2
// (1x1) and the sigmoid:
//   q(p)   = ReLU(b_R1 + sum over (dy, dx) in {-1, 0, 1}^2 of W_(dy,dx) y(p + (dy, dx)))
//   rgb(p) = sigmoid(W_R2 q(p) + b_R2)
// with y = 0 outside the frame.  y comes from the fused kernel as BF16 in
// the layout [h][H/8][w][8] (8-channel chunks of one image row contiguous).
//
// Tiles are 128 consecutive pixels of one image row (M = 128 = TMEM lanes);
// a pass runs two vertically adjacent tiles (rows y, y + 1) into two
// H-column FP32 accumulators, so every tap's weights serve 256 pixels.  The
// 3x3 kernel is 9 taps x H/16 K steps of tcgen05 BF16 MMAs per accumulator.
// The A operand of tap (dy, dx) is a shifted view of a shared-memory halo:
// halo row r holds the columns x0 - 1 .. x0 + 128 as [H/8 chunks][130
// columns][8 channels], 16 bytes per pixel and chunk, so 8 consecutive
// pixels of a chunk form one core matrix and the tap is the descriptor
// started dx + 1 columns into row y + dy (leading byte offset 130 * 16
// between chunks, stride byte offset 128 between groups of 8 pixels).  Halo
// rows live in a ring of 5 slots: a CTA runs consecutive passes of one
// 128-column strip, so a pass reads 4 rows of which it loads 2 new ones, the
// first while the previous pass runs and the second (needed only by the
// taps with dy = +1) once that pass has released its oldest row.  Weights
// stream from L2 through a ring of 3 stages of half a tap (K = 64) each.
//
// Warps: 0-3 epilogue (TMEM lane quadrant = warp), 4 MMA, 5 weight loads,
// 6 row loads.  The epilogue turns each accumulator into q = BF16(ReLU(D +
// b_R1)) 16 columns at a time and applies R2 (3 outputs) on the CUDA cores
// in FP32 with the BF16-rounded R2 weights, then the sigmoid, then stores
// the RGB of its pixel.  Accumulator pairs are double buffered, so a pass's
// epilogue overlaps the next pass's MMAs.  Every wait gives up after 1 s
// (error bit, common exit), as in the fused kernel.
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
  static constexpr int kSlots = 5;
  static constexpr int kStageChunks = 8;                  // K = 64 per weight stage
  static constexpr uint32_t kStageBytes = kStageChunks * H * 16;
  static constexpr int kStagesPerTap = (H / 8) / kStageChunks;
  static constexpr int kStages = 3;
  static constexpr uint32_t kTapBytes = H * H * 2;        // [H/8][H][8] bf16
  static constexpr uint32_t kTailBytes = (H + 3 * H + 4) * 4;  // b_R1 [H], W_R2 [3][H], b_R2 [4]
  // shared memory
  static constexpr uint32_t rows = 0;
  static constexpr uint32_t wst = rows + kSlots * kRowBytes;
  static constexpr uint32_t tail = wst + kStages * kStageBytes;
  static constexpr uint32_t smem_bytes = tail + kTailBytes;
  // device image: the 9 taps (t = (dy + 1) * 3 + dx + 1), then the tail
  static constexpr uint32_t img_tail = 9 * kTapBytes;
  static constexpr uint32_t img_bytes = img_tail + kTailBytes;
  // TMEM: two buffers of two H-column accumulators (rows y, y + 1)
  static constexpr uint32_t tcols = 4 * H;
  static_assert(tcols == 256 || tcols == 512, "TMEM allocation must be a power of two");
  static_assert(smem_bytes <= 232448, "conv operands exceed shared memory");
  static_assert(kTailBytes % 16 == 0 && kStageBytes % 16 == 0, "bulk copies move 16-byte units");
  static_assert(kStagesPerTap * kStageChunks * 8 == H, "weight stages must tile a tap");
};

struct ConvParams {
  const uint16_t* phi;  // [h][H/8][w][8] bf16
  float* out;           // [3][h][w]
  uint32_t* err;
  int h, w, hp, passes;  // hp = passes per strip = ceil(h / 2)
};

constexpr int kSlotsC = 5, kStagesC = 3;
enum : int {
  C_TAIL = 0,                     // biases and R2 copied
  C_FULL = 1,                     // + slot: halo row loaded
  C_FREE = C_FULL + kSlotsC,      // + slot: halo row no longer read (commit)
  C_WFULL = C_FREE + kSlotsC,     // + stage: weights loaded
  C_WEMPTY = C_WFULL + kStagesC,  // + stage: weights consumed (commit)
  C_DFULL = C_WEMPTY + kStagesC,  // + buffer: accumulator pair ready (commit)
  C_DFREE = C_DFULL + 2,          // + buffer: accumulator pair read (epilogue warps)
  C_DRAIN = C_DFREE + 2,          // the exit path's last commit
  C_COUNT = C_DRAIN + 1
};

constexpr int kConvEpi = 4, kConvMma = 4, kConvWLoad = 5, kConvRLoad = 6, kConvThreads = 7 * 32;

// Pass i (strip-major): strip s = i / hp, rows y = 2 (i % hp) and y + 1.
// Halo-row loads are numbered in issue order; a pass reads loads base ..
// base + 3 (rows y - 1 .. y + 2).  A pass that starts a strip (or the CTA's
// range) loads all four, the next pass of the same strip two.
struct PassSeq {
  int s = 0, y = 0, base = 0;
  bool fresh = true;
};
__device__ __forceinline__ PassSeq next_pass(const PassSeq& prev, int i, int hp, bool first) {
  PassSeq t;
  t.s = i / hp;
  t.y = 2 * (i - t.s * hp);
  t.fresh = first || t.y == 0;
  t.base = first ? 0 : prev.base + (t.fresh ? 4 : 2);
  return t;
}

template <int H>
__global__ void __launch_bounds__(kConvThreads, 1)
    conv_r3_kernel(const __grid_constant__ ConvParams prm, const uint8_t* __restrict__ img) {
  using L = ConvLayout<H>;
  static_assert(L::kSlots == kSlotsC && L::kStages == kStagesC, "barrier slots");
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[C_COUNT];
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar_base = smem_u32(&bars[0]);
  auto bar = [&](int i) { return bar_base + static_cast<uint32_t>(i) * 8u; };
  // this CTA's passes: a contiguous range of the strip-major order
  const int G = gridDim.x;
  const int t0 = static_cast<int>(static_cast<long long>(prm.passes) * blockIdx.x / G);
  const int t1 = static_cast<int>(static_cast<long long>(prm.passes) * (blockIdx.x + 1) / G);
  const int n = t1 - t0;

  if (tid == 0) {
    mbar_init(bar(C_TAIL), 1);
    for (int i = 0; i < kSlotsC; ++i) {
      mbar_init(bar(C_FULL + i), 1);
      mbar_init(bar(C_FREE + i), 1);
    }
    for (int i = 0; i < kStagesC; ++i) {
      mbar_init(bar(C_WFULL + i), 1);
      mbar_init(bar(C_WEMPTY + i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar(C_DFULL + i), 1);
      mbar_init(bar(C_DFREE + i), kConvEpi);
    }
    mbar_init(bar(C_DRAIN), 1);
    s_abort = 0;
    fence_mbar_init();
  }
  // the last copy each loader warp issued per weight stage / halo slot (the
  // exit path waits for them)
  int last_wg[kStagesC], last_l[kSlotsC];
  for (int i = 0; i < kStagesC; ++i) last_wg[i] = -1;
  for (int i = 0; i < kSlotsC; ++i) last_l[i] = -1;
  if (warp == kConvMma) {
    tmem_alloc(smem_u32(&s_tmem), L::tcols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = s_tmem;
  // the halo-row slot of load l
  auto slot_addr = [&](int l) {
    return sbase + L::rows + static_cast<uint32_t>(l % kSlotsC) * L::kRowBytes;
  };

  if (warp == kConvWLoad) {
    // ---------------------------------------------------- weight stream
    if (lane == 0) {
      mbar_arrive_expect_tx(bar(C_TAIL), L::kTailBytes);
      bulk_g2s(sbase + L::tail, img + L::img_tail, L::kTailBytes, bar(C_TAIL));
    }
    __syncwarp();
    for (int j = 0; j < n; ++j)
      for (int tap = 0; tap < 9; ++tap)
        for (int q = 0; q < L::kStagesPerTap; ++q) {
          const int g = (j * 9 + tap) * L::kStagesPerTap + q, st = g % kStagesC, u = g / kStagesC;
          if (u > 0 && !warp_wait(bar(C_WEMPTY + st), (u - 1) & 1, &s_abort)) goto done;
          last_wg[st] = g;
          if (lane == 0) {
            mbar_arrive_expect_tx(bar(C_WFULL + st), L::kStageBytes);
            bulk_g2s(sbase + L::wst + static_cast<uint32_t>(st) * L::kStageBytes,
                     img + static_cast<size_t>(tap) * L::kTapBytes + static_cast<size_t>(q) * L::kStageBytes,
                     L::kStageBytes, bar(C_WFULL + st));
          }
          __syncwarp();
        }
  } else if (warp == kConvRLoad) {
    // ------------------------------------------------------- halo rows
    const int h = prm.h, w = prm.w;
    // halo row yy of strip s into the slot of load l
    auto load_row = [&](int l, int s, int yy) -> bool {
      const int sl = l % kSlotsC;
      if (l >= kSlotsC && !warp_wait(bar(C_FREE + sl), ((l / kSlotsC) - 1) & 1, &s_abort))
        return false;
      const uint32_t dst = slot_addr(l);
      last_l[sl] = l;
      if (yy < 0 || yy >= h) {  // outside the frame: zeros
        for (uint32_t o = static_cast<uint32_t>(lane) * 16u; o < L::kRowBytes; o += 32u * 16u)
          sts128(dst + o, 0u, 0u, 0u, 0u);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(C_FULL + sl));
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
      if (lane == 0) mbar_arrive_expect_tx(bar(C_FULL + sl), (H / 8) * bytes);
      __syncwarp();
      if (lane < H / 8) {
        const uint16_t* src = prm.phi + ((static_cast<size_t>(yy) * (H / 8) + lane) * w + cs) * 8;
        bulk_g2s(dst + static_cast<uint32_t>(lane) * L::kChunkBytes + off, src, bytes,
                 bar(C_FULL + sl));
      }
      return true;
    };
    PassSeq ps;
    for (int j = 0; j < n; ++j) {
      ps = next_pass(ps, t0 + j, prm.hp, j == 0);
      if (ps.fresh && (!load_row(ps.base, ps.s, ps.y - 1) || !load_row(ps.base + 1, ps.s, ps.y)))
        goto done;
      if (!load_row(ps.base + 2, ps.s, ps.y + 1) || !load_row(ps.base + 3, ps.s, ps.y + 2)) goto done;
    }
  } else if (warp == kConvMma) {
    // -------------------------------------------------------------- MMA
    constexpr uint32_t idH = make_idesc(128, H, kFmtBF16);
    constexpr uint64_t kA16 = (2 * L::kChunkBytes) >> 4;  // one K step of an A operand
    constexpr uint64_t kB16 = (2 * H * 16) >> 4;          // one K step of a weight stage
    PassSeq ps;
    for (int j = 0; j < n; ++j) {
      ps = next_pass(ps, t0 + j, prm.hp, j == 0);
      const int d = j & 1;
      if (j >= 2 && !warp_wait(bar(C_DFREE + d), ((j >> 1) - 1) & 1, &s_abort)) goto done;
      const uint32_t Da = tbase + static_cast<uint32_t>(d) * 2 * H, Db = Da + H;
      for (int ky = 0; ky < 3; ++ky) {
        // rows y - 1 + ky (output row y) and y + ky (output row y + 1)
        for (int r = 0; r < 2; ++r) {
          const int l = ps.base + ky + r;
          if (!warp_wait(bar(C_FULL + l % kSlotsC), (l / kSlotsC) & 1, &s_abort)) goto done;
        }
        tc_fence_after();
        for (int kx = 0; kx < 3; ++kx) {
          const int tap = ky * 3 + kx;
          const uint64_t a0 = make_sdesc(slot_addr(ps.base + ky) + static_cast<uint32_t>(kx) * 16u,
                                         L::kChunkBytes, 128);
          const uint64_t b0 = make_sdesc(slot_addr(ps.base + ky + 1) + static_cast<uint32_t>(kx) * 16u,
                                         L::kChunkBytes, 128);
          for (int q = 0; q < L::kStagesPerTap; ++q) {
            const int g = (j * 9 + tap) * L::kStagesPerTap + q, st = g % kStagesC;
            if (!warp_wait(bar(C_WFULL + st), (g / kStagesC) & 1, &s_abort)) goto done;
            tc_fence_after();
            const uint64_t w0 =
                make_sdesc(sbase + L::wst + static_cast<uint32_t>(st) * L::kStageBytes, H * 16, 128);
#pragma unroll
            for (int kc = 0; kc < L::kStageChunks / 2; ++kc) {
              const uint64_t ko = static_cast<uint64_t>(q * (L::kStageChunks / 2) + kc) * kA16;
              const uint32_t acc = (tap > 0 || q > 0 || kc > 0) ? 1u : 0u;
              mma_f16_ss_e(Da, a0 + ko, w0 + static_cast<uint64_t>(kc) * kB16, idH, acc);
              mma_f16_ss_e(Db, b0 + ko, w0 + static_cast<uint64_t>(kc) * kB16, idH, acc);
            }
            mma_commit_e(bar(C_WEMPTY + st));
            __syncwarp();
          }
        }
      }
      mma_commit_e(bar(C_DFULL + d));
      // halo rows no later pass of this CTA reads
      const bool cont = j + 1 < n && (t0 + j + 1) % prm.hp != 0;
      mma_commit_e(bar(C_FREE + ps.base % kSlotsC));
      mma_commit_e(bar(C_FREE + (ps.base + 1) % kSlotsC));
      if (!cont) {
        mma_commit_e(bar(C_FREE + (ps.base + 2) % kSlotsC));
        mma_commit_e(bar(C_FREE + (ps.base + 3) % kSlotsC));
      }
      __syncwarp();
    }
  } else if (warp < kConvEpi) {
    // --------------------------------------------------------- epilogue
    const int row = warp * 32 + lane;
    const uint32_t tl = tbase + (static_cast<uint32_t>(warp * 32) << 16);
    const float* b_r1 = reinterpret_cast<const float*>(smem + L::tail);
    const float* w_r2 = b_r1 + H;  // [3][H], BF16-rounded
    const float* b_r2 = w_r2 + 3 * H;
    if (!warp_wait(bar(C_TAIL), 0, &s_abort)) goto done;
    const size_t P = static_cast<size_t>(prm.h) * prm.w;
    PassSeq ps;
    for (int j = 0; j < n; ++j) {
      ps = next_pass(ps, t0 + j, prm.hp, j == 0);
      const int d = j & 1;
      if (!warp_wait(bar(C_DFULL + d), (j >> 1) & 1, &s_abort)) goto done;
      tc_fence_after();
#pragma unroll 1
      for (int r = 0; r < 2; ++r) {
        const uint32_t src = tl + static_cast<uint32_t>(d * 2 + r) * H;
        float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f;
        uint32_t ra[16], rb[16];
        tmem_ld16_async(src, ra);
        tmem_wait_ld_tied(ra);
#pragma unroll
        for (int cb = 0; cb < H / 16; ++cb) {
          uint32_t(&cur)[16] = (cb & 1) ? rb : ra;
          uint32_t(&nxt)[16] = (cb & 1) ? ra : rb;
          if (cb + 1 < H / 16) tmem_ld16_async(src + (cb + 1) * 16, nxt);
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            const int k = cb * 16 + i;
            float v0, v1;
            fadd2_rn(v0, v1, __uint_as_float(cur[i]), __uint_as_float(cur[i + 1]), b_r1[k], b_r1[k + 1]);
            const uint32_t qb = pack_bf16_relu(v0, v1);  // q, rounded to BF16 as R2's operand
            const float q0 = __uint_as_float(qb << 16), q1 = __uint_as_float(qb & 0xffff0000u);
            o0 = fmaf(q1, w_r2[k + 1], fmaf(q0, w_r2[k], o0));
            o1 = fmaf(q1, w_r2[H + k + 1], fmaf(q0, w_r2[H + k], o1));
            o2 = fmaf(q1, w_r2[2 * H + k + 1], fmaf(q0, w_r2[2 * H + k], o2));
          }
          if (cb + 1 < H / 16) tmem_wait_ld_tied(nxt);
        }
        const int y = ps.y + r, x = ps.s * 128 + row;
        if (y < prm.h && x < prm.w) {
          float* o = prm.out + static_cast<size_t>(y) * prm.w + x;
          o[0] = 1.0f / (1.0f + expf(-(o0 + b_r2[0])));
          o[P] = 1.0f / (1.0f + expf(-(o1 + b_r2[1])));
          o[2 * P] = 1.0f / (1.0f + expf(-(o2 + b_r2[2])));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(C_DFREE + d));
    }
  }
done:
  tc_fence_before();
  __syncthreads();  // every warp is here: s_abort is final
  if (s_abort) {
    // nothing of this CTA may be in flight when it leaves: each loader warp
    // waits (bounded) for the last copy it issued per stage or slot, the MMA
    // warp commits every MMA it issued and waits for that
    if (warp == kConvWLoad && lane == 0) {
      mbar_wait(bar(C_TAIL), 0, kWaitNs);
      for (int st = 0; st < kStagesC; ++st)
        if (last_wg[st] >= 0) mbar_wait(bar(C_WFULL + st), (last_wg[st] / kStagesC) & 1, kWaitNs);
    }
    if (warp == kConvRLoad && lane == 0)
      for (int sl = 0; sl < kSlotsC; ++sl)
        if (last_l[sl] >= 0) mbar_wait(bar(C_FULL + sl), (last_l[sl] / kSlotsC) & 1, kWaitNs);
    if (warp == kConvMma) {
      mma_commit_e(bar(C_DRAIN));
      __syncwarp();
      mbar_wait(bar(C_DRAIN), 0, kWaitNs);
      __syncwarp();
    }
    if (tid == 0) report_timeout(prm.err, s_abort, bar_base, kKernelConvR3, 0);
    __syncthreads();
  }
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
  p.hp = (h + 1) / 2;
  p.passes = ((w + 127) / 128) * p.hp;
  const int grid = p.passes < device_sm_count() ? p.passes : device_sm_count();
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

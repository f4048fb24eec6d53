// Compacted ragged-layer kernel (BF16, H = 64, no encoding, 1x1 R): the
// layer work of a block of 256 pixels runs in 128-row layer tiles that hold
// valid (pixel, layer) rows only, so no tile runs a layer slot for a pixel
// that has no such layer (Eq. 5 pools over each pixel's own layers).
//
// Arithmetic: the one-stream kernel's (fused_bf16.cu) step for step, so a
// frame comes out bit-identical to it: per valid (pixel, layer) row
// U = bf16 ReLU(phi1) and u = bf16 ReLU(phi2 U + b); pool = [max ; mean] (or
// the sum tau) of each pixel's u; then rho, B1, B2, R1, R2 and the sigmoid.
//
// Layer rows.  A block is half of a plan window: up to two 128-pixel tiles of
// one frame in pixel order (the plan's identity mode).  Its rows are the
// pairs (slot k, pixel p) with k < c_p, slot-major: slot 0's pixels in block
// order, then slot 1's, and so on; R rows in ceil(R / 128) layer tiles.  Only
// the last layer tile of a block has empty rows: about 64 of ~770 at
// Poisson(3) counts (1.08 executed rows per valid row, against 1.42 for the
// count-sorted tiles of the one-stream kernel).
//
// Pooling in shared memory.  Row r of a layer tile need not be TMEM lane r's
// pixel in the next layer tile, so the pool cannot stay in registers: it is
// kept channel-major in shared memory for the block's 256 pixels (the running
// max as the bits of the non-negative bf16 u, and the fixed-point sum), and
// each valid row updates its pixel's entries with shared-memory reductions.
// Both are order-independent: the max by nature; the sum because every
// addend is first truncated to the quantum 2^-12 (u added to 2^11 rounding
// toward zero, minus 2^11, both exact), and sums of such multiples in
// [2^11, 2^12) are exact in FP32 in any order.  The register form adds u to
// its running sum rounding toward zero, which gives the same multiples of
// 2^-12, so a pixel's pool matches it bit for bit; a sum that leaves
// [2^11, 2^12) sets the range error bit in both forms.
//
// Pixel layers.  After a block's last layer tile the epilogue turns each
// pixel's entries into rho's A operand in TMEM ([max ; mean] as bf16, lane =
// the pixel's row in its tile), resets them, and the per-pixel layers run
// tile by tile as in the one-stream kernel.
//
// Roles (11 warps): 8 epilogue warps (TMEM lane quadrant w % 4, accumulator
// columns 32 (w / 4) .. + 31), the MMA warp, 2 loader warps.  TMEM: three
// H-column accumulators rotating over the layer tiles (phi1 two tiles ahead
// of phi2) and U double buffered, reused by the per-pixel layers.  Shared
// memory: the operand image, a second G-buffer operand and the pool (128 KB),
// 205 KB; one CTA per SM.  Every wait is bounded (1 s).
#include <cuda_bf16.h>

#include "fused_common.cuh"

namespace gn {
namespace {
using namespace fused;

constexpr int HC = 64;
constexpr int kBlockTiles = 2;                  // pixel tiles per block (half a plan window)
constexpr int kBlockPx = kBlockTiles * kTile;   // 256
constexpr int kEpiC = 8;                        // epilogue warps 0-7
constexpr int kMmaC = kEpiC;                    // warp 8
constexpr int kLoadC0 = kEpiC + 1;              // warps 9, 10
constexpr int kLoadCW = 2;
constexpr int kRplC = kTile / (kLoadCW * 32);   // rows per loader lane (2)
constexpr int kThreadsC = (kEpiC + 1 + kLoadCW) * 32;
constexpr int CHc = HC / 2;                     // channels per epilogue thread (32)

using LC = FusedLayout<HC, false>;

// Shared memory beyond the operand image (bytes).
struct CS {
  static constexpr uint32_t ag1 = (LC::smem_bytes + 127) / 128 * 128;  // tile 1's G-buffer operand
  static constexpr uint32_t pmax = ag1 + 16 * 256;                      // u32 [HC][kBlockPx]
  static constexpr uint32_t psum = pmax + HC * kBlockPx * 4;            // f32 [HC][kBlockPx]
  static constexpr uint32_t bytes = psum + HC * kBlockPx * 4;
  static_assert(bytes + 8192 <= 232448, "shared memory");
};

// mbarrier slots beyond the common ones (B_SCHED's two slots are B_SETUP here).
constexpr int B_SETUP = B_SCHED;     // + parity: block set up by loader warp 0
constexpr int B_HC = B_COUNT;        // + half: K half of the next per-pixel A operand written
constexpr int B_ES = B_COUNT + 2;    // + n & 1: epilogue warps' sync
constexpr int B_STALLC = B_COUNT + 4;
constexpr int B_DRAINC = B_COUNT + 5;
constexpr int B_COUNT_C = B_COUNT + 6;

// TMEM as the one-stream kernel at H = 64: buffers 0..2 at b H, U at 3H, 3H + H/2.
constexpr uint32_t AU0c = 3 * HC, AU1c = 3 * HC + HC / 2, APOOLc = AU0c, NCOLSc = 4 * HC;

// A block as loader warp 0 publishes it, double buffered by block parity.
struct BlockShared {
  int blk[2];
  int tile0[2];
  int ntiles[2];
  int P[2];
  float* out[2];
  const float* fold[2];
  int off[2][kMaxK + 1];            // first row of each slot; off[kMaxK] = R
  uint32_t ent[2][kBlockPx];        // the block's plan entries
  uint8_t list[2][kMaxK][kBlockPx]; // slot k's entries in block order
};

__device__ __forceinline__ void red_max_u32(uint32_t addr, uint32_t v) {
  asm volatile("red.shared.max.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ void red_add_f32(uint32_t addr, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// D (+)= A (TMEM, K/2 columns from a_tmem) x B^T, B [K/8][N][8] bf16 from
// descriptor d0; one K step of 16 advances B by 2 N 16 bytes.
template <int N, int K>
__device__ __forceinline__ void gemm_t(uint32_t d_tmem, uint32_t a_tmem, uint64_t d0, uint32_t idesc,
                                       bool accumulate = false) {
  constexpr uint32_t step = (2 * N * 16) >> 4;
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks)
    mma_f16_ts_e(d_tmem, a_tmem + ks * 8, d0 + static_cast<uint64_t>(step) * ks, idesc,
                 (ks > 0 || accumulate) ? 1u : 0u);
}

// Block b: half (b & 1) of plan window b / 2, i.e. its tiles 2 (b & 1) and
// 2 (b & 1) + 1 that exist (none for the second half of a short window).
__device__ __forceinline__ void block_tiles(const FusedParams& prm, int b, int& fi, int& tile0,
                                            int& ntiles) {
  const int w = b >> 1;
  fi = 0;
  while (fi + 1 < prm.nframes && w >= prm.f[fi + 1].win0) ++fi;
  const FusedFrame& F = prm.f[fi];
  const int tiles_f = (F.P + kTile - 1) / kTile;
  const int first = (w - F.win0) * prm.win_tiles + (b & 1) * kBlockTiles;
  tile0 = F.tile0 + first;
  ntiles = max(0, min(kBlockTiles, tiles_f - first));
}

// Row r of a block's layer rows: its entry in the block (0..255) and slot,
// or -1 past the block's last row.
__device__ __forceinline__ int row_entry(const BlockShared& bs, int par, int r, int& k) {
  k = 0;
  if (r >= bs.off[par][kMaxK]) return -1;
  while (k + 1 < kMaxK && bs.off[par][k + 1] <= r) ++k;
  return bs.list[par][k][r - bs.off[par][k]];
}

// ---------------------------------------------------------------- loaders
// Loader warp 0 takes blocks from the global counter and sets each one up
// (entries, slot lists, row offsets); both warps then gather the block's
// G-buffer rows and fill the layer operands tile by tile (two buffers,
// released by the phi1 MMAs) and the two G-buffer operands (released by the
// block's last B1).  That release also paces the set-up: a block's shared
// data (parity buffer) is rewritten two blocks later, after every role is
// done with it.
__device__ __forceinline__ void loader_c(const FusedParams& prm, uint32_t sbase, uint32_t bar_base,
                                         BlockShared& bs, volatile int* abort_flag, int li, int lane) {
  auto bar = [&](int i) { return bar_base + static_cast<uint32_t>(i) * 8u; };
  const int row0 = li * (32 * kRplC) + lane;
  const int total_blocks = 2 * prm.total_windows;
  uint32_t lc = 0, n_ag = 0;
  for (uint32_t tb = 0;; ++tb) {
    const int par = tb & 1;
    if (li == 0) {
      int b, fi = 0, tile0 = 0, ntiles = 0;
      do {
        b = 0;
        if (lane == 0) b = static_cast<int>(atomicAdd(prm.next_tile, 1u));
        b = __shfl_sync(0xffffffffu, b, 0);
        if (b < total_blocks) block_tiles(prm, b, fi, tile0, ntiles);
      } while (b < total_blocks && ntiles == 0);
      if (b < total_blocks) {
        // entries 8 lane .. 8 lane + 7, then slot-major row lists
        int c[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int e = 8 * lane + i;
          const uint32_t en = e < ntiles * kTile ? __ldg(prm.plan + static_cast<size_t>(tile0) * kTile + e)
                                                 : kPlanEmpty;
          bs.ent[par][e] = en;
          c[i] = en == kPlanEmpty ? 0 : static_cast<int>(en >> 28);
        }
        int off = 0;
#pragma unroll 1
        for (int k = 0; k < kMaxK; ++k) {
          int mine = 0;
#pragma unroll
          for (int i = 0; i < 8; ++i) mine += c[i] > k ? 1 : 0;
          int incl = mine;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
          }
          int pos = incl - mine;
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (c[i] > k) bs.list[par][k][pos++] = static_cast<uint8_t>(8 * lane + i);
          if (lane == 0) bs.off[par][k] = off;
          off += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
          bs.off[par][kMaxK] = off;
          bs.tile0[par] = tile0;
          bs.ntiles[par] = ntiles;
          bs.out[par] = prm.f[fi].out;
          bs.fold[par] = prm.f[fi].fold;
          bs.P[par] = prm.f[fi].P;
        }
      }
      if (lane == 0) bs.blk[par] = b;
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_SETUP + par));
    } else if (!warp_wait(bar(B_SETUP + par), (tb >> 1) & 1, abort_flag)) {
      return;
    }
    // both loader warps publish the block to the MMA and epilogue warps
    __syncwarp();
    if (lane == 0) mbar_arrive(bar(B_TILE + par));
    const int b = *reinterpret_cast<volatile int*>(&bs.blk[par]);
    if (b >= total_blocks) return;
    const int R = bs.off[par][kMaxK];
    const int ns = (R + kTile - 1) / kTile;
    int fi, tile0_unused, nt_unused;
    block_tiles(prm, b, fi, tile0_unused, nt_unused);
    const FusedFrame& F = prm.f[fi];
    const uint32_t P = static_cast<uint32_t>(F.P);

    // the G-buffer rows of both pixel tiles, loads in flight now
    float gv[kBlockTiles][kRplC][kGC];
#pragma unroll
    for (int t = 0; t < kBlockTiles; ++t)
#pragma unroll
      for (int i = 0; i < kRplC; ++i) {
        const uint32_t en = bs.ent[par][t * kTile + row0 + 32 * i];
        const bool has = en != kPlanEmpty;
        const uint32_t pix = has ? (en & kPlanPixelMask) : 0u;
#pragma unroll
        for (int ch = 0; ch < kGC; ++ch)
          gv[t][i][ch] = has ? __ldg(F.gbuf + (static_cast<uint32_t>(ch) * P + pix)) : 0.0f;
      }
    auto put_ag = [&]() -> bool {
      if (!warp_wait(bar(B_AG_E), (n_ag & 1) ^ 1, abort_flag)) return false;
      ++n_ag;
      const uint32_t one = pack_bf16(1.0f, 1.0f);
#pragma unroll
      for (int t = 0; t < kBlockTiles; ++t)
#pragma unroll
        for (int i = 0; i < kRplC; ++i) {
          const uint32_t r = sbase + (t ? CS::ag1 : LC::ag) + static_cast<uint32_t>(row0 + 32 * i) * 16u;
          const float(&g)[kGC] = gv[t][i];
          sts128(r, pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]),
                 pack_bf16(g[6], g[7]));
          sts128(r + 2048u, pack_bf16(g[8], g[9]), pack_bf16(g[10], g[11]), pack_bf16(g[12], g[13]),
                 one);
        }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_AG_F));
      return true;
    };
    // layer rows of layer tile t: 12 channels of (slot k, entry e), zeros past R
    auto load_rows = [&](int t, float(&x)[kRplC][kTC]) {
#pragma unroll
      for (int i = 0; i < kRplC; ++i) {
        int k;
        const int e = row_entry(bs, par, t * kTile + row0 + 32 * i, k);
        const uint32_t pix = e < 0 ? 0u : (bs.ent[par][e] & kPlanPixelMask);
        const uint32_t o = static_cast<uint32_t>(k) * kTC * P + pix;
#pragma unroll
        for (int ch = 0; ch < kTC; ++ch) x[i][ch] = e >= 0 ? __ldg(F.tbuf + (o + ch * P)) : 0.0f;
      }
    };
    float x[kRplC][kTC], y[kRplC][kTC];
    if (ns > 0) load_rows(0, x);
    if (ns == 0 && !put_ag()) return;
    for (int t = 0; t < ns; ++t, ++lc) {
      if (t + 1 < ns) load_rows(t + 1, y);
      const int bb = lc & 1;
      if (!warp_wait(bar(B_AT_E + bb), ((lc >> 1) & 1) ^ 1, abort_flag)) return;
      const uint32_t base = sbase + (bb ? LC::at1 : LC::at0);
      const uint32_t one = pack_bf16(1.0f, 1.0f);
#pragma unroll
      for (int i = 0; i < kRplC; ++i) {
        const uint32_t r = base + static_cast<uint32_t>(row0 + 32 * i) * 16u;
        sts128(r, pack_bf16(x[i][0], x[i][1]), pack_bf16(x[i][2], x[i][3]),
               pack_bf16(x[i][4], x[i][5]), pack_bf16(x[i][6], x[i][7]));
        sts128(r + 2048u, pack_bf16(x[i][8], x[i][9]), pack_bf16(x[i][10], x[i][11]), one, 0u);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_AT_F + bb));
      if (t == 0 && !put_ag()) return;
#pragma unroll
      for (int i = 0; i < kRplC; ++i)
#pragma unroll
        for (int ch = 0; ch < kTC; ++ch) x[i][ch] = y[i][ch];
    }
  }
}

// ------------------------------------------------------------------ kernel
template <bool Sum>
__global__ void __launch_bounds__(kThreadsC, 1)
    fused_compact_kernel(const __grid_constant__ FusedParams prm, const uint8_t* __restrict__ wimg) {
  constexpr int H = HC;
  using L = LC;
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[B_COUNT_C];
  __shared__ uint32_t s_tmem;
  __shared__ BlockShared s_bs;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar_base = smem_u32(&bars[0]);
  auto bar = [&](int i) { return bar_base + static_cast<uint32_t>(i) * 8u; };
  const int total_blocks = 2 * prm.total_windows;
  const uint32_t pmax = sbase + CS::pmax, psum = sbase + CS::psum;

  if (tid == 0) {
    mbar_init(bar(B_W), 1);
    mbar_init(bar(B_DP), 1);
    mbar_init(bar(B_DR2), 1);
    mbar_init(bar(B_AG_F), kLoadCW);
    mbar_init(bar(B_AG_E), 1);
    mbar_init(bar(B_STALLC), 1);
    mbar_init(bar(B_DRAINC), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(B_IN + b), kEpiC);
      mbar_init(bar(B_AT_F + b), kLoadCW);
      mbar_init(bar(B_AT_E + b), 1);
      mbar_init(bar(B_TILE + b), kLoadCW);
      mbar_init(bar(B_SETUP + b), 1);
      mbar_init(bar(B_HC + b), kEpiC);
      mbar_init(bar(B_ES + b), kEpiC);
    }
    for (int b = 0; b < 3; ++b) {
      mbar_init(bar(B_D1 + b), 1);
      mbar_init(bar(B_D2 + b), 1);
      mbar_init(bar(B_BE + b), kEpiC);
    }
    s_abort = 0;
    fence_mbar_init();
  }
  // pool start values (max 0, sum 2^11), by every thread
  for (uint32_t i = tid; i < HC * kBlockPx / 4; i += kThreadsC) {
    const uint32_t s0 = __float_as_uint(kSumBase);
    sts128(pmax + i * 16u, 0u, 0u, 0u, 0u);
    sts128(psum + i * 16u, s0, s0, s0, s0);
  }
  if (warp == kMmaC) {
    tmem_alloc(smem_u32(&s_tmem), NCOLSc);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = s_tmem;

  // Block number t of this CTA as the loaders published it.
  auto take_block = [&](uint32_t t, int& blk, int& ns, int& ntiles) -> bool {
    if (!warp_wait(bar(B_TILE + (t & 1)), (t >> 1) & 1, &s_abort)) return false;
    blk = *reinterpret_cast<volatile int*>(&s_bs.blk[t & 1]);
    ns = blk < total_blocks ? (s_bs.off[t & 1][kMaxK] + kTile - 1) / kTile : 0;
    ntiles = blk < total_blocks ? s_bs.ntiles[t & 1] : 0;
    return true;
  };

  if (warp >= kLoadC0) {
    // --------------------------------------------------------------- loaders
    for (int r = (warp - kLoadC0) * 32 + lane; r < kTile; r += kLoadCW * 32) {
      sts128(sbase + L::aone + r * 16u, pack_bf16(1.0f, 1.0f), 0u, 0u, 0u);
      sts128(sbase + L::aone + 2048u + r * 16u, 0u, 0u, 0u, 0u);
    }
    fence_proxy_async_smem();
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the plan is complete
    loader_c(prm, sbase, bar_base, s_bs, &s_abort, warp - kLoadC0, lane);
  } else if (warp == kMmaC) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      mbar_arrive_expect_tx(bar(B_W), L::bytes);
      for (uint32_t off = 0; off < L::bytes; off += 32768u) {
        const uint32_t n = L::bytes - off < 32768u ? L::bytes - off : 32768u;
        bulk_g2s(sbase + off, wimg + off, n, bar(B_W));
      }
    }
    __syncwarp();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    constexpr uint32_t idH = make_idesc(128, H, kFmtBF16);
    constexpr uint32_t id16 = make_idesc(128, 16, kFmtBF16);
    const uint64_t dsc_phi1 = make_sdesc(sbase + L::phi1, H * 16, 128);
    const uint64_t dsc_phi2 = make_sdesc(sbase + L::phi2, H * 16, 128);
    const uint64_t dsc_phi2b = make_sdesc(sbase + L::phi2b, H * 16, 128);
    const uint64_t dsc_rho = make_sdesc(sbase + L::rho, H * 16, 128);
    const uint64_t dsc_b1 = make_sdesc(sbase + L::b1, H * 16, 128);
    const uint64_t dsc_b2 = make_sdesc(sbase + L::b2, H * 16, 128);
    const uint64_t dsc_r1 = make_sdesc(sbase + L::r1, H * 16, 128);
    const uint64_t dsc_r2 = make_sdesc(sbase + L::r2, 16 * 16, 128);
    const uint64_t dsc_at0 = make_sdesc(sbase + L::at0, 128 * 16, 128);
    const uint64_t dsc_at1 = make_sdesc(sbase + L::at1, 128 * 16, 128);
    const uint64_t dsc_one = make_sdesc(sbase + L::aone, 128 * 16, 128);
    const uint64_t dsc_ag0 = make_sdesc(sbase + L::ag, 128 * 16, 128);
    const uint64_t dsc_ag1 = make_sdesc(sbase + CS::ag1, 128 * 16, 128);
    const uint64_t dsc_b1r = dsc_b1 + static_cast<uint64_t>((2 * H * 16) >> 4);
    constexpr uint64_t kHalfK = static_cast<uint64_t>(H / 32) * ((2 * H * 16) >> 4);
    SlotPos p1, p2;
    uint32_t g1 = 0, n_in = 0, n_agf = 0, n_pt = 0, n_h[2] = {0, 0};
    const float* cur_fold = nullptr;
    auto phi1 = [&]() -> bool {
      if (!warp_wait(bar(B_BE + p1.b), (p1.u & 1) ^ 1, &s_abort)) return false;
      const int a = g1 & 1;
      if (!warp_wait(bar(B_AT_F + a), (g1 >> 1) & 1, &s_abort)) return false;
      tc_fence_after();
      mma_f16_ss_e(tbase + p1.b * H, a ? dsc_at1 : dsc_at0, dsc_phi1, idH, 0u);
      mma_commit_e(bar(B_D1 + p1.b));
      mma_commit_e(bar(B_AT_E + a));
      __syncwarp();
      ++g1;
      p1.next();
      return true;
    };
    auto wait_in = [&]() -> bool {
      if (!warp_wait(bar(B_IN + (n_in & 1)), (n_in >> 1) & 1, &s_abort)) return false;
      ++n_in;
      tc_fence_after();
      return true;
    };
    auto wait_h = [&](int h) -> bool {
      if (!warp_wait(bar(B_HC + h), n_h[h] & 1, &s_abort)) return false;
      ++n_h[h];
      tc_fence_after();
      return true;
    };
    // per-scene folded biases -> the constant-one rows of phi1 and B1 (no MMA
    // reads the previous ones any more)
    auto patch_fold = [&](const float* fold) {
      for (int i = lane; i < 2 * H; i += 32) {
        const int n = i < H ? i : i - H;
        const float cv = fold[i];
        const float hi = bf16_value(cv);
        const uint32_t packed = static_cast<uint32_t>(bf16_bits(hi)) |
                                (static_cast<uint32_t>(bf16_bits(cv - hi)) << 16);
        const uint32_t off = i < H ? L::phi1 + ((H + n) * 8 + 4) * 2 : L::b1 + ((H + n) * 8 + 6) * 2;
        *reinterpret_cast<uint32_t*>(smem + off) = packed;
      }
      fence_proxy_async_smem();
      __syncwarp();
      cur_fold = fold;
    };
    int blk, ns, ntiles;
    if (!warp_wait(bar(B_W), 0, &s_abort)) goto done;
    // test hook: a wait that nothing ends (glassnet_debug_stall_next_render)
    if (prm.stall_ns > 0 && !warp_wait(bar(B_STALLC), 0, &s_abort, prm.stall_ns)) goto done;
    if (!take_block(0, blk, ns, ntiles)) goto done;
    if (blk < total_blocks) {
      patch_fold(s_bs.fold[0]);
      for (int k = 0; k < ns && k < 2; ++k)
        if (!phi1()) goto done;
    }
    for (uint32_t tb = 0; blk < total_blocks; ++tb) {
      for (int k = 0; k < ns; ++k) {
        if (!wait_in()) goto done;
        {
          const uint32_t d = tbase + p2.b * H;
          gemm_t<H, H>(d, tbase + (k & 1 ? AU1c : AU0c), dsc_phi2, idH);
          mma_f16_ss_e(d, dsc_one, dsc_phi2b, idH, 1u);
          mma_commit_e(bar(B_D2 + p2.b));
        }
        __syncwarp();
        p2.next();
        if (k + 2 < ns && !phi1()) goto done;
      }
      // The block's pixel tiles; accumulators X, Y, Z and A operands lo / hi
      // as in the one-stream kernel: rho X <- [max ; mean]; B1 Y <- [g ; r =
      // lo]; B2 X <- y = hi; R1 Y <- y2 = lo; R2 Z <- q = hi.
      const uint32_t X = tbase + p1.b * H;
      const uint32_t Y = tbase + (p1.b == 2 ? 0 : p1.b + 1) * H;
      const uint32_t Z = tbase + (p1.b == 0 ? 2 : p1.b - 1) * H;
      const uint32_t A_LO = tbase + APOOLc, A_HI = tbase + APOOLc + H / 2;
      if (!warp_wait(bar(B_AG_F), n_agf & 1, &s_abort)) goto done;
      ++n_agf;
      for (int pt = 0; pt < ntiles; ++pt, ++n_pt) {
        if constexpr (!Sum) {
          if (!wait_h(0)) goto done;
          gemm_t<H, H>(X, A_LO, dsc_rho, idH);
          if (!wait_h(1)) goto done;
          gemm_t<H, H>(X, A_HI, dsc_rho + 2 * kHalfK, idH, true);
          mma_commit_e(bar(B_DP));
          __syncwarp();
        }
        if (!wait_h(0)) goto done;
        mma_f16_ss_e(Y, pt ? dsc_ag1 : dsc_ag0, dsc_b1, idH, 0u);
        gemm_t<H, H / 2>(Y, A_LO, dsc_b1r, idH, true);
        if (!wait_h(1)) goto done;
        gemm_t<H, H / 2>(Y, A_LO + H / 4, dsc_b1r + kHalfK, idH, true);
        mma_commit_e(bar(B_DP));
        if (pt + 1 == ntiles) mma_commit_e(bar(B_AG_E));  // both G-buffer operands read
        __syncwarp();
        if (!wait_h(0)) goto done;
        gemm_t<H, H / 2>(X, A_HI, dsc_b2, idH);
        if (!wait_h(1)) goto done;
        gemm_t<H, H / 2>(X, A_HI + H / 4, dsc_b2 + kHalfK, idH, true);
        mma_commit_e(bar(B_DP));
        __syncwarp();
        if (!wait_h(0)) goto done;
        gemm_t<H, H / 2>(Y, A_LO, dsc_r1, idH);
        if (!wait_h(1)) goto done;
        gemm_t<H, H / 2>(Y, A_LO + H / 4, dsc_r1 + kHalfK, idH, true);
        mma_commit_e(bar(B_DP));
        __syncwarp();
        if (!wait_h(0) || !wait_h(1)) goto done;
        gemm_t<16, H>(Z, A_HI, dsc_r2, id16);
        mma_commit_e(bar(B_DR2));
        __syncwarp();
      }
      // the next block's first two phi1 right behind R2 (they write X and Y)
      if (!take_block(tb + 1, blk, ns, ntiles)) goto done;
      if (blk < total_blocks) {
        const float* fold = s_bs.fold[(tb + 1) & 1];
        if (fold != cur_fold) {
          // every MMA so far (B1 reads the bias rows) has completed
          if (n_pt > 0 && !warp_wait(bar(B_DR2), (n_pt - 1) & 1, &s_abort)) goto done;
          patch_fold(fold);
        }
        for (int k = 0; k < ns && k < 2; ++k)
          if (!phi1()) goto done;
      }
    }
  } else {
    // ------------------------------------------------------- epilogue warps
    const int q = warp & 3, g = warp >> 2;
    const int row = q * 32 + lane;
    const uint32_t tl = tbase + (static_cast<uint32_t>(q * 32) << 16);
    const float* b_rho = reinterpret_cast<const float*>(smem + L::bias_rho);
    const float* b_b2 = reinterpret_cast<const float*>(smem + L::bias_b2);
    const float* b_r1 = reinterpret_cast<const float*>(smem + L::bias_r1);
    const float* b_r2 = reinterpret_cast<const float*>(smem + L::bias_r2);
    uint32_t gs = 0, n_in = 0, n_dp = 0, n_pt = 0, n_es = 0;
    auto arrive_h = [&](int h) {
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_HC + h));
    };
    auto arrive_in = [&]() {
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_IN + (n_in & 1)));
      ++n_in;
    };
    // every epilogue warp's shared-memory pool accesses so far are visible
    // to all of them (two alternating barriers)
    auto epi_sync = [&]() -> bool {
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_ES + (n_es & 1)));
      const bool ok = warp_wait(bar(B_ES + (n_es & 1)), (n_es >> 1) & 1, &s_abort);
      ++n_es;
      return ok;
    };
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (!warp_wait(bar(B_W), 0, &s_abort)) goto done;
    {
      int blk, ns, ntiles;
      if (!take_block(0, blk, ns, ntiles)) goto done;
      for (uint32_t tb = 0; blk < total_blocks; ++tb) {
        const int bp = tb & 1;
        // phi1(k) accumulator -> U(k) = ReLU as bf16
        auto epi1 = [&](int k) -> bool {
          const uint32_t gk = gs + k, b = gk % 3u;
          if (!warp_wait(bar(B_D1 + b), (gk / 3u) & 1, &s_abort)) return false;
          tc_fence_after();
          const uint32_t src = tl + b * H + g * CHc;
          const uint32_t dst = tl + (k & 1 ? AU1c : AU0c) + g * (CHc / 2);
          uint32_t ra[16], rb[16];
          tmem_ld16_async(src, ra);
          tmem_wait_ld_tied(ra);
#pragma unroll
          for (int hh = 0; hh < CHc / 16; ++hh) {
            uint32_t(&cur)[16] = (hh & 1) ? rb : ra;
            uint32_t(&nxt)[16] = (hh & 1) ? ra : rb;
            if (hh + 1 < CHc / 16) tmem_ld16_async(src + (hh + 1) * 16, nxt);
            uint32_t u[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
              u[i] = pack_bf16_relu(__uint_as_float(cur[2 * i]), __uint_as_float(cur[2 * i + 1]));
            tmem_st8(dst + hh * 8, u);
            if (hh + 1 < CHc / 16) tmem_wait_ld_tied(nxt);
          }
          arrive_in();
          return true;
        };
        // phi2(k) accumulator -> the row's pixel's pool entries
        auto epi2 = [&](int k) -> bool {
          int slot;
          const int e = row_entry(s_bs, bp, k * kTile + row, slot);
          const uint32_t gk = gs + k, b = gk % 3u;
          if (!warp_wait(bar(B_D2 + b), (gk / 3u) & 1, &s_abort)) return false;
          tc_fence_after();
          const uint32_t src = tl + b * H + g * CHc;
          uint32_t ra[16], rb[16];
          tmem_ld16_async(src, ra);
          tmem_wait_ld_tied(ra);
#pragma unroll
          for (int hh = 0; hh < CHc / 16; ++hh) {
            uint32_t(&cur)[16] = (hh & 1) ? rb : ra;
            uint32_t(&nxt)[16] = (hh & 1) ? ra : rb;
            if (hh + 1 < CHc / 16) {
              tmem_ld16_async(src + (hh + 1) * 16, nxt);
            } else {
              // every column of this buffer is in registers: release it
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(bar(B_BE + b));
            }
            if (e >= 0) {
#pragma unroll
              for (int i = 0; i < 16; i += 2) {
                const uint32_t ch = static_cast<uint32_t>(g * CHc + hh * 16 + i);
                const uint32_t u =
                    pack_bf16_relu(__uint_as_float(cur[i]), __uint_as_float(cur[i + 1]));
                const uint32_t a0 = (ch * kBlockPx + static_cast<uint32_t>(e)) * 4u;
                const uint32_t a1 = a0 + kBlockPx * 4u;
                float t0 = kSumBase, t1 = kSumBase;
                add_bf16x2_rz(t0, t1, u);  // 2^11 + u truncated to the quantum
                float d0, d1;
                fadd2_rn(d0, d1, t0, t1, -kSumBase, -kSumBase);  // exact
                if constexpr (!Sum) {
                  // non-negative bf16 (a -0 taken as +0): unsigned order is value order
                  red_max_u32(pmax + a0, u & 0x7fffu);
                  red_max_u32(pmax + a1, (u >> 16) & 0x7fffu);
                }
                red_add_f32(psum + a0, d0);
                red_add_f32(psum + a1, d1);
              }
            }
            if (hh + 1 < CHc / 16) tmem_wait_ld_tied(nxt);
          }
          return true;
        };
        for (int k = -1; k < ns; ++k) {
          if (k + 1 < ns && !epi1(k + 1)) goto done;
          if (k >= 0 && !epi2(k)) goto done;
        }
        gs += ns;
        if (!epi_sync()) goto done;  // every reduction of the block has landed

        const uint32_t r3 = gs % 3u;
        const uint32_t X = tl + r3 * H;
        const uint32_t Y = tl + (r3 == 2 ? 0 : r3 + 1) * H;
        const uint32_t Z = tl + (r3 == 0 ? 2 : r3 - 1) * H;
        const uint32_t A_LO = tl + APOOLc, A_HI = tl + APOOLc + H / 2;
        constexpr int PC = H / 4;  // accumulator columns of this warp per pass (16)
        float* const out = s_bs.out[bp];
        const size_t P = static_cast<size_t>(s_bs.P[bp]);
        const int tile0 = s_bs.tile0[bp];
        for (int pt = 0; pt < ntiles; ++pt, ++n_pt) {
          const uint32_t e = static_cast<uint32_t>(pt * kTile + row);
          const uint32_t ent = __ldg(prm.plan + static_cast<size_t>(tile0 + pt) * kTile + row);
          const int c = ent == kPlanEmpty ? 0 : static_cast<int>(ent >> 28);
          // this thread's pool entries -> rho's A operand (or tau -> B1's r
          // block), each entry reset to its start value
          {
            const float off = kSumBase - static_cast<float>(c) * kHalfQuantum;
            const float rcp = c > 0 ? __frcp_rn(static_cast<float>(c)) : 0.0f;
            bool over = false;
            uint32_t mx[CHc / 2], pa[CHc / 2];
#pragma unroll
            for (int j = 0; j < CHc / 2; ++j) {
              const uint32_t ch = static_cast<uint32_t>(g * CHc + 2 * j);
              const uint32_t a0 = (ch * kBlockPx + e) * 4u, a1 = a0 + kBlockPx * 4u;
              const float s0 = __uint_as_float(lds32(psum + a0));
              const float s1 = __uint_as_float(lds32(psum + a1));
              over |= !(fmaxf(s0, s1) < kSumLimit);
              float v0, v1;
              fadd2_rn(v0, v1, s0, s1, -off, -off);
              pa[j] = Sum ? pack_bf16(v0, v1) : pack_bf16(v0 * rcp, v1 * rcp);
              sts32(psum + a0, __float_as_uint(kSumBase));
              sts32(psum + a1, __float_as_uint(kSumBase));
              if constexpr (!Sum) {
                mx[j] = lds32(pmax + a0) | (lds32(pmax + a1) << 16);
                sts32(pmax + a0, 0u);
                sts32(pmax + a1, 0u);
              }
            }
            if (over && c > 0) atomicOr(prm.err, kErrRange);
            if constexpr (Sum) {
              // tau -> lo; B1 reads it in K halves, this warp's channels are half g
              if (g == 1) arrive_h(0);
#pragma unroll
              for (int hh = 0; hh < CHc / 16; ++hh) {
                uint32_t w8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) w8[i] = pa[hh * 8 + i];
                tmem_st8(A_LO + g * (CHc / 2) + hh * 8, w8);
              }
              if (g == 0) arrive_h(0);
              arrive_h(1);
            } else {
#pragma unroll
              for (int hh = 0; hh < CHc / 16; ++hh) {
                uint32_t w8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) w8[i] = mx[hh * 8 + i];
                tmem_st8(A_LO + g * (CHc / 2) + hh * 8, w8);
              }
              arrive_h(0);
#pragma unroll
              for (int hh = 0; hh < CHc / 16; ++hh) {
                uint32_t w8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) w8[i] = pa[hh * 8 + i];
                tmem_st8(A_HI + g * (CHc / 2) + hh * 8, w8);
              }
              arrive_h(1);
            }
          }
          // rho -> r (zero without layers) -> lo;  B1 -> y -> hi;
          // B2 -> y2 -> lo;  R1 -> q -> hi; two passes of 16 columns each
#pragma unroll
          for (int l = Sum ? 1 : 0; l < 4; ++l) {
            if (!warp_wait(bar(B_DP), n_dp & 1, &s_abort)) goto done;
            ++n_dp;
            tc_fence_after();
            const float* bl = l == 0 ? b_rho : (l == 2 ? b_b2 : b_r1);
            const uint32_t acc = (l & 1) ? Y : X;
            const uint32_t dst = (l & 1) ? A_HI : A_LO;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int c0 = h * (H / 2) + g * PC;
              uint32_t ra[16];
              tmem_ld16_async(acc + c0, ra);
              tmem_wait_ld_tied(ra);
              uint32_t u[8];
              if (l == 1) {  // B1's bias is folded into its GEMM
#pragma unroll
                for (int i = 0; i < 8; ++i)
                  u[i] = pack_bf16_relu(__uint_as_float(ra[2 * i]), __uint_as_float(ra[2 * i + 1]));
              } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  float v0, v1;
                  fadd2_rn(v0, v1, __uint_as_float(ra[2 * i]), __uint_as_float(ra[2 * i + 1]),
                           bl[c0 + 2 * i], bl[c0 + 2 * i + 1]);
                  u[i] = (l == 0 && c == 0) ? 0u : pack_bf16_relu(v0, v1);
                }
              }
              tmem_st8(dst + c0 / 2, u);
              arrive_h(h);
            }
          }
          // R2 + sigmoid -> out (column group 0 stores); every warp waits for
          // R2 before the next pool conversion overwrites lo
          if (!warp_wait(bar(B_DR2), n_pt & 1, &s_abort)) goto done;
          if (g == 0) {
            tc_fence_after();
            uint32_t r[4];
            tmem_ld4(Z, r);
            if (ent != kPlanEmpty) {
              const uint32_t pix = ent & kPlanPixelMask;
#pragma unroll
              for (int j = 0; j < kOut; ++j) {
                const float yv = __uint_as_float(r[j]) + b_r2[j];
                out[j * P + pix] = 1.0f / (1.0f + expf(-yv));
              }
            }
          }
        }
        if (!epi_sync()) goto done;  // the reset entries before the next block's reductions
        if (!take_block(tb + 1, blk, ns, ntiles)) goto done;
      }
    }
  }
done:
  tc_fence_before();
  __syncthreads();  // every warp is here: s_abort is final
  if (s_abort) {
    if (warp == kMmaC) drain_async(bar(B_W), bar(B_DRAINC));
    if (tid == 0) report_timeout(prm.err, s_abort, bar_base, kKernelCompact, 0);
  }
  if (warp == kMmaC) {
    tc_fence_after();
    tmem_dealloc(tbase, NCOLSc);
  }
}

template <bool Sum>
cudaError_t prepare_c() {
  static bool done = false;  // per process: the attribute holds for every later launch
  if (done) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fused_compact_kernel<Sum>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(CS::bytes));
  if (e == cudaSuccess) done = true;
  return e;
}

template <bool Sum>
cudaError_t launch_c(const void* wimg, const FusedParams& p, cudaStream_t s) {
  cudaError_t e = prepare_c<Sum>();
  if (e != cudaSuccess) return e;
  const int blocks = 2 * p.total_windows;
  const int sms = device_sm_count();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks < sms ? blocks : sms);
  cfg.blockDim = dim3(kThreadsC);
  cfg.dynamicSmemBytes = CS::bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fused_compact_kernel<Sum>, p, static_cast<const uint8_t*>(wimg));
}

}  // namespace

cudaError_t prepare_fused_compact() {
  device_sm_count();
  const cudaError_t e = prepare_c<false>();
  return e == cudaSuccess ? prepare_c<true>() : e;
}

cudaError_t launch_fused_compact(const void* wimg, const FusedParams& params, cudaStream_t s) {
  if (params.total_tiles <= 0) return cudaSuccess;
  FusedParams p = params;
  p.plan_identity = 1;  // blocks are pixel tiles in pixel order
  cudaError_t e = launch_plan(p, s);
  if (e != cudaSuccess) return e;
  if (p.win_tiles != 2 * kBlockTiles) return cudaErrorInvalidValue;  // blocks are half windows
  return p.pool_sum ? launch_c<true>(wimg, p, s) : launch_c<false>(wimg, p, s);
}

}  // namespace gn

// Fused GlassNet forward pass on sm_103a: a count-sorting plan kernel, then
// one persistent kernel over 128-pixel tiles in which every layer is a
// tcgen05 BF16 GEMM with FP32 accumulators in TMEM.
//
// Per tile (Sec. 3.3-3.4, Eq. 5), with the scene latent folded into per-scene
// biases (c_phi, c_B) that enter the GEMMs through two constant-one input
// columns (a hi/lo BF16 split of each bias, so the fold keeps ~16 bits):
//   for each layer slot k < max count in the tile:
//     U   = ReLU([t_k, 1, 1, 0, 0] W_phi1'^T)            (K = 16)
//     V   = [U, 1, 1, 0..] [W_phi2, b_phi2 hi, lo]^T     (K = H + 16)
//     u   = bf16(ReLU(V));  max = max(max, u);  sum += u   for pixels with k < c_p
//   pool  = [max ; mean], mean = sum / c_p               (exact, see below)
//   r     = ReLU(pool W_rho^T + b_rho), r = 0 if c_p = 0
//   y     = ReLU([g, 1, 1, r] W_B1'^T)                   (K = 16 + H)
//   y2    = ReLU(y W_B2^T + b_B2);  q = ReLU(y2 W_R1^T + b_R1)
//   rgb   = sigmoid(q W_R2^T + b_R2)                     (N padded to 16)
//
// Tile plan and schedule.  Eq. 5 pools over each pixel's own layers, so a
// tile must run as many layer slots as its largest count.  The plan kernel
// sorts the pixels of every window of 4 tiles (512 pixels) by layer count,
// largest first (stable in pixel index), so the tiles of a window hold pixels
// of similar counts and the slots run per tile come closer to the mean count.
// A pixel's result does not depend on its tile or row, so the order changes
// nothing but the work.  Tiles are handed out dynamically (a global counter),
// in plan order: tiles of very different cost then balance over the CTAs, and
// the tiles of one window, which gather from the same 512-pixel stretch of
// every plane, run at about the same time.  Small windows trade some
// compaction for gathers that stay within fewer cache lines (measured at 512^2,
// K = 8, Poisson(3) counts: 4 tiles beat 8, 16 and 32).
//
// Exact, order-independent set pooling: each valid layer contributes
// u = bf16(ReLU(V)); the running max starts at 0 (which is also the ReLU) and
// is kept as bf16 pairs; the sum is a fixed-point accumulator held in an FP32
// significand: s starts at 2^11 and every addition of u (exact in FP32) is
// rounded toward zero, so while s < 2^12 each add contributes exactly
// floor(u / 2^-12) quanta, whatever the order of the layers.
// mean = (s - 2^11 + c 2^-13) * (1/c) (the c 2^-13 term centres the
// truncation).  A pixel whose sum reaches 2^12 sets the range error bit.
// Hence the output is bit-identical under any permutation of a pixel's valid
// layers.  The adds use the mixed-precision add.rz.f32.bf16 (FMA pipe), the
// max uses max.bf16x2 on the pair that the ReLU conversion produced.
//
// Warp roles (11 warps, at most three per SM sub-partition, 168 registers):
//  - warps 0-7 (epilogue): warp w serves TMEM lane quadrant q = w % 4 (pixel
//    rows 32q..32q+31) and accumulator columns [g H/2, (g+1) H/2), g = w / 4.
//    They run every epilogue (ReLU, pooling, biases, sigmoid) and hold the
//    pool state (H/2 sums and H/4 packed maxima per thread) in registers.
//  - warp 8 (MMA): allocates TMEM, patches the per-scene bias rows, issues
//    every tcgen05.mma (one elected lane of the converged warp).
//  - warps 9-10 (loaders, 64 pixel rows each): read each tile's plan entries,
//    gather its G-buffer and layers, convert them to BF16 and write the
//    shared-memory A operands, running up to two layer slots ahead.  With
//    positional encoding at H = 64 there are four loader warps (9-12, 32
//    rows each) that also compute the encoded bands (13 warps); at H = 128
//    the two loader warps encode, and warp 11 fills the ring through which
//    the per-pixel weights stream (12 warps, FusedLayout<128, true>).
// The base widths without encoding (H = 64) run one epilogue warp per lane
// quadrant instead (warps 0-3, all H columns; MMA warp 4; loaders 5-6), at
// two CTAs per SM (128 registers a thread).
//
// Layer-slot pipeline.  Three TMEM accumulator buffers rotate over the global
// sequence of layer slots: phi1(k) writes buffer k mod 3, the epilogue turns
// it into U(k) (TMEM, double buffered), then phi2(k) overwrites the same
// buffer.  The MMA warp issues phi1 two slots ahead of phi2, so the tensor
// pipe always holds the next phi1 while the epilogue works:
//   tensor pipe:  phi2(k-1) phi1(k+1) phi2(k) phi1(k+2) ...
//   epilogue:     epi1(k+1) epi2(k) epi1(k+2) epi2(k+1) ...
// Hand-offs are mbarriers: the MMA warp commits accumulators and consumed
// operands (tcgen05.commit); the epilogue warps arrive once per warp when an
// A operand is written (two alternating barriers, so a warp that runs ahead
// cannot complete the phase of a slower one) or an accumulator has been read;
// the loaders arrive when an operand is filled.  After the last slot the
// per-pixel layers reuse the three buffers; the next tile's first two phi1
// are issued right behind R2.  The MMA and epilogue warps take the next
// tile's slot count and frame (which the loaders publish in shared memory,
// four tiles deep) while the per-pixel layers run, and the epilogue loads
// each row's plan entry for the store before them, so little but the R2
// epilogue separates two tiles.  Every device-side wait gives up after 1 s,
// sets the timeout error bit and makes all warps leave through the common
// exit.
#include <cuda_bf16.h>

#include "fused_common.cuh"

namespace gn {
namespace {
using namespace fused;

// Per-pixel layers: the epilogue writes each layer's output A operand in two
// halves of K, arriving on one barrier per half, so the next layer's MMAs
// over the first half run while the second half is produced.
constexpr int B_H = B_COUNT;  // + half: K half of the next per-pixel A operand written
constexpr int B_STALL = B_COUNT + 2;  // never arrived on: the stall that tests the timeout path
constexpr int B_DRAIN = B_COUNT + 3;  // the exit path's last commit
// Streamed per-pixel weights (doubled widths with encoding): + stage (2).
constexpr int B_WF = B_COUNT + 4;  // ring stage filled (transaction count)
constexpr int B_WE = B_COUNT + 6;  // ring stage read by its MMAs (commit)
constexpr int B_COUNT_B = B_COUNT + 8;

// TMEM column map (128 lanes x 4H columns of 32 bits): three accumulator
// buffers of H columns, then U (H bf16 = H/2 columns) double buffered.  The
// per-pixel layers of a tile use, with r = (first global slot of the next
// tile) mod 3:  X = buffer r (their accumulator), Y = buffer r + 1 (r, then y
// and q), Z = buffer r + 2 (y2, and R2's accumulator), and the U region for
// the pooled [max ; mean].  The next tile's phi1 for its first two slots
// write X and Y, issued after R2 (which reads Y); Z is written again only
// after every epilogue warp has read R2.
template <int H>
struct TMap {
  static constexpr uint32_t AU0 = 3 * H;
  static constexpr uint32_t AU1 = 3 * H + H / 2;
  static constexpr uint32_t APOOL = AU0;  // rho A: [max ; mean] (H columns)
  static constexpr uint32_t NCOLS = 4 * H;
  static __device__ __forceinline__ uint32_t buf(uint32_t b) { return b * H; }
  static_assert(NCOLS == 256 || NCOLS == 512, "TMEM allocation must be a power of two");
};

// D (+)= A (TMEM, K/2 columns from a_tmem) x B^T, B stored [K/8][N][8] bf16
// and described by `d0` (its K = 0 column).  Each K step of 16 advances the
// start address by two core-matrix columns (2 N 16 bytes), i.e. (2 N 16) >> 4
// in the descriptor's 14-bit address field (shared-memory addresses stay
// < 256 KB, so the field never carries into the next one).  Issued by the
// whole warp (one elected lane), eight K steps per statement.
template <int N, int K>
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, uint32_t a_tmem, uint64_t d0,
                                           uint32_t idesc, bool accumulate = false) {
  constexpr uint32_t step = (2 * N * 16) >> 4;
  if constexpr (K % 128 == 0) {
#pragma unroll
    for (int kb = 0; kb < K / 128; ++kb)
      mma8_f16_ts_e<step>(d_tmem, a_tmem + kb * 64, d0 + static_cast<uint64_t>(8 * step) * kb,
                          idesc, (kb > 0 || accumulate) ? 1u : 0u);
  } else {
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks)
      mma_f16_ts_e(d_tmem, a_tmem + ks * 8, d0 + static_cast<uint64_t>(step) * ks, idesc,
                   (ks > 0 || accumulate) ? 1u : 0u);
  }
}

// Layer k of the lane's rows: 12 channels each, zeros where the slot is not
// valid.  Element offsets fit in 32 bits: the host requires 12 K h w < 2^31.
template <int RPL>
__device__ __forceinline__ void load_slot(const FusedFrame& F, int k, const uint32_t (&pix)[RPL],
                                          const int (&cnt)[RPL], float (&x)[RPL][kTC]) {
  const uint32_t P = static_cast<uint32_t>(F.P);
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const bool v = k < cnt[i];
    const uint32_t o = static_cast<uint32_t>(k) * kTC * P + pix[i];
#pragma unroll
    for (int ch = 0; ch < kTC; ++ch) x[i][ch] = v ? __ldg(F.tbuf + (o + ch * P)) : 0.0f;
  }
}

// Writes rows row0 + 32 i of a [2][128][8] bf16 operand: K entries 0..11 from
// x, then the constant-one columns [1, 1, 0, 0].
template <int RPL>
__device__ __forceinline__ void store_slot(uint32_t base, int row0, const float (&x)[RPL][kTC]) {
  const uint32_t one = pack_bf16(1.0f, 1.0f);
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const uint32_t r = base + static_cast<uint32_t>(row0 + 32 * i) * 16u;
    sts128(r, pack_bf16(x[i][0], x[i][1]), pack_bf16(x[i][2], x[i][3]), pack_bf16(x[i][4], x[i][5]),
           pack_bf16(x[i][6], x[i][7]));
    sts128(r + 2048u, pack_bf16(x[i][8], x[i][9]), pack_bf16(x[i][10], x[i][11]), one, 0u);
  }
}

// One 16-byte chunk (8 K values, one core-matrix column of one row) holding
// N <= 8 values and zeros.
template <int N>
__device__ __forceinline__ void sts_chunk(uint32_t a, const float (&v)[N]) {
  uint32_t q[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) q[j] = 2 * j < N ? pack_bf16(v[2 * j], v[2 * j + 1 < N ? 2 * j + 1 : 2 * j]) : 0u;
  if constexpr (N % 2 == 1) q[N / 2] = pack_bf16(v[N - 1], 0.0f);
  sts128(a, q[0], q[1], q[2], q[3]);
}
// Bands 1 .. 2 nf of N consecutive channels whose band-0 chunk is at `a`:
// band t is 16 K columns (4096 bytes of a [K/8][128][8] operand) further on.
template <int N>
__device__ __forceinline__ void pe_chunks(uint32_t a, const float (&v)[N], int nf) {
  float sn[N], cs[N];
  pe_first(v, sn, cs);
  for (int f = 0; f < nf; ++f) {
    if (f > 0) pe_double(sn, cs);
    sts_chunk(a + static_cast<uint32_t>(2 * f + 1) * 4096u, sn);
    sts_chunk(a + static_cast<uint32_t>(2 * f + 2) * 4096u, cs);
  }
}

// Encoded layer operand: band 0 as store_slot writes it (channels 0-7, then
// 8-11 and the constant-one pair), then the nf frequencies' sine and cosine
// bands, one core-matrix column of channels at a time.  The encoding's code
// is kept small, so that the loaders do not evict the epilogue's loops from
// the instruction cache (the same code unrolled over two rows per lane
// measured 40 % slower at H = 64): one row per lane there, with four loader
// warps, one per SM sub-partition, sharing the encoding work; with two rows
// per lane (the doubled widths) a loop over the rows, each row's values
// picked by selects (an indexed register array would go to local memory).
template <int RPL>
__device__ __forceinline__ void store_slot_pe(uint32_t base, int row0, const float (&x)[RPL][kTC],
                                              int nf) {
  static_assert(RPL == 1 || RPL == 2, "one or two rows per loader lane with encoding");
  const uint32_t one = pack_bf16(1.0f, 1.0f);
#pragma unroll 1
  for (int i = 0; i < RPL; ++i) {
    const uint32_t r = base + static_cast<uint32_t>(row0 + 32 * i) * 16u;
    float lo[8], hi[4];
#pragma unroll
    for (int j = 0; j < 8; ++j) lo[j] = i == 0 ? x[0][j] : x[RPL - 1][j];
#pragma unroll
    for (int j = 0; j < 4; ++j) hi[j] = i == 0 ? x[0][8 + j] : x[RPL - 1][8 + j];
    sts_chunk(r, lo);
    sts128(r + 2048u, pack_bf16(hi[0], hi[1]), pack_bf16(hi[2], hi[3]), one, 0u);
    pe_chunks(r, lo, nf);
    pe_chunks(r + 2048u, hi, nf);
  }
}

// Launch modes: a whole frame (plan sorted by count, every layer slot, the
// per-pixel layers), one streamed layer accumulated into a pool state in
// device memory (one slot per tile, no per-pixel layers), or the per-pixel
// layers of a pool state (no slots).  The arithmetic of each step is the same
// code in all three, so a streamed frame resolves to the same bits.
enum : int { kModeFrame = 0, kModeAccumulate = 1, kModeResolve = 2 };

// Warp counts: 2 loader warps (2 rows per lane), or 4 (1 row per lane) when
// the loaders also encode the inputs.  The base widths (H = 64, no
// encoding) run one epilogue warp per TMEM lane quadrant (7 warps) and two
// CTAs per SM: each CTA holds 74 KB of shared memory and 256 TMEM columns,
// and the SM interleaves two tiles' hand-off chains.
//
// The doubled widths with encoding stream their per-pixel weights (kStream,
// FusedLayout<128, true>): two loader warps that also encode (two rows per
// lane), and one more warp that fills the weight ring (12 warps, three per
// SM sub-partition, as the pool state of two epilogue warps per lane
// quadrant needs).
template <int H, bool PE>
struct Roles {
  static constexpr bool kPair = H == 64 && !PE;
  static constexpr bool kStream = FusedLayout<H, PE>::kStream;
  static constexpr int EW = kPair ? 1 : kEW;  // epilogue warps per lane quadrant
  static constexpr int EPI = 4 * EW;          // epilogue warps 0 .. EPI - 1
  static constexpr int MMA = 4 * EW;          // the MMA warp
  static constexpr int LOAD0 = 4 * EW + 1;    // the first loader warp
  static constexpr int LW = PE && !kStream ? 4 : kLoadWarps;
  static constexpr int PROD = kStream ? LOAD0 + LW : -1;  // the weight-ring warp
  static constexpr int RPL = kTile / (LW * 32);
  static constexpr int kThreads = (4 * EW + 1 + LW + (kStream ? 1 : 0)) * 32;
  static constexpr int kCtasPerSm = kPair ? 2 : 1;
  static_assert(LW <= kMaxLoadWarps && RPL * LW * 32 == kTile, "loader rows must cover the tile");
};

// Loader warps: per tile, read the plan entries of their rows and publish the
// slot count, then fill the layer operands slot by slot (two buffers, released
// by the phi1 MMAs that read them) and B1's G-buffer operand (released by B1
// of the previous tile).
template <int H, int Mode, bool PE>
__device__ __forceinline__ void loader_loop(const FusedParams& prm, uint32_t sbase,
                                            uint32_t bar_base, LoaderShared& ls,
                                            volatile int* abort_flag, int li, int lane) {
  using L = FusedLayout<H, PE>;
  constexpr int RPL = Roles<H, PE>::RPL, LW = Roles<H, PE>::LW;
  constexpr bool kOol = true;  // the waits' polling loop out of line (warp_wait)
  const int nf = PE ? prm.pe_freqs : 0;  // positional-encoding frequencies
  auto bar = [&](int i) { return bar_base + static_cast<uint32_t>(i) * 8u; };
  const int row0 = li * (32 * RPL) + lane;
  uint32_t lc = 0, n_ag = 0;
  for (uint32_t tb = 0;; ++tb) {
    // Dynamic schedule: loader warp 0 takes the next tile from the global
    // counter (which the plan kernel zeroed) and hands it to loader warp 1;
    // an index past the last tile ends every role's loop.
    int tile;
    if (li == 0) {
      if (lane == 0) ls.tile[tb & 1] = schedule_tile(prm, atomicAdd(prm.next_tile, 1u));
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_SCHED + (tb & 1)));
    } else if (!warp_wait<kOol>(bar(B_SCHED + (tb & 1)), (tb >> 1) & 1, abort_flag)) {
      return;
    }
    tile = *reinterpret_cast<volatile int*>(&ls.tile[tb & 1]);
    if (tile >= prm.total_tiles) {
      if (lane == 0) {
        ls.ns[tb & 1][li] = 0;
        mbar_arrive(bar(B_TILE + (tb & 1)));
      }
      return;
    }
    const FusedFrame& F = frame_of(prm, tile);
    const uint32_t* ent = prm.plan + static_cast<size_t>(tile) * kTile;
    uint32_t pix[RPL];
    int cnt[RPL];
    bool has[RPL];
    int cmax = 0;
#pragma unroll
    for (int i = 0; i < RPL; ++i) {
      const uint32_t e = __ldg(ent + row0 + 32 * i);
      has[i] = e != kPlanEmpty;
      pix[i] = has[i] ? (e & kPlanPixelMask) : 0u;
      cnt[i] = has[i] ? static_cast<int>(e >> 28) : 0;
      cmax = max(cmax, cnt[i]);
      ls.cnt[tb & 1][row0 + 32 * i] = static_cast<uint8_t>(cnt[i]);
    }
    const int wmax = __reduce_max_sync(0xffffffffu, cmax);
    if (lane == 0) {
      ls.ns[tb & 1][li] = Mode == kModeResolve ? 0 : wmax;  // resolve: no layer slots
      if (li == 0) {
        ls.out[tb & 3] = F.out;
        ls.fold[tb & 3] = F.fold;
        ls.P[tb & 3] = F.P;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(bar(B_TILE + (tb & 1)));
    // the tile's slot count is the max over both loader warps
    if (!warp_wait<kOol>(bar(B_TILE + (tb & 1)), (tb >> 1) & 1, abort_flag)) return;
    int ns = 0;
#pragma unroll
    for (int w = 0; w < LW; ++w) ns = max(ns, ls.ns[tb & 1][w]);
    if (Mode == kModeResolve || (Mode == kModeAccumulate && ns > 0 && !prm.pool_fresh)) {
      // Streaming launches: the pool state of this warp's rows (row0 + 32 i:
      // 32 consecutive pixels, one 128-byte line in each of the tile's H/2 + H
      // planes) into L2 ahead of the epilogue's loads, for the lines that
      // hold a pixel whose state is read.
      const uint32_t* blk =
          prm.pool_st + static_cast<size_t>(tile - F.tile0) * ((H / 2 + H) * kTile) + li * (32 * RPL);
#pragma unroll
      for (int i = 0; i < RPL; ++i) {
        if (!__any_sync(0xffffffffu, has[i] && cnt[i] > 0)) continue;
        for (int pl = lane; pl < H / 2 + H; pl += 32)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(blk + pl * kTile + 32 * i));
      }
    }

    // G-buffer block [g0..g13, 1, 1] of the lane's rows, loads in flight now
    // (accumulate launches run no B1)
    float gv[RPL][kGC] = {};
    auto load_g = [&]() {
      const uint32_t P = static_cast<uint32_t>(F.P);
#pragma unroll
      for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int ch = 0; ch < kGC; ++ch)
          gv[i][ch] = has[i] ? __ldg(F.gbuf + (static_cast<uint32_t>(ch) * P + pix[i])) : 0.0f;
    };
    if constexpr (Mode != kModeAccumulate) load_g();
    // The operand's release (B_AG_E) also paces the loaders: they are at most
    // one tile ahead, as the two tile-publication barriers need.  Accumulate
    // launches run no B1 and write no operand: the loaders still arrive on
    // B_AG_F once per tile after their wait, and the MMA warp waits for that
    // arrival before it commits B_AG_E for the tile.  Each commit then follows
    // the loaders' wait for the previous one, so B_AG_E never completes two
    // phases ahead of the loaders' parity wait (without the arrival a tile
    // with no covered pixel let the MMA warp commit two tiles in a row before
    // the loaders looked, and their wait then missed the phase).
    auto put_ag = [&]() -> bool {
      if (!warp_wait<kOol>(bar(B_AG_E), (n_ag & 1) ^ 1, abort_flag)) return false;
      ++n_ag;
      if constexpr (Mode == kModeAccumulate) {
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_AG_F));
        return true;
      }
      const uint32_t one = pack_bf16(1.0f, 1.0f);
      if constexpr (PE) {
        // a loop over the rows, each row's values picked by selects, as in
        // store_slot_pe: one copy of the encoding code
        static_assert(RPL == 1 || RPL == 2, "one or two rows per loader lane with encoding");
#pragma unroll 1
        for (int i = 0; i < RPL; ++i) {
          const uint32_t r = sbase + L::ag + static_cast<uint32_t>(row0 + 32 * i) * 16u;
          float g[kGC];
#pragma unroll
          for (int c = 0; c < kGC; ++c) g[c] = i == 0 ? gv[0][c] : gv[RPL - 1][c];
          sts128(r, pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]),
                 pack_bf16(g[6], g[7]));
          sts128(r + 2048u, pack_bf16(g[8], g[9]), pack_bf16(g[10], g[11]),
                 pack_bf16(g[12], g[13]), one);
          const float lo[8] = {g[0], g[1], g[2], g[3], g[4], g[5], g[6], g[7]};
          const float hi[6] = {g[8], g[9], g[10], g[11], g[12], g[13]};
          pe_chunks(r, lo, nf);
          pe_chunks(r + 2048u, hi, nf);
        }
      } else {
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          const uint32_t r = sbase + L::ag + static_cast<uint32_t>(row0 + 32 * i) * 16u;
          const float (&g)[kGC] = gv[i];
          sts128(r, pack_bf16(g[0], g[1]), pack_bf16(g[2], g[3]), pack_bf16(g[4], g[5]),
                 pack_bf16(g[6], g[7]));
          sts128(r + 2048u, pack_bf16(g[8], g[9]), pack_bf16(g[10], g[11]),
                 pack_bf16(g[12], g[13]), one);
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_AG_F));
      return true;
    };

    float x[RPL][kTC], y[RPL][kTC];
    if (ns > 0) load_slot(F, 0, pix, cnt, x);
    const int ag_after = min(ns, 2) - 1;  // B1's operand after the first slots
    if (ag_after < 0 && !put_ag()) return;
    for (int k = 0; k < ns; ++k, ++lc) {
      if (k + 1 < ns) load_slot(F, k + 1, pix, cnt, y);
      const int b = lc & 1;
      if (!warp_wait<kOol>(bar(B_AT_E + b), ((lc >> 1) & 1) ^ 1, abort_flag)) return;
      if constexpr (PE)
        store_slot_pe(sbase + (b ? L::at1 : L::at0), row0, x, nf);
      else
        store_slot(sbase + (b ? L::at1 : L::at0), row0, x);
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_AT_F + b));
      if (k == ag_after && !put_ag()) return;
#pragma unroll
      for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int ch = 0; ch < kTC; ++ch) x[i][ch] = y[i][ch];
    }
  }
}

// Ring stage s of the streamed per-pixel weights (FusedLayout<128, true>).
template <class L>
__device__ __forceinline__ uint32_t ring_stage(int s) {
  if constexpr (L::kStream) return s ? L::ring1 : L::ring0;
  else return 0;
}

// Weight-ring warp of the streamed layout: per tile, the per-pixel weight
// chunks in the order the MMA warp consumes them (rho's four K = 64 chunks
// unless Sum; B1's G-buffer bands 1.. (four bands a chunk) and its two r
// chunks; B2's two; R1's two and R2 unless R3), each into the next of the two
// stages once the MMAs that read that stage's previous chunk have completed.
// It follows the tiles the loaders publish and ends with the last; every
// copy it issued has landed before it leaves, so none is in flight when the
// CTA exits.
template <int H, bool Sum, bool R3>
__device__ __forceinline__ void ring_loop(const FusedParams& prm, const uint8_t* wimg,
                                          uint32_t sbase, uint32_t bar_base, LoaderShared& ls,
                                          volatile int* abort_flag, int lane) {
  using L = FusedLayout<H, true>;
  auto bar = [&](int i) { return bar_base + static_cast<uint32_t>(i) * 8u; };
  const int nb = 1 + 2 * prm.pe_freqs;
  uint32_t n = 0, last[2] = {0, 0};
  bool used[2] = {false, false};
  auto fill = [&](uint32_t off, uint32_t bytes) -> bool {
    const uint32_t st = n & 1;
    if (!warp_wait(bar(B_WE + st), ((n >> 1) & 1) ^ 1, abort_flag)) return false;
    if (lane == 0) {
      mbar_arrive_expect_tx(bar(B_WF + st), bytes);
      bulk_g2s(sbase + ring_stage<L>(st), wimg + off, bytes, bar(B_WF + st));
    }
    __syncwarp();
    last[st] = n;
    used[st] = true;
    ++n;
    return true;
  };
  bool ok = true;
  for (uint32_t tb = 0; ok; ++tb) {
    if (!warp_wait(bar(B_TILE + (tb & 1)), (tb >> 1) & 1, abort_flag)) break;
    if (*reinterpret_cast<volatile int*>(&ls.tile[tb & 1]) >= prm.total_tiles) break;
    if constexpr (!Sum)
      for (uint32_t q = 0; ok && q < 4; ++q) ok = fill(L::img_rho + q * L::kChunk, L::kChunk);
    for (int t0 = 1; ok && t0 < nb; t0 += 4)
      ok = fill(L::img_b1g + static_cast<uint32_t>((t0 - 1) / 4) * L::kChunk,
                static_cast<uint32_t>(min(4, nb - t0)) * 4096u);
    for (uint32_t q = 0; ok && q < 2; ++q) ok = fill(L::img_b1r + q * L::kChunk, L::kChunk);
    for (uint32_t q = 0; ok && q < 2; ++q) ok = fill(L::img_b2 + q * L::kChunk, L::kChunk);
    if constexpr (!R3) {
      for (uint32_t q = 0; ok && q < 2; ++q) ok = fill(L::img_r1 + q * L::kChunk, L::kChunk);
      if (ok) ok = fill(L::img_r2, H * L::NR2 * 2);
    }
  }
  for (int st = 0; st < 2; ++st)
    if (used[st]) mbar_wait(bar(B_WF + st), (last[st] >> 1) & 1, kWaitNs);
  __syncwarp();
}

// ------------------------------------------------------------------ kernel
// Sum: the paper's own form of Eq. 5, tau = sum of the valid layers' phi
// outputs entering B1 directly (no rho).  tau is the same fixed-point sum as
// the mean's, tau = s - 2^11 + c 2^-13 (0 without layers), so it is
// bit-identical under any order of the layers; the max is not kept.
// PE: the inputs are positionally encoded (H = 64 layout, 1 + 2 pe_freqs
// bands of 16 K columns in phi1's and B1's first operands).
// R3: R's first layer is a 3x3 kernel over the frame (conv_r3.cu): the tile
// ends after B2 and writes the neural buffer y (BF16, layout
// [y][H/8][x][8], one buffer per frame of the launch) to device memory
// instead of running R.
template <int H, int Mode, bool Sum, bool PE, bool R3>
__global__ void __launch_bounds__(Roles<H, PE>::kThreads, Roles<H, PE>::kCtasPerSm)
    fused_bf16_kernel(const __grid_constant__ FusedParams prm, const uint8_t* __restrict__ wimg) {
  static_assert(!Sum || Mode != kModeAccumulate, "accumulation does not depend on the pooling");
  static_assert(!R3 || Mode != kModeAccumulate, "accumulation does not depend on R");
  using L = FusedLayout<H, PE>;
  using T = TMap<H>;
  using R = Roles<H, PE>;
  // the epilogue waits' polling loop out of line (warp_wait); the MMA warp's
  // always
  constexpr bool kOol = R::kPair || PE;
  constexpr int kEW = R::EW;  // epilogue warps per lane quadrant
  constexpr int CH = H / kEW;  // accumulator columns per epilogue thread
  constexpr int CHC = CH / 2;  // TMEM columns of CH bf16 values
  static_assert(CH % 16 == 0, "accumulator columns per thread must be a multiple of 16");

  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[B_COUNT_B];
  __shared__ uint32_t s_tmem;
  __shared__ LoaderShared s_ld;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar_base = smem_u32(&bars[0]);
  auto bar = [&](int i) { return bar_base + static_cast<uint32_t>(i) * 8u; };

  if (tid == 0) {
    mbar_init(bar(B_W), 1);
    mbar_init(bar(B_DP), 1);
    mbar_init(bar(B_DR2), 1);
    mbar_init(bar(B_STALL), 1);
    mbar_init(bar(B_DRAIN), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(B_WF + b), 1);
      mbar_init(bar(B_WE + b), 1);
    }
    mbar_init(bar(B_AG_F), Roles<H, PE>::LW);
    mbar_init(bar(B_AG_E), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(B_IN + b), R::EPI);
      mbar_init(bar(B_AT_F + b), Roles<H, PE>::LW);
      mbar_init(bar(B_AT_E + b), 1);
      mbar_init(bar(B_TILE + b), Roles<H, PE>::LW);
      mbar_init(bar(B_SCHED + b), 1);
      mbar_init(bar(B_H + b), R::EPI);
    }
    for (int b = 0; b < 3; ++b) {
      mbar_init(bar(B_D1 + b), 1);
      mbar_init(bar(B_D2 + b), 1);
      mbar_init(bar(B_BE + b), R::EPI);
    }
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == R::MMA) {
    tmem_alloc(smem_u32(&s_tmem), T::NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = s_tmem;

  if (warp >= R::LOAD0 && warp < R::LOAD0 + R::LW) {
    // the constant [1, 1, 0, ...] operand that multiplies phi2's bias rows
    for (int r = (warp - R::LOAD0) * 32 + lane; r < kTile; r += Roles<H, PE>::LW * 32) {
      sts128(sbase + L::aone + r * 16u, pack_bf16(1.0f, 1.0f), 0u, 0u, 0u);
      sts128(sbase + L::aone + 2048u + r * 16u, 0u, 0u, 0u, 0u);
    }
    fence_proxy_async_smem();
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the tile plan is complete
    loader_loop<H, Mode, PE>(prm, sbase, bar_base, s_ld, &s_abort, warp - R::LOAD0, lane);
  } else if (R::kStream && warp == R::PROD) {
    // ------------------------------------------------------ weight-ring warp
    if constexpr (R::kStream && Mode != kModeAccumulate)
      ring_loop<H, Sum, R3>(prm, wimg, sbase, bar_base, s_ld, &s_abort, lane);
  } else if (warp == R::MMA) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      mbar_arrive_expect_tx(bar(B_W), L::bytes);
      for (uint32_t off = 0; off < L::bytes; off += 32768u) {
        const uint32_t n = L::bytes - off < 32768u ? L::bytes - off : 32768u;
        bulk_g2s(sbase + off, wimg + off, n, bar(B_W));
      }
    }
    __syncwarp();
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the tile plan is complete
    constexpr uint32_t idH = make_idesc(128, H, kFmtBF16);
    constexpr uint32_t id16 = make_idesc(128, 16, kFmtBF16);
    const uint64_t dsc_phi1 = make_sdesc(sbase + L::phi1, H * 16, 128);
    const uint64_t dsc_phi2 = make_sdesc(sbase + L::phi2, H * 16, 128);
    const uint64_t dsc_phi2b = make_sdesc(sbase + L::phi2b, H * 16, 128);
    const uint64_t dsc_b1 = make_sdesc(sbase + L::b1, H * 16, 128);
    // per-pixel weights: resident, or (streamed layout) the ring's two stages
    uint64_t dsc_rho = 0, dsc_b2 = 0, dsc_r1 = 0, dsc_r2 = 0;
    if constexpr (!L::kStream) {
      dsc_rho = make_sdesc(sbase + L::rho, H * 16, 128);
      dsc_b2 = make_sdesc(sbase + L::b2, H * 16, 128);
      dsc_r1 = make_sdesc(sbase + L::r1, H * 16, 128);
      dsc_r2 = make_sdesc(sbase + L::r2, 16 * 16, 128);
    }
    const uint64_t dsc_ring[2] = {make_sdesc(sbase + ring_stage<L>(0), H * 16, 128),
                                  make_sdesc(sbase + ring_stage<L>(1), H * 16, 128)};
    const uint64_t dsc_ring16[2] = {make_sdesc(sbase + ring_stage<L>(0), 16 * 16, 128),
                                    make_sdesc(sbase + ring_stage<L>(1), 16 * 16, 128)};
    uint32_t n_ck = 0;  // ring chunks taken
    // the next chunk is in its stage: its descriptor (N = H, or N = 16 for R2)
    auto ck_wait = [&](uint64_t& d, bool n16) -> bool {
      const uint32_t st = n_ck & 1;
      if (!warp_wait<true>(bar(B_WF + st), (n_ck >> 1) & 1, &s_abort)) return false;
      d = n16 ? dsc_ring16[st] : dsc_ring[st];
      return true;
    };
    // its MMAs are issued: the stage is free once they complete
    auto ck_done = [&]() {
      mma_commit_e(bar(B_WE + (n_ck & 1)));
      __syncwarp();
      ++n_ck;
    };
    const uint64_t dsc_at0 = make_sdesc(sbase + L::at0, 128 * 16, 128);
    const uint64_t dsc_at1 = make_sdesc(sbase + L::at1, 128 * 16, 128);
    const uint64_t dsc_one = make_sdesc(sbase + L::aone, 128 * 16, 128);
    const uint64_t dsc_ag = make_sdesc(sbase + L::ag, 128 * 16, 128);
    // bands of phi1's and B1's first operands (16 K columns each); B1's
    // weights for r start after the last G-buffer band.  A K step of 16 is
    // 4096 bytes of an A operand and 2 H 16 bytes of a weight operand.
    const int nb = PE ? 1 + 2 * prm.pe_freqs : 1;
    const uint64_t dsc_b1r = dsc_b1 + static_cast<uint64_t>(nb) * ((2 * H * 16) >> 4);
    auto mma_bands = [&](uint32_t d, uint64_t a0, uint64_t b0) {
      if constexpr (PE) {
        for (int t = 0; t < nb; ++t)
          mma_f16_ss_e(d, a0 + static_cast<uint64_t>(t) * 256u,
                       b0 + static_cast<uint64_t>(t) * ((2 * H * 16) >> 4), idH, t > 0 ? 1u : 0u);
      } else {
        mma_f16_ss_e(d, a0, b0, idH, 0u);
      }
    };
    SlotPos p1, p2;  // next phi1 / phi2 buffer
    uint32_t g1 = 0, n_in = 0, n_agf = 0;
    const int total_tiles = prm.total_tiles;
    const float* cur_fold = nullptr;
    // phi1 for the next global layer slot, into its rotating buffer
    auto phi1 = [&]() -> bool {
      // the buffer's previous phi2 accumulator has been read
      if (!warp_wait<true>(bar(B_BE + p1.b), (p1.u & 1) ^ 1, &s_abort)) return false;
      const int a = g1 & 1;
      if (!warp_wait<true>(bar(B_AT_F + a), (g1 >> 1) & 1, &s_abort)) return false;
      tc_fence_after();
      mma_bands(tbase + T::buf(p1.b), a ? dsc_at1 : dsc_at0, dsc_phi1);
      mma_commit_e(bar(B_D1 + p1.b));
      mma_commit_e(bar(B_AT_E + a));
      __syncwarp();
      ++g1;
      p1.next();
      return true;
    };
    // the epilogue warps have written the next A operand in TMEM
    uint32_t n_h[2] = {0, 0};
    auto wait_h = [&](int h) -> bool {
      if (!warp_wait<true>(bar(B_H + h), n_h[h] & 1, &s_abort)) return false;
      ++n_h[h];
      tc_fence_after();
      return true;
    };
    auto wait_in = [&]() -> bool {
      if (!warp_wait<true>(bar(B_IN + (n_in & 1)), (n_in >> 1) & 1, &s_abort)) return false;
      ++n_in;
      tc_fence_after();
      return true;
    };
    // Tile number t of this CTA as the loaders published it: global index
    // (>= total_tiles ends the loop), slot count and the frame's biases.
    auto take_tile = [&](uint32_t t, int& tile, int& ns, const float*& fold) -> bool {
      if (!warp_wait<true>(bar(B_TILE + (t & 1)), (t >> 1) & 1, &s_abort)) return false;
      tile = *reinterpret_cast<volatile int*>(&s_ld.tile[t & 1]);
      ns = 0;
#pragma unroll
      for (int w = 0; w < Roles<H, PE>::LW; ++w) ns = max(ns, s_ld.ns[t & 1][w]);
      fold = tile < total_tiles ? s_ld.fold[t & 3] : nullptr;
      return true;
    };
    // Per-scene folded biases -> the constant-one rows of phi1 and B1.  The
    // caller makes sure that no MMA can still read the previous ones.
    auto patch_fold = [&](const float* fold) {
      for (int i = lane; i < 2 * H; i += 32) {
        const int n = i < H ? i : i - H;
        const float cv = fold[i];
        const float hi = bf16_value(cv);
        const uint32_t packed = static_cast<uint32_t>(bf16_bits(hi)) |
                                (static_cast<uint32_t>(bf16_bits(cv - hi)) << 16);
        const uint32_t off = i < H ? L::phi1 + ((H + n) * 8 + 4) * 2
                                   : L::b1 + ((H + n) * 8 + 6) * 2;
        *reinterpret_cast<uint32_t*>(smem + off) = packed;
      }
      fence_proxy_async_smem();
      __syncwarp();
      cur_fold = fold;
    };
    int tile, ns;
    const float* fold;
    if (!warp_wait<true>(bar(B_W), 0, &s_abort)) goto done;
    // Test hook (stall_ns > 0, set by glassnet_debug_stall_next_render): wait
    // on a barrier that nothing arrives on, before any MMA is issued, so that
    // the wait gives up and every warp takes the timeout exit.
    if (prm.stall_ns > 0 && !warp_wait<true>(bar(B_STALL), 0, &s_abort, prm.stall_ns)) goto done;
    if (!take_tile(0, tile, ns, fold)) goto done;
    if (tile < total_tiles) {
      patch_fold(fold);
      for (int k = 0; k < ns && k < 2; ++k)
        if (!phi1()) goto done;
    }
    for (uint32_t tb = 0; tile < total_tiles; ++tb) {
      for (int k = 0; k < ns; ++k) {
        if (!wait_in()) goto done;  // U(k) written, its buffer read
        {
          const uint32_t d = tbase + T::buf(p2.b);
          issue_gemm<H, H>(d, tbase + (k & 1 ? T::AU1 : T::AU0), dsc_phi2, idH);
          mma_f16_ss_e(d, dsc_one, dsc_phi2b, idH, 1u);
          mma_commit_e(bar(B_D2 + p2.b));
        }
        __syncwarp();
        p2.next();
        if (k + 2 < ns && !phi1()) goto done;
      }
      int next_tile, next_ns;
      const float* next_fold;
      if constexpr (Mode == kModeAccumulate) {
        // no per-pixel layers: the pool state goes back to device memory;
        // B_AG_E paces the loaders (see loader_loop), once every epilogue
        // warp has taken this tile (a tile without covered pixels involves
        // no epilogue work, and the loaders must not get two tiles ahead of
        // the epilogue either) and the loaders have passed their wait for
        // the previous commit (B_AG_F)
        // (two alternating barriers: the epilogue cannot take tile tb + 2
        // before this commit, so neither runs two phases ahead)
        if (!warp_wait<true>(bar(B_H + (tb & 1)), (tb >> 1) & 1, &s_abort)) goto done;
        if (!warp_wait<true>(bar(B_AG_F), n_agf & 1, &s_abort)) goto done;
        ++n_agf;
        mma_commit_e(bar(B_AG_E));
        __syncwarp();
        if (!take_tile(tb + 1, next_tile, next_ns, next_fold)) goto done;
      } else {
        // Per-pixel layers.  Accumulators alternate X / Y (a layer never
        // overwrites the accumulator its input is being read from), A operands
        // live in the U region (lo = first H/2 columns, hi = last H/2):
        //   rho: X <- [max ; mean];  B1: Y <- [g ; r = lo];  B2: X <- y = hi;
        //   R1: Y <- y2 = lo;  R2: Z <- q = hi.
        // The sum form has no rho: B1 reads tau from lo.
        // Each GEMM is issued in two K halves, each as soon as the epilogue
        // half that produces it has arrived.
        const uint32_t X = tbase + T::buf(p1.b);
        const uint32_t Y = tbase + T::buf(p1.b == 2 ? 0 : p1.b + 1);
        const uint32_t Z = tbase + T::buf(p1.b == 0 ? 2 : p1.b - 1);
        const uint32_t A_LO = tbase + T::APOOL, A_HI = tbase + T::APOOL + H / 2;
        constexpr uint64_t kHalfK = static_cast<uint64_t>(H / 32) * ((2 * H * 16) >> 4);
        if constexpr (L::kStream) {
        // The same GEMMs with the weights from the ring, one K = 64 chunk per
        // half of a K half (the producer's order, ring_loop).  B1's G-buffer
        // band 0 (with the folded bias) is resident.
        auto half = [&](uint32_t acc, uint32_t a, bool accum) -> bool {
          uint64_t d;
          if (!ck_wait(d, false)) return false;
          issue_gemm<H, H / 2>(acc, a, d, idH, accum);
          ck_done();
          return true;
        };
        if constexpr (!Sum) {
          if (!wait_h(0) || !half(X, A_LO, false) || !half(X, A_LO + H / 4, true)) goto done;
          if (!wait_h(1) || !half(X, A_HI, true) || !half(X, A_HI + H / 4, true)) goto done;
          mma_commit_e(bar(B_DP));
          __syncwarp();
        }
        if (!take_tile(tb + 1, next_tile, next_ns, next_fold)) goto done;
        if (!wait_h(0)) goto done;
        if (!warp_wait<true>(bar(B_AG_F), n_agf & 1, &s_abort)) goto done;
        ++n_agf;
        tc_fence_after();
        mma_f16_ss_e(Y, dsc_ag, dsc_b1, idH, 0u);
        for (int t0 = 1; t0 < nb; t0 += 4) {
          uint64_t d;
          if (!ck_wait(d, false)) goto done;
          for (int t = t0; t < nb && t < t0 + 4; ++t)
            mma_f16_ss_e(Y, dsc_ag + static_cast<uint64_t>(t) * 256u,
                         d + static_cast<uint64_t>(t - t0) * ((2 * H * 16) >> 4), idH, 1u);
          ck_done();
        }
        if (!half(Y, A_LO, true) || !wait_h(1) || !half(Y, A_LO + H / 4, true)) goto done;
        mma_commit_e(bar(B_DP));
        mma_commit_e(bar(B_AG_E));
        __syncwarp();
        if (!wait_h(0) || !half(X, A_HI, false) || !wait_h(1) || !half(X, A_HI + H / 4, true))
          goto done;
        mma_commit_e(bar(B_DP));
        __syncwarp();
        if constexpr (R3) {
          if (!wait_h(0) || !wait_h(1)) goto done;
          mma_commit_e(bar(B_DR2));
          __syncwarp();
        } else {
          if (!wait_h(0) || !half(Y, A_LO, false) || !wait_h(1) || !half(Y, A_LO + H / 4, true))
            goto done;
          mma_commit_e(bar(B_DP));
          __syncwarp();
          if (!wait_h(0) || !wait_h(1)) goto done;
          uint64_t d;
          if (!ck_wait(d, true)) goto done;
          issue_gemm<16, H>(Z, A_HI, d, id16);
          ck_done();
          mma_commit_e(bar(B_DR2));
          __syncwarp();
        }
        } else {
        if constexpr (!Sum) {
          if (!wait_h(0)) goto done;
          issue_gemm<H, H>(X, A_LO, dsc_rho, idH);
          if (!wait_h(1)) goto done;
          issue_gemm<H, H>(X, A_HI, dsc_rho + 2 * kHalfK, idH, true);
          mma_commit_e(bar(B_DP));
          __syncwarp();
        }
        // the next tile, read while the per-pixel layers run (the loaders
        // publish it once this tile's layer operands are written)
        if (!take_tile(tb + 1, next_tile, next_ns, next_fold)) goto done;
        if (!wait_h(0)) goto done;
        if (!warp_wait<true>(bar(B_AG_F), n_agf & 1, &s_abort)) goto done;
        ++n_agf;
        tc_fence_after();
        mma_bands(Y, dsc_ag, dsc_b1);
        issue_gemm<H, H / 2>(Y, A_LO, dsc_b1r, idH, true);
        if (!wait_h(1)) goto done;
        issue_gemm<H, H / 2>(Y, A_LO + H / 4, dsc_b1r + kHalfK, idH, true);
        mma_commit_e(bar(B_DP));
        mma_commit_e(bar(B_AG_E));
        __syncwarp();
        if (!wait_h(0)) goto done;
        issue_gemm<H, H / 2>(X, A_HI, dsc_b2, idH);
        if (!wait_h(1)) goto done;
        issue_gemm<H, H / 2>(X, A_HI + H / 4, dsc_b2 + kHalfK, idH, true);
        mma_commit_e(bar(B_DP));
        __syncwarp();
        if constexpr (R3) {
          // y goes to device memory: the epilogue's B2 passes arrive as they
          // would for R1 (X is read before the next tile's phi1 writes it)
          if (!wait_h(0) || !wait_h(1)) goto done;
          mma_commit_e(bar(B_DR2));
          __syncwarp();
        } else {
        if (!wait_h(0)) goto done;
        issue_gemm<H, H / 2>(Y, A_LO, dsc_r1, idH);
        if (!wait_h(1)) goto done;
        issue_gemm<H, H / 2>(Y, A_LO + H / 4, dsc_r1 + kHalfK, idH, true);
        mma_commit_e(bar(B_DP));
        __syncwarp();
        if (!wait_h(0) || !wait_h(1)) goto done;
        issue_gemm<16, H>(Z, A_HI, dsc_r2, id16);
        mma_commit_e(bar(B_DR2));
        __syncwarp();
        }  // R1, R2
        }  // resident per-pixel weights
      }
      // the next tile's first two phi1 right behind R2 (they write X and Y)
      tile = next_tile;
      ns = next_ns;
      if (tile < total_tiles) {
        if (next_fold != cur_fold) {
          // every MMA of this tile (B1 reads the old bias rows) has completed
          if (!warp_wait<true>(bar(B_DR2), tb & 1, &s_abort)) goto done;
          patch_fold(next_fold);
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
    uint32_t gs = 0;  // global index of the tile's first layer slot
    uint32_t n_in = 0, n_dp = 0, tb = 0;
    auto arrive_h = [&](int h) {
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_H + h));
    };
    auto arrive_in = [&]() {
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_IN + (n_in & 1)));
      ++n_in;
    };
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the tile plan is complete
    if (!warp_wait<kOol>(bar(B_W), 0, &s_abort)) goto done;
    {
      const int total_tiles = prm.total_tiles;
      // Tile number t of this CTA as the loaders published it.
      int tile, ns, c;
      auto take_tile = [&](uint32_t t) -> bool {
        if (!warp_wait<kOol>(bar(B_TILE + (t & 1)), (t >> 1) & 1, &s_abort)) return false;
        tile = *reinterpret_cast<volatile int*>(&s_ld.tile[t & 1]);
        ns = 0;
#pragma unroll
      for (int w = 0; w < Roles<H, PE>::LW; ++w) ns = max(ns, s_ld.ns[t & 1][w]);
        c = s_ld.cnt[t & 1][row];
        return true;
      };
      if (!take_tile(0)) goto done;
      // R2's output of the previous tile, read from TMEM but not yet stored:
      // the column-group-0 warps store it after their first phi1 epilogue of
      // the next tile, so that the sigmoid and the global stores are not
      // between that tile's first phi2 and the previous tile's R2.
      float pend_y[kOut] = {};
      float* pend_out = nullptr;
      size_t pend_P = 0;
      uint32_t pend_pix = 0;
      auto flush_store = [&]() {
        if (pend_out) {
#pragma unroll
          for (int j = 0; j < kOut; ++j)
            pend_out[j * pend_P + pend_pix] = 1.0f / (1.0f + expf(-pend_y[j]));
          pend_out = nullptr;
        }
      };
      for (; tile < total_tiles; ++tb) {
        uint32_t mx[CHC];  // running max, bf16 pairs
        float sm[CH];      // fixed-point sums
#pragma unroll
        for (int j = 0; j < CHC; ++j) mx[j] = 0u;
#pragma unroll
        for (int j = 0; j < CH; ++j) sm[j] = kSumBase;
        // Streaming launches: a pixel that has layers starts from its pool
        // state (planes of the pixel's channel pairs and channels).
        uint32_t* st = nullptr;  // this row's word in plane 0 of the tile's state block
        if constexpr (Mode == kModeAccumulate) {
          if (lane == 0) mbar_arrive(bar(B_H + (tb & 1)));  // this tile is taken (paces the loaders)
        }
        if constexpr (Mode != kModeFrame) {
          // pixel order: row `row` of the tile is its pixel
          st = prm.pool_st + static_cast<size_t>(tile - prm.f[0].tile0) * ((H / 2 + H) * kTile) + row;
          if (c > 0 && !prm.pool_fresh) {
#pragma unroll
            for (int j = 0; j < CHC; ++j) mx[j] = Sum ? 0u : st[(g * CHC + j) * kTile];
#pragma unroll
            for (int j = 0; j < CH; ++j) sm[j] = __uint_as_float(st[(H / 2 + g * CH + j) * kTile]);
          }
        }

        // phi1(k) accumulator -> U(k) = ReLU as bf16.  16-column TMEM loads
        // are double buffered: block hh + 1 is in flight while hh is packed.
        auto epi1 = [&](int k) -> bool {
          const uint32_t gk = gs + k, b = gk % 3u;
          if (!warp_wait<kOol>(bar(B_D1 + b), (gk / 3u) & 1, &s_abort)) return false;
          tc_fence_after();
          const uint32_t src = tl + T::buf(b) + g * CH;
          const uint32_t dst = tl + (k & 1 ? T::AU1 : T::AU0) + g * CHC;
          uint32_t ra[16], rb[16];
          tmem_ld16_async(src, ra);
          tmem_wait_ld_tied(ra);
#pragma unroll
          for (int hh = 0; hh < CH / 16; ++hh) {
            uint32_t(&cur)[16] = (hh & 1) ? rb : ra;
            uint32_t(&nxt)[16] = (hh & 1) ? ra : rb;
            if (hh + 1 < CH / 16) tmem_ld16_async(src + (hh + 1) * 16, nxt);
            uint32_t u[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
              u[i] = pack_bf16_relu(__uint_as_float(cur[2 * i]), __uint_as_float(cur[2 * i + 1]));
            tmem_st8(dst + hh * 8, u);
            if (hh + 1 < CH / 16) tmem_wait_ld_tied(nxt);
          }
          arrive_in();
          return true;
        };
        // phi2(k) accumulator -> pool update for pixels with k < c.
        auto epi2 = [&](int k) -> bool {
          const uint32_t gk = gs + k, b = gk % 3u;
          if (!warp_wait<kOol>(bar(B_D2 + b), (gk / 3u) & 1, &s_abort)) return false;
          tc_fence_after();
          const uint32_t src = tl + T::buf(b) + g * CH;
          uint32_t ra[16], rb[16];
          tmem_ld16_async(src, ra);
          tmem_wait_ld_tied(ra);
#pragma unroll
          for (int hh = 0; hh < CH / 16; ++hh) {
            uint32_t(&cur)[16] = (hh & 1) ? rb : ra;
            uint32_t(&nxt)[16] = (hh & 1) ? ra : rb;
            if (hh + 1 < CH / 16) {
              tmem_ld16_async(src + (hh + 1) * 16, nxt);
            } else {
              // every column of this buffer is in registers: release it
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(bar(B_BE + b));
            }
            if (k < c) {
#pragma unroll
              for (int i = 0; i < 16; i += 2) {
                const int j = hh * 16 + i;
                const uint32_t u =
                    pack_bf16_relu(__uint_as_float(cur[i]), __uint_as_float(cur[i + 1]));
                if constexpr (!Sum) mx[j / 2] = bmax2(mx[j / 2], u);
                add_bf16x2_rz(sm[j], sm[j + 1], u);
              }
            }
            if (hh + 1 < CH / 16) tmem_wait_ld_tied(nxt);
          }
          return true;
        };

        // epi1(k + 1) runs ahead of epi2(k); one call site each
        for (int k = -1; k < ns; ++k) {
          if (k + 1 < ns && !epi1(k + 1)) goto done;
          if (k < 0) flush_store();  // the previous tile's RGB
          if (k >= 0 && !epi2(k)) goto done;
        }
        if constexpr (Mode == kModeAccumulate) {
          // the covered pixels' state back to device memory, one more layer
          if (c > 0) {
#pragma unroll
            for (int j = 0; j < CHC; ++j) st[(g * CHC + j) * kTile] = mx[j];
#pragma unroll
            for (int j = 0; j < CH; ++j) st[(H / 2 + g * CH + j) * kTile] = __float_as_uint(sm[j]);
            if (g == 0) {
              const size_t pix = static_cast<size_t>(tile - prm.f[0].tile0) * kTile + row;
              prm.pool_cnt[pix] = static_cast<uint8_t>(prm.pool_cnt[pix] + 1);
            }
          }
          gs += ns;
          if (!take_tile(tb + 1)) goto done;
        } else {
        if constexpr (Sum) {
        // tau -> lo (bf16, H values = H/2 columns), B1's K half by K half.
        // This warp's channels lie in one half (all of them for kEW = 1): it
        // arrives on the other half's barrier without writing.
        const bool first_half = g * CH < H / 2;
        if (!first_half) arrive_h(0);
        {
          const float off = kSumBase - static_cast<float>(c) * kHalfQuantum;
          bool over = false;
#pragma unroll
          for (int hh = 0; hh < CHC / 8; ++hh) {
            uint32_t pa[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int jj = hh * 8 + j;
              over |= !(fmaxf(sm[2 * jj], sm[2 * jj + 1]) < kSumLimit);
              float a0, a1;
              fadd2_rn(a0, a1, sm[2 * jj], sm[2 * jj + 1], -off, -off);
              pa[j] = pack_bf16(a0, a1);
            }
            tmem_st8(tl + T::APOOL + g * CHC + hh * 8, pa);
          }
          if (over && c > 0) atomicOr(prm.err, kErrRange);
        }
        if (first_half) arrive_h(0);
        arrive_h(1);
        } else {
        // pool = [max ; mean] -> the U region (bf16, 2H values = H columns):
        // the max half first (rho's first K half can start), then the mean.
#pragma unroll
        for (int hh = 0; hh < CHC / 8; ++hh) {
          uint32_t pm[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) pm[j] = mx[hh * 8 + j];
          tmem_st8(tl + T::APOOL + g * CHC + hh * 8, pm);
        }
        arrive_h(0);
        {
          const float rcp = c > 0 ? __frcp_rn(static_cast<float>(c)) : 0.0f;
          const float off = kSumBase - static_cast<float>(c) * kHalfQuantum;
          bool over = false;
#pragma unroll
          for (int hh = 0; hh < CHC / 8; ++hh) {
            uint32_t pa[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int jj = hh * 8 + j;
              over |= !(fmaxf(sm[2 * jj], sm[2 * jj + 1]) < kSumLimit);
              float a0, a1;
              fadd2_rn(a0, a1, sm[2 * jj], sm[2 * jj + 1], -off, -off);
              pa[j] = pack_bf16(a0 * rcp, a1 * rcp);
            }
            tmem_st8(tl + T::APOOL + H / 2 + g * CHC + hh * 8, pa);
          }
          if (over && c > 0) atomicOr(prm.err, kErrRange);
        }
        arrive_h(1);
        }  // max + mean

        // the row's plan entry (pixel index) for the store, loaded while the
        // per-pixel layers run
        const uint32_t ent = (g == 0 || R3)
                                 ? __ldg(prm.plan + static_cast<size_t>(tile) * kTile + row)
                                 : kPlanEmpty;
        // 3x3 R: this row's pixel in the neural buffer (chunk c of 8 channels
        // at phi_px + c w)
        uint4* phi_px = nullptr;
        uint32_t fw = 0;
        if constexpr (R3) {
          const FusedFrame& Fr = frame_of(prm, tile);
          fw = static_cast<uint32_t>(Fr.w);
          if (ent != kPlanEmpty) {
            const uint32_t pix = ent & kPlanPixelMask;
            const uint32_t py = pix / fw;
            phi_px = reinterpret_cast<uint4*>(Fr.phi) + static_cast<size_t>(py) * (H / 8) * fw +
                     (pix - py * fw);
          }
        }

        // rho -> r (zero without layers) -> lo;  B1 -> y -> hi;  B2 -> y2 -> lo;
        // R1 -> q -> hi.  Accumulators X, Y, X, Y.  Each layer in two passes of
        // H/2 accumulator columns (this warp: H/(2 kEW) of them), one arrival each.
        gs += ns;
        const uint32_t r3 = gs % 3u;
        const uint32_t X = tl + T::buf(r3);
        const uint32_t Y = tl + T::buf(r3 == 2 ? 0 : r3 + 1);
        const uint32_t Z = tl + T::buf(r3 == 0 ? 2 : r3 - 1);
        const uint32_t A_LO = tl + T::APOOL, A_HI = tl + T::APOOL + H / 2;
        constexpr int PC = H / (2 * kEW);  // accumulator columns of this warp per pass
        static_assert(PC % 16 == 0, "per-pixel passes load 16 accumulator columns at a time");
#pragma unroll
        for (int l = Sum ? 1 : 0; l < (R3 ? 3 : 4); ++l) {
          if (!warp_wait<kOol>(bar(B_DP), n_dp & 1, &s_abort)) goto done;
          ++n_dp;
          tc_fence_after();
          const float* bl = l == 0 ? b_rho : (l == 2 ? b_b2 : b_r1);
          const uint32_t acc = (l & 1) ? Y : X;
          const uint32_t dst = (l & 1) ? A_HI : A_LO;
#pragma unroll 1
          for (int h = 0; h < 2; ++h) {
            const int c0 = h * (H / 2) + g * PC;  // first accumulator column of this pass
            uint32_t ra[16], rb[16];
            tmem_ld16_async(acc + c0, ra);
            tmem_wait_ld_tied(ra);
#pragma unroll
            for (int hh = 0; hh < PC / 16; ++hh) {
              uint32_t(&cur)[16] = (hh & 1) ? rb : ra;
              uint32_t(&nxt)[16] = (hh & 1) ? ra : rb;
              if (hh + 1 < PC / 16) tmem_ld16_async(acc + c0 + (hh + 1) * 16, nxt);
              uint32_t u[8];
              if (l == 1) {  // B1's bias is folded into its GEMM
#pragma unroll
                for (int i = 0; i < 8; ++i)
                  u[i] = pack_bf16_relu(__uint_as_float(cur[2 * i]), __uint_as_float(cur[2 * i + 1]));
              } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  float v0, v1;
                  fadd2_rn(v0, v1, __uint_as_float(cur[2 * i]), __uint_as_float(cur[2 * i + 1]),
                           bl[c0 + hh * 16 + 2 * i], bl[c0 + hh * 16 + 2 * i + 1]);
                  u[i] = (l == 0 && c == 0) ? 0u : pack_bf16_relu(v0, v1);
                }
              }
              if (R3 && l == 2) {  // y -> the neural buffer
                if (phi_px) {
                  const size_t c8 = static_cast<size_t>(c0 + hh * 16) / 8;
                  phi_px[c8 * fw] = make_uint4(u[0], u[1], u[2], u[3]);
                  phi_px[(c8 + 1) * fw] = make_uint4(u[4], u[5], u[6], u[7]);
                }
              } else {
                tmem_st8(dst + c0 / 2 + hh * 8, u);
              }
              if (hh + 1 < PC / 16) tmem_wait_ld_tied(nxt);
            }
            arrive_h(h);
          }
        }
        // R2 -> registers (column group 0), stored by flush_store after the
        // next tile's first phi1 epilogue (or after the last tile).  Every warp
        // waits for R2: the next tile's phi1 for its third slot writes Z, and
        // it is issued only after every warp's first phi1 epilogue of that
        // tile, which follows this TMEM read.  The next tile is taken first.
        if (!take_tile(tb + 1)) goto done;
        if (!warp_wait<kOol>(bar(B_DR2), tb & 1, &s_abort)) goto done;
        if (!R3 && g == 0) {
          tc_fence_after();
          uint32_t r[4];
          tmem_ld4(Z, r);
          if (ent != kPlanEmpty) {
            pend_out = s_ld.out[tb & 3];
            pend_P = static_cast<size_t>(s_ld.P[tb & 3]);
            pend_pix = ent & kPlanPixelMask;
#pragma unroll
            for (int j = 0; j < kOut; ++j) pend_y[j] = __uint_as_float(r[j]) + b_r2[j];
          }
        }
        }  // frame and resolve launches: the per-pixel layers
      }
      flush_store();  // the last tile's RGB
    }
  }
done:
  tc_fence_before();
  __syncthreads();  // every warp is here: s_abort is final
  if (s_abort) {
    if (warp == R::MMA) drain_async(bar(B_W), bar(B_DRAIN));
    if (tid == 0) report_timeout(prm.err, s_abort, bar_base, kKernelFusedBf16, Mode);
  }
  if (warp == R::MMA) {
    tc_fence_after();
    tmem_dealloc(tbase, TMap<H>::NCOLS);
  }
}

template <int H, int Mode, bool Sum, bool PE, bool R3 = false>
cudaError_t prepare_h() {
  static bool done = false;  // per process: the attribute holds for every later launch
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fused_bf16_kernel<H, Mode, Sum, PE, R3>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       FusedLayout<H, PE>::smem_bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int H, int Mode, bool Sum, bool PE, bool R3 = false>
cudaError_t launch_h(const void* wimg, const FusedParams& p, cudaStream_t s, int grid) {
  constexpr int smem = FusedLayout<H, PE>::smem_bytes;
  cudaError_t e = prepare_h<H, Mode, Sum, PE, R3>();
  if (e != cudaSuccess) return e;
  // Programmatic dependent launch: the CTAs may start while the plan kernel
  // is still running; they wait on the grid dependency before the plan reads.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(Roles<H, PE>::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fused_bf16_kernel<H, Mode, Sum, PE, R3>, p,
                            static_cast<const uint8_t*>(wimg));
}

template <int H, bool PE>
cudaError_t prepare_all() {
  cudaError_t e = prepare_h<H, kModeFrame, false, PE>();
  if (e == cudaSuccess) e = prepare_h<H, kModeAccumulate, false, PE>();
  if (e == cudaSuccess) e = prepare_h<H, kModeResolve, false, PE>();
  if (e == cudaSuccess) e = prepare_h<H, kModeFrame, true, PE>();
  if (e == cudaSuccess) e = prepare_h<H, kModeResolve, true, PE>();
  if (e == cudaSuccess) e = prepare_h<H, kModeFrame, false, PE, true>();
  if (e == cudaSuccess) e = prepare_h<H, kModeFrame, true, PE, true>();
  if (e == cudaSuccess) e = prepare_h<H, kModeResolve, false, PE, true>();
  if (e == cudaSuccess) e = prepare_h<H, kModeResolve, true, PE, true>();
  return e;
}

template <int H, bool PE>
cudaError_t launch_mode(int mode, const void* wimg, const FusedParams& p, cudaStream_t s,
                        int grid) {
  // accumulation is the same for both poolings (the state holds max and sum)
  if (mode == kModeAccumulate) return launch_h<H, kModeAccumulate, false, PE>(wimg, p, s, grid);
  if (p.f[0].phi) {  // the neural buffer out, for the 3x3 R (frames and resolves)
    if (mode == kModeResolve)
      return p.pool_sum ? launch_h<H, kModeResolve, true, PE, true>(wimg, p, s, grid)
                        : launch_h<H, kModeResolve, false, PE, true>(wimg, p, s, grid);
    return p.pool_sum ? launch_h<H, kModeFrame, true, PE, true>(wimg, p, s, grid)
                      : launch_h<H, kModeFrame, false, PE, true>(wimg, p, s, grid);
  }
  if (p.pool_sum)
    return mode == kModeResolve ? launch_h<H, kModeResolve, true, PE>(wimg, p, s, grid)
                                : launch_h<H, kModeFrame, true, PE>(wimg, p, s, grid);
  return mode == kModeResolve ? launch_h<H, kModeResolve, false, PE>(wimg, p, s, grid)
                              : launch_h<H, kModeFrame, false, PE>(wimg, p, s, grid);
}

}  // namespace

cudaError_t prepare_fused_bf16(int H) {
  device_sm_count();
  if (H == 128) {
    cudaError_t e = prepare_all<128, false>();
    return e == cudaSuccess ? prepare_all<128, true>() : e;
  }
  cudaError_t e = prepare_all<64, false>();
  return e == cudaSuccess ? prepare_all<64, true>() : e;
}

cudaError_t launch_fused_bf16(int H, const void* wimg, const FusedParams& params,
                              cudaStream_t s, int mode) {
  if (params.total_tiles <= 0) return cudaSuccess;
  FusedParams p = params;
  cudaError_t e = launch_plan(p, s);
  if (e != cudaSuccess) return e;
  // persistent CTAs take tiles from the plan's counter: as many as fit
  const int per_sm = (H == 64 && p.pe_freqs == 0) ? Roles<64, false>::kCtasPerSm : 1;
  const int slots = per_sm * device_sm_count();
  const int grid = p.total_tiles < slots ? p.total_tiles : slots;
  if (p.pe_freqs > 0) {
    // the encoded operands are sized for kMaxPeFreqsFused (the loader refuses more)
    if (p.pe_freqs > kMaxPeFreqsFused) return cudaErrorInvalidValue;
    return H == 128 ? launch_mode<128, true>(mode, wimg, p, s, grid)
                    : launch_mode<64, true>(mode, wimg, p, s, grid);
  }
  return H == 128 ? launch_mode<128, false>(mode, wimg, p, s, grid)
                  : launch_mode<64, false>(mode, wimg, p, s, grid);
}

}  // namespace gn

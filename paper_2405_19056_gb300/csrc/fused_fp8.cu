// Fused GlassNet forward pass with E4M3 operands (FP8 variant): the same
// pipeline as the BF16 kernel (tile plan, warp roles, three rotating TMEM
// accumulators, phi1 two slots ahead, exact pooling), with every layer's
// GEMM a tcgen05 kind::f8f6f4 MMA (K = 32 per instruction, FP32 accumulate).
//
// Quantisation (static, per tensor for activations, per output channel for
// weights): a layer computes acc = sum_k xq[k] wq[n][k] with E4M3 codes, and
// its epilogue maps acc to the next layer's code with one FMA per element,
//   next = e4m3(ReLU(acc * s[n] + b[n])),   s[n] = s_in s_w[n] / s_out,
// or to real units where the value is not re-quantised (phi2's output, which
// feeds the exact pooling, and R2's, which feeds the sigmoid).  The per-scene
// folded biases c_phi and c_B (Sec. 3.4 latent, folded exactly) are too fine
// for E4M3: they enter the accumulator through one BF16 MMA of a constant
// [1, 1, 0, ...] operand against their hi / lo BF16 split, pre-divided by
// s_in s_w[n] so that they land in accumulator units.
//
// Pooling is exactly the BF16 kernel's (max of bf16(ReLU(v)) pairs, exact
// fixed-point sum), on the dequantised v; the pooled [max ; mean] is then
// quantised for rho.  The output is therefore bit-identical under any
// permutation of a pixel's valid layers, as in the BF16 kernel.
#include "fused_common.cuh"

namespace gn {
namespace {
using namespace fused;

constexpr int B_STALL8 = B_COUNT;      // never arrived on: the stall that tests the timeout path
constexpr int B_DRAIN8 = B_COUNT + 1;  // the exit path's last commit
constexpr int B_COUNT_F8 = B_COUNT + 2;

// TMEM column map (128 lanes x 4H columns): three accumulator buffers of H
// columns, then U (H e4m3 = H/4 columns) double buffered; the pooled
// [max ; mean] (2H e4m3 = H/2 columns) reuses the U region.  The per-pixel
// layers use X / Y / Z exactly as in the BF16 kernel.
template <int H>
struct TMapF8 {
  static constexpr uint32_t AU0 = 3 * H;
  static constexpr uint32_t AU1 = 3 * H + H / 4;
  static constexpr uint32_t APOOL = AU0;
  static constexpr uint32_t NCOLS = 4 * H;
  static __device__ __forceinline__ uint32_t buf(uint32_t b) { return b * H; }
};

// D (+)= A (TMEM, K e4m3 = K/4 columns from a_tmem) x B^T, B stored
// [K/16][N][16] bytes and described by `d0`.  Each K step of 32 advances A by
// 8 columns and B by two core-matrix columns ((2 N 16) >> 4 in the
// descriptor's address field).
template <int N, int K>
__device__ __forceinline__ void issue_gemm_f8(uint32_t d_tmem, uint32_t a_tmem, uint64_t d0,
                                              uint32_t idesc, bool accumulate = false) {
  constexpr uint32_t step = (2 * N * 16) >> 4;
  if constexpr (K % 128 == 0) {
#pragma unroll
    for (int kb = 0; kb < K / 128; ++kb)
      mma4_f8_ts_e<step>(d_tmem, a_tmem + kb * 32, d0 + static_cast<uint64_t>(4 * step) * kb,
                         idesc, (kb > 0 || accumulate) ? 1u : 0u);
  } else {
#pragma unroll
    for (int ks = 0; ks < K / 32; ++ks)
      mma_f8_ts_e(d_tmem, a_tmem + ks * 8, d0 + static_cast<uint64_t>(step) * ks, idesc,
                  (ks > 0 || accumulate) ? 1u : 0u);
  }
}

// (a0, a1) * (s0, s1) + (b0, b1), round to nearest even, two lanes per op.
__device__ __forceinline__ void ffma2(float& r0, float& r1, float a0, float a1, float s0, float s1,
                                      float b0, float b1) {
  asm("{.reg .b64 p, q, c, r;\n\tmov.b64 p, {%2, %3};\n\tmov.b64 q, {%4, %5};\n\t"
      "mov.b64 c, {%6, %7};\n\tfma.rn.f32x2 r, p, q, c;\n\tmov.b64 {%0, %1}, r;}"
      : "=f"(r0), "=f"(r1)
      : "f"(a0), "f"(a1), "f"(s0), "f"(s1), "f"(b0), "f"(b1));
}

// 16 accumulator columns -> 16 E4M3 codes of ReLU(acc * s + b) in 4 TMEM
// columns (4 codes per column, lowest column index in the low byte).
__device__ __forceinline__ void quant16(const uint32_t (&acc)[16], const float* s, const float* b,
                                        bool zero, uint32_t (&q)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float y[4];
#pragma unroll
    for (int i = 0; i < 4; i += 2)
      ffma2(y[i], y[i + 1], __uint_as_float(acc[4 * j + i]), __uint_as_float(acc[4 * j + i + 1]),
            s[4 * j + i], s[4 * j + i + 1], b ? b[4 * j + i] : 0.0f, b ? b[4 * j + i + 1] : 0.0f);
    q[j] = zero ? 0u : pack_u16x2(pack_e4m3_relu(y[0], y[1]), pack_e4m3_relu(y[2], y[3]));
  }
}

// ---------------------------------------------------------------- loader
// Layer k of the lane's rows: 12 channels each, zeros where the slot is not
// valid.  Element offsets fit in 32 bits: the host requires 12 K h w < 2^31.
__device__ __forceinline__ void load_slot_f8(const FusedFrame& F, int k,
                                             const uint32_t (&pix)[kRowsPerLoadLane],
                                             const int (&cnt)[kRowsPerLoadLane],
                                             float (&x)[kRowsPerLoadLane][kTC]) {
  const uint32_t P = static_cast<uint32_t>(F.P);
#pragma unroll
  for (int i = 0; i < kRowsPerLoadLane; ++i) {
    const bool v = k < cnt[i];
    const uint32_t o = static_cast<uint32_t>(k) * kTC * P + pix[i];
#pragma unroll
    for (int ch = 0; ch < kTC; ++ch) x[i][ch] = v ? __ldg(F.tbuf + (o + ch * P)) : 0.0f;
  }
}

// x[c] / s[c] for N input channels, each channel with its own calibrated
// scale; `sat` is set when a value lies beyond the largest E4M3 code (the
// conversion clamps it).
template <int N>
__device__ __forceinline__ void scale_inputs(const float (&x)[N], const float (&inv_s)[N],
                                             float (&v)[N], bool& sat) {
#pragma unroll
  for (int c = 0; c < N; ++c) {
    v[c] = x[c] * inv_s[c];
    sat |= fabsf(v[c]) > 448.0f;
  }
}

// Writes K block 0 of rows row0 + 32 i of a [2][128][16]-byte operand: the
// 12 channels as E4M3 codes of x[c] / s_t[c], then zeros (block 1 stays zero).
__device__ __forceinline__ void store_slot_f8(uint32_t base, int row0, const float (&inv_s)[kTC],
                                              const float (&x)[kRowsPerLoadLane][kTC], bool& sat) {
#pragma unroll
  for (int i = 0; i < kRowsPerLoadLane; ++i) {
    float v[kTC];
    scale_inputs(x[i], inv_s, v, sat);
    uint32_t w[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      w[j] = pack_u16x2(pack_e4m3(v[4 * j], v[4 * j + 1]), pack_e4m3(v[4 * j + 2], v[4 * j + 3]));
    sts128(base + static_cast<uint32_t>(row0 + 32 * i) * 16u, w[0], w[1], w[2], 0u);
  }
}

// Positional encoding (Sec. 3.4) of one row of N input channels (12 for a
// layer, 14 for the G-buffer) as a K = 128 E4M3 operand row: band-major, code
// k = N t + c of band t; band 0 the code of x[c] / s[c] (calibrated channel
// scale), bands 2f + 1 and 2f + 2 the codes of sin and cos(2^f pi x[c]) times
// kFp8BandCode; zeros from k = N (1 + 2 nf) on.  Channel pairs fill 16-bit
// halves (N t + c is even for even c).
// The channel scales 1 / s[c] are read from shared memory at `inv_s` (a
// volatile load per use: the encoder's registers go to the bands).
__device__ __forceinline__ float lds_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
template <int N>
__device__ __forceinline__ void encode_row_f8(const float (&x)[N], uint32_t inv_s, int nf,
                                              uint32_t (&w)[32], bool& sat) {
  static_assert(N % 2 == 0 && N * (1 + 2 * kMaxPeFreqsFused) <= 128, "bands must fit K = 128");
#pragma unroll
  for (int j = 0; j < 32; ++j) w[j] = 0u;
  auto put = [&](int h, uint16_t v) {  // codes 2h and 2h + 1 of the row
    w[h >> 1] |= (h & 1) ? static_cast<uint32_t>(v) << 16 : static_cast<uint32_t>(v);
  };
#pragma unroll
  for (int p = 0; p < N / 2; ++p) {
    const float x0 = x[2 * p], x1 = x[2 * p + 1];
    const float v0 = x0 * lds_f32(inv_s + 8u * p), v1 = x1 * lds_f32(inv_s + 8u * p + 4u);
    sat |= fabsf(v0) > 448.0f || fabsf(v1) > 448.0f;
    put(p, pack_e4m3(v0, v1));
    // the bands times kFp8BandCode = 2^8 throughout: the double-angle steps
    // on scaled values (2 s c = (2 / 2^8) s' c', 1 - 2 s^2 = 2^8 - (2 / 2^8)
    // s'^2 in units of 2^-8) differ from the unscaled ones only by the
    // exact power-of-two factors
    float sn[2], cs[2];
    const float xs[2] = {x0, x1};
    pe_first(xs, sn, cs);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      sn[j] *= kFp8BandCode;
      cs[j] *= kFp8BandCode;
    }
    constexpr float k2 = 2.0f / kFp8BandCode;
#pragma unroll
    for (int f = 0; f < kMaxPeFreqsFused; ++f) {
      if (f < nf) {
        if (f > 0) {
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const float a = sn[j];
            sn[j] = k2 * a * cs[j];
            cs[j] = fmaf(-k2 * a, a, kFp8BandCode);
          }
        }
        put((N / 2) * (2 * f + 1) + p, pack_e4m3(sn[0], sn[1]));
        put((N / 2) * (2 * f + 2) + p, pack_e4m3(cs[0], cs[1]));
      }
    }
  }
}

// The 8 core-matrix columns (16 codes each) of row `row` of a [8][128][16]
// operand.
__device__ __forceinline__ void store_row_k128(uint32_t base, int row, const uint32_t (&w)[32]) {
#pragma unroll
  for (int j = 0; j < 8; ++j)
    sts128(base + static_cast<uint32_t>(j) * 2048u + static_cast<uint32_t>(row) * 16u, w[4 * j],
           w[4 * j + 1], w[4 * j + 2], w[4 * j + 3]);
}

template <int H, bool PE>
__device__ __forceinline__ void loader_loop_f8(const FusedParams& prm, const uint8_t* wimg,
                                               uint32_t sbase, uint32_t bar_base,
                                               LoaderShared& ls, volatile int* abort_flag, int li,
                                               int lane) {
  using L = FusedLayoutF8<H, PE>;
  const int nf = PE ? prm.pe_freqs : 0;  // positional-encoding frequencies
  auto bar = [&](int i) { return bar_base + static_cast<uint32_t>(i) * 8u; };
  const float* cst = reinterpret_cast<const float*>(wimg + L::cst);
  float inv_s_t[kTC], inv_s_g[kGC];  // per-channel input scales (inputs as given)
  // encoded inputs: the scales stay in the shared-memory copy of the
  // constants, which is there once the weights have landed
  const uint32_t inv_s_t_sm = sbase + L::cst + 4u * L::INV_S_TCH;
  const uint32_t inv_s_g_sm = sbase + L::cst + 4u * L::INV_S_GCH;
  if constexpr (PE) {
    if (!warp_wait<true>(bar(B_W), 0, abort_flag)) return;
  } else {
#pragma unroll
    for (int c = 0; c < kTC; ++c) inv_s_t[c] = __ldg(cst + L::INV_S_TCH + c);
#pragma unroll
    for (int c = 0; c < kGC; ++c) inv_s_g[c] = __ldg(cst + L::INV_S_GCH + c);
  }
  bool sat = false;  // an input of this warp's rows was clamped
  // reported once per tile, by the warp's lane 0
  auto report_sat = [&]() {
    if (__any_sync(0xffffffffu, sat) && lane == 0) atomicOr(prm.err, kErrSaturated);
    sat = false;
  };
  const int row0 = li * 64 + lane;
  uint32_t lc = 0, n_ag = 0;
  for (uint32_t tb = 0;; ++tb) {
    int tile;
    if (li == 0) {
      if (lane == 0) ls.tile[tb & 1] = schedule_tile(prm, atomicAdd(prm.next_tile, 1u));
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_SCHED + (tb & 1)));
    } else if (!warp_wait<true>(bar(B_SCHED + (tb & 1)), (tb >> 1) & 1, abort_flag)) {
      return;
    }
    tile = *reinterpret_cast<volatile int*>(&ls.tile[tb & 1]);
    report_sat();  // the previous tile's inputs
    if (tile >= prm.total_tiles) {
      if (lane == 0) {
        ls.ns[tb & 1][li] = 0;
        mbar_arrive(bar(B_TILE + (tb & 1)));
      }
      return;
    }
    const FusedFrame& F = frame_of(prm, tile);
    const uint32_t* ent = prm.plan + static_cast<size_t>(tile) * kTile;
    uint32_t pix[kRowsPerLoadLane];
    int cnt[kRowsPerLoadLane];
    bool has[kRowsPerLoadLane];
    int cmax = 0;
#pragma unroll
    for (int i = 0; i < kRowsPerLoadLane; ++i) {
      const uint32_t e = __ldg(ent + row0 + 32 * i);
      has[i] = e != kPlanEmpty;
      pix[i] = has[i] ? (e & kPlanPixelMask) : 0u;
      cnt[i] = has[i] ? static_cast<int>(e >> 28) : 0;
      cmax = max(cmax, cnt[i]);
      ls.cnt[tb & 1][row0 + 32 * i] = static_cast<uint8_t>(cnt[i]);
    }
    const int wmax = __reduce_max_sync(0xffffffffu, cmax);
    if (lane == 0) ls.ns[tb & 1][li] = wmax;
    __syncwarp();
    if (lane == 0) mbar_arrive(bar(B_TILE + (tb & 1)));
    if (!warp_wait<true>(bar(B_TILE + (tb & 1)), (tb >> 1) & 1, abort_flag)) return;
    const int ns = max(ls.ns[tb & 1][0], ls.ns[tb & 1][1]);

    // the G-buffer rows, loads in flight now (encoded inputs: loaded when
    // B1's operand is written, which keeps the slot loop's registers free)
    float gv[kRowsPerLoadLane][kGC];
    auto load_g = [&]() {
      const uint32_t P = static_cast<uint32_t>(F.P);
#pragma unroll
      for (int i = 0; i < kRowsPerLoadLane; ++i)
#pragma unroll
        for (int ch = 0; ch < kGC; ++ch)
          gv[i][ch] = has[i] ? __ldg(F.gbuf + (static_cast<uint32_t>(ch) * P + pix[i])) : 0.0f;
    };
    if constexpr (!PE) load_g();
    // B1's G-buffer operand: the 14 channels as codes of g[c] / s_g[c], then zeros
    auto put_ag = [&]() -> bool {
      if constexpr (PE) load_g();
      if (!warp_wait<true>(bar(B_AG_E), (n_ag & 1) ^ 1, abort_flag)) return false;
      ++n_ag;
      // with encoding a loop over the rows, each row's values picked by
      // selects: one copy of the (long) encoding code, which keeps the
      // loaders from evicting the other warps' loops from the instruction
      // cache (an indexed register array would go to local memory)
      static_assert(kRowsPerLoadLane == 2, "the row selects below assume two rows per lane");
      if constexpr (PE) {
#pragma unroll 1
        for (int i = 0; i < kRowsPerLoadLane; ++i) {
          float g[kGC];
#pragma unroll
          for (int c = 0; c < kGC; ++c) g[c] = i == 0 ? gv[0][c] : gv[1][c];
          uint32_t w[32];
          encode_row_f8(g, inv_s_g_sm, nf, w, sat);
          store_row_k128(sbase + L::ag, row0 + 32 * i, w);
        }
      } else {
#pragma unroll
        for (int i = 0; i < kRowsPerLoadLane; ++i) {
          float v[kGC];
          scale_inputs(gv[i], inv_s_g, v, sat);
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 3; ++j)
            w[j] = pack_u16x2(pack_e4m3(v[4 * j], v[4 * j + 1]), pack_e4m3(v[4 * j + 2], v[4 * j + 3]));
          w[3] = pack_u16x2(pack_e4m3(v[12], v[13]), 0);
          sts128(sbase + L::ag + static_cast<uint32_t>(row0 + 32 * i) * 16u, w[0], w[1], w[2], w[3]);
        }
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_AG_F));
      return true;
    };

    float x[kRowsPerLoadLane][kTC], y[kRowsPerLoadLane][kTC];
    if (ns > 0) load_slot_f8(F, 0, pix, cnt, x);
    const int ag_after = min(ns, 2) - 1;
    if (ag_after < 0 && !put_ag()) return;
    for (int k = 0; k < ns; ++k, ++lc) {
      if (k + 1 < ns) load_slot_f8(F, k + 1, pix, cnt, y);
      const int b = lc & 1;
      if (!warp_wait<true>(bar(B_AT_E + b), ((lc >> 1) & 1) ^ 1, abort_flag)) return;
      if constexpr (PE) {
#pragma unroll 1
        for (int i = 0; i < kRowsPerLoadLane; ++i) {  // one copy of the code (see put_ag)
          uint32_t w[32];
          if (__any_sync(0xffffffffu, k < (i == 0 ? cnt[0] : cnt[1]))) {
            float xr[kTC];
#pragma unroll
            for (int c = 0; c < kTC; ++c) xr[c] = i == 0 ? x[0][c] : x[1][c];
            encode_row_f8(xr, inv_s_t_sm, nf, w, sat);
          } else {  // no row of this warp has slot k: zeros (the loaded values are zeros)
#pragma unroll
            for (int j = 0; j < 32; ++j) w[j] = 0u;
          }
          store_row_k128(sbase + (b ? L::at1 : L::at0), row0 + 32 * i, w);
        }
      } else {
        store_slot_f8(sbase + (b ? L::at1 : L::at0), row0, inv_s_t, x, sat);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_AT_F + b));
      if (k == ag_after && !put_ag()) return;
#pragma unroll
      for (int i = 0; i < kRowsPerLoadLane; ++i)
#pragma unroll
        for (int ch = 0; ch < kTC; ++ch) x[i][ch] = y[i][ch];
    }
  }
}

// ------------------------------------------------------------------ kernel
// Sum: the paper's sum form of Eq. 5.  tau = s - 2^11 + c 2^-13 (the exact
// fixed-point sum) goes straight to B1's r operand as codes of tau / s_r,
// where rho's output would go; rho's GEMM and its epilogue pass are skipped
// and the max is not kept.
// R3: R's first layer is a 3x3 kernel over the frame (conv_r3.cu): the tile
// ends after B2, whose output goes to the frame's neural buffer as BF16 in
// real units ((acc s_B2 + b_B2) s_y2, ReLU) instead of R1's E4M3 operand.
template <int H, bool Sum, bool R3, bool PE>
__global__ void __launch_bounds__(kThreadsF, 1)
    fused_fp8_kernel(const __grid_constant__ FusedParams prm, const uint8_t* __restrict__ wimg) {
  static_assert(!(PE && R3), "the encoded inputs are built with the 1x1 R");
  using L = FusedLayoutF8<H, PE>;
  using T = TMapF8<H>;
  constexpr int CH = H / kEW;  // accumulator columns per epilogue thread
  constexpr int CHQ = CH / 4;  // TMEM columns of CH e4m3 values
  constexpr int CHC = CH / 2;  // bf16 pairs of the running max
  static_assert(CH % 16 == 0, "accumulator columns per thread must be a multiple of 16");

  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[B_COUNT_F8];
  __shared__ uint32_t s_tmem;
  __shared__ LoaderShared s_ld;
  __shared__ volatile int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar_base = smem_u32(&bars[0]);
  auto bar = [&](int i) { return bar_base + static_cast<uint32_t>(i) * 8u; };
  const float* cst = reinterpret_cast<const float*>(smem + L::cst);

  if (tid == 0) {
    mbar_init(bar(B_W), 1);
    mbar_init(bar(B_DP), 1);
    mbar_init(bar(B_DR2), 1);
    mbar_init(bar(B_AG_F), kLoadWarps);
    mbar_init(bar(B_AG_E), 1);
    mbar_init(bar(B_STALL8), 1);
    mbar_init(bar(B_DRAIN8), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(B_IN + b), kEpiWarps);
      mbar_init(bar(B_AT_F + b), kLoadWarps);
      mbar_init(bar(B_AT_E + b), 1);
      mbar_init(bar(B_TILE + b), kLoadWarps);
      mbar_init(bar(B_SCHED + b), 1);
    }
    for (int b = 0; b < 3; ++b) {
      mbar_init(bar(B_D1 + b), 1);
      mbar_init(bar(B_D2 + b), 1);
      mbar_init(bar(B_BE + b), kEpiWarps);
    }
    s_abort = 0;
    fence_mbar_init();
  }
  if (warp == kMmaWarp) {
    tmem_alloc(smem_u32(&s_tmem), T::NCOLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = s_tmem;

  if (warp >= kLoadWarp0) {
    // constant operands: K block 1 of the E4M3 A operands is zero; the BF16
    // [1, 1, 0, ...] operand multiplies the per-scene bias rows
    for (int r = (warp - kLoadWarp0) * 32 + lane; r < kTile; r += kLoadWarps * 32) {
      sts128(sbase + L::at0 + 2048u + r * 16u, 0u, 0u, 0u, 0u);
      sts128(sbase + L::at1 + 2048u + r * 16u, 0u, 0u, 0u, 0u);
      sts128(sbase + L::ag + 2048u + r * 16u, 0u, 0u, 0u, 0u);
      sts128(sbase + L::aone + r * 16u, pack_bf16(1.0f, 1.0f), 0u, 0u, 0u);
      sts128(sbase + L::aone + 2048u + r * 16u, 0u, 0u, 0u, 0u);
    }
    fence_proxy_async_smem();
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the tile plan is complete
    loader_loop_f8<H, PE>(prm, wimg, sbase, bar_base, s_ld, &s_abort, warp - kLoadWarp0, lane);
  } else if (warp == kMmaWarp) {
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
    constexpr uint32_t id8 = make_idesc(128, H, kFmtE4M3);
    constexpr uint32_t id816 = make_idesc(128, 16, kFmtE4M3);
    constexpr uint32_t idb = make_idesc(128, H, kFmtBF16);
    const uint64_t dsc_phi1 = make_sdesc(sbase + L::phi1, H * 16, 128);
    const uint64_t dsc_phi1b = make_sdesc(sbase + L::phi1b, H * 16, 128);
    const uint64_t dsc_phi2 = make_sdesc(sbase + L::phi2, H * 16, 128);
    const uint64_t dsc_rho = make_sdesc(sbase + L::rho, H * 16, 128);
    const uint64_t dsc_b1 = make_sdesc(sbase + L::b1, H * 16, 128);
    const uint64_t dsc_b1b = make_sdesc(sbase + L::b1b, H * 16, 128);
    const uint64_t dsc_b2 = make_sdesc(sbase + L::b2, H * 16, 128);
    const uint64_t dsc_r1 = make_sdesc(sbase + L::r1, H * 16, 128);
    const uint64_t dsc_r2 = make_sdesc(sbase + L::r2, 16 * 16, 128);
    const uint64_t dsc_at0 = make_sdesc(sbase + L::at0, 128 * 16, 128);
    const uint64_t dsc_at1 = make_sdesc(sbase + L::at1, 128 * 16, 128);
    const uint64_t dsc_one = make_sdesc(sbase + L::aone, 128 * 16, 128);
    const uint64_t dsc_ag = make_sdesc(sbase + L::ag, 128 * 16, 128);
    // B1's weights for r start after its 32-wide G-buffer block
    const uint64_t dsc_b1r = dsc_b1 + static_cast<uint64_t>(L::KG / 32) * ((2 * H * 16) >> 4);
    // D (+)= A (shared memory, K codes) x B^T: K / 32 steps, each advancing A
    // by two core-matrix columns of 128 rows (4096 bytes) and B by two of N
    // rows
    auto mma_ss_k = [&](uint32_t d, uint64_t a0, uint64_t b0, int K, uint32_t acc) {
      for (int t = 0; t < K / 32; ++t)
        mma_f8_ss_e(d, a0 + static_cast<uint64_t>(t) * (4096u >> 4),
                    b0 + static_cast<uint64_t>(t) * ((2 * H * 16) >> 4), id8, (t > 0 || acc) ? 1u : 0u);
    };
    SlotPos p1, p2;
    uint32_t g1 = 0, n_in = 0, n_agf = 0, tb = 0;
    const float* cur_fold = nullptr;
    auto phi1 = [&]() -> bool {
      if (!warp_wait<true>(bar(B_BE + p1.b), (p1.u & 1) ^ 1, &s_abort)) return false;
      const int a = g1 & 1;
      if (!warp_wait<true>(bar(B_AT_F + a), (g1 >> 1) & 1, &s_abort)) return false;
      tc_fence_after();
      const uint32_t d = tbase + T::buf(p1.b);
      mma_ss_k(d, a ? dsc_at1 : dsc_at0, dsc_phi1, L::KT, 0u);
      mma_f16_ss_e(d, dsc_one, dsc_phi1b, idb, 1u);
      mma_commit_e(bar(B_D1 + p1.b));
      mma_commit_e(bar(B_AT_E + a));
      __syncwarp();
      ++g1;
      p1.next();
      return true;
    };
    auto wait_in = [&]() -> bool {
      if (!warp_wait<true>(bar(B_IN + (n_in & 1)), (n_in >> 1) & 1, &s_abort)) return false;
      ++n_in;
      tc_fence_after();
      return true;
    };
    if (!warp_wait<true>(bar(B_W), 0, &s_abort)) goto done;
    // Test hook (stall_ns > 0, set by glassnet_debug_stall_next_render): a
    // wait on a barrier that nothing arrives on, before any MMA is issued.
    if (prm.stall_ns > 0 && !warp_wait<true>(bar(B_STALL8), 0, &s_abort, prm.stall_ns)) goto done;
    for (;; ++tb) {
      if (!warp_wait<true>(bar(B_TILE + (tb & 1)), (tb >> 1) & 1, &s_abort)) goto done;
      const int tile = *reinterpret_cast<volatile int*>(&s_ld.tile[tb & 1]);
      if (tile >= prm.total_tiles) break;
      const int ns = max(s_ld.ns[tb & 1][0], s_ld.ns[tb & 1][1]);
      const FusedFrame& F = frame_of(prm, tile);
      if (F.fold != cur_fold) {
        // Per-scene biases in accumulator units -> the BF16 bias operands,
        // once no MMA of the previous tile can still read them.
        if (tb > 0 && !warp_wait<true>(bar(B_DR2), (tb - 1) & 1, &s_abort)) goto done;
        for (int i = lane; i < 2 * H; i += 32) {
          const int n = i < H ? i : i - H;
          const float cv = F.fold[i] * cst[(i < H ? L::U_PHI1 : L::U_B1) + n];
          const float hi = bf16_value(cv);
          const uint32_t packed = static_cast<uint32_t>(bf16_bits(hi)) |
                                  (static_cast<uint32_t>(bf16_bits(cv - hi)) << 16);
          *reinterpret_cast<uint32_t*>(smem + (i < H ? L::phi1b : L::b1b) + n * 16) = packed;
        }
        fence_proxy_async_smem();
        __syncwarp();
        cur_fold = F.fold;
      }
      for (int k = 0; k < ns && k < 2; ++k)
        if (!phi1()) goto done;
      for (int k = 0; k < ns; ++k) {
        if (!wait_in()) goto done;  // U(k) written, its buffer read
        issue_gemm_f8<H, H>(tbase + T::buf(p2.b), tbase + (k & 1 ? T::AU1 : T::AU0), dsc_phi2,
                            id8);
        mma_commit_e(bar(B_D2 + p2.b));
        __syncwarp();
        p2.next();
        if (k + 2 < ns && !phi1()) goto done;
      }
      const uint32_t X = tbase + T::buf(p1.b);
      const uint32_t Y = tbase + T::buf(p1.b == 2 ? 0 : p1.b + 1);
      const uint32_t Z = tbase + T::buf(p1.b == 0 ? 2 : p1.b - 1);
#pragma unroll
      for (int l = Sum ? 1 : 0; l < (R3 ? 3 : 4); ++l) {
        if (!wait_in()) goto done;
        if (l == 1) {
          if (!warp_wait<true>(bar(B_AG_F), n_agf & 1, &s_abort)) goto done;
          ++n_agf;
          tc_fence_after();
        }
        if (l == 0) issue_gemm_f8<H, 2 * H>(X, tbase + T::APOOL, dsc_rho, id8);
        if (l == 1) {
          mma_ss_k(X, dsc_ag, dsc_b1, L::KG, 0u);
          issue_gemm_f8<H, H>(X, Y, dsc_b1r, id8, true);
          mma_f16_ss_e(X, dsc_one, dsc_b1b, idb, 1u);
        }
        if (l == 2) issue_gemm_f8<H, H>(X, Y + H / 2, dsc_b2, id8);
        if (l == 3) issue_gemm_f8<H, H>(X, Z, dsc_r1, id8);
        mma_commit_e(bar(B_DP));
        if (l == 1) mma_commit_e(bar(B_AG_E));
        __syncwarp();
      }
      if (!wait_in()) goto done;  // R2's operand written (3x3 R: B2's accumulator read)
      if constexpr (!R3) issue_gemm_f8<16, H>(Z + H / 2, Y + H / 2, dsc_r2, id816);
      mma_commit_e(bar(B_DR2));
      __syncwarp();
    }
  } else {
    // ------------------------------------------------------- epilogue warps
    const int q = warp & 3, g = warp >> 2;
    const int row = q * 32 + lane;
    const uint32_t tl = tbase + (static_cast<uint32_t>(q * 32) << 16);
    const float* s_phi1 = cst + L::S_PHI1 + g * CH;
    const float* s_phi2 = cst + L::S_PHI2 + g * CH;
    const float* b_phi2 = cst + L::B_PHI2 + g * CH;
    uint32_t gs = 0;
    uint32_t n_in = 0, n_dp = 0, tb = 0;
    auto arrive_in = [&]() {
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_IN + (n_in & 1)));
      ++n_in;
    };
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the tile plan is complete
    if (!warp_wait<true>(bar(B_W), 0, &s_abort)) goto done;
    {
      const float inv_s_pool = cst[L::INV_S_POOL];
      for (;; ++tb) {
        if (!warp_wait<true>(bar(B_TILE + (tb & 1)), (tb >> 1) & 1, &s_abort)) goto done;
        const int tile = *reinterpret_cast<volatile int*>(&s_ld.tile[tb & 1]);
        if (tile >= prm.total_tiles) break;
        const int ns = max(s_ld.ns[tb & 1][0], s_ld.ns[tb & 1][1]);
        const int c = s_ld.cnt[tb & 1][row];

        uint32_t mx[CHC];
        float sm[CH];
#pragma unroll
        for (int j = 0; j < CHC; ++j) mx[j] = 0u;
#pragma unroll
        for (int j = 0; j < CH; ++j) sm[j] = kSumBase;

        // phi1(k) accumulator -> U(k) codes (the bias is in the accumulator)
        auto epi1 = [&](int k) -> bool {
          const uint32_t gk = gs + k, b = gk % 3u;
          if (!warp_wait<true>(bar(B_D1 + b), (gk / 3u) & 1, &s_abort)) return false;
          tc_fence_after();
          const uint32_t src = tl + T::buf(b) + g * CH;
          const uint32_t dst = tl + (k & 1 ? T::AU1 : T::AU0) + g * CHQ;
          uint32_t ra[16], rb[16];
          tmem_ld16_async(src, ra);
          tmem_wait_ld_tied(ra);
#pragma unroll
          for (int hh = 0; hh < CH / 16; ++hh) {
            uint32_t(&cur)[16] = (hh & 1) ? rb : ra;
            uint32_t(&nxt)[16] = (hh & 1) ? ra : rb;
            if (hh + 1 < CH / 16) tmem_ld16_async(src + (hh + 1) * 16, nxt);
            uint32_t u[4];
            quant16(cur, s_phi1 + hh * 16, nullptr, false, u);
            tmem_st4(dst + hh * 4, u);
            if (hh + 1 < CH / 16) tmem_wait_ld_tied(nxt);
          }
          arrive_in();
          return true;
        };
        // phi2(k) accumulator -> v = acc s + b (real units) -> pool update
        auto epi2 = [&](int k) -> bool {
          const uint32_t gk = gs + k, b = gk % 3u;
          if (!warp_wait<true>(bar(B_D2 + b), (gk / 3u) & 1, &s_abort)) return false;
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
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(bar(B_BE + b));
            }
            if (k < c) {
#pragma unroll
              for (int i = 0; i < 16; i += 2) {
                const int j = hh * 16 + i;
                float v0, v1;
                ffma2(v0, v1, __uint_as_float(cur[i]), __uint_as_float(cur[i + 1]), s_phi2[j],
                      s_phi2[j + 1], b_phi2[j], b_phi2[j + 1]);
                const uint32_t u = pack_bf16_relu(v0, v1);
                if constexpr (!Sum) mx[j / 2] = bmax2(mx[j / 2], u);
                add_bf16x2_rz(sm[j], sm[j + 1], u);
              }
            }
            if (hh + 1 < CH / 16) tmem_wait_ld_tied(nxt);
          }
          return true;
        };

        if (ns > 0 && !epi1(0)) goto done;
        for (int k = 0; k < ns; ++k) {
          if (k + 1 < ns && !epi1(k + 1)) goto done;
          if (!epi2(k)) goto done;
        }

        if constexpr (Sum) {
          // tau -> the r operand of B1 (buffer Y, see below) as codes of
          // tau / s_r
          const uint32_t Yr = tl + T::buf((gs + ns) % 3u == 2 ? 0 : (gs + ns) % 3u + 1);
          const float inv_s_r = cst[L::INV_S_R];
          const float off = kSumBase - static_cast<float>(c) * kHalfQuantum;
          bool over = false;
#pragma unroll
          for (int hh = 0; hh < CH / 16; ++hh) {
            uint32_t u[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              float a[4];
#pragma unroll
              for (int t = 0; t < 4; t += 2) {
                const int e = hh * 16 + 4 * j + t;
                over |= !(fmaxf(sm[e], sm[e + 1]) < kSumLimit);
                float d0, d1;
                fadd2_rn(d0, d1, sm[e], sm[e + 1], -off, -off);
                a[t] = d0 * inv_s_r;
                a[t + 1] = d1 * inv_s_r;
              }
              u[j] = pack_u16x2(pack_e4m3_relu(a[0], a[1]), pack_e4m3_relu(a[2], a[3]));
            }
            tmem_st4(Yr + g * CHQ + hh * 4, u);
          }
          if (over && c > 0) atomicOr(prm.err, kErrRange);
        } else
        // pool = [max ; mean] -> APOOL as codes of pool / s_pool
        {
          const float rcp = c > 0 ? __frcp_rn(static_cast<float>(c)) : 0.0f;
          const float off = kSumBase - static_cast<float>(c) * kHalfQuantum;
          bool over = false;
#pragma unroll
          for (int hh = 0; hh < CHQ / 4; ++hh) {
            uint32_t pm[4], pa[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int e = hh * 16 + 4 * j;  // first of 4 pooled values
              float a[4], m[4];
#pragma unroll
              for (int t = 0; t < 4; t += 2) {
                over |= !(fmaxf(sm[e + t], sm[e + t + 1]) < kSumLimit);
                float d0, d1;
                fadd2_rn(d0, d1, sm[e + t], sm[e + t + 1], -off, -off);
                a[t] = d0 * rcp * inv_s_pool;
                a[t + 1] = d1 * rcp * inv_s_pool;
                const uint32_t mp = mx[(e + t) / 2];
                m[t] = __uint_as_float(mp << 16) * inv_s_pool;
                m[t + 1] = __uint_as_float(mp & 0xffff0000u) * inv_s_pool;
              }
              pm[j] = pack_u16x2(pack_e4m3_relu(m[0], m[1]), pack_e4m3_relu(m[2], m[3]));
              pa[j] = pack_u16x2(pack_e4m3_relu(a[0], a[1]), pack_e4m3_relu(a[2], a[3]));
            }
            tmem_st4(tl + T::APOOL + g * CHQ + hh * 4, pm);
            tmem_st4(tl + T::APOOL + H / 4 + g * CHQ + hh * 4, pa);
          }
          if (over && c > 0) atomicOr(prm.err, kErrRange);
        }
        arrive_in();

        // rho -> r (zero without layers) -> Y;  B1 -> y -> Y + H/2;
        // B2 -> y2 -> Z;  R1 -> q -> Y + H/2.  Accumulator X.
        gs += ns;
        const uint32_t r3 = gs % 3u;
        const uint32_t X = tl + T::buf(r3);
        const uint32_t Y = tl + T::buf(r3 == 2 ? 0 : r3 + 1);
        const uint32_t Z = tl + T::buf(r3 == 0 ? 2 : r3 - 1);
        // 3x3 R: this row's pixel in its frame's neural buffer (chunk c of 8
        // channels at phi_px + c w)
        uint4* phi_px = nullptr;
        uint32_t fw = 0;
        if constexpr (R3) {
          const FusedFrame& Fr = frame_of(prm, tile);
          fw = static_cast<uint32_t>(Fr.w);
          const uint32_t e = __ldg(prm.plan + static_cast<size_t>(tile) * kTile + row);
          if (e != kPlanEmpty) {
            const uint32_t pix = e & kPlanPixelMask;
            const uint32_t py = pix / fw;
            phi_px = reinterpret_cast<uint4*>(Fr.phi) + static_cast<size_t>(py) * (H / 8) * fw +
                     (pix - py * fw);
          }
        }
#pragma unroll
        for (int l = Sum ? 1 : 0; l < (R3 ? 3 : 4); ++l) {
          if (!warp_wait<true>(bar(B_DP), n_dp & 1, &s_abort)) goto done;
          ++n_dp;
          tc_fence_after();
          const float* sl = cst + (l == 0 ? L::S_RHO : l == 1 ? L::S_B1 : l == 2 ? L::S_B2 : L::S_R1) + g * CH;
          const float* bl = l == 1 ? nullptr
                                   : cst + (l == 0 ? L::B_RHO : l == 2 ? L::B_B2 : L::B_R1) + g * CH;
          const uint32_t src = X + g * CH;
          const uint32_t dst = (l == 0 ? Y : (l == 2 ? Z : Y + H / 2)) + g * CHQ;
          uint32_t ra[16], rb[16];
          tmem_ld16_async(src, ra);
          tmem_wait_ld_tied(ra);
#pragma unroll
          for (int hh = 0; hh < CH / 16; ++hh) {
            uint32_t(&cur)[16] = (hh & 1) ? rb : ra;
            uint32_t(&nxt)[16] = (hh & 1) ? ra : rb;
            if (hh + 1 < CH / 16) tmem_ld16_async(src + (hh + 1) * 16, nxt);
            if (R3 && l == 2) {  // y2 in real units -> the neural buffer (BF16)
              if (phi_px) {
                const float s_y2 = cst[L::S_Y2];
                uint32_t v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                  float y0, y1;
                  ffma2(y0, y1, __uint_as_float(cur[2 * i]), __uint_as_float(cur[2 * i + 1]),
                        sl[hh * 16 + 2 * i], sl[hh * 16 + 2 * i + 1], bl[hh * 16 + 2 * i],
                        bl[hh * 16 + 2 * i + 1]);
                  v[i] = pack_bf16_relu(y0 * s_y2, y1 * s_y2);
                }
                const size_t c8 = static_cast<size_t>(g * CH + hh * 16) / 8;
                phi_px[c8 * fw] = make_uint4(v[0], v[1], v[2], v[3]);
                phi_px[(c8 + 1) * fw] = make_uint4(v[4], v[5], v[6], v[7]);
              }
            } else {
              uint32_t u[4];
              quant16(cur, sl + hh * 16, bl ? bl + hh * 16 : nullptr, l == 0 && c == 0, u);
              tmem_st4(dst + hh * 4, u);
            }
            if (hh + 1 < CH / 16) tmem_wait_ld_tied(nxt);
          }
          arrive_in();
        }
        // R2 + sigmoid -> out (column group 0 stores)
        const uint32_t ent = g == 0 ? __ldg(prm.plan + static_cast<size_t>(tile) * kTile + row)
                                    : kPlanEmpty;
        if (!warp_wait<true>(bar(B_DR2), tb & 1, &s_abort)) goto done;
        if (!R3 && g == 0) {
          tc_fence_after();
          uint32_t r[4];
          tmem_ld4(Z + H / 2, r);
          if (ent != kPlanEmpty) {
            const FusedFrame& F = frame_of(prm, tile);
            const uint32_t pix = ent & kPlanPixelMask;
#pragma unroll
            for (int j = 0; j < kOut; ++j) {
              const float y = fmaf(__uint_as_float(r[j]), cst[L::S_R2 + j], cst[L::B_R2 + j]);
              F.out[static_cast<size_t>(j) * F.P + pix] = 1.0f / (1.0f + expf(-y));
            }
          }
        }
      }
    }
  }
done:
  tc_fence_before();
  __syncthreads();  // every warp is here: s_abort is final
  if (s_abort) {
    // nothing of this CTA may be in flight when its TMEM is freed
    if (warp == kMmaWarp) drain_async(bar(B_W), bar(B_DRAIN8));
    if (tid == 0) report_timeout(prm.err, s_abort, bar_base, kKernelFusedFp8, 0);
  }
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tbase, TMapF8<H>::NCOLS);
  }
}

template <int H, bool Sum, bool R3, bool PE = false>
cudaError_t prepare_f8() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fused_fp8_kernel<H, Sum, R3, PE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       FusedLayoutF8<H, PE>::smem_bytes);
  if (e == cudaSuccess) done = true;
  return e;
}

template <int H, bool Sum, bool R3, bool PE = false>
cudaError_t launch_f8(const void* wimg, const FusedParams& p, cudaStream_t s, int grid) {
  cudaError_t e = prepare_f8<H, Sum, R3, PE>();
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreadsF);
  cfg.dynamicSmemBytes = FusedLayoutF8<H, PE>::smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fused_fp8_kernel<H, Sum, R3, PE>, p,
                            static_cast<const uint8_t*>(wimg));
}

template <int H>
cudaError_t prepare_all_f8() {
  cudaError_t e = prepare_f8<H, false, false>();
  if (e == cudaSuccess) e = prepare_f8<H, true, false>();
  if (e == cudaSuccess) e = prepare_f8<H, false, true>();
  if (e == cudaSuccess) e = prepare_f8<H, true, true>();
  if (e == cudaSuccess) e = prepare_f8<H, false, false, true>();
  if (e == cudaSuccess) e = prepare_f8<H, true, false, true>();
  return e;
}

template <int H>
cudaError_t launch_h_f8(const void* wimg, const FusedParams& p, cudaStream_t s, int grid) {
  if (p.pe_freqs > 0) {  // encoded inputs (1x1 R only; the loader encodes up to 4 frequencies)
    if (p.f[0].phi || p.pe_freqs > kMaxPeFreqsFused) return cudaErrorInvalidValue;
    return p.pool_sum ? launch_f8<H, true, false, true>(wimg, p, s, grid)
                      : launch_f8<H, false, false, true>(wimg, p, s, grid);
  }
  if (p.f[0].phi)  // 3x3 R: the neural buffer out
    return p.pool_sum ? launch_f8<H, true, true>(wimg, p, s, grid)
                      : launch_f8<H, false, true>(wimg, p, s, grid);
  return p.pool_sum ? launch_f8<H, true, false>(wimg, p, s, grid)
                    : launch_f8<H, false, false>(wimg, p, s, grid);
}

}  // namespace

cudaError_t prepare_fused_fp8(int H) {
  device_sm_count();
  return H == 128 ? prepare_all_f8<128>() : prepare_all_f8<64>();
}

cudaError_t launch_fused_fp8(int H, const void* wimg, const FusedParams& params, cudaStream_t s) {
  if (params.total_tiles <= 0) return cudaSuccess;
  FusedParams p = params;
  cudaError_t e = launch_plan(p, s);
  if (e != cudaSuccess) return e;
  const int grid = p.total_tiles < device_sm_count() ? p.total_tiles : device_sm_count();
  return H == 128 ? launch_h_f8<128>(wimg, p, s, grid) : launch_h_f8<64>(wimg, p, s, grid);
}

}  // namespace gn

// C ABI of the GlassNet library: argument checks, weight-blob validation and
// packing, model / latent objects, and dispatch to the kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace {

thread_local std::string g_last_error;

// The BF16 neural buffer of a 3x3 R render: [h][H/8][w][8], 256-byte rounded.
size_t phi_bytes(const gn_model* m, int h, int w) {
  return (static_cast<size_t>(h) * w * m->H * 2 + 255) / 256 * 256;
}

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(GN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

uint64_t fnv1a64(const uint8_t* p, size_t n) {
  uint64_t h = 0xcbf29ce484222325ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001b3ull;
  }
  return h;
}

// Round-to-nearest-even float -> bf16 bits (host).
uint16_t bf16_rne(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;  // NaN
  const uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
  return static_cast<uint16_t>(r >> 16);
}

// Element (n, k) of an N x K operand in the [K/8][N][8] core-matrix layout.
inline size_t core_idx(int N, int n, int k) {
  return (static_cast<size_t>(k / 8) * N + n) * 8 + (k % 8);
}

// With positional encoding, band t of phi1's input (12 encoded values) and of
// B1's G-buffer block (14) go to K columns 16 t .. (FusedLayout); r follows
// the last band.
template <int H, bool PE>
std::vector<uint8_t> pack_fused_bf16(const float* w, const gn::WeightIndex& wi) {
  using L = gn::FusedLayout<H, PE>;
  const int nb = wi.bands();
  std::vector<uint8_t> img(L::bytes, 0);
  auto put = [&](uint32_t off, int N, int n, int k, float v) {
    uint16_t b = bf16_rne(v);
    std::memcpy(img.data() + off + core_idx(N, n, k) * 2, &b, 2);
  };
  auto W = [&](int l, int n, int j) { return w[wi.w[l] + static_cast<size_t>(n) * wi.in[l] + j]; };
  for (int n = 0; n < H; ++n) {
    for (int t = 0; t < nb; ++t)
      for (int k = 0; k < gn::kTC; ++k) put(L::phi1, H, n, 16 * t + k, W(gn::LPHI1, n, t * gn::kTC + k));
    for (int k = 0; k < H; ++k) put(L::phi2, H, n, k, W(gn::LPHI2, n, k));
    for (int k = 0; k < 2 * H; ++k) put(L::rho, H, n, k, W(gn::LRHO, n, k));
    for (int t = 0; t < nb; ++t)
      for (int k = 0; k < gn::kGC; ++k) put(L::b1, H, n, 16 * t + k, W(gn::LB1, n, t * gn::kGC + k));
    for (int k = 0; k < H; ++k) put(L::b1, H, n, 16 * nb + k, W(gn::LB1, n, wi.gc_enc() + k));
    for (int k = 0; k < H; ++k) put(L::b2, H, n, k, W(gn::LB2, n, k));
    for (int k = 0; k < H; ++k) put(L::r1, H, n, k, W(gn::LR1, n, k));
  }
  for (int n = 0; n < gn::kOut; ++n)
    for (int k = 0; k < H; ++k) put(L::r2, 16, n, k, W(gn::LR2, n, k));
  for (int n = 0; n < H; ++n) {  // phi2 bias as hi + lo BF16 rows of a K = 16 operand
    const float b = w[wi.b[gn::LPHI2] + n];
    uint16_t hb = bf16_rne(b);
    uint32_t hu = static_cast<uint32_t>(hb) << 16;
    float hf;
    std::memcpy(&hf, &hu, 4);
    put(L::phi2b, H, n, 0, hf);
    put(L::phi2b, H, n, 1, b - hf);
  }
  float* bias = reinterpret_cast<float*>(img.data() + L::bias);
  for (int n = 0; n < H; ++n) {
    bias[n] = w[wi.b[gn::LPHI2] + n];
    bias[H + n] = w[wi.b[gn::LRHO] + n];
    bias[2 * H + n] = w[wi.b[gn::LB2] + n];
    bias[3 * H + n] = w[wi.b[gn::LR1] + n];
  }
  for (int n = 0; n < gn::kOut; ++n) bias[4 * H + n] = w[wi.b[gn::LR2] + n];
  return img;
}

// Image of the doubled widths with positional encoding (FusedLayout<128,
// true>): the resident block (phi1 with every band, phi2, band 0 of B1's
// G-buffer block, phi2b, the biases), then the per-pixel weights in chunks of
// K = 64 rows, each chunk the slice [8 k0 / 64 ...][N][8] of the layer's
// [K/8][N][8] operand, streamed through the kernel's shared-memory ring.
std::vector<uint8_t> pack_fused_bf16_stream(const float* w, const gn::WeightIndex& wi) {
  using L = gn::FusedLayout<128, true>;
  constexpr int H = 128;
  const int nb = wi.bands();
  std::vector<uint8_t> img(L::img_bytes, 0);
  auto put = [&](uint32_t off, int N, int n, int k, float v) {
    uint16_t b = bf16_rne(v);
    std::memcpy(img.data() + off + core_idx(N, n, k) * 2, &b, 2);
  };
  // K row k of a chunked operand starting at `base`
  auto put_chunked = [&](uint32_t base, int n, int k, float v) {
    put(base + static_cast<uint32_t>(k / 64) * L::kChunk, H, n, k % 64, v);
  };
  auto W = [&](int l, int n, int j) { return w[wi.w[l] + static_cast<size_t>(n) * wi.in[l] + j]; };
  for (int n = 0; n < H; ++n) {
    for (int t = 0; t < nb; ++t)
      for (int k = 0; k < gn::kTC; ++k) put(L::phi1, H, n, 16 * t + k, W(gn::LPHI1, n, t * gn::kTC + k));
    for (int k = 0; k < H; ++k) put(L::phi2, H, n, k, W(gn::LPHI2, n, k));
    for (int k = 0; k < gn::kGC; ++k) put(L::b1, H, n, k, W(gn::LB1, n, k));
    for (int k = 0; k < 2 * H; ++k) put_chunked(L::img_rho, n, k, W(gn::LRHO, n, k));
    for (int t = 1; t < nb; ++t)  // band t at K 16 (t - 1) of the bands' chunks
      for (int k = 0; k < gn::kGC; ++k)
        put_chunked(L::img_b1g, n, 16 * (t - 1) + k, W(gn::LB1, n, t * gn::kGC + k));
    for (int k = 0; k < H; ++k) put_chunked(L::img_b1r, n, k, W(gn::LB1, n, wi.gc_enc() + k));
    for (int k = 0; k < H; ++k) put_chunked(L::img_b2, n, k, W(gn::LB2, n, k));
    for (int k = 0; k < H; ++k) put_chunked(L::img_r1, n, k, W(gn::LR1, n, k));
  }
  for (int n = 0; n < gn::kOut; ++n)
    for (int k = 0; k < H; ++k) put(L::img_r2, 16, n, k, W(gn::LR2, n, k));
  for (int n = 0; n < H; ++n) {  // phi2 bias as hi + lo BF16 rows of a K = 16 operand
    const float b = w[wi.b[gn::LPHI2] + n];
    uint16_t hb = bf16_rne(b);
    uint32_t hu = static_cast<uint32_t>(hb) << 16;
    float hf;
    std::memcpy(&hf, &hu, 4);
    put(L::phi2b, H, n, 0, hf);
    put(L::phi2b, H, n, 1, b - hf);
  }
  float* bias = reinterpret_cast<float*>(img.data() + L::bias);
  for (int n = 0; n < H; ++n) {
    bias[n] = w[wi.b[gn::LPHI2] + n];
    bias[H + n] = w[wi.b[gn::LRHO] + n];
    bias[2 * H + n] = w[wi.b[gn::LB2] + n];
    bias[3 * H + n] = w[wi.b[gn::LR1] + n];
  }
  for (int n = 0; n < gn::kOut; ++n) bias[4 * H + n] = w[wi.b[gn::LR2] + n];
  return img;
}

// Image of the 3x3 R kernel (conv_r3.cu): per tap t = (dy + 1) 3 + dx + 1
// the [H/8][H][8] BF16 B operand of W_R1[:, :, dy + 1, dx + 1] (the blob
// stores R1 as [H][H 9], column k 9 + t), then in FP32 b_R1 [H], W_R2 [3][H]
// (rounded to BF16, the precision of every other weight operand) and b_R2
// [4] (3 used).
std::vector<uint8_t> pack_conv_r3(const float* w, const gn::WeightIndex& wi) {
  const int H = wi.H;
  std::vector<uint8_t> img(gn::conv_r3_image_bytes(H), 0);
  const size_t tap_bytes = static_cast<size_t>(H) * H * 2;
  auto put = [&](size_t off, int N, int n, int k, float v) {
    uint16_t b = bf16_rne(v);
    std::memcpy(img.data() + off + core_idx(N, n, k) * 2, &b, 2);
  };
  const float* W1 = w + wi.w[gn::LR1];
  for (int t = 0; t < 9; ++t)
    for (int n = 0; n < H; ++n)
      for (int k = 0; k < H; ++k) put(t * tap_bytes, H, n, k, W1[static_cast<size_t>(n) * 9 * H + k * 9 + t]);
  float* tail = reinterpret_cast<float*>(img.data() + 9 * tap_bytes);
  for (int n = 0; n < H; ++n) tail[n] = w[wi.b[gn::LR1] + n];
  for (int n = 0; n < gn::kOut; ++n)
    for (int k = 0; k < H; ++k) {
      const uint32_t u = static_cast<uint32_t>(bf16_rne(w[wi.w[gn::LR2] + static_cast<size_t>(n) * H + k])) << 16;
      std::memcpy(&tail[H + n * H + k], &u, 4);
    }
  for (int n = 0; n < gn::kOut; ++n) tail[4 * H + n] = w[wi.b[gn::LR2] + n];
  return img;
}

// Round-to-nearest-even float -> E4M3 code (1 sign, 4 exponent bits with bias
// 7, 3 mantissa bits; largest finite 448, no infinities), saturating to
// +-448 (the satfinite rule).  NaN -> 0x7f.
uint8_t e4m3_rne(float f) {
  if (std::isnan(f)) return 0x7f;
  const uint8_t sign = std::signbit(f) ? 0x80 : 0x00;
  const double a = std::fabs(static_cast<double>(f));
  if (a >= 448.0) return sign | 0x7e;
  int code;
  if (a < std::ldexp(1.0, -6)) {
    code = static_cast<int>(std::nearbyint(a / std::ldexp(1.0, -9)));  // subnormal steps of 2^-9
  } else {
    int e;
    const double m = std::frexp(a, &e);  // a = m 2^e, m in [0.5, 1)
    // a = (1 + f) 2^(e-1): mantissa steps of 2^(e-4)
    double q = std::nearbyint(a / std::ldexp(1.0, e - 4));  // in [8, 16]
    int ex = e - 1;
    if (q >= 16.0) {
      q = 8.0;
      ex += 1;
    }
    const int field = ex + 7;
    code = (field << 3) | (static_cast<int>(q) - 8);
    (void)m;
  }
  if (code > 0x7e) code = 0x7e;
  return sign | static_cast<uint8_t>(code);
}

// Element (n, k) of an N x K E4M3 operand in the [K/16][N][16] layout.
inline size_t core_idx8(int N, int n, int k) {
  return (static_cast<size_t>(k / 16) * N + n) * 16 + (k % 16);
}

// FP8 image (FusedLayoutF8) from the concat-form weights and the activation
// scales act[kFp8Acts] (per-channel t and g, then U, pool, r, y, y2, q).
template <int H, bool PE = false>
std::vector<uint8_t> pack_fused_fp8(const float* w, const gn::WeightIndex& wi, const float* act) {
  using L = gn::FusedLayoutF8<H, PE>;
  std::vector<uint8_t> img(L::bytes, 0);
  auto W = [&](int l, int n, int j) { return w[wi.w[l] + static_cast<size_t>(n) * wi.in[l] + j]; };
  auto Bv = [&](int l, int n) { return w[wi.b[l] + n]; };
  // per-output-channel weight scale over the columns that stay in the GEMM
  auto wscale = [&](int l, int n, int j0, int j1) {
    float m = 0.0f;
    for (int j = j0; j < j1; ++j) m = std::max(m, std::fabs(W(l, n, j)));
    return m > 0.0f ? m / 448.0f : 1.0f;
  };
  auto put = [&](uint32_t off, int N, int n, int k, float v) {
    img[off + core_idx8(N, n, k)] = e4m3_rne(v);
  };
  const float* s_t = act + gn::FP8_T0;
  const float* s_g = act + gn::FP8_G0;
  const float s_u = act[gn::FP8_U], s_pool = act[gn::FP8_POOL], s_r = act[gn::FP8_R],
              s_y = act[gn::FP8_Y], s_y2 = act[gn::FP8_Y2], s_q = act[gn::FP8_Q];
  float* c = reinterpret_cast<float*>(img.data() + L::cst);
  // Input column k of phi1's (B1's) first block is channel k % 12 (k % 14) of
  // band k / 12 (k / 14): band 0 enters as x / s[c], the sine and cosine bands
  // as v kFp8BandCode, so the column carries s[c] or 1 / kFp8BandCode.
  const int tce = wi.tc_enc(), gce = wi.gc_enc();
  auto col_t = [&](int k) { return k < gn::kTC ? s_t[k] : 1.0f / gn::kFp8BandCode; };
  auto col_g = [&](int k) { return k < gn::kGC ? s_g[k] : 1.0f / gn::kFp8BandCode; };
  for (int n = 0; n < H; ++n) {
    // phi1: column c of the weights carries the input channel's scale
    float m1 = 0.0f;
    for (int k = 0; k < tce; ++k) m1 = std::max(m1, std::fabs(W(gn::LPHI1, n, k) * col_t(k)));
    const float w1 = m1 > 0.0f ? m1 / 448.0f : 1.0f;
    for (int k = 0; k < tce; ++k) put(L::phi1, H, n, k, W(gn::LPHI1, n, k) * col_t(k) / w1);
    c[L::S_PHI1 + n] = w1 / s_u;
    c[L::U_PHI1 + n] = 1.0f / w1;
    const float w2 = wscale(gn::LPHI2, n, 0, H);
    for (int k = 0; k < H; ++k) put(L::phi2, H, n, k, W(gn::LPHI2, n, k) / w2);
    c[L::S_PHI2 + n] = s_u * w2;
    c[L::B_PHI2 + n] = Bv(gn::LPHI2, n);
    const float wr = wscale(gn::LRHO, n, 0, 2 * H);
    for (int k = 0; k < 2 * H; ++k) put(L::rho, H, n, k, W(gn::LRHO, n, k) / wr);
    c[L::S_RHO + n] = s_pool * wr / s_r;
    c[L::B_RHO + n] = Bv(gn::LRHO, n) / s_r;
    // B1: the G-buffer columns carry their channels' scales, the r columns s_r
    float mb = 0.0f;
    for (int k = 0; k < gce; ++k) mb = std::max(mb, std::fabs(W(gn::LB1, n, k) * col_g(k)));
    for (int k = 0; k < H; ++k) mb = std::max(mb, std::fabs(W(gn::LB1, n, gce + k) * s_r));
    const float wb1 = mb > 0.0f ? mb / 448.0f : 1.0f;
    for (int k = 0; k < gce; ++k) put(L::b1, H, n, k, W(gn::LB1, n, k) * col_g(k) / wb1);
    for (int k = 0; k < H; ++k) put(L::b1, H, n, L::KG + k, W(gn::LB1, n, gce + k) * s_r / wb1);
    c[L::S_B1 + n] = wb1 / s_y;
    c[L::U_B1 + n] = 1.0f / wb1;
    const float wb2 = wscale(gn::LB2, n, 0, H);
    for (int k = 0; k < H; ++k) put(L::b2, H, n, k, W(gn::LB2, n, k) / wb2);
    c[L::S_B2 + n] = s_y * wb2 / s_y2;
    c[L::B_B2 + n] = Bv(gn::LB2, n) / s_y2;
    const float wq1 = wscale(gn::LR1, n, 0, H);
    for (int k = 0; k < H; ++k) put(L::r1, H, n, k, W(gn::LR1, n, k) / wq1);
    c[L::S_R1 + n] = s_y2 * wq1 / s_q;
    c[L::B_R1 + n] = Bv(gn::LR1, n) / s_q;
  }
  for (int n = 0; n < gn::kOut; ++n) {
    const float wq2 = wscale(gn::LR2, n, 0, H);
    for (int k = 0; k < H; ++k) put(L::r2, 16, n, k, W(gn::LR2, n, k) / wq2);
    c[L::S_R2 + n] = s_q * wq2;
    c[L::B_R2 + n] = Bv(gn::LR2, n);
  }
  c[L::INV_S_R] = 1.0f / s_r;
  c[L::INV_S_POOL] = 1.0f / s_pool;
  c[L::S_Y2] = s_y2;
  for (int k = 0; k < gn::kTC; ++k) c[L::INV_S_TCH + k] = 1.0f / s_t[k];
  for (int k = 0; k < gn::kGC; ++k) c[L::INV_S_GCH + k] = 1.0f / s_g[k];
  return img;
}

bool aligned4(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) == 0; }

int check_frame(const gn_model* m, const gn_latent* lat, const float* gbuf, const float* tbuf,
                const uint8_t* cnt, int K, int h, int w, const float* out) {
  if (!m) return fail(GN_EINVAL, "model is NULL");
  if (!lat) return fail(GN_EINVAL, "latent is NULL");
  if (lat->H != m->H || lat->Z != m->Z)
    return fail(GN_EINVAL, "latent widths (%d, %d) do not match the model (%d, %d)", lat->H,
                lat->Z, m->H, m->Z);
  if (K < 0 || K > gn::kMaxK) return fail(GN_EINVAL, "K = %d outside 0..%d", K, gn::kMaxK);
  if (h < 1 || w < 1) return fail(GN_EINVAL, "frame %d x %d is empty", h, w);
  if (static_cast<long long>(h) * w * gn::kTC * (K > 0 ? K : 1) >= (1ll << 31))
    return fail(GN_EINVAL, "frame %d x %d x K=%d too large (12*K*h*w must be < 2^31)", h, w, K);
  if (!gbuf || !cnt || !out) return fail(GN_EINVAL, "gbuf, layer_count and out must be non-NULL");
  if (K > 0 && !tbuf) return fail(GN_EINVAL, "tbuf is NULL with K = %d", K);
  if (!aligned4(gbuf) || !aligned4(out) || (tbuf && !aligned4(tbuf)))
    return fail(GN_EINVAL, "gbuf, tbuf and out must be 4-byte aligned");
  return GN_OK;
}

}  // namespace

namespace gn {
// Records an error message for glassnet_last_error() from other translation units.
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace gn

extern "C" {

const char* glassnet_last_error(void) { return g_last_error.c_str(); }

int glassnet_load_weights(const void* blob, size_t nbytes, int precision, gn_model** out) {
  const gn_model_config cfg = {precision, GN_POOL_MAX_MEAN, 0, 1};
  return glassnet_load_weights_ex(blob, nbytes, &cfg, out);
}

namespace {
int load_weights_impl(const void* blob, size_t nbytes, const gn_model_config* cfg, gn_model** out,
                      gn_model** partial);
}  // namespace

// Host allocations (the weights' copy, the packed images) may fail with
// std::bad_alloc; nothing is thrown across the ABI.
int glassnet_load_weights_ex(const void* blob, size_t nbytes, const gn_model_config* cfg,
                             gn_model** out) {
  gn_model* partial = nullptr;
  try {
    return load_weights_impl(blob, nbytes, cfg, out, &partial);
  } catch (const std::bad_alloc&) {
    glassnet_free_model(partial);
    if (out) *out = nullptr;
    return fail(GN_ENOMEM, "host allocation failed");
  }
}

namespace {
int load_weights_impl(const void* blob, size_t nbytes, const gn_model_config* cfg, gn_model** out,
                      gn_model** partial) {
  if (!blob || !cfg || !out) return fail(GN_EINVAL, "blob, config and out must be non-NULL");
  *out = nullptr;
  const int precision = cfg->precision, pooling = cfg->pooling, pe = cfg->pe_freqs;
  const int rk = cfg->r_kernel == 0 ? 1 : cfg->r_kernel;
  if (rk != 1 && rk != 3) return fail(GN_EINVAL, "r_kernel %d is neither 1 nor 3", cfg->r_kernel);
  if (precision != GN_FP32_PLAIN && precision != GN_BF16_FUSED && precision != GN_FP8_FUSED)
    return fail(GN_EINVAL, "unknown precision %d", precision);
  if (pooling != GN_POOL_MAX_MEAN && pooling != GN_POOL_SUM)
    return fail(GN_EINVAL, "unknown pooling %d", pooling);
  if (pe < 0 || pe > gn::kMaxPeFreqs)
    return fail(GN_EINVAL, "pe_freqs %d outside 0..%d", pe, gn::kMaxPeFreqs);
  if (precision == GN_FP8_FUSED && pe > 0 && (pe > gn::kMaxPeFreqsFused || rk != 1))
    return fail(GN_EUNSUPPORTED,
                "positional encoding in the FP8 kernel is built for pe_freqs 1..%d with a 1x1 R; "
                "pe_freqs = %d, r_kernel = %d", gn::kMaxPeFreqsFused, pe, rk);
  if (nbytes < sizeof(gn_blob_header))
    return fail(GN_EFORMAT, "blob of %zu bytes is shorter than its header", nbytes);
  gn_blob_header hd;
  std::memcpy(&hd, blob, sizeof(hd));
  if (hd.magic != GN_BLOB_MAGIC) return fail(GN_EFORMAT, "bad magic 0x%08x", hd.magic);
  if (hd.version != GN_BLOB_VERSION) return fail(GN_EFORMAT, "unsupported version %u", hd.version);
  if (hd.scene_dim != gn::kScene || hd.tbuf_channels != gn::kTC || hd.gbuf_channels != gn::kGC ||
      hd.out_channels != gn::kOut)
    return fail(GN_EFORMAT, "channel counts (%u, %u, %u, %u) differ from (32, 12, 14, 3)",
                hd.scene_dim, hd.tbuf_channels, hd.gbuf_channels, hd.out_channels);
  if (hd.hidden > 4096 || hd.latent > 4096) return fail(GN_EFORMAT, "implausible widths");
  gn::WeightIndex wi;
  wi.build(static_cast<int>(hd.hidden), static_cast<int>(hd.latent), pe, rk);
  if (hd.payload_floats != wi.total)
    return fail(GN_EFORMAT,
                "payload holds %llu floats, widths (%u, %u) with pe_freqs %d, r_kernel %d need %zu",
                static_cast<unsigned long long>(hd.payload_floats), hd.hidden, hd.latent, pe, rk,
                wi.total);
  if (nbytes != sizeof(gn_blob_header) + wi.total * sizeof(float))
    return fail(GN_EFORMAT, "blob size %zu != %zu", nbytes,
                sizeof(gn_blob_header) + wi.total * sizeof(float));
  const uint8_t* payload = static_cast<const uint8_t*>(blob) + sizeof(gn_blob_header);
  if (fnv1a64(payload, wi.total * sizeof(float)) != hd.checksum)
    return fail(GN_EFORMAT, "payload checksum mismatch");
  const bool ok_widths = (hd.hidden == 64 && hd.latent == 128) || (hd.hidden == 128 && hd.latent == 256);
  if (!ok_widths)
    return fail(GN_EUNSUPPORTED, "widths (H, Z) = (%u, %u); the library provides (64, 128) and (128, 256)",
                hd.hidden, hd.latent);
  if (precision == GN_BF16_FUSED && pe > gn::kMaxPeFreqsFused)
    return fail(GN_EUNSUPPORTED,
                "positional encoding in the fused BF16 kernel is built for pe_freqs 1..%d (its "
                "encoded operands are sized for them); pe_freqs = %d",
                gn::kMaxPeFreqsFused, pe);

  std::vector<float> w(wi.total);
  std::memcpy(w.data(), payload, wi.total * sizeof(float));
  gn_model* m = new (std::nothrow) gn_model();
  if (!m) return fail(GN_ENOMEM, "host allocation failed");
  *partial = m;  // freed by the caller if a host allocation throws below
  m->H = wi.H;
  m->Z = wi.Z;
  m->precision = precision;
  m->pooling = pooling;
  m->wi = wi;
  cudaGetDevice(&m->device);
  cudaError_t e;
  if ((e = cudaMalloc(&m->w32, wi.total * sizeof(float))) != cudaSuccess) {
    glassnet_free_model(m);
    return fail(GN_ENOMEM, "cudaMalloc weights: %s", cudaGetErrorString(e));
  }
  if ((e = cudaMemcpy(m->w32, w.data(), wi.total * sizeof(float), cudaMemcpyHostToDevice)) !=
      cudaSuccess) {
    glassnet_free_model(m);
    return cuda_fail(e, "upload weights");
  }
  if ((e = cudaMalloc(&m->err, 256)) != cudaSuccess ||
      (e = cudaMemset(m->err, 0, 256)) != cudaSuccess) {
    glassnet_free_model(m);
    return fail(GN_ENOMEM, "cudaMalloc error word: %s", cudaGetErrorString(e));
  }
  if (precision == GN_FP32_PLAIN && (e = gn::setup_static_scratch(m->device)) != cudaSuccess) {
    glassnet_free_model(m);
    return fail(GN_ENOMEM, "static scratch of glassnet_render_fp32_static: %s",
                cudaGetErrorString(e));
  }
  if (precision == GN_FP8_FUSED) {
    // packed by glassnet_calibrate_fp8 once activation scales are known
    m->host_w = static_cast<float*>(std::malloc(wi.total * sizeof(float)));
    if (!m->host_w) {
      glassnet_free_model(m);
      return fail(GN_ENOMEM, "host allocation failed");
    }
    std::memcpy(m->host_w, w.data(), wi.total * sizeof(float));
  }
  if (precision == GN_BF16_FUSED) {
    std::vector<uint8_t> img = wi.H == 128 ? (wi.L > 0 ? pack_fused_bf16_stream(w.data(), wi)
                                                       : pack_fused_bf16<128, false>(w.data(), wi))
                               : wi.L > 0  ? pack_fused_bf16<64, true>(w.data(), wi)
                                           : pack_fused_bf16<64, false>(w.data(), wi);
    m->fused_bytes = img.size();
    if ((e = cudaMalloc(&m->fused, img.size())) != cudaSuccess) {
      glassnet_free_model(m);
      return fail(GN_ENOMEM, "cudaMalloc packed weights: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemcpy(m->fused, img.data(), img.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess) {
      glassnet_free_model(m);
      return cuda_fail(e, "upload packed weights");
    }
  }
  if (rk == 3 && precision != GN_FP32_PLAIN) {  // the 3x3 R kernel's image (BF16)
    std::vector<uint8_t> cimg = pack_conv_r3(w.data(), wi);
    if ((e = cudaMalloc(&m->conv, cimg.size())) != cudaSuccess) {
      glassnet_free_model(m);
      return fail(GN_ENOMEM, "cudaMalloc 3x3 R weights: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemcpy(m->conv, cimg.data(), cimg.size(), cudaMemcpyHostToDevice)) != cudaSuccess) {
      glassnet_free_model(m);
      return cuda_fail(e, "upload 3x3 R weights");
    }
  }
  *partial = nullptr;
  *out = m;
  return GN_OK;
}
}  // namespace

int glassnet_model_info(const gn_model* m, int* hidden, int* latent, int* precision) {
  if (!m) return fail(GN_EINVAL, "model is NULL");
  if (hidden) *hidden = m->H;
  if (latent) *latent = m->Z;
  if (precision) *precision = m->precision;
  return GN_OK;
}

int glassnet_model_config(const gn_model* m, gn_model_config* cfg) {
  if (!m || !cfg) return fail(GN_EINVAL, "model and config must be non-NULL");
  cfg->precision = m->precision;
  cfg->pooling = m->pooling;
  cfg->pe_freqs = m->wi.L;
  cfg->r_kernel = m->wi.RK;
  return GN_OK;
}

int glassnet_encode_scene_device(gn_model* m, const float* scene_dev, gn_latent* lat,
                                 cudaStream_t s) {
  if (!m || !scene_dev || !lat) return fail(GN_EINVAL, "model, scene and latent must be non-NULL");
  if (lat->H != m->H || lat->Z != m->Z) return fail(GN_EINVAL, "latent widths differ from model");
  cudaError_t e = gn::launch_encode(m->w32, m->wi, scene_dev, lat->d, s);
  if (e != cudaSuccess) return cuda_fail(e, "encode launch");
  return GN_OK;
}

int glassnet_encode_scene(gn_model* m, const float* scene, gn_latent** out, cudaStream_t s) {
  if (!m || !scene || !out) return fail(GN_EINVAL, "model, scene and out must be non-NULL");
  *out = nullptr;
  gn_latent* lat = new (std::nothrow) gn_latent();
  if (!lat) return fail(GN_ENOMEM, "host allocation failed");
  lat->H = m->H;
  lat->Z = m->Z;
  const size_t n = static_cast<size_t>(m->Z) + 2 * m->H + gn::kScene;
  cudaError_t e = cudaMalloc(&lat->d, n * sizeof(float));
  if (e != cudaSuccess) {
    delete lat;
    return fail(GN_ENOMEM, "cudaMalloc latent: %s", cudaGetErrorString(e));
  }
  // The scene vector travels with the latent; a synchronous copy so the
  // caller's host buffer may be reused as soon as this returns.
  if ((e = cudaMemcpyAsync(lat->scene(), scene, gn::kScene * sizeof(float),
                           cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    glassnet_free_latent(lat);
    return cuda_fail(e, "upload scene");
  }
  int rc = glassnet_encode_scene_device(m, lat->scene(), lat, s);
  if (rc != GN_OK) {
    glassnet_free_latent(lat);
    return rc;
  }
  *out = lat;
  return GN_OK;
}

int glassnet_latent_read(const gn_latent* lat, float* sigma, float* c_phi, float* c_b,
                         cudaStream_t s) {
  if (!lat) return fail(GN_EINVAL, "latent is NULL");
  cudaError_t e = cudaSuccess;
  if (sigma && e == cudaSuccess)
    e = cudaMemcpyAsync(sigma, lat->d, lat->Z * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (c_phi && e == cudaSuccess)
    e = cudaMemcpyAsync(c_phi, lat->d + lat->Z, lat->H * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (c_b && e == cudaSuccess)
    e = cudaMemcpyAsync(c_b, lat->d + lat->Z + lat->H, lat->H * sizeof(float),
                        cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "latent copy");
  return GN_OK;
}

int glassnet_workspace_bytes(const gn_model* m, int K, int h, int w, size_t* bytes) {
  if (!m || !bytes) return fail(GN_EINVAL, "model and bytes must be non-NULL");
  if (K < 0 || K > gn::kMaxK || h < 1 || w < 1) return fail(GN_EINVAL, "bad frame size");
  const long long tiles = (static_cast<long long>(h) * w + gn::kTile - 1) / gn::kTile;
  *bytes = m->precision == GN_FP32_PLAIN ? gn::plain_workspace_bytes(m->H, K, h * w)
                                         : gn::fused_plan_bytes(tiles);
  if (m->precision != GN_FP32_PLAIN && m->wi.RK == 3)  // plan, then the neural buffer
    *bytes = (*bytes + 255) / 256 * 256 + phi_bytes(m, h, w);
  return GN_OK;
}

namespace {
// Grows a model-owned device buffer to `need` bytes; a growing call
// synchronises the device first (the old buffer may be in use).
int grow_buffer(void*& buf, size_t& bytes, size_t need, const char* what) {
  if (bytes >= need) return GN_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess)
    return fail(GN_ECUDA, "synchronise before growing the %s: %s", what, cudaGetErrorString(e));
  if (buf) cudaFree(buf);
  buf = nullptr;
  bytes = 0;
  if ((e = cudaMalloc(&buf, need)) != cudaSuccess)
    return fail(GN_ENOMEM, "cudaMalloc %s (%zu bytes): %s", what, need, cudaGetErrorString(e));
  bytes = need;
  return GN_OK;
}

// Fills the frame table's first-tile offsets and the tile total.
void number_tiles(gn::FusedParams& p) {
  long long tiles = 0;
  for (int i = 0; i < p.nframes; ++i) {
    p.f[i].tile0 = static_cast<int>(tiles);
    tiles += (static_cast<long long>(p.f[i].P) + gn::kTile - 1) / gn::kTile;
  }
  p.total_tiles = static_cast<int>(tiles);
}
}  // namespace

}  // extern "C"

namespace gn {

int build_batch(const gn_model* m, const gn_frame* frames, int n, FusedParams* out) {
  if (!m || !frames || !out) return fail(GN_EINVAL, "model and frames must be non-NULL");
  if (n < 1 || n > kMaxBatch) return fail(GN_EINVAL, "batch of %d frames outside 1..%d", n, kMaxBatch);
  if (m->precision == GN_FP32_PLAIN)
    return fail(GN_EUNSUPPORTED, "batched launch needs a fused precision");
  if (m->precision == GN_FP8_FUSED && !m->fp8_ready)
    return fail(GN_EINVAL, "FP8 model is not calibrated (glassnet_calibrate_fp8)");
  FusedParams& p = *out;
  std::memset(&p, 0, sizeof(p));
  p.nframes = n;
  p.err = m->err;
  long long tiles = 0;
  for (int i = 0; i < n; ++i) {
    const gn_frame& f = frames[i];
    int rc = check_frame(m, f.latent, f.gbuf, f.tbuf, f.layer_count, f.K, f.h, f.w, f.out);
    if (rc != GN_OK) {
      const std::string msg = g_last_error;
      return fail(rc, "frame %d: %s", i, msg.c_str());
    }
    const int P = f.h * f.w;
    p.f[i] = FusedFrame{f.gbuf, f.tbuf, f.layer_count, f.out, f.latent->fold(), f.K, P, 0, 0};
    p.f[i].w = f.w;
    tiles += (P + kTile - 1) / kTile;
    if (tiles >= (1ll << 24)) return fail(GN_EINVAL, "batch too large");
  }
  number_tiles(p);
  return GN_OK;
}

cudaError_t launch_fused(const gn_model* m, const FusedParams& p, cudaStream_t s) {
  if (m->precision == GN_FP8_FUSED) {
    FusedParams q = p;
    q.pool_sum = m->pooling == GN_POOL_SUM;
    q.pe_freqs = m->wi.L;
    q.stall_ns = m->stall_ns;  // the test hook holds for one launch
    const_cast<gn_model*>(m)->stall_ns = 0;
    return launch_fused_fp8(m->H, m->fused, q, s);
  }
  if (m->pooling == GN_POOL_SUM || m->wi.L > 0 || m->stall_ns > 0 ||
      m->schedule == GN_SCHEDULE_COMPACT) {
    FusedParams q = p;
    q.pool_sum = m->pooling == GN_POOL_SUM;
    q.pe_freqs = m->wi.L;
    q.stall_ns = m->stall_ns;  // the test hook holds for one launch
    const_cast<gn_model*>(m)->stall_ns = 0;
    if (m->schedule == GN_SCHEDULE_COMPACT) return launch_fused_compact(m->fused, q, s);
    return launch_fused_bf16(m->H, m->fused, q, s);
  }
  return launch_fused_bf16(m->H, m->fused, p, s);
}

cudaError_t prepare_fused(const gn_model* m) {
  cudaError_t e = m->precision == GN_FP8_FUSED ? prepare_fused_fp8(m->H) : prepare_fused_bf16(m->H);
  if (e == cudaSuccess && m->schedule == GN_SCHEDULE_COMPACT) e = prepare_fused_compact();
  return e == cudaSuccess && m->wi.RK == 3 ? prepare_conv_r3(m->H) : e;
}

void bind_plan(FusedParams& p, void* ws) {
  p.next_tile = static_cast<uint32_t*>(ws);
  p.plan = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(ws) + kPlanHeader);
}

size_t batch_ws_bytes(const gn_model* m, const FusedParams& p) {
  size_t b = (fused_plan_bytes(p.total_tiles) + 255) / 256 * 256;
  if (m->wi.RK == 3)
    for (int i = 0; i < p.nframes; ++i) b += phi_bytes(m, p.f[i].P / p.f[i].w, p.f[i].w);
  return b;
}

void bind_batch_ws(const gn_model* m, FusedParams& p, void* ws) {
  bind_plan(p, ws);
  if (m->wi.RK != 3) return;
  uint8_t* at = static_cast<uint8_t*>(ws) + (fused_plan_bytes(p.total_tiles) + 255) / 256 * 256;
  for (int i = 0; i < p.nframes; ++i) {
    p.f[i].phi = reinterpret_cast<uint16_t*>(at);
    at += phi_bytes(m, p.f[i].P / p.f[i].w, p.f[i].w);
  }
}

cudaError_t launch_render(const gn_model* m, const FusedParams& p, cudaStream_t s) {
  cudaError_t e = launch_fused(m, p, s);
  if (e != cudaSuccess || m->wi.RK != 3) return e;
  for (int i = 0; i < p.nframes && e == cudaSuccess; ++i)
    e = launch_conv_r3(m->H, m->conv, p.f[i].phi, p.f[i].out, p.f[i].P / p.f[i].w, p.f[i].w, m->err, s);
  return e;
}

}  // namespace gn

extern "C" {

int glassnet_render_ws(const gn_model* m, const gn_latent* lat, const float* gbuf,
                       const float* tbuf, const uint8_t* cnt, int K, int h, int w, float* out,
                       void* ws, size_t ws_bytes, cudaStream_t s) {
  int rc = check_frame(m, lat, gbuf, tbuf, cnt, K, h, w, out);
  if (rc != GN_OK) return rc;
  const int P = h * w;
  cudaError_t e;
  if (m->precision == GN_FP32_PLAIN) {
    const size_t need = gn::plain_workspace_bytes(m->H, K, P);
    if (!ws || ws_bytes < need)
      return fail(GN_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, need);
    if (reinterpret_cast<uintptr_t>(ws) & 255u)
      return fail(GN_EINVAL, "workspace must be 256-byte aligned");
    e = gn::launch_plain_fp32(m->w32, m->wi, lat->d, gbuf, tbuf, cnt, K, P, out, ws, m->err, s,
                              m->pooling == GN_POOL_SUM, w);
    if (e != cudaSuccess) return cuda_fail(e, "FP32 plain launch");
    return GN_OK;
  }
  if (m->precision == GN_FP8_FUSED && !m->fp8_ready)
    return fail(GN_EINVAL, "FP8 model is not calibrated (glassnet_calibrate_fp8)");
  gn::FusedParams p;
  std::memset(&p, 0, sizeof(p));
  p.nframes = 1;
  p.err = m->err;
  p.f[0] = gn::FusedFrame{gbuf, tbuf, cnt, out, lat->fold(), K, P, 0, 0};
  p.f[0].w = w;
  number_tiles(p);
  const size_t need = gn::batch_ws_bytes(m, p);  // = glassnet_workspace_bytes
  if (!ws || ws_bytes < need)
    return fail(GN_EINVAL, "workspace of %zu bytes, %zu needed", ws_bytes, need);
  if (reinterpret_cast<uintptr_t>(ws) & 255u)
    return fail(GN_EINVAL, "workspace must be 256-byte aligned");
  // the plan (and, for a 3x3 R, the neural buffer the fused kernel stops at)
  gn::bind_batch_ws(m, p, ws);
  e = gn::launch_render(m, p, s);
  if (e != cudaSuccess) return cuda_fail(e, "fused launch");
  return GN_OK;
}

int glassnet_render(const gn_model* m, const gn_latent* lat, const float* gbuf, const float* tbuf,
                    const uint8_t* cnt, int K, int h, int w, float* out, cudaStream_t s) {
  int rc = check_frame(m, lat, gbuf, tbuf, cnt, K, h, w, out);
  if (rc != GN_OK) return rc;
  gn_model* mm = const_cast<gn_model*>(m);
  size_t need = 0;
  glassnet_workspace_bytes(m, K, h, w, &need);
  if (m->precision != GN_FP32_PLAIN) {
    if ((rc = grow_buffer(mm->plan, mm->plan_bytes, need, "tile plan")) != GN_OK) return rc;
    return glassnet_render_ws(m, lat, gbuf, tbuf, cnt, K, h, w, out, mm->plan, mm->plan_bytes, s);
  }
  if ((rc = grow_buffer(mm->ws, mm->ws_bytes, need, "workspace")) != GN_OK) return rc;
  return glassnet_render_ws(m, lat, gbuf, tbuf, cnt, K, h, w, out, mm->ws, mm->ws_bytes, s);
}

int glassnet_render_host(gn_model* m, const gn_latent* lat, const float* gbuf_h,
                         const float* tbuf_h, const uint8_t* cnt_h, int K, int h, int w,
                         float* out_h, cudaStream_t s) {
  int rc = check_frame(m, lat, gbuf_h, tbuf_h, cnt_h, K, h, w, out_h);
  if (rc != GN_OK) return rc;
  const size_t P = static_cast<size_t>(h) * w;
  const size_t b_g = P * gn::kGC * 4, b_t = P * gn::kTC * 4 * K, b_o = P * gn::kOut * 4;
  const size_t b_c = (P + 255) / 256 * 256;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t need = up(b_g) + up(b_t) + up(b_o) + b_c;
  cudaError_t e;
  if (m->stage_bytes < need) {
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "synchronise");
    if (m->stage) cudaFree(m->stage);
    m->stage = nullptr;
    m->stage_bytes = 0;
    if ((e = cudaMalloc(&m->stage, need)) != cudaSuccess)
      return fail(GN_ENOMEM, "cudaMalloc staging (%zu bytes): %s", need, cudaGetErrorString(e));
    m->stage_bytes = need;
  }
  uint8_t* base = static_cast<uint8_t*>(m->stage);
  float* d_g = reinterpret_cast<float*>(base);
  float* d_t = reinterpret_cast<float*>(base + up(b_g));
  float* d_o = reinterpret_cast<float*>(base + up(b_g) + up(b_t));
  uint8_t* d_c = base + up(b_g) + up(b_t) + up(b_o);
  if ((e = cudaMemcpyAsync(d_g, gbuf_h, b_g, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (K > 0 && (e = cudaMemcpyAsync(d_t, tbuf_h, b_t, cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
      (e = cudaMemcpyAsync(d_c, cnt_h, P, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e, "host to device copy");
  rc = glassnet_render(m, lat, d_g, K > 0 ? d_t : nullptr, d_c, K, h, w, d_o, s);
  if (rc != GN_OK) return rc;
  if ((e = cudaMemcpyAsync(out_h, d_o, b_o, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "device to host copy");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "synchronise");
  return GN_OK;
}

int glassnet_render_batch(const gn_model* m, const gn_frame* frames, int n, cudaStream_t s) {
  gn::FusedParams p;
  int rc = gn::build_batch(m, frames, n, &p);
  if (rc != GN_OK) return rc;
  gn_model* mm = const_cast<gn_model*>(m);
  rc = grow_buffer(mm->plan, mm->plan_bytes, gn::batch_ws_bytes(m, p), "tile plan");
  if (rc != GN_OK) return rc;
  gn::bind_batch_ws(m, p, mm->plan);
  cudaError_t e = gn::launch_render(m, p, s);
  if (e != cudaSuccess) return cuda_fail(e, "batched fused launch");
  return GN_OK;
}

// Scales = headroom |max| / 448 over the calibration render, per channel for
// the two input tensors (the transparency layers and the G-buffer, whose
// channels range from [0, 1] to log-normal lighting) and per tensor for the
// hidden activations (internal.h gives the headroom factors).  With one
// scale for all input channels and one binade of headroom, a 93,639-pixel
// frame clipped a lighting value at 2x its calibration maximum and its
// hidden activations went past 2x theirs.

namespace {
int calibrate_fp8_impl(gn_model* m, const gn_latent* lat, const float* gbuf, const float* tbuf,
                       const uint8_t* cnt, int K, int h, int w, cudaStream_t s);
}  // namespace

int glassnet_calibrate_fp8(gn_model* m, const gn_latent* lat, const float* gbuf, const float* tbuf,
                           const uint8_t* cnt, int K, int h, int w, cudaStream_t s) {
  try {
    return calibrate_fp8_impl(m, lat, gbuf, tbuf, cnt, K, h, w, s);
  } catch (const std::bad_alloc&) {
    return fail(GN_ENOMEM, "host allocation failed");
  }
}

namespace {
int calibrate_fp8_impl(gn_model* m, const gn_latent* lat, const float* gbuf, const float* tbuf,
                       const uint8_t* cnt, int K, int h, int w, cudaStream_t s) {
  if (!m) return fail(GN_EINVAL, "model is NULL");
  if (m->precision != GN_FP8_FUSED) return fail(GN_EINVAL, "model precision is not GN_FP8_FUSED");
  const int P = h * w;
  int rc = check_frame(m, lat, gbuf, tbuf, cnt, K, h, w, gbuf);
  if (rc != GN_OK) return rc;
  const size_t need = gn::plain_workspace_bytes(m->H, K, P);
  if ((rc = grow_buffer(m->ws, m->ws_bytes, need, "workspace")) != GN_OK) return rc;
  void* tmp = nullptr;  // RGB of the calibration render, then the amax words
  const size_t out_bytes = (static_cast<size_t>(P) * gn::kOut * sizeof(float) + 255) / 256 * 256;
  cudaError_t e = cudaMalloc(&tmp, out_bytes + 256);
  if (e != cudaSuccess) return fail(GN_ENOMEM, "cudaMalloc calibration scratch");
  float* out = static_cast<float*>(tmp);
  uint32_t* amax = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(tmp) + out_bytes);
  uint32_t bits[gn::kFp8Acts] = {};
  e = gn::launch_plain_fp32(m->w32, m->wi, lat->d, gbuf, tbuf, cnt, K, P, out, m->ws, m->err, s,
                            m->pooling == GN_POOL_SUM, w);
  if (e == cudaSuccess)
    e = gn::launch_fp8_act_amax(m->ws, gbuf, tbuf, cnt, m->H, K, P, amax, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bits, amax, sizeof(bits), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "calibration render");
  float act[gn::kFp8Acts];
  for (int i = 0; i < gn::kFp8Acts; ++i) {
    float a;
    std::memcpy(&a, &bits[i], 4);
    const float headroom = i < gn::FP8_U ? gn::kFp8InputHeadroom : gn::kFp8HiddenHeadroom;
    act[i] = (a > 0.0f && std::isfinite(a)) ? a * headroom / 448.0f : 1.0f;
  }
  const bool pe = m->wi.L > 0;
  std::vector<uint8_t> img = m->H == 128 ? (pe ? pack_fused_fp8<128, true>(m->host_w, m->wi, act)
                                                : pack_fused_fp8<128>(m->host_w, m->wi, act))
                                         : (pe ? pack_fused_fp8<64, true>(m->host_w, m->wi, act)
                                                : pack_fused_fp8<64>(m->host_w, m->wi, act));
  if (!m->fused) {
    if ((e = cudaMalloc(&m->fused, img.size())) != cudaSuccess)
      return fail(GN_ENOMEM, "cudaMalloc packed weights: %s", cudaGetErrorString(e));
    m->fused_bytes = img.size();
  }
  if ((e = cudaMemcpy(m->fused, img.data(), img.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "upload packed FP8 weights");
  std::memcpy(m->fp8_act, act, sizeof(act));
  m->fp8_ready = true;
  return GN_OK;
}
}  // namespace

int glassnet_fp8_scales(const gn_model* m, float* scales) {
  if (!m || !scales) return fail(GN_EINVAL, "model and scales must be non-NULL");
  if (m->precision != GN_FP8_FUSED || !m->fp8_ready)
    return fail(GN_EINVAL, "not a calibrated GN_FP8_FUSED model");
  std::memcpy(scales, m->fp8_act, sizeof(m->fp8_act));
  return GN_OK;
}

int glassnet_debug_stall_next_render(gn_model* m, uint64_t stall_ns) {
  if (!m) return fail(GN_EINVAL, "model is NULL");
  if (m->precision == GN_FP32_PLAIN)
    return fail(GN_EINVAL, "the stall hook is in the fused kernels (BF16, FP8)");
  if (stall_ns == 0 || stall_ns > 1000000000ull)
    return fail(GN_EINVAL, "stall of %llu ns outside 1 ns .. 1 s", static_cast<unsigned long long>(stall_ns));
  m->stall_ns = stall_ns;
  return GN_OK;
}

int glassnet_set_layer_schedule(gn_model* m, int schedule) {
  if (!m) return fail(GN_EINVAL, "model is NULL");
  if (schedule != GN_SCHEDULE_SORTED && schedule != GN_SCHEDULE_COMPACT)
    return fail(GN_EINVAL, "unknown schedule %d", schedule);
  if (schedule == GN_SCHEDULE_COMPACT) {
    if (m->precision != GN_BF16_FUSED || m->H != 64 || m->wi.L > 0 || m->wi.RK != 1)
      return fail(GN_EUNSUPPORTED,
                  "the compacted layer schedule is built for GN_BF16_FUSED at H = 64 without "
                  "positional encoding and with a 1x1 R");
    const cudaError_t e = gn::prepare_fused_compact();
    if (e != cudaSuccess) return cuda_fail(e, "compacted kernel attributes");
  }
  m->schedule = schedule;
  return GN_OK;
}

int glassnet_check(const gn_model* m, cudaStream_t s) {
  if (!m) return fail(GN_EINVAL, "model is NULL");
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream");
  uint32_t words[2] = {0, 0};  // error bits; which wait timed out (report_timeout)
  if ((e = cudaMemcpy(words, m->err, 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "read error word");
  const uint32_t bits = words[0];
  if (bits || words[1]) {
    if ((e = cudaMemset(m->err, 0, 8)) != cudaSuccess) return cuda_fail(e, "clear error word");
  }
  if (bits & gn::kErrTimeout) {
    const uint32_t w = words[1];
    if (!(w >> 31)) return fail(GN_ETIMEOUT, "a device-side wait timed out");
    static const char* const kernels[] = {"?", "fused BF16", "fused FP8", "compacted", "3x3 R"};
    static const char* const modes[] = {"frame", "accumulate", "resolve"};
    const uint32_t k = (w >> 16) & 0x7fffu, md = (w >> 8) & 0xffu, slot = w & 0xffu;
    return fail(GN_ETIMEOUT, "a device-side wait timed out (%s kernel, %s launch, mbarrier slot %u)",
                k < 5 ? kernels[k] : "?", md < 3 ? modes[md] : "?", slot);
  }
  if (bits & gn::kErrCount) return fail(GN_EINVAL, "a layer count exceeded K");
  if (bits & gn::kErrRange) return fail(GN_ERANGE, "an exact set-sum left its fixed-point range");
  if (bits & gn::kErrSaturated)
    return fail(GN_ESATURATED, "an FP8 input was beyond its calibrated range and was clamped");
  return GN_OK;
}

void glassnet_free_latent(gn_latent* lat) {
  if (!lat) return;
  if (lat->d) cudaFree(lat->d);
  delete lat;
}

}  // extern "C"

// ------------------------------------------------------------- streaming
struct gn_pool {
  int h = 0, w = 0, H = 0, RK = 1;  // frame, widths and R1's kernel size of its model
  void* dev = nullptr;  // state blocks (tile-major, see FusedParams), then counts [P] u8
  uint32_t* st = nullptr;
  size_t st_words = 0;
  uint8_t* cnt = nullptr;
  void* plan = nullptr;  // tile plan of the pool's launches, then (3x3 R) the neural buffer
  uint16_t* phi = nullptr;
  int layers = 0;        // accumulate calls since the last reset
};

namespace {
// Empty pool: running max 0 (the ReLU floor), sums at 2^11 (the fixed-point
// base of the exact pooling), no layers.  Word w of the state lies in plane
// (w / 128) mod (H/2 + H) of its tile's block: the first H/2 planes hold the
// max pairs, the others the sums.
__global__ void pool_reset_kernel(uint32_t* st, size_t n_st, int planes, int mx_planes,
                                  uint8_t* cnt, size_t n_cnt) {
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n_st; i += stride) {
    const int pl = static_cast<int>((i / gn::kTile) % static_cast<size_t>(planes));
    st[i] = pl < mx_planes ? 0u : 0x45000000u;  // 2048.0f
    if (i < n_cnt) cnt[i] = 0u;
  }
}

// One-frame fused parameters of a pool launch (pixel-order plan, the pool's
// state and plan workspace).
gn::FusedParams pool_params(const gn_model* m, const gn_latent* lat, const gn_pool* pool,
                            const float* gbuf, const float* tbuf, const uint8_t* cnt, int K,
                            float* out) {
  gn::FusedParams p;
  std::memset(&p, 0, sizeof(p));
  p.nframes = 1;
  p.err = m->err;
  p.f[0] = gn::FusedFrame{gbuf, tbuf, cnt, out, lat->fold(), K, pool->h * pool->w, 0, 0};
  number_tiles(p);
  p.plan_identity = 1;
  p.pool_sum = m->pooling == GN_POOL_SUM;
  p.pe_freqs = m->wi.L;
  p.pool_st = pool->st;
  p.pool_cnt = pool->cnt;
  gn::bind_plan(p, pool->plan);
  return p;
}

int check_pool_call(const gn_model* m, const gn_latent* lat, const gn_pool* pool) {
  if (!m) return fail(GN_EINVAL, "model is NULL");
  if (!lat) return fail(GN_EINVAL, "latent is NULL");
  if (!pool) return fail(GN_EINVAL, "pool is NULL");
  if (m->precision != GN_BF16_FUSED)
    return fail(GN_EUNSUPPORTED, "streaming needs a GN_BF16_FUSED model");
  if (lat->H != m->H || lat->Z != m->Z)
    return fail(GN_EINVAL, "latent widths (%d, %d) do not match the model (%d, %d)", lat->H,
                lat->Z, m->H, m->Z);
  if (pool->H != m->H) return fail(GN_EINVAL, "pool of width %d, model of width %d", pool->H, m->H);
  if (pool->RK != m->wi.RK)
    return fail(GN_EINVAL, "pool made for a %dx%d R, model with a %dx%d R", pool->RK, pool->RK,
                m->wi.RK, m->wi.RK);
  return GN_OK;
}
}  // namespace

extern "C" {

int glassnet_pool_create(const gn_model* m, int h, int w, gn_pool** out) {
  if (!m || !out) return fail(GN_EINVAL, "model and out must be non-NULL");
  *out = nullptr;
  if (m->precision != GN_BF16_FUSED)
    return fail(GN_EUNSUPPORTED, "streaming needs a GN_BF16_FUSED model");
  if (h < 1 || w < 1) return fail(GN_EINVAL, "frame %d x %d is empty", h, w);
  const long long P = static_cast<long long>(h) * w;
  if (P * gn::kTC >= (1ll << 31)) return fail(GN_EINVAL, "frame %d x %d too large", h, w);
  cudaError_t e = gn::prepare_fused(m);
  if (e != cudaSuccess) return cuda_fail(e, "fused kernel attributes");
  gn_pool* pool = new (std::nothrow) gn_pool;
  if (!pool) return fail(GN_ENOMEM, "host allocation failed");
  pool->h = h;
  pool->w = w;
  pool->H = m->H;
  pool->RK = m->wi.RK;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const long long tiles = (P + gn::kTile - 1) / gn::kTile;
  pool->st_words = static_cast<size_t>(tiles) * (m->H / 2 + m->H) * gn::kTile;
  const size_t b_st = up(pool->st_words * 4), b_cnt = up(static_cast<size_t>(P));
  if (cudaMalloc(&pool->dev, b_st + b_cnt) != cudaSuccess) {
    delete pool;
    return fail(GN_ENOMEM, "cudaMalloc pool state (%zu bytes)", b_st + b_cnt);
  }
  uint8_t* base = static_cast<uint8_t*>(pool->dev);
  pool->st = reinterpret_cast<uint32_t*>(base);
  pool->cnt = base + b_st;
  const size_t b_plan = up(gn::fused_plan_bytes(tiles));
  const size_t b_phi = m->wi.RK == 3 ? phi_bytes(m, h, w) : 0;
  if (cudaMalloc(&pool->plan, b_plan + b_phi) != cudaSuccess) {
    cudaFree(pool->dev);
    delete pool;
    return fail(GN_ENOMEM, "cudaMalloc pool tile plan");
  }
  if (b_phi) pool->phi = reinterpret_cast<uint16_t*>(static_cast<uint8_t*>(pool->plan) + b_plan);
  int rc = glassnet_pool_reset(pool, nullptr);
  if (rc == GN_OK && (e = cudaStreamSynchronize(nullptr)) != cudaSuccess) rc = cuda_fail(e, "pool reset");
  if (rc != GN_OK) {
    glassnet_pool_free(pool);
    return rc;
  }
  *out = pool;
  return GN_OK;
}

int glassnet_pool_reset(gn_pool* pool, cudaStream_t s) {
  if (!pool) return fail(GN_EINVAL, "pool is NULL");
  const size_t P = static_cast<size_t>(pool->h) * pool->w;
  pool_reset_kernel<<<std::min<size_t>((pool->st_words + 255) / 256, 4096), 256, 0, s>>>(
      pool->st, pool->st_words, pool->H / 2 + pool->H, pool->H / 2, pool->cnt, P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pool reset launch");
  pool->layers = 0;
  return GN_OK;
}

int glassnet_accumulate_layer(const gn_model* m, const gn_latent* lat, gn_pool* pool,
                              const float* layer, const uint8_t* covered, cudaStream_t s) {
  int rc = check_pool_call(m, lat, pool);
  if (rc != GN_OK) return rc;
  if (!layer) return fail(GN_EINVAL, "layer is NULL");
  if (!aligned4(layer)) return fail(GN_EINVAL, "layer must be 4-byte aligned");
  if (pool->layers >= gn::kMaxK)
    return fail(GN_EINVAL, "the pool already holds %d layers (at most %d)", pool->layers, gn::kMaxK);
  gn::FusedParams p = pool_params(m, lat, pool, nullptr, layer, covered, 1, nullptr);
  p.pool_fresh = pool->layers == 0;  // after a reset the state need not be read
  cudaError_t e = gn::launch_fused_bf16(m->H, m->fused, p, s, 1);
  if (e != cudaSuccess) return cuda_fail(e, "accumulate launch");
  ++pool->layers;
  return GN_OK;
}

int glassnet_resolve(const gn_model* m, const gn_latent* lat, const gn_pool* pool,
                     const float* gbuf, float* out, cudaStream_t s) {
  int rc = check_pool_call(m, lat, pool);
  if (rc != GN_OK) return rc;
  if (!gbuf || !out) return fail(GN_EINVAL, "gbuf and out must be non-NULL");
  if (!aligned4(gbuf) || !aligned4(out)) return fail(GN_EINVAL, "gbuf and out must be 4-byte aligned");
  gn::FusedParams p = pool_params(m, lat, pool, gbuf, nullptr, pool->cnt, gn::kMaxK, out);
  if (pool->phi) {  // 3x3 R: the resolve stops at the neural buffer, the 3x3 kernel follows
    p.f[0].phi = pool->phi;
    p.f[0].w = pool->w;
  }
  cudaError_t e = gn::launch_fused_bf16(m->H, m->fused, p, s, 2);
  if (e == cudaSuccess && pool->phi)
    e = gn::launch_conv_r3(m->H, m->conv, pool->phi, out, pool->h, pool->w, m->err, s);
  if (e != cudaSuccess) return cuda_fail(e, "resolve launch");
  return GN_OK;
}

void glassnet_pool_free(gn_pool* pool) {
  if (!pool) return;
  if (pool->dev) cudaFree(pool->dev);
  if (pool->plan) cudaFree(pool->plan);
  delete pool;
}

void glassnet_free_model(gn_model* m) {
  if (!m) return;
  if (m->w32) cudaFree(m->w32);
  if (m->fused) cudaFree(m->fused);
  if (m->err) cudaFree(m->err);
  if (m->ws) cudaFree(m->ws);
  if (m->conv) cudaFree(m->conv);
  if (m->stage) cudaFree(m->stage);
  if (m->plan) cudaFree(m->plan);
  std::free(m->host_w);
  delete m;
}

}  // extern "C"

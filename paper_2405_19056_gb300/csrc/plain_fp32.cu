// FP32 plain form of the GlassNet forward pass: the concat-form network as
// written, one kernel per layer, intermediates in a device workspace, FP32
// FMA on CUDA cores (no tensor cores, no TF32, no folding).  It is the
// same-GPU baseline for the fused kernels.
//
// Layers (Sec. 3.3-3.4, Eq. 5), inputs b_k and g positionally encoded when
// the weights have L > 0 frequencies (bands computed as the GEMM reads them):
//   U = ReLU(W_phi1 [b_k ; sigma] + b)    rows (k, p) with k < c_p
//   V = ReLU(W_phi2 U + b)
//   pool_p = [max_k V ; (sum_k V) / c_p]   FP32 sum in slot order
//   R = ReLU(W_rho pool + b), R = 0 when c_p = 0
//   (sum form of Eq. 5: R = sum_k V over the valid layers, no rho)
//   Y = ReLU(W_B2 ReLU(W_B1 [g ; R ; sigma] + b) + b)
//   out = sigmoid(W_R2 ReLU(W_R1 Y + b) + b)
//   (with a 3x3 R1, W_R1 reads the 3x3 neighbourhood of Y, zero outside the frame)
#include "internal.h"

namespace gn {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// Input row assemblers: x(r, j) is element j of input row r; valid(r) tells
// whether row r is computed (invalid rows are written as 0 and never read).
struct PhiIn {  // [gamma_L(b_k) (12 (1 + 2L)) ; sigma (Z)]
  const float* tbuf;
  const float* sigma;
  const uint8_t* counts;
  int P, L;
  __device__ bool valid(int r) const { return (r / P) < counts[r % P]; }
  __device__ float x(int r, int j) const {
    const int k = r / P, p = r % P;
    const int tce = kTC * (1 + 2 * L);
    if (j >= tce) return sigma[j - tce];
    return pe_band_value(tbuf[(static_cast<size_t>(k) * kTC + j % kTC) * P + p], j / kTC);
  }
};
struct RowsIn {  // row-major [M][Kx]; validity from the layer counts (rows (k, p))
  const float* X;
  const uint8_t* counts;
  int P, Kx;
  __device__ bool valid(int r) const { return counts == nullptr || (r / P) < counts[r % P]; }
  __device__ float x(int r, int j) const { return X[static_cast<size_t>(r) * Kx + j]; }
};
struct ConvIn {  // R1 with a 3x3 kernel: j = k * 9 + (dy + 1) * 3 + (dx + 1), zero outside the frame
  const float* Y;  // [P][H] neural buffer, pixel p = y w + x
  int h, w, H;
  __device__ bool valid(int) const { return true; }
  __device__ float x(int r, int j) const {
    const int k = j / 9, t = j % 9;
    const int yy = r / w + t / 3 - 1, xx = r % w + t % 3 - 1;
    if (yy < 0 || yy >= h || xx < 0 || xx >= w) return 0.0f;
    return Y[static_cast<size_t>(yy * w + xx) * H + k];
  }
};
struct RhoIn {  // pool rows; a pixel without valid layers gets r = 0
  const float* pool;
  const uint8_t* counts;
  int Kx;
  __device__ bool valid(int r) const { return counts[r] > 0; }
  __device__ float x(int r, int j) const { return pool[static_cast<size_t>(r) * Kx + j]; }
};
struct BIn {  // [gamma_L(g) (14 (1 + 2L)) ; r (H) ; sigma (Z)]
  const float* gbuf;
  const float* R;
  const float* sigma;
  int P, H, L;
  __device__ bool valid(int) const { return true; }
  __device__ float x(int r, int j) const {
    const int gce = kGC * (1 + 2 * L);
    if (j < gce) return pe_band_value(gbuf[static_cast<size_t>(j % kGC) * P + r], j / kGC);
    if (j < gce + H) return R[static_cast<size_t>(r) * H + (j - gce)];
    return sigma[j - gce - H];
  }
};

// Y = act(X W^T + b) for one 64x64 output tile; 256 threads, 4x4 outputs each.
// SIGMOID_SOA: sigmoid activation and output stored as [N][M] (RGB planes).
template <class In, bool SIGMOID_SOA>
__global__ void __launch_bounds__(256) linear_kernel(In in, const float* __restrict__ W,
                                                     const float* __restrict__ b, float* Y, int M,
                                                     int N, int Kx) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  __shared__ unsigned char s_valid[BM];
  const int t = threadIdx.x;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  int any = 0;
  if (t < BM) {
    const int r = m0 + t;
    const int v = (r < M) && in.valid(r);
    s_valid[t] = static_cast<unsigned char>(v);
    any = v;
  }
  if (!__syncthreads_or(any)) {
    // every row invalid: write zeros (hidden layers only)
    if (!SIGMOID_SOA) {
      for (int e = t; e < BM * BN; e += 256) {
        const int r = m0 + e / BN, n = n0 + e % BN;
        if (r < M && n < N) Y[static_cast<size_t>(r) * N + n] = 0.0f;
      }
    }
    return;
  }
  const int tr = (t / 16) * 4, tc = (t % 16) * 4;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < Kx; k0 += BK) {
    for (int e = t; e < BM * BK; e += 256) {
      const int mm = e / BK, kk = e % BK;
      const int r = m0 + mm, j = k0 + kk;
      As[kk][mm] = (s_valid[mm] && j < Kx) ? in.x(r, j) : 0.0f;
    }
    for (int e = t; e < BN * BK; e += 256) {
      const int nn = e / BK, kk = e % BK;
      const int n = n0 + nn, j = k0 + kk;
      Bs[kk][nn] = (n < N && j < Kx) ? W[static_cast<size_t>(n) * Kx + j] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], w[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + i];
#pragma unroll
      for (int i = 0; i < 4; ++i) w[i] = Bs[kk][tc + i];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + tr + i;
    if (r >= M) continue;
    const bool v = s_valid[tr + i];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tc + j;
      if (n >= N) continue;
      const float y = acc[i][j] + b[n];
      if (SIGMOID_SOA) {
        Y[static_cast<size_t>(n) * M + r] = 1.0f / (1.0f + expf(-y));
      } else {
        Y[static_cast<size_t>(r) * N + n] = v ? fmaxf(y, 0.0f) : 0.0f;
      }
    }
  }
}

// pool[p] = [max_k V ; (sum_k V) / c_p] over k < c_p (zeros when c_p = 0), or
// with `tau` set, R[p] = sum_k V (Eq. 5's sum form, zero when c_p = 0).
__global__ void pool_kernel(const float* __restrict__ V, const uint8_t* __restrict__ counts,
                            float* pool, float* tau, int P, int K, int H, uint32_t* err) {
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<size_t>(P) * H) return;
  const int p = static_cast<int>(i / H), n = static_cast<int>(i % H);
  int c = counts[p];
  if (c > K) {
    if (n == 0) atomicOr(err, kErrCount);
    c = K;
  }
  float mx = 0.0f, s = 0.0f;
  for (int k = 0; k < c; ++k) {
    const float v = V[(static_cast<size_t>(k) * P + p) * H + n];
    mx = fmaxf(mx, v);
    s += v;
  }
  if (tau) {
    tau[static_cast<size_t>(p) * H + n] = s;
    return;
  }
  pool[static_cast<size_t>(p) * 2 * H + n] = mx;
  pool[static_cast<size_t>(p) * 2 * H + H + n] = c > 0 ? s / static_cast<float>(c) : 0.0f;
}

template <class In, bool S>
cudaError_t run_linear(const In& in, const float* W, const float* b, float* Y, int M, int N,
                       int Kx, cudaStream_t s) {
  if (M == 0) return cudaSuccess;
  dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
  linear_kernel<In, S><<<grid, 256, 0, s>>>(in, W, b, Y, M, N, Kx);
  return cudaGetLastError();
}

}  // namespace

// |x| max of n floats into *slot (as ordered uint bits of a non-negative float).
__global__ void amax_kernel(const float* __restrict__ x, size_t n, uint32_t* slot) {
  float m = 0.0f;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, __float_as_uint(m));
}
// |t| max of channel `ch` over the valid layer slots (k < c_p) of a
// transparency buffer.
__global__ void amax_layers_kernel(const float* __restrict__ tbuf, const uint8_t* __restrict__ counts,
                                   int K, int P, int ch, uint32_t* slot) {
  float m = 0.0f;
  const size_t n = static_cast<size_t>(K) * P;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int p = static_cast<int>(i % P);
    const int k = static_cast<int>(i / P);
    if (k < counts[p]) m = fmaxf(m, fabsf(tbuf[(static_cast<size_t>(k) * kTC + ch) * P + p]));
  }
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 16));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 8));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
  m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
  if ((threadIdx.x & 31) == 0) atomicMax(slot, __float_as_uint(m));
}

size_t plain_workspace_bytes(int H, int K, int P) {
  const size_t rows = static_cast<size_t>(K) * P;
  // U, V: [K*P][H]; pool [P][2H]; R, Y1, Y2, Q: [P][H]
  size_t f = 2 * rows * H + static_cast<size_t>(P) * 2 * H + 4 * static_cast<size_t>(P) * H;
  return ((f * sizeof(float)) + 255) / 256 * 256;
}

cudaError_t launch_plain_fp32(const float* w32, const WeightIndex& wi, const float* latent,
                              const float* gbuf, const float* tbuf, const uint8_t* counts, int K,
                              int P, float* out, void* ws, uint32_t* err, cudaStream_t s,
                              int pool_sum, int w) {
  const int H = wi.H, Z = wi.Z;
  const size_t rows = static_cast<size_t>(K) * P;
  float* U = static_cast<float*>(ws);
  float* V = U + rows * H;
  float* pool = V + rows * H;
  float* R = pool + static_cast<size_t>(P) * 2 * H;
  float* Y1 = R + static_cast<size_t>(P) * H;
  float* Y2 = Y1 + static_cast<size_t>(P) * H;
  float* Q = Y2 + static_cast<size_t>(P) * H;
  const float* sigma = latent;  // latent starts with sigma [Z]
  auto W = [&](int l) { return w32 + wi.w[l]; };
  auto B = [&](int l) { return w32 + wi.b[l]; };
  cudaError_t e = cudaSuccess;
  if (K > 0) {
    e = run_linear<PhiIn, false>(PhiIn{tbuf, sigma, counts, P, wi.L}, W(LPHI1), B(LPHI1), U,
                                 static_cast<int>(rows), H, wi.tc_enc() + Z, s);
    if (e != cudaSuccess) return e;
    e = run_linear<RowsIn, false>(RowsIn{U, counts, P, H}, W(LPHI2), B(LPHI2), V,
                                  static_cast<int>(rows), H, H, s);
    if (e != cudaSuccess) return e;
    const size_t n = static_cast<size_t>(P) * H;
    pool_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
        V, counts, pool, pool_sum ? R : nullptr, P, K, H, err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!pool_sum)
      e = run_linear<RhoIn, false>(RhoIn{pool, counts, 2 * H}, W(LRHO), B(LRHO), R, P, H, 2 * H, s);
  } else {
    e = cudaMemsetAsync(R, 0, static_cast<size_t>(P) * H * sizeof(float), s);
  }
  if (e != cudaSuccess) return e;
  e = run_linear<BIn, false>(BIn{gbuf, R, sigma, P, H, wi.L}, W(LB1), B(LB1), Y1, P, H,
                             wi.gc_enc() + H + Z, s);
  if (e != cudaSuccess) return e;
  e = run_linear<RowsIn, false>(RowsIn{Y1, nullptr, P, H}, W(LB2), B(LB2), Y2, P, H, H, s);
  if (e != cudaSuccess) return e;
  if (wi.RK == 3)
    e = run_linear<ConvIn, false>(ConvIn{Y2, P / w, w, H}, W(LR1), B(LR1), Q, P, H, 9 * H, s);
  else
    e = run_linear<RowsIn, false>(RowsIn{Y2, nullptr, P, H}, W(LR1), B(LR1), Q, P, H, H, s);
  if (e != cudaSuccess) return e;
  return run_linear<RowsIn, true>(RowsIn{Q, nullptr, P, H}, W(LR2), B(LR2), out, P, kOut, H, s);
}

cudaError_t launch_fp8_act_amax(const void* ws, const float* gbuf, const float* tbuf,
                                const uint8_t* counts, int H, int K, int P, uint32_t* amax,
                                cudaStream_t s) {
  const size_t rows = static_cast<size_t>(K) * P;
  const float* U = static_cast<const float*>(ws);
  const float* pool = U + 2 * rows * H;
  const float* R = pool + static_cast<size_t>(P) * 2 * H;
  const float* Y1 = R + static_cast<size_t>(P) * H;
  const float* Y2 = Y1 + static_cast<size_t>(P) * H;
  const float* Q = Y2 + static_cast<size_t>(P) * H;
  cudaError_t e = cudaMemsetAsync(amax, 0, kFp8Acts * sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  const size_t ph = static_cast<size_t>(P) * H;
  auto run = [&](const float* x, size_t n, int slot) {
    if (n == 0) return;
    const unsigned blocks = static_cast<unsigned>(n / 256 + 1 < 2048 ? n / 256 + 1 : 2048);
    amax_kernel<<<blocks, 256, 0, s>>>(x, n, amax + slot);
  };
  if (K > 0) {
    for (int ch = 0; ch < kTC; ++ch)
      amax_layers_kernel<<<512, 256, 0, s>>>(tbuf, counts, K, P, ch, amax + FP8_T0 + ch);
    run(U, rows * H, FP8_U);
    run(pool, ph * 2, FP8_POOL);
  }
  for (int ch = 0; ch < kGC; ++ch) run(gbuf + static_cast<size_t>(ch) * P, P, FP8_G0 + ch);
  run(R, ph, FP8_R);
  run(Y1, ph, FP8_Y);
  run(Y2, ph, FP8_Y2);
  run(Q, ph, FP8_Q);
  return cudaGetLastError();
}

}  // namespace gn

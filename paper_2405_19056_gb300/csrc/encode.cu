// Scene encoder F and the per-scene folded biases (once per scene).
//
// F (Sec. 3.4): sigma = ReLU(W_F2 ReLU(W_F1 s' + b_F1) + b_F2), s = 32 floats,
// s' = s or, with positional encoding, its 32 (1 + 2L) encoded values.
// The latent enters phi1 and B1 only through a matrix-vector product that is
// the same for every pixel, so it is folded into two bias vectors:
//   c_phi = W_phi1[:, 12 e:] sigma + b_phi1      (H)
//   c_B   = W_B1[:, 14 e + H:] sigma + b_B1      (H)
// (e = 1 + 2L bands) which is exact algebra of the concat form W [x ; sigma] + b.
#include "internal.h"

namespace gn {

void WeightIndex::build(int H_, int Z_, int L_, int RK_) {
  H = H_;
  Z = Z_;
  L = L_;
  RK = RK_;
  const int o[kLayers] = {Z, Z, H, H, H, H, H, H, kOut};
  const int i[kLayers] = {sc_enc(), Z, tc_enc() + Z, H, 2 * H, gc_enc() + H + Z, H, H * RK * RK, H};
  size_t at = 0;
  for (int l = 0; l < kLayers; ++l) {
    out[l] = o[l];
    in[l] = i[l];
    w[l] = at;
    at += static_cast<size_t>(o[l]) * i[l];
    b[l] = at;
    at += o[l];
  }
  total = at;
}

struct EncodeArgs {
  const float *Wf1, *bf1, *Wf2, *bf2, *Wp, *bp, *Wb, *bb;
  const float* scene;
  float* latent;
  int H, Z, L;
};

// One CTA of 256 threads; every dot product is a sequential FP32 sum in
// index order.
__global__ void __launch_bounds__(256) encode_kernel(EncodeArgs a) {
  __shared__ float s_in[kScene * (1 + 2 * kMaxPeFreqs)];
  __shared__ float s_h1[256];
  __shared__ float s_z[256];
  const int t = threadIdx.x;
  const int n_in = kScene * (1 + 2 * a.L);  // band b of channel c at b * 32 + c
  for (int i = t; i < n_in; i += blockDim.x) s_in[i] = pe_band_value(a.scene[i % kScene], i / kScene);
  __syncthreads();
  if (t < a.Z) {
    float acc = a.bf1[t];
    const float* row = a.Wf1 + static_cast<size_t>(t) * n_in;
    for (int i = 0; i < n_in; ++i) acc = fmaf(row[i], s_in[i], acc);
    s_h1[t] = fmaxf(acc, 0.0f);
  }
  __syncthreads();
  if (t < a.Z) {
    float acc = a.bf2[t];
    const float* row = a.Wf2 + static_cast<size_t>(t) * a.Z;
    for (int i = 0; i < a.Z; ++i) acc = fmaf(row[i], s_h1[i], acc);
    s_z[t] = fmaxf(acc, 0.0f);
    a.latent[t] = s_z[t];
  }
  __syncthreads();
  if (t < a.H) {
    float acc = a.bp[t];
    const int tce = kTC * (1 + 2 * a.L);
    const float* row = a.Wp + static_cast<size_t>(t) * (tce + a.Z) + tce;
    for (int i = 0; i < a.Z; ++i) acc = fmaf(row[i], s_z[i], acc);
    a.latent[a.Z + t] = acc;
  } else if (t < 2 * a.H) {
    const int n = t - a.H;
    float acc = a.bb[n];
    const int gce = kGC * (1 + 2 * a.L);
    const float* row = a.Wb + static_cast<size_t>(n) * (gce + a.H + a.Z) + gce + a.H;
    for (int i = 0; i < a.Z; ++i) acc = fmaf(row[i], s_z[i], acc);
    a.latent[a.Z + a.H + n] = acc;
  }
}

cudaError_t launch_encode(const float* w32, const WeightIndex& wi, const float* scene_dev,
                          float* latent_dev, cudaStream_t s) {
  EncodeArgs a;
  a.Wf1 = w32 + wi.w[LF1];
  a.bf1 = w32 + wi.b[LF1];
  a.Wf2 = w32 + wi.w[LF2];
  a.bf2 = w32 + wi.b[LF2];
  a.Wp = w32 + wi.w[LPHI1];
  a.bp = w32 + wi.b[LPHI1];
  a.Wb = w32 + wi.w[LB1];
  a.bb = w32 + wi.b[LB1];
  a.scene = scene_dev;
  a.latent = latent_dev;
  a.H = wi.H;
  a.Z = wi.Z;
  a.L = wi.L;
  encode_kernel<<<1, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace gn

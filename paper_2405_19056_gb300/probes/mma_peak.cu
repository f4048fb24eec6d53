// Tensor-core peak probe: cycles per tcgen05.mma (M = 128; kind::f16 with BF16
// operands, K = 16, or kind::f8f6f4 with E4M3 operands, K = 32) for shared- or
// TMEM-resident A and several N, back to back into one TMEM tile; one CTA per
// SM.  It measures the instruction rate only (no operand traffic), the upper
// bound for the fused kernels' GEMMs.
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        -o /tmp/mma_peak paper_2405_19056_gb300/probes/mma_peak.cu && /tmp/mma_peak
#include <cstdint>
#include <cstdio>
#include "../csrc/tc_ptx.cuh"
using namespace gn;

template <int N, bool TS, bool F8>
__global__ void bench(unsigned long long* out, int iters) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t slot;
  __shared__ __align__(8) uint64_t bar;
  const int warp = threadIdx.x / 32;
  // A: 128 x 64 bf16 (16 KB), B: N x 64 bf16, no swizzle, zero-filled
  for (int i = threadIdx.x; i < (128 + N) * 64 * 2 / 4; i += blockDim.x) ((uint32_t*)smem)[i] = (F8 ? 0x38383838u : 0x3f803f80u);
  fence_proxy_async_smem();
  if (warp == 0) { tmem_alloc(smem_u32(&slot), 512); tmem_relinquish(); }
  if (threadIdx.x == 0) { mbar_init(smem_u32(&bar), 1); fence_mbar_init(); }
  tc_fence_before(); __syncthreads(); tc_fence_after();
  const uint32_t tb = slot;
  if (threadIdx.x == 0) {
    const uint32_t sa = smem_u32(smem), sb = sa + 128 * 64 * 2;
    const uint32_t idesc = make_idesc(128, N, F8 ? kFmtE4M3 : kFmtBF16);
    uint64_t ad[4], bd[4];
    for (int k = 0; k < 4; ++k) { ad[k] = make_sdesc(sa + k * 2 * 128 * 16, 128 * 16, 128); bd[k] = make_sdesc(sb + k * 2 * N * 16, N * 16, 128); }
    // warm-up
    for (int i = 0; i < 8; ++i) { if (F8) { if (TS) mma_f8_ts(tb, tb + 256 + (i & 3) * 8, bd[i & 3], idesc, 1); else mma_f8_ss(tb, ad[i & 3], bd[i & 3], idesc, 1); } else { if (TS) mma_f16_ts(tb, tb + 256 + (i & 3) * 8, bd[i & 3], idesc, 1); else mma_f16_ss(tb, ad[i & 3], bd[i & 3], idesc, 1); } }
    mma_commit(smem_u32(&bar));
    mbar_wait(smem_u32(&bar), 0, 1000000000ull);
    unsigned long long t0 = clock64();
    for (int i = 0; i < iters; i += 4) {
#pragma unroll
      for (int k = 0; k < 4; ++k) { if (F8) { if (TS) mma_f8_ts(tb, tb + 256 + k * 8, bd[k], idesc, 1); else mma_f8_ss(tb, ad[k], bd[k], idesc, 1); } else { if (TS) mma_f16_ts(tb, tb + 256 + k * 8, bd[k], idesc, 1); else mma_f16_ss(tb, ad[k], bd[k], idesc, 1); } }
    }
    unsigned long long t1 = clock64();
    mma_commit(smem_u32(&bar));
    mbar_wait(smem_u32(&bar), 1, 1000000000ull);
    unsigned long long t2 = clock64();
    if (blockIdx.x == 0) { out[0] = t1 - t0; out[1] = t2 - t0; }
  }
  tc_fence_before(); __syncthreads();
  if (warp == 0) { tc_fence_after(); tmem_dealloc(tb, 512); }
}

template <int N, bool TS, bool F8>
void run(unsigned long long* d, int grid, int iters) {
  int smem = (128 + N) * 64 * 2;
  cudaFuncSetAttribute(bench<N, TS, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  bench<N, TS, F8><<<grid, 128, smem>>>(d, iters);
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0);
  bench<N, TS, F8><<<grid, 128, smem>>>(d, iters);
  cudaEventRecord(e1); cudaEventSynchronize(e1);
  float ms; cudaEventElapsedTime(&ms, e0, e1);
  unsigned long long h[2]; cudaMemcpy(h, d, 16, cudaMemcpyDeviceToHost);
  double flop_per_mma = 2.0 * 128 * N * (F8 ? 32 : 16);
  printf("%s N=%3d %s grid=%3d: issue %.1f clk/mma, complete %.1f clk/mma -> %.0f FLOP/clk/SM; wall %.3f ms -> %.1f TFLOP/s\n",
         F8 ? "e4m3" : "bf16", N, TS ? "TS" : "SS", grid, (double)h[0] / iters, (double)h[1] / iters, flop_per_mma * iters / h[1],
         ms, flop_per_mma * iters * grid / (ms * 1e-3) / 1e12);
}

int main() {
  unsigned long long* d; cudaMalloc(&d, 64);
  int iters = 1 << 16;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  for (int grid : {1, sms}) {
    run<128, false, false>(d, grid, iters); run<128, true, false>(d, grid, iters);
    run<256, false, false>(d, grid, iters);
    run<128, false, true>(d, grid, iters); run<128, true, true>(d, grid, iters);
    run<256, false, true>(d, grid, iters);
  }
  cudaError_t e = cudaDeviceSynchronize();
  printf("status: %s\n", cudaGetErrorString(e));
  return e != cudaSuccess;
}

// MMA issue probe: tcgen05.mma kind::f16 (BF16, M = 128, N = 128, K = 16)
// with A in TMEM, for several placements of the A and accumulator columns in
// a 512-column allocation: cycles per MMA while issuing, cycles per MMA to
// completion, and the round trip of 8 MMAs + commit + mbarrier wait (the
// hand-off unit of the fused kernels).
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        -o /tmp/mma_issue paper_2405_19056_gb300/probes/mma_issue.cu && /tmp/mma_issue
#include <cstdint>
#include <cstdio>
#include "../csrc/tc_ptx.cuh"
using namespace gn;

__global__ void bench(unsigned long long* out, int iters, int colD, int colA) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t slot;
  __shared__ __align__(8) uint64_t bar;
  const int warp = threadIdx.x / 32;
  constexpr int N = 128;
  // B: N x 64 bf16 (16 KB), no swizzle
  for (int i = threadIdx.x; i < N * 64 * 2 / 4; i += blockDim.x) ((uint32_t*)smem)[i] = 0x3f803f80u;
  fence_proxy_async_smem();
  if (warp == 0) { tmem_alloc(smem_u32(&slot), 512); tmem_relinquish(); }
  if (threadIdx.x == 0) { mbar_init(smem_u32(&bar), 1); fence_mbar_init(); }
  tc_fence_before(); __syncthreads(); tc_fence_after();
  const uint32_t tb = slot;
  if (threadIdx.x == 0) {
    const uint32_t sb = smem_u32(smem);
    const uint32_t idesc = make_idesc(128, N, kFmtBF16);
    uint64_t bd[4];
    for (int k = 0; k < 4; ++k) bd[k] = make_sdesc(sb + k * 2 * N * 16, N * 16, 128);
    for (int i = 0; i < 8; ++i) mma_f16_ts(tb + colD, tb + colA + (i & 3) * 8, bd[i & 3], idesc, 1);
    mma_commit(smem_u32(&bar));
    mbar_wait(smem_u32(&bar), 0, 1000000000ull);
    unsigned long long t0 = clock64();
    for (int i = 0; i < iters; i += 4) {
#pragma unroll
      for (int k = 0; k < 4; ++k) mma_f16_ts(tb + colD, tb + colA + k * 8, bd[k], idesc, 1);
    }
    unsigned long long t1 = clock64();
    mma_commit(smem_u32(&bar));
    mbar_wait(smem_u32(&bar), 1, 1000000000ull);
    unsigned long long t2 = clock64();
    // round trips: 8 MMAs + commit + wait
    unsigned long long t3 = clock64();
    for (int r = 0; r < 64; ++r) {
#pragma unroll
      for (int k = 0; k < 8; ++k) mma_f16_ts(tb + colD, tb + colA + (k & 3) * 8, bd[k & 3], idesc, 1);
      mma_commit(smem_u32(&bar));
      mbar_wait(smem_u32(&bar), r & 1, 1000000000ull);
    }
    unsigned long long t4 = clock64();
    if (blockIdx.x == 0) { out[0] = t1 - t0; out[1] = t2 - t0; out[2] = t4 - t3; }
  }
  tc_fence_before(); __syncthreads();
  if (warp == 0) { tc_fence_after(); tmem_dealloc(tb, 512); }
}

int main() {
  unsigned long long* d; cudaMalloc(&d, 64);
  const int iters = 1 << 14;
  const int smem = 128 * 64 * 2;
  cudaFuncSetAttribute(bench, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int place[][2] = {{0, 256}, {0, 128}, {256, 384}, {384, 320}, {384, 256}, {128, 448}, {0, 448}, {256, 0}};
  for (int grid : {1, 152}) {
    for (auto& p : place) {
      bench<<<grid, 128, smem>>>(d, iters, p[0], p[1]);
      unsigned long long h[3];
      cudaMemcpy(h, d, 24, cudaMemcpyDeviceToHost);
      printf("grid=%3d D=%3d A=%3d: issue %.1f clk/mma, complete %.1f clk/mma, round trip (8 MMAs + commit + wait) %.0f clk\n",
             grid, p[0], p[1], (double)h[0] / iters, (double)h[1] / iters, (double)h[2] / 64);
    }
  }
  cudaError_t e = cudaDeviceSynchronize();
  printf("status: %s\n", cudaGetErrorString(e));
  return e != cudaSuccess;
}

// TMEM contention probe: tcgen05.mma rate (BF16, M = 128, N = 128, K = 16)
// with A in TMEM (TS) or shared memory (SS) while W other warps stream
// tcgen05.ld (and tcgen05.st) over other TMEM columns of their lane quadrant,
// and the load loop's rate per warp (16-column loads, one in flight).
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 \
//        -o /tmp/tmem_contend paper_2405_19056_gb300/probes/tmem_contend.cu && /tmp/tmem_contend
#include <cstdint>
#include <cstdio>
#include "../csrc/tc_ptx.cuh"
using namespace gn;

template <bool TS>
__global__ void bench(unsigned long long* out, int iters, int nw_ld, int st) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t slot;
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int stop;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  constexpr int N = 128;
  for (int i = threadIdx.x; i < (128 + N) * 64 * 2 / 4; i += blockDim.x) ((uint32_t*)smem)[i] = 0x3f803f80u;
  fence_proxy_async_smem();
  if (warp == 0) { tmem_alloc(smem_u32(&slot), 512); tmem_relinquish(); }
  if (threadIdx.x == 0) { mbar_init(smem_u32(&bar), 1); fence_mbar_init(); stop = 0; }
  tc_fence_before(); __syncthreads(); tc_fence_after();
  const uint32_t tb = slot;
  if (warp == 0) {
    if (lane == 0) {
      const uint32_t sa = smem_u32(smem), sb = sa + 128 * 64 * 2;
      const uint32_t idesc = make_idesc(128, N, kFmtBF16);
      uint64_t ad[4], bd[4];
      for (int k = 0; k < 4; ++k) { ad[k] = make_sdesc(sa + k * 2 * 128 * 16, 128 * 16, 128); bd[k] = make_sdesc(sb + k * 2 * N * 16, N * 16, 128); }
      unsigned long long t0 = clock64();
      for (int i = 0; i < iters; i += 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) { if (TS) mma_f16_ts(tb, tb + 256 + k * 8, bd[k], idesc, 1); else mma_f16_ss(tb, ad[k], bd[k], idesc, 1); }
      }
      mma_commit(smem_u32(&bar));
      mbar_wait(smem_u32(&bar), 0, 1000000000ull);
      unsigned long long t1 = clock64();
      if (blockIdx.x == 0) out[0] = t1 - t0;
      stop = 1;
    }
    __syncwarp();
  } else if (warp <= nw_ld) {
    // TMEM traffic on columns 384..511 of this warp's lane quadrant
    const uint32_t q = warp & 3;
    const uint32_t base = tb + (q * 32 << 16) + 384;
    uint32_t r[16], acc = 0;
    long long n = 0;
    while (!stop && n < (1 << 22)) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        tmem_ld16_async(base + c * 16, r);
        tmem_wait_ld_tied(r);
        acc += r[0] ^ r[15];
        if (st) {
          uint32_t u[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) u[i] = r[2 * i] + r[2 * i + 1];
          tmem_st8(base + 64 + (c & 3) * 8, u);
        }
      }
      if (st) tmem_wait_st();
      ++n;
    }
    if (acc == 12345u) out[3] = acc;
    if (blockIdx.x == 0 && warp == 1 && lane == 0) out[1] = n;
  }
  tc_fence_before(); __syncthreads();
  if (warp == 0) { tc_fence_after(); tmem_dealloc(tb, 512); }
}

int main() {
  unsigned long long* d; cudaMalloc(&d, 64);
  const int iters = 1 << 14;
  const int smem = (128 + 128) * 64 * 2;
  cudaFuncSetAttribute(bench<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(bench<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  for (int st = 0; st < 2; ++st)
    for (int nw : {0, 4, 8, 12}) {
      for (int ts = 0; ts < 2; ++ts) {
        cudaMemset(d, 0, 64);
        if (ts) bench<true><<<152, 32 * 13, smem>>>(d, iters, nw, st);
        else bench<false><<<152, 32 * 13, smem>>>(d, iters, nw, st);
        unsigned long long h[2];
        cudaMemcpy(h, d, 16, cudaMemcpyDeviceToHost);
        printf("%s ld%s warps=%2d: %.1f clk/mma (ld loop iters %llu)\n", ts ? "TS" : "SS", st ? "+st" : "   ", nw,
               (double)h[0] / iters, h[1]);
      }
    }
  cudaError_t e = cudaDeviceSynchronize();
  printf("status: %s\n", cudaGetErrorString(e));
  return e != cudaSuccess;
}

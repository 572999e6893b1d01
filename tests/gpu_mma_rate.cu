// Issue rate of tcgen05.mma (M = 128, K = 16, bf16 inputs, float32 accumulator) for N = 64, 128
// and 256: one CTA per SM issues back-to-back MMAs from fixed, zeroed shared-memory tiles into one
// TMEM accumulator and times them with clock64; prints cycles per MMA and flops per clock per SM.
// Run by tests/test_gpu_mma_rate.py.
#include <cuda.h>
#include <cstdio>
#include <cstdint>
#include "../paper_1107_4192_gb300/csrc/tc_ptx.cuh"
using namespace kfm;

template <int NN>
__global__ void __launch_bounds__(128, 1) rate_kernel(int reps, long long* out, int* flag) {
  extern __shared__ __align__(1024) uint8_t sm[];
  // A: 128 rows x 32 B (4 KB) at 0; B: NN rows x 32 B at 4096; zero-filled
  for (int i = threadIdx.x; i < (4096 + NN * 32) / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(sm)[i] = 0u;
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const uint32_t base = smem_u32(sm);
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&tslot)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  if (threadIdx.x == 0) {
    const uint64_t ad = smem_desc_sw(base, 256, kLayoutSw32);
    const uint64_t bd = smem_desc_sw(base + 4096, 256, kLayoutSw32);
    long long t0 = clock64();
    for (int r = 0; r < reps; ++r) mma_bf16(tmem, ad, bd, IDESC, r > 0 ? 1u : 0u);
    mma_commit(smem_u32(&bar));
    volatile int never = 0;
    const bool ok = mbar_wait(smem_u32(&bar), 0, &never);
    long long t1 = clock64();
    if (!ok) *flag = 1;
    out[blockIdx.x] = t1 - t0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
  }
}

template <int NN>
void run(int reps) {
  long long* d; int* f;
  cudaMalloc(&d, 152 * sizeof(long long)); cudaMalloc(&f, 4); cudaMemset(f, 0, 4);
  const int smem = 4096 + NN * 32 + 1024;
  cudaFuncSetAttribute(rate_kernel<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  rate_kernel<NN><<<152, 128, smem>>>(reps, d, f);
  cudaError_t e = cudaDeviceSynchronize();
  long long h[152]; int hf = 0;
  cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost); cudaMemcpy(&hf, f, 4, cudaMemcpyDeviceToHost);
  long long mx = 0; for (int i = 0; i < 152; ++i) mx = h[i] > mx ? h[i] : mx;
  printf("N=%d: %s timeout=%d  %.1f cycles per MMA (128x%dx16), %.0f flop/clk/SM\n", NN, cudaGetErrorString(e), hf,
         (double)mx / reps, NN, 2.0 * 128 * NN * 16 * reps / (double)mx);
  cudaFree(d); cudaFree(f);
}

int main() {
  for (int i = 0; i < 2; ++i) { run<64>(4096); run<128>(4096); run<256>(4096); }
  return 0;
}

// Microbenchmarks of the B300 resources the DSES kernels are bound by:
// shared-memory atomic increments (random bins of a vote-sized histogram,
// bank-distinct bins, one shared bin), FP32 FMA issue, and random 4-byte and
// 16-byte gathers from L2-resident tables. Each returns operations per second
// measured with CUDA events; used to state roofline fractions.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 1024;
constexpr int kAddrPerThread = 16;

// mode 0: random bins in [0, nbins); 1: bin = lane + 32 k (one per bank);
// 2: every lane the same bin
__global__ void __launch_bounds__(kThreads, 1) smem_atomic_kernel(int nbins, int mode, int reps,
                                                                  unsigned long long* sink) {
  extern __shared__ uint32_t hist[];
  for (int i = threadIdx.x; i < nbins; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  uint32_t addr[kAddrPerThread];
  uint32_t x = 0x9E3779B9u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(hist);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kAddrPerThread; ++k) {
    x ^= x << 13; x ^= x >> 17; x ^= x << 5;
    uint32_t b;
    if (mode == 0) b = x % (uint32_t)nbins;
    else if (mode == 1) b = (uint32_t)((lane + 32 * (warp * kAddrPerThread + k)) % nbins);
    else b = 0;
    addr[k] = base + 4u * b;
  }
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int k = 0; k < kAddrPerThread; ++k) asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr[k]));
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(sink, (unsigned long long)hist[0]);
}

__global__ void __launch_bounds__(kThreads, 1) ffma_kernel(int reps, float* sink) {
  float a0 = threadIdx.x * 1e-7f, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
        a7 = a0 + 7;
  const float m = 0.999999f, c = 1e-7f;
  for (int r = 0; r < reps; ++r) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fmaf(a0, m, c); a1 = fmaf(a1, m, c); a2 = fmaf(a2, m, c); a3 = fmaf(a3, m, c);
      a4 = fmaf(a4, m, c); a5 = fmaf(a5, m, c); a6 = fmaf(a6, m, c); a7 = fmaf(a7, m, c);
    }
  }
  const float s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 12345.678f) *sink = s;
}

__global__ void l2_gather_kernel(const float* __restrict__ table, uint32_t n, int reps, float* sink) {
  uint32_t x = 0x2545F491u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
  float acc = 0.f;
  for (int r = 0; r < reps; ++r) {
#pragma unroll 8
    for (int k = 0; k < 8; ++k) {
      x ^= x << 13; x ^= x >> 17; x ^= x << 5;
      acc += __ldcg(table + (x % n));
    }
  }
  if (acc == 12345.678f) *sink = acc;
}

__global__ void l2_gather16_kernel(const float4* __restrict__ table, uint32_t n, int reps, float* sink) {
  uint32_t x = 0x2545F491u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
  float acc = 0.f;
  for (int r = 0; r < reps; ++r) {
#pragma unroll 8
    for (int k = 0; k < 8; ++k) {
      x ^= x << 13; x ^= x >> 17; x ^= x << 5;
      const float4 v = __ldcg(table + (x % n));
      acc += v.x + v.w;
    }
  }
  if (acc == 12345.678f) *sink = acc;
}

float time_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace

// out[0..2]: shared atomics/s (random, bank-distinct, same bin) over a
// histogram of nbins 32-bit words; out[3]: FP32 FMA/s; out[4]: random 4-byte
// L2 gathers/s from a table of table_bytes; out[5]: random 16-byte (aligned)
// L2 gathers/s from a table of table16_bytes. Returns 0 or a cudaError_t.
extern "C" int dses_peaks_run(int device, int nbins, size_t table_bytes, size_t table16_bytes, double* out) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return (int)e;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  unsigned long long* sink = nullptr;
  float* fsink = nullptr;
  float* table = nullptr;
  float4* table16 = nullptr;
  const uint32_t n = (uint32_t)(table_bytes / 4), n16 = (uint32_t)(table16_bytes / 16);
  if ((e = cudaMalloc(&sink, 8)) != cudaSuccess) return (int)e;
  if ((e = cudaMalloc(&fsink, 8)) != cudaSuccess) return (int)e;
  if ((e = cudaMalloc(&table, (size_t)n * 4)) != cudaSuccess) return (int)e;
  cudaMemset(table, 0, (size_t)n * 4);
  if ((e = cudaMalloc(&table16, (size_t)n16 * 16)) != cudaSuccess) return (int)e;
  cudaMemset(table16, 0, (size_t)n16 * 16);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int smem = nbins * 4;
  cudaFuncSetAttribute(smem_atomic_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int reps = 2000;
  for (int mode = 0; mode < 3; ++mode) {
    const int rr = mode == 2 ? reps / 16 : reps;
    smem_atomic_kernel<<<sms, kThreads, smem>>>(nbins, mode, 10, sink);  // warm-up
    cudaEventRecord(a);
    smem_atomic_kernel<<<sms, kThreads, smem>>>(nbins, mode, rr, sink);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    out[mode] = (double)sms * kThreads * kAddrPerThread * rr / (time_ms(a, b) * 1e-3);
  }
  const int freps = 4000;
  ffma_kernel<<<sms, kThreads>>>(10, fsink);
  cudaEventRecord(a);
  ffma_kernel<<<sms, kThreads>>>(freps, fsink);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  out[3] = (double)sms * kThreads * 8 * 16 * freps / (time_ms(a, b) * 1e-3);
  const int greps = 256, gblocks = sms * 8;
  l2_gather_kernel<<<gblocks, 256>>>(table, n, 4, fsink);
  cudaEventRecord(a);
  l2_gather_kernel<<<gblocks, 256>>>(table, n, greps, fsink);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  out[4] = (double)gblocks * 256 * 8 * greps / (time_ms(a, b) * 1e-3);
  l2_gather16_kernel<<<gblocks, 256>>>(table16, n16, 4, fsink);
  cudaEventRecord(a);
  l2_gather16_kernel<<<gblocks, 256>>>(table16, n16, greps, fsink);
  cudaEventRecord(b);
  cudaEventSynchronize(b);
  out[5] = (double)gblocks * 256 * 8 * greps / (time_ms(a, b) * 1e-3);
  e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  cudaFree(fsink);
  cudaFree(table);
  cudaFree(table16);
  return (int)e;
}

// Peak-rate microbenchmarks of this GPU (measurement only, not part of the
// amplitude path; built into its own library, libpeps_peaks.so):
//   * FP32 FMA rate of the CUDA cores (the ceiling of the FP32 CUDA-core
//     contraction form): 8 independent FMA chains per thread;
//   * dense tensor-core rate of tcgen05.mma for kind::f16 and kind::tf32
//     (the ceilings of the FP16/BF16 and TF32 forms): one CTA per SM, one
//     thread issuing M = 128, N = 256 MMAs back to back on operands held in
//     shared memory, accumulating into TMEM.  No global memory traffic, so
//     the rate is the tensor pipe's.
// Every wait is bounded (a %globaltimer deadline); an expired wait sets the
// error flag and the kernel still releases its TMEM.
#include <cuda_runtime.h>
#include <stdint.h>

#define PEAKS_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr int MMA_M = 128, MMA_N = 256;
constexpr int ROWB = 128;             // bytes of K per smem row (128-byte swizzle)
constexpr int KSTEPS = ROWB / 32;     // 32 bytes of K per MMA (16 f16 or 8 tf32)
constexpr int THREADS = 128;
constexpr uint64_t WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(256) k_fma(int iters, float *sink) {
  float a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 1.0f + 1e-3f * (float)((threadIdx.x + j) & 15);
  const float b = 0.9999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fmaf(a[j], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == -1.0f) sink[0] = s;  // never true; keeps the chains live
}

// K-major 128-byte-swizzled tile descriptor (8-row groups 1024 bytes apart).
__device__ __forceinline__ uint64_t sdesc128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)((8u * ROWB) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

template <int TF32>
__global__ void __launch_bounds__(THREADS, 1) k_mma(int iters, int *err) {
  extern __shared__ __align__(1024) unsigned char raw[];
  unsigned char *sm = (unsigned char *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sa = sm;                          // 128 rows x 128 B
  unsigned char *sb = sm + MMA_M * ROWB;           // 256 rows x 128 B
  uint64_t *bar = (uint64_t *)(sb + MMA_N * ROWB);
  uint32_t *tslot = (uint32_t *)(bar + 1);
  const int warp = threadIdx.x >> 5;

  // operands: finite values of both signs in [1, 2), from a hash of the index
  uint32_t *wa = (uint32_t *)sm;
  const int words = (MMA_M + MMA_N) * ROWB / 4;
  for (int i = threadIdx.x; i < words; i += THREADS) {
    uint32_t h = (uint32_t)i * 2654435761u ^ (blockIdx.x * 40503u);
    h ^= h >> 13;
    h *= 0x5bd1e995u;
    h ^= h >> 15;
    if (TF32) {
      wa[i] = 0x3F800000u | (h & 0x807FE000u);
    } else {
      const uint32_t lo = 0x3C00u | (h & 0x83FFu), hi = 0x3C00u | ((h >> 16) & 0x83FFu);
      wa[i] = lo | (hi << 16);
    }
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
        smem_u32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (threadIdx.x == 32) {
    const uint32_t ab = TF32 ? 2u : 0u;  // operand format: F16 = 0, TF32 = 2
    const uint32_t idesc = (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(MMA_N >> 3) << 17) |
                           ((uint32_t)(MMA_M >> 4) << 24);
    const uint64_t da = sdesc128(smem_u32(sa)), db = sdesc128(smem_u32(sb));
    for (int i = 0; i < iters; ++i) {
      const uint32_t d = tmem + (uint32_t)((i & 1) * MMA_N);
#pragma unroll
      for (int ks = 0; ks < KSTEPS; ++ks) {
        const uint64_t a = da + (uint64_t)(ks * 2), b = db + (uint64_t)(ks * 2);
        const uint32_t acc = (i > 1 || ks > 0) ? 1u : 0u;
        if (TF32)
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
              "l"(a), "l"(b), "r"(idesc), "r"(acc));
        else
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
              "l"(a), "l"(b), "r"(idesc), "r"(acc));
      }
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
  }
  // everyone waits for the MMAs to retire (bounded)
  if (threadIdx.x % 32 == 0) {
    const uint64_t deadline = globaltimer() + WAIT_NS;
    uint32_t ok = 0;
    while (!ok) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(smem_u32(bar))
          : "memory");
      if (!ok && globaltimer() > deadline) {
        atomicExch(err, 1);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return n;
}

template <typename F>
int time_ms(F launch, float *ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1;
  if (cudaEventCreate(&e1) != cudaSuccess) return -1;
  launch();  // warm-up
  cudaEventRecord(e0);
  launch();
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e == cudaSuccess ? 0 : -2;
}

}  // namespace

// FP32 FMA rate in TFLOP/s (2 flops per FMA) over `iters` loop trips.
PEAKS_API int peaks_fma_tflops(int iters, double *tflops, double *ms_out) {
  const int sms = sm_count();
  if (sms <= 0 || iters <= 0 || !tflops) return -1;
  float *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return -3;
  const int blocks = sms * 8, threads = 256;
  float ms = 0.f;
  const int rc = time_ms([&] { k_fma<<<blocks, threads>>>(iters, sink); }, &ms);
  cudaFree(sink);
  if (rc) return rc;
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return 0;
}

// Dense tcgen05 rate in TFLOP/s: kind = 0 for kind::f16, 1 for kind::tf32.
PEAKS_API int peaks_mma_tflops(int kind, int iters, double *tflops, double *ms_out) {
  const int sms = sm_count();
  if (sms <= 0 || iters <= 1 || !tflops || (kind != 0 && kind != 1)) return -1;
  int *err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return -3;
  cudaMemset(err, 0, sizeof(int));
  const size_t smem = 1024 + (size_t)(MMA_M + MMA_N) * ROWB + 16;
  auto kern = kind ? k_mma<1> : k_mma<0>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaFree(err);
    return -4;
  }
  float ms = 0.f;
  const int rc = time_ms([&] { kern<<<sms, THREADS, smem>>>(iters, err); }, &ms);
  int h_err = 0;
  cudaMemcpy(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (rc) return rc;
  if (h_err) return -5;
  const double k_per_mma = kind ? 8.0 : 16.0;
  const double flops = 2.0 * MMA_M * MMA_N * k_per_mma * KSTEPS * (double)iters * sms;
  *tflops = flops / (ms * 1e-3) / 1e12;
  if (ms_out) *ms_out = ms;
  return 0;
}

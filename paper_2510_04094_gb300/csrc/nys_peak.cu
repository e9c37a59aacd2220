// Arithmetic-peak probes (declared in include/nys_peak.h): the denominators of
// the roofline fractions, measured on the device instead of taken from a data
// sheet.  Each probe keeps one pipe busy with independent work and reports the
// operations it performed; the caller times the launch with CUDA events.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nys_peak.h"
#include "nys_tc.cuh"

namespace {

using namespace nys;

constexpr int kFmaThreads = 256;
constexpr int kFmaChains = 8;     // independent accumulators per thread
constexpr int kFmaUnroll = 16;

// FP32 / FP64 FMA chains: a <- a * b + c with |b| < 1, kFmaChains independent
// chains per thread; the result feeds a store under a runtime flag (always 0),
// so the compiler cannot drop the chains.
__device__ double g_peak_sink[kFmaThreads];

template <typename T>
__global__ void __launch_bounds__(kFmaThreads)
k_peak_fma(int iters, T b, T c, int keep) {
  T a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kFmaUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += a[k];
  if (keep) g_peak_sink[threadIdx.x] = (double)s;
}

// Instruction descriptor of kind::f16 with bf16 A and B (both K-major), F32 D:
// D type at bits 4-5 (1 = F32), A type bits 7-9 and B type bits 10-12
// (1 = BF16), N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ inline uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}

constexpr int kMmaM = 128, kMmaN = 256;
constexpr int kMmaThreads = 128;
constexpr int kTileA = kMmaM * 128;          // bytes: 128 rows x 128-byte swizzled K row
constexpr int kTileB = kMmaN * 128;
constexpr int kMmaSmem = kTileA + kTileB + 1024;
constexpr int kMmaWaitIter = 1 << 22;        // polls of <= 1 us each

// One CTA per SM: warp 0 holds kMmaN tensor-memory columns (one FP32
// accumulator of 128 lanes x 256 columns); one thread issues 4 K steps per
// trip (the 128-byte operand row holds 32 TF32 or 64 bf16 values) back to back
// into it, commits once and waits (bounded) for completion.  The operands are
// small finite values; the results are never read.
template <bool kBf16>
__global__ void __launch_bounds__(kMmaThreads, 1)
k_peak_mma(int iters, int32_t* __restrict__ err) {
  extern __shared__ unsigned char pk_raw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(pk_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t s_done;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < (kTileA + kTileB) / 4; e += kMmaThreads) {
    const float v = 0.25f + 0.001f * (float)(e & 63);
    uint32_t w = __float_as_uint(v);
    if (kBf16) {   // two bf16 copies of v (the high halves of its FP32 pattern)
      const uint32_t h = w >> 16;
      w = (h << 16) | h;
    }
    reinterpret_cast<uint32_t*>(sm)[e] = w;
  }
  if (warp == 0) tmem_alloc(smem_u32(&s_tmem), (uint32_t)kMmaN);
  if (tid == 0) {
    mbar_init(smem_u32(&s_done), 1);
    mbar_fence_init();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  if (tid == 0) {
    const uint32_t a0 = smem_u32(sm), b0 = a0 + (uint32_t)kTileA;
    const uint32_t idesc = kBf16 ? idesc_bf16(kMmaM, kMmaN) : tc_idesc_tf32(kMmaM, kMmaN);
    uint32_t acc = 0;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const uint64_t da = tc_desc_sw128(a0 + 32u * t), db = tc_desc_sw128(b0 + 32u * t);
        if (kBf16) mma_bf16(tmem, da, db, idesc, acc);
        else tc_mma_tf32(tmem, da, db, idesc, acc);
        acc = 1;
      }
    }
    tc_commit(smem_u32(&s_done));
    if (!mbar_wait_bounded(smem_u32(&s_done), 0, kMmaWaitIter) && err) atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)kMmaN);
}

}  // namespace

extern "C" int32_t nys_peak_launch(int32_t kind, int32_t iters, void* stream, int32_t* err_word,
                                   double* flops_out) {
  if (iters <= 0 || kind < NYS_PEAK_FFMA || kind > NYS_PEAK_BF16_MMA) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -3;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -3;
  double flops = 0.0;
  if (kind == NYS_PEAK_FFMA || kind == NYS_PEAK_DFMA) {
    const int grid = 4 * sms;
    const double per_thread = 2.0 * kFmaChains * kFmaUnroll * (double)iters;
    flops = per_thread * (double)grid * kFmaThreads;
    if (kind == NYS_PEAK_FFMA)
      k_peak_fma<float><<<grid, kFmaThreads, 0, st>>>(iters, 0.9999999f, 1e-7f, 0);
    else
      k_peak_fma<double><<<grid, kFmaThreads, 0, st>>>(iters, 0.9999999999, 1e-12, 0);
  } else {
    const bool bf16 = (kind == NYS_PEAK_BF16_MMA);
    const double k_per_trip = bf16 ? 64.0 : 32.0;   // 4 K steps of 16 (bf16) or 8 (tf32)
    flops = 2.0 * kMmaM * kMmaN * k_per_trip * (double)iters * sms;
    cudaError_t e;
    if (bf16) {
      e = cudaFuncSetAttribute(k_peak_mma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem);
      if (e == cudaSuccess) k_peak_mma<true><<<sms, kMmaThreads, kMmaSmem, st>>>(iters, err_word);
    } else {
      e = cudaFuncSetAttribute(k_peak_mma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMmaSmem);
      if (e == cudaSuccess) k_peak_mma<false><<<sms, kMmaThreads, kMmaSmem, st>>>(iters, err_word);
    }
    if (e != cudaSuccess) return -3;
  }
  if (cudaGetLastError() != cudaSuccess) return -3;
  if (flops_out) *flops_out = flops;
  return 0;
}

// Throughput probes of this device's arithmetic pipes, used as the peaks of
// the roofline fractions the library reports: FP64 and FP32 fused multiply-add
// on the CUDA cores, the special-function unit's exp2, and dense tcgen05
// products of FP16 and TF32 operands with FP32 accumulation (the form of the
// tensor-core sketch: operand A in tensor memory, B in shared memory).
//
// Each probe launches a fixed amount of independent work on every SM, times
// the launch with CUDA events on the caller's stream and returns the best of
// a few launches.  Inputs are constants; the results are kept alive by a
// store that never happens (the value cannot equal the sentinel).
#include <cuda_fp16.h>

#include <algorithm>

#include "h2_internal.cuh"
#include "tc_ptx.cuh"

namespace h2 {
namespace {

constexpr int kChains = 8;   // independent dependency chains per thread

template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T a, T b, T *sink) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == (T)-12345.0) sink[threadIdx.x] = s;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One special-function operation per step and chain: OP 0 exp2 (x <- 2^-x
// stays in [0.5, 1]), 1 square root and 2 reciprocal square root (x <-
// op(x + 1) stays in [1, 2]).
template <int OP>
__global__ void __launch_bounds__(256) k_sfu_peak(int iters, float *sink) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 0.5f + 0.01f * c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (OP == 0) x[c] = ex2_approx(-x[c]);
      else if constexpr (OP == 1) x[c] = sqrt_approx(x[c] + 1.f);
      else x[c] = rsqrt_approx(x[c] + 1.f);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -12345.f) sink[threadIdx.x] = s;
}

// One CTA per SM, 4 warps.  Thread 0 issues `iters` x 4 K-steps of
// D(128 x 256, FP32, TMEM) += A(128 x K, TMEM) * B(K x 256, shared memory,
// K-major 128-byte swizzle); K = 16 FP16 or 8 TF32 values per step.  All
// operands are zero.  The waits are bounded; a timeout sets *err.
constexpr int kPeakN = 256;
constexpr uint32_t kPeakB = kPeakN * 128;   // one 128-byte row per column of B

template <bool F16>
__global__ void __launch_bounds__(128, 1) k_mma_peak(int iters, int *err) {
  extern __shared__ unsigned char smem_dyn[];
  unsigned char *sB = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  __shared__ uint64_t done;
  __shared__ uint32_t tmem_base;
  const int t = threadIdx.x, warp = t >> 5;
  for (uint32_t q = t; q < kPeakB / 16; q += blockDim.x)
    reinterpret_cast<uint4 *>(sB)[q] = make_uint4(0u, 0u, 0u, 0u);
  if (t == 0) {
    mbar_init(saddr(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     saddr(&tmem_base)),
                 "n"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // shared-memory writes become visible to the tensor core's async proxy
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t a_col = tbase + kPeakN;   // A: 32 columns after the accumulator
  {
    // zero this warp's 32 lanes of the A columns
    uint32_t z[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    const uint32_t lane_addr = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int c = 0; c < 32; c += 8) tmem_st8(a_col + lane_addr + c, z);
    tmem_st_wait();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (t == 0) {
    constexpr uint32_t idesc = idesc_mma(F16, 128, kPeakN);
    const uint32_t b0 = saddr(sB);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        mma_ts<F16>(tbase, a_col + ks * 8, desc_sw128(b0 + ks * 32), idesc,
                    (i | ks) ? 1u : 0u);
    }
    mma_commit(saddr(&done));
    if (!mbar_wait(saddr(&done), 0u)) {
      atomicExch(err, 1);
      mbar_wait(saddr(&done), 0u);   // once more before the memory is released
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase),
                 "n"(512));
}

template <typename F>
double best_ms(cudaStream_t s, int reps, F &&launch) {
  cudaEvent_t e0, e1;
  H2_CUDA(cudaEventCreate(&e0));
  H2_CUDA(cudaEventCreate(&e1));
  launch();   // warm-up
  H2_CUDA(cudaStreamSynchronize(s));
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    H2_CUDA(cudaEventRecord(e0, s));
    launch();
    H2_CUDA(cudaEventRecord(e1, s));
    H2_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    H2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace
}  // namespace h2

using namespace h2;

extern "C" h2_status h2_measure_peak(int which, h2_stream_t stream, double *value) {
  if (!value || which < 0 || which > 6) return fail(H2_ERR_ARG, "h2_measure_peak: bad arguments");
  try {
    cudaStream_t s = (cudaStream_t)stream;
    const int sms = device_sm_count();
    const int reps = 5;
    if (which <= 1) {   // FMA: 2 flops each
      const int blocks = sms * 8, threads = 256, iters = which == 0 ? 2048 : 16384;
      DBuf<double> sink;
      sink.alloc(256);
      double ms = best_ms(s, reps, [&]() {
        if (which == 0)
          k_fma_peak<double><<<blocks, threads, 0, s>>>(iters, 0.999999, 1e-7, sink.p);
        else
          k_fma_peak<float><<<blocks, threads, 0, s>>>(iters, 0.999f, 1e-4f,
                                                       reinterpret_cast<float *>(sink.p));
        count_launch();
        H2_CHECK_LAUNCH();
      });
      const double flops = 2.0 * kChains * (double)iters * blocks * threads;
      *value = flops / (ms * 1e-3) / 1e12;   // TFLOP/s
    } else if (which == 2 || which >= 5) {   // special-function operations per second
      const int blocks = sms * 8, threads = 256, iters = 4096;
      DBuf<float> sink;
      sink.alloc(256);
      auto kern = which == 2 ? k_sfu_peak<0> : (which == 5 ? k_sfu_peak<1> : k_sfu_peak<2>);
      double ms = best_ms(s, reps, [&]() {
        kern<<<blocks, threads, 0, s>>>(iters, sink.p);
        count_launch();
        H2_CHECK_LAUNCH();
      });
      *value = (double)kChains * iters * blocks * threads / (ms * 1e-3) / 1e9;   // Gop/s
    } else {   // tensor cores: 3 = FP16, 4 = TF32
      const bool f16 = which == 3;
      const int iters = 2048;
      DBuf<int> err;
      err.alloc_zero(1, s);
      // 129 KB of shared memory: one CTA per SM, so each SM gets its own
      const size_t smem = 128 * 1024 + 1024;
      auto kern = f16 ? k_mma_peak<true> : k_mma_peak<false>;
      H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      double ms = best_ms(s, reps, [&]() {
        kern<<<sms, 128, smem, s>>>(iters, err.p);
        count_launch();
        H2_CHECK_LAUNCH();
      });
      if (to_host(err.p, 1, s)[0] != 0)
        return fail(H2_ERR_TIMEOUT, "h2_measure_peak: a tensor-core wait ran out");
      const double k = f16 ? 16.0 : 8.0;
      const double flops = 2.0 * 128 * kPeakN * k * 4 * (double)iters * sms;
      *value = flops / (ms * 1e-3) / 1e12;   // TFLOP/s
    }
    return H2_OK;
  } catch (const Error &e) {
    return fail(e.code, e.msg);
  }
}

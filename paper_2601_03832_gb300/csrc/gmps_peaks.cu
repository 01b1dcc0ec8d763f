// Peak-rate microbenchmarks of the units the iterative-Grover kernels are
// bound by (libgmps_peaks.so, declared in include/gmps_peaks.h): FP64 FMA
// and FP32 FMA issue over the whole chip, and shared-memory read bandwidth.
// They are the denominators of the reported roofline fractions; the caller
// times each launch with CUDA events on the stream it passes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gmps_peaks.h"

namespace {

constexpr int kChains = 8;   // independent FMA chains per thread
constexpr int kUnroll = 4;   // chain rounds per loop trip

// kChains independent a <- a*b + c chains per thread (b < 1, c > 0 keep the
// values finite and normal); the sum is stored only if it matches an
// impossible value, so the work cannot be dropped.
template <class T>
__global__ void __launch_bounds__(256) fma_chains(long long trips, T b, T c, T* sink) {
  T a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (long long i = 0; i < trips; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
    }
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == (T)-1) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Every thread reads 16-byte words of a 32 KiB shared buffer, consecutive
// threads consecutive words (no bank conflicts), `trips` rounds of 8 reads.
__global__ void __launch_bounds__(256) smem_reads(long long trips, float* sink) {
  constexpr int kWords = 2048;  // 32 KiB of float4
  __shared__ float4 buf[kWords];
  for (int i = threadIdx.x; i < kWords; i += blockDim.x) buf[i] = make_float4(i, i + 1, i + 2, i + 3);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int idx = threadIdx.x;
  for (long long t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float4 v = buf[(idx + u * 256) & (kWords - 1)];
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    idx = (idx + 32) & (kWords - 1);
  }
  const float s = acc.x + acc.y + acc.z + acc.w;
  if (s == -1.f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int gmps_peak_launch(int kind, int blocks, int threads, long long trips, void* stream, void* sink,
                                double* work) {
  if (blocks < 1 || threads < 32 || threads > 256 || threads % 32 || trips < 1 || !work) return 1;
  cudaStream_t s = (cudaStream_t)stream;
  const double nthreads = (double)blocks * threads;
  switch (kind) {
    case GMPS_PEAK_FP64_FMA:
      fma_chains<double><<<blocks, threads, 0, s>>>(trips, 0.999999, 1e-6, (double*)sink);
      *work = 2.0 * kChains * kUnroll * (double)trips * nthreads;
      break;
    case GMPS_PEAK_FP32_FMA:
      fma_chains<float><<<blocks, threads, 0, s>>>(trips, 0.999999f, 1e-6f, (float*)sink);
      *work = 2.0 * kChains * kUnroll * (double)trips * nthreads;
      break;
    case GMPS_PEAK_SMEM_READ:
      if (threads != 256) return 1;
      smem_reads<<<blocks, threads, 0, s>>>(trips, (float*)sink);
      *work = 16.0 * 8 * (double)trips * nthreads;
      break;
    default:
      return 1;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

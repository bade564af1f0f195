// Arithmetic peak probes (not part of the method): the FP32 FFMA and FP64 DFMA issue rates of the
// GPU, measured by kernels of independent FMA chains over every SM, so that the ALU-bound stages
// can be quoted against a measured peak as well as the one derived from unit counts and clocks.
// Each thread runs kChains independent chains of `iters` dependent FMAs whose result is written
// out (so nothing is optimised away); flops = 2 x threads x kChains x iters (x 2 for the paired
// FP32 form, mode 2).
#include "doa_internal.cuh"

namespace doa {
namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(int iters, T *out) {
  T a[kChains];
  const T x = (T)1.0000001, y = (T)0.9999999;
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Paired FP32 form (fma.rn.f32x2: two FP32 FMAs per instruction): kChains chains of float pairs.
__global__ void __launch_bounds__(kProbeThreads) fma2_probe_kernel(int iters, float *out) {
  unsigned long long a[kChains];
  const float2 xf = make_float2(1.0000001f, 1.0000001f), yf = make_float2(0.9999999f, 0.9999999f);
  const unsigned long long x = *reinterpret_cast<const unsigned long long *>(&xf);
  const unsigned long long y = *reinterpret_cast<const unsigned long long *>(&yf);
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    const float2 v = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x + 2 * c));
    a[c] = *reinterpret_cast<const unsigned long long *>(&v);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[c]) : "l"(x), "l"(y));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    const float2 v = *reinterpret_cast<const float2 *>(&a[c]);
    s += v.x + v.y;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace doa

using namespace doa;

extern "C" doa_status doa_probe_fma(int fp64, int blocks, int iters, void *out, double *flops, void *stream) {
  if (!out || !flops || blocks < 1 || iters < 1) return DOA_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (fp64 == 1)
    fma_probe_kernel<double><<<blocks, kProbeThreads, 0, s>>>(iters, static_cast<double *>(out));
  else if (fp64 == 2)
    fma2_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(iters, static_cast<float *>(out));
  else
    fma_probe_kernel<float><<<blocks, kProbeThreads, 0, s>>>(iters, static_cast<float *>(out));
  *flops = (fp64 == 2 ? 4.0 : 2.0) * blocks * kProbeThreads * (double)kChains * iters;
  return cudaGetLastError() == cudaSuccess ? DOA_OK : DOA_ECUDA;
}

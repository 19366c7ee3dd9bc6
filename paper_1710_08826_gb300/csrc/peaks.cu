// peaks.cu -- FMA-pipe micro-benchmark: the denominators of the arithmetic rooflines.
//
// The FP64 likelihood kernels of this library are bound by GB300's FP64 pipe, whose rate is
// not in any published sheet for this part, and the FP32 kernels by instruction issue.  This
// kernel measures the sustained fused-multiply-add rate of one pipe: every thread runs
// kChains independent dependency chains x <- x * a + b for `iters` rounds of kUnroll steps,
// so that the pipe, not the latency of one chain, bounds the rate.  Three forms:
//   GOO_PEAK_F64    fma.rn.f64
//   GOO_PEAK_F32    fma.rn.f32
//   GOO_PEAK_F32X2  fma.rn.f32x2 (two lanes per instruction)
// The result counts FMAs (one per lane), so FLOP/s = 2 x the returned rate.
#include <cuda_runtime.h>

#include "common.cuh"

namespace goo {

constexpr int kPeakChains = 8;
constexpr int kPeakUnroll = 16;
constexpr int kPeakBlock = 256;
constexpr int kPeakBlocksPerSm = 4;

template <typename T>
__global__ void __launch_bounds__(kPeakBlock) peak_fma_kernel(T a, T b, int iters, T* sink) {
  T x[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) x[j] = T(threadIdx.x) * T(1e-6) + T(j);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kPeakChains; ++j) x[j] = fma(x[j], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += x[j];
  if (s == T(-1.25e-30)) *sink = s;  // never true; keeps the chains alive
}

__global__ void __launch_bounds__(kPeakBlock) peak_fma2_kernel(float a, float b, int iters, float* sink) {
  float2 x[kPeakChains];
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) x[j] = make_float2(threadIdx.x * 1e-6f + j, threadIdx.x * 2e-6f + j);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int j = 0; j < kPeakChains; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kPeakChains; ++j) s += x[j].x + x[j].y;
  if (s == -1.25e-30f) *sink = s;
}

}  // namespace goo

using namespace goo;

extern "C" int goo_peak_fma(goo_ctx* ctx, int kind, int iters, double* fma_per_s, double* ms_out) {
  if (!ctx || !fma_per_s) return set_error(GOO_ERR_ARG, "goo_peak_fma: NULL argument");
  if (kind != GOO_PEAK_F64 && kind != GOO_PEAK_F32 && kind != GOO_PEAK_F32X2)
    return set_error(GOO_ERR_ARG, "goo_peak_fma: kind %d", kind);
  if (iters < 1 || iters > (1 << 24)) return set_error(GOO_ERR_ARG, "goo_peak_fma: iters %d (1 .. 2^24)", iters);
  GOO_CUDA_TRY(cudaSetDevice(ctx->device));
  const int nb = ctx->num_sms * kPeakBlocksPerSm;
  double* sink = ctx->scratch.result;  // never written (the kernels' guard is never true)
  cudaEvent_t e0, e1;
  GOO_CUDA_TRY(cudaEventCreate(&e0));
  GOO_CUDA_TRY(cudaEventCreate(&e1));
  auto launch = [&]() {
    LaunchScope ls(ctx, kind == GOO_PEAK_F64 ? "peak_fma_f64" : kind == GOO_PEAK_F32 ? "peak_fma_f32" : "peak_fma_f32x2");
    if (kind == GOO_PEAK_F64)
      peak_fma_kernel<double><<<nb, kPeakBlock, 0, ctx->stream>>>(0.999999, 1e-7, iters, sink);
    else if (kind == GOO_PEAK_F32)
      peak_fma_kernel<float><<<nb, kPeakBlock, 0, ctx->stream>>>(0.9999f, 1e-4f, iters, (float*)sink);
    else
      peak_fma2_kernel<<<nb, kPeakBlock, 0, ctx->stream>>>(0.9999f, 1e-4f, iters, (float*)sink);
  };
  launch();  // warm-up (clocks, instruction cache)
  cudaEventRecord(e0, ctx->stream);
  launch();
  cudaEventRecord(e1, ctx->stream);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return set_error(GOO_ERR_CUDA, "goo_peak_fma: %s", cudaGetErrorString(e));
  const double lanes = kind == GOO_PEAK_F32X2 ? 2.0 : 1.0;
  const double fmas = (double)nb * kPeakBlock * (double)iters * kPeakUnroll * kPeakChains * lanes;
  *fma_per_s = fmas / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return GOO_OK;
}

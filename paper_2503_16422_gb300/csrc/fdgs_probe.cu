// FP32 FMA throughput probe: the denominator of the blend's FP32 roofline, measured on the
// device that runs the blend instead of derived from unit counts and the nominal clock.
// Every thread runs kChains independent fma chains (scalar fma.rn.f32, or fma.rn.f32x2 on
// pairs of them), enough resident warps to cover the pipe latency, and the launch is timed
// with events on the caller's stream; FLOP = 2 per lane fma.
#include <algorithm>

#include "fdgs.h"
#include "fdgs_internal.h"

namespace {

constexpr int kChains = 16;          // independent accumulators per thread (8 pairs)
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8; // 2048 threads an SM

template <bool kPair>
__global__ void __launch_bounds__(kProbeThreads, kProbeBlocksPerSm)
    k_fma_probe(float *out, int iters, float a, float b) {
  float acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = (float)threadIdx.x * 1e-3f + (float)i;
  for (int it = 0; it < iters; ++it) {
    if constexpr (kPair) {
#pragma unroll
      for (int i = 0; i < kChains; i += 2) {
        const float2 v = __ffma2_rn(make_float2(acc[i], acc[i + 1]), make_float2(a, a),
                                    make_float2(b, b));
        acc[i] = v.x;
        acc[i + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = __fmaf_rn(acc[i], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  if (s == -1.f) out[blockIdx.x] = s;   // never true for these inputs; keeps the chains live
}

}  // namespace

extern "C" int fdgs_measure_fp32_peak(int paired, double *tflops_out, fdgs_stream stream) {
  if (!tflops_out || (paired != 0 && paired != 1)) {
    fdgs::set_error_message("fdgs_measure_fp32_peak: null output or paired not 0/1");
    return FDGS_ERR_INVALID;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = fdgs::num_sms() * kProbeBlocksPerSm;
  const int iters = 1 << 16;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float *sink = nullptr;
  double best_ms = 0.0;
  cudaError_t e = cudaMalloc(&sink, (size_t)grid * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // one untimed launch, then the fastest of three
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, st);
    if (paired)
      k_fma_probe<true><<<grid, kProbeThreads, 0, st>>>(sink, iters, 0.999f, 1e-3f);
    else
      k_fma_probe<false><<<grid, kProbeThreads, 0, st>>>(sink, iters, 0.999f, 1e-3f);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && e == cudaSuccess && (best_ms == 0.0 || ms < best_ms)) best_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess || best_ms <= 0.0) {
    fdgs::set_error_message(e != cudaSuccess ? cudaGetErrorString(e) : "probe not timed");
    return FDGS_ERR_CUDA;
  }
  const double flop = 2.0 * kChains * (double)iters * (double)grid * kProbeThreads;
  *tflops_out = flop / (best_ms * 1e-3) / 1e12;
  return FDGS_OK;
}

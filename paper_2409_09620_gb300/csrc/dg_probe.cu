// dg_probe.cu -- FMA throughput of this GPU in FP64 and FP32, measured with
// CUDA events.  The FP64 stage kernels are bound by the FP64 pipe (GB300 runs
// DFMA at a small fraction of its FP32 rate), so the roofline of the solver's
// FP64 path is this measured rate, not a memory bandwidth.
#include <cuda_runtime.h>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace dg {

constexpr int PROBE_THREADS = 256;

__device__ double g_probe_sink;   // written only if a chain ends on an impossible value

// Each thread runs CH independent chains x <- x * m + c for iters rounds of 4:
// 2 flops per FMA.  m and c are launch arguments, so nothing folds.
template <typename T, int CH>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(int64_t iters, T m, T c) {
  T x[CH];
#pragma unroll
  for (int j = 0; j < CH; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < CH; ++j) x[j] = fma(x[j], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < CH; ++j) s += x[j];
  if (s == T(-12345.678)) g_probe_sink = double(s);
}

}  // namespace dg

using namespace dg;

extern "C" int32_t dg_probe_fma_peak(int32_t precision, double *tflops, double *ms, void *cuda_stream) {
  if (!tflops || (precision != DG_PREC_FP64 && precision != DG_PREC_MIXED))
    return set_error(DG_EINVAL, "bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  // about 20 ms per launch at the expected rates (FP64 ~1.2, FP32 ~70 TFLOP/s)
  const int64_t iters = precision == DG_PREC_FP64 ? 2048 : 2048 * 48;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  double best = 0.0;
  float best_ms = 0.0f;
  // two shapes (8 or 16 chains per thread, 4 or 8 blocks of 256 threads per
  // SM); for each the best of three launches after a warm-up
  for (int shape = 0; shape < 2 && e == cudaSuccess; ++shape) {
    const int ch = shape == 0 ? 8 : 16, bps = shape == 0 ? 8 : 4;
    const unsigned grid = (unsigned)(nsm * bps);
    const double flops = 2.0 * 4.0 * ch * (double)iters * PROBE_THREADS * grid;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(ev[0], s);
      if (e != cudaSuccess) break;
      if (precision == DG_PREC_FP64) {
        if (ch == 8) k_probe_fma<double, 8><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999999, 1e-9);
        else k_probe_fma<double, 16><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999999, 1e-9);
      } else {
        if (ch == 8) k_probe_fma<float, 8><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999f, 1e-6f);
        else k_probe_fma<float, 16><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999f, 1e-6f);
      }
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
      float t = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
      const double tf = flops / (double(t) * 1e-3) / 1e12;
      if (e == cudaSuccess && rep > 0 && t > 0.0f && tf > best) { best = tf; best_ms = t; }
    }
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  *tflops = best;
  if (ms) *ms = best_ms;
  return DG_OK;
}

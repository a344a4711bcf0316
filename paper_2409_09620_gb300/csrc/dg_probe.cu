// dg_probe.cu -- FMA throughput of this GPU in FP64 and FP32, measured with
// CUDA events.  The FP64 stage kernels are bound by the FP64 pipe (GB300 runs
// DFMA at a small fraction of its FP32 rate), so the roofline of the solver's
// FP64 path is this measured rate, not a memory bandwidth.
#include <cuda_runtime.h>

#include "../../include/dg.h"
#include "dg_internal.h"

namespace dg {

constexpr int PROBE_CHAINS = 8;        // independent FMA chains per thread
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 4;

__device__ double g_probe_sink;   // written only if a chain ends on an impossible value

// Each thread runs PROBE_CHAINS independent chains x <- x * m + c for iters
// rounds: 2 flops per FMA.  m and c are launch arguments, so nothing folds.
template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_fma(int64_t iters, T m, T c) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int j = 0; j < PROBE_CHAINS; ++j) x[j] = fma(x[j], m, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += x[j];
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
  const unsigned grid = (unsigned)(nsm * PROBE_BLOCKS_PER_SM);
  // about 20 ms per launch at the expected rates (FP64 ~1.2, FP32 ~70 TFLOP/s)
  const int64_t iters = precision == DG_PREC_FP64 ? 4096 : 4096 * 48;
  const double flops = 2.0 * 4.0 * PROBE_CHAINS * (double)iters * PROBE_THREADS * grid;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  float best = 0.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch is a warm-up
    e = cudaEventRecord(ev[0], s);
    if (e != cudaSuccess) break;
    if (precision == DG_PREC_FP64) k_probe_fma<double><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999999, 1e-9);
    else k_probe_fma<float><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999f, 1e-6f);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float t = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
    if (e == cudaSuccess && rep > 0 && (best == 0.0f || t < best)) best = t;
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return DG_OK;
}

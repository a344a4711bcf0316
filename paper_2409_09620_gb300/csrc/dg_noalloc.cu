// dg_noalloc.cu -- dg_stats_noalloc: the OE global statistics (domain means
// and sup deviations at the volume points) computed without allocating any
// device memory.  The per-block partial results live in a fixed file-scope
// device array instead of buffers from cudaMalloc.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it (2.36 MB) until the process exits.  All calls on a device
// share it and it keeps the last call's contents, so calls whose kernels
// overlap on the same GPU (for example on two streams) race on it.
#include <mutex>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg_stage.cuh"

namespace dg {
namespace {

// Largest mesh accepted: 2^22 cells -> 32768 blocks of TPB = 128 cells.
constexpr int64_t NA_MAX_CELLS = int64_t(1) << 22;
constexpr int64_t NA_MAX_BLOCKS = NA_MAX_CELLS / TPB;
// Layout: [0, 4 B) block sums of |K| u^(0); [4 B, 9 B) block maxima of the
// five deviations; [9 B, 9 B + 4) domain means (B = NA_MAX_BLOCKS).
constexpr int64_t NA_OFF_DEV = 4 * NA_MAX_BLOCKS;
constexpr int64_t NA_OFF_MEAN = 9 * NA_MAX_BLOCKS;
constexpr int64_t NA_SLOTS = 9 * NA_MAX_BLOCKS + 4;

static __device__ __align__(256) double g_na_scratch[NA_SLOTS];

// host-side cache of the scratch array's device address, per device
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
double *g_na_ptr[NA_MAX_DEVICES] = {};

// coefficient (c, l) of cell K in the public layout [4][nb][nt]
__device__ __forceinline__ double coef(const double *u, int nb, int64_t nt, int c, int l, int64_t K) {
  return u[((int64_t)c * nb + l) * nt + K];
}

// pass 1: block sums of |K| u^(0)
template <int K>
__global__ void __launch_bounds__(TPB) k_na_sum(int64_t nt, const double *__restrict__ area,
                                                const double *__restrict__ u, double *scratch) {
  constexpr int NB = Deg<K>::NB;
  const int64_t Kc = (int64_t)blockIdx.x * TPB + threadIdx.x;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  if (Kc < nt) {
    const double a = area[Kc];
#pragma unroll
    for (int c = 0; c < 4; ++c) s[c] = a * coef(u, NB, nt, c, 0, Kc);
  }
  block_reduce<4>(s, scratch + 4 * blockIdx.x, OpSum());
}

// fixed-order reduction of the block partials by one block of FIN_THREADS
template <int N, typename Op>
__device__ void na_fin_reduce(const double *part, int nblk, double init, Op op, double out[N]) {
  __shared__ double sh[FIN_THREADS][N];
  double acc[N];
#pragma unroll
  for (int q = 0; q < N; ++q) acc[q] = init;
  for (int b = threadIdx.x; b < nblk; b += FIN_THREADS)
#pragma unroll
    for (int q = 0; q < N; ++q) acc[q] = op(acc[q], part[b * N + q]);
#pragma unroll
  for (int q = 0; q < N; ++q) sh[threadIdx.x][q] = acc[q];
  __syncthreads();
  for (int st = FIN_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
#pragma unroll
      for (int q = 0; q < N; ++q) sh[threadIdx.x][q] = op(sh[threadIdx.x][q], sh[threadIdx.x + st][q]);
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < N; ++q) out[q] = sh[0][q];
}

__global__ void k_na_mean(int nblk, double area_total, double *scratch) {
  double r[4];
  na_fin_reduce<4>(scratch, nblk, 0.0, OpSum(), r);
  if (threadIdx.x == 0)
    for (int c = 0; c < 4; ++c) scratch[NA_OFF_MEAN + c] = r[c] / area_total;
}

// pass 2: block maxima of |rho - mean|, |m - mean m|, |E - mean|, |m1 - mean|, |m2 - mean|
template <int K>
__global__ void __launch_bounds__(TPB) k_na_dev(int64_t nt, const double *__restrict__ u, double *scratch) {
  constexpr int NB = Deg<K>::NB, NV = Deg<K>::NV;
  const int64_t Kc = (int64_t)blockIdx.x * TPB + threadIdx.x;
  double d[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (Kc < nt) {
    double off[4];
    double hi[4][NB];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      off[c] = coef(u, NB, nt, c, 0, Kc) - scratch[NA_OFF_MEAN + c];
      hi[c][0] = 0.0;
#pragma unroll
      for (int l = 1; l < NB; ++l) hi[c][l] = coef(u, NB, nt, c, l, Kc);
    }
#pragma unroll
    for (int mu = 0; mu < NV; ++mu) {
      double v[4];
      eval_fixed<double, NB>(off, hi, vol_xi(NV, mu), vol_eta(NV, mu), v);
      d[0] = fmax(d[0], fabs(v[0]));
      d[1] = fmax(d[1], sqrt(v[1] * v[1] + v[2] * v[2]));
      d[2] = fmax(d[2], fabs(v[3]));
      d[3] = fmax(d[3], fabs(v[1]));
      d[4] = fmax(d[4], fabs(v[2]));
    }
  }
  block_reduce<5>(d, scratch + NA_OFF_DEV + 5 * blockIdx.x, OpMaxNN());
}

__global__ void k_na_fin(int nblk, double area_total, double *scratch, double *out) {
  double r[5];
  na_fin_reduce<5>(scratch + NA_OFF_DEV, nblk, 0.0, OpMaxNN(), r);
  if (threadIdx.x == 0) {
    for (int c = 0; c < 4; ++c) out[c] = scratch[NA_OFF_MEAN + c];
    out[4] = r[0];
    out[5] = r[1];
    out[6] = r[2];
    out[7] = area_total;
    out[8] = r[3];
    out[9] = r[4];
  }
}

}  // namespace
}  // namespace dg

extern "C" int32_t dg_stats_noalloc(const dg_mesh *mesh, int32_t k, const double *coeffs, double *stats,
                                    void *cuda_stream) {
  using namespace dg;
  if (!mesh || !coeffs || !stats) return set_error(DG_EINVAL, "dg_stats_noalloc: NULL argument");
  if (k != 1 && k != 2) return set_error(DG_EINVAL, "dg_stats_noalloc: k must be 1 or 2");
  int64_t nt = 0;
  const double *area = nullptr;
  double area_total = 0.0;
  mesh_view(mesh, &nt, &area, &area_total);
  if (nt > NA_MAX_CELLS)
    return set_error(DG_EINVAL, "dg_stats_noalloc: the mesh has more cells than the fixed scratch allows "
                                      "(limit 4194304 cells)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return set_error(DG_EINVAL, "dg_stats_noalloc: device id too large");
  if (dev != mesh_device(mesh))
    return set_error(DG_EINVAL, "dg_stats_noalloc: the current device is not the one that holds the mesh");
  double *scratch = nullptr;
  {
    // once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_na_scratch);
      if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
      g_na_ptr[dev] = static_cast<double *>(p);
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const unsigned nblk = (unsigned)((nt + TPB - 1) / TPB);
  // every partial slot read below is written earlier in this call: nothing to clear
  if (k == 1) k_na_sum<1><<<nblk, TPB, 0, s>>>(nt, area, coeffs, scratch);
  else k_na_sum<2><<<nblk, TPB, 0, s>>>(nt, area, coeffs, scratch);
  k_na_mean<<<1, FIN_THREADS, 0, s>>>((int)nblk, area_total, scratch);
  if (k == 1) k_na_dev<1><<<nblk, TPB, 0, s>>>(nt, coeffs, scratch);
  else k_na_dev<2><<<nblk, TPB, 0, s>>>(nt, coeffs, scratch);
  k_na_fin<<<1, FIN_THREADS, 0, s>>>((int)nblk, area_total, scratch, stats);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
  return DG_OK;
}

// dg_batch.cu -- many independent solves advanced together over a work list
// of (solve, tile range) chunks.  A stage has three phases (flux + means;
// deviations, edge records and OE normalisers; RIOE + limiter + alpha).  They
// run either as one persistent cooperative launch per stage with grid
// barriers between the phases, or as one ordinary launch per phase, each at
// the occupancy of the per-solve kernel of that phase; the autotuner picks.
// Each phase finalises its reductions in the block that completes them, in
// the same fixed order as the per-solve kernels.
//
// Every solve keeps its own buffers, scalars (t, dt, alpha, normalisers) and
// per-tile partials; tiles never straddle solves and partials are per TPB
// cells from each solve's first cell, so a solve's arithmetic does not depend
// on the other solves, the chunk size or the launch form: results are bitwise
// those of the same solve run alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg_stage.cuh"

namespace dg {

struct SolveDev {
  MeshDev mesh;
  Phys ph;
  double *avg[3];   // u_n, u_h, u_s
  void *hi[3];
  void *tr, *vd, *hs, *ej;
  double *part_sum, *part_dev, *part_alpha;
  long long *part_cnt;
  FinBufs fin;
  Scalars *sc;
  int k, oe, bp, pad;
  int64_t ntiles;
};

struct WorkItem {
  int solve;
  int pad;
  int64_t first_tile, ntiles;
};

// Grid barrier of the cooperative form.  count and gen are the barrier;
// error is set by a block whose wait ran out; extra phantom arrivals (0 in
// normal use) raise the count the barrier waits for, so that a test can make
// every wait run out; timeout_ns bounds each wait.
struct BarrierState {
  unsigned int count;
  unsigned int gen;
  int error;
  unsigned int extra;
  unsigned long long timeout_ns;
};
constexpr unsigned long long BARRIER_TIMEOUT_NS = 2000000000ull;

__constant__ double kRK_A[3] = {0.0, 0.75, 1.0 / 3.0};
__constant__ double kRK_B[3] = {1.0, 0.25, 2.0 / 3.0};
__constant__ double kC_IN[3] = {0.0, 1.0, 0.5};
__constant__ double kC_OUT[3] = {1.0, 0.5, 1.0};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch (all blocks resident).  The wait
// is bounded: after timeout_ns (or, should the global timer not advance, a
// number of polls far beyond it) the block records an error and leaves; a
// waiting block also leaves as soon as another block has recorded one.
// Every block then returns false and the kernel ends early (the host reports
// DG_ETIMEOUT).
__device__ __forceinline__ bool grid_sync(BarrierState *b, unsigned nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *vgen = &b->gen;
    volatile int *verr = &b->error;
    const unsigned target = nblocks + *(volatile unsigned *)&b->extra;
    const unsigned long long limit = *(volatile unsigned long long *)&b->timeout_ns;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&b->count, 1u);
    if (arrived == target - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      const unsigned long long max_polls = limit / 16 + 1000000ull;   // a poll takes far longer than 16 ns
      unsigned long long polls = 0;
      while (*vgen == g && *verr == 0) {
        if (global_ns() - t0 > limit || ++polls > max_polls) {
          atomicExch(&b->error, 1);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = *verr == 0;
  }
  __syncthreads();
  return s_ok;
}

// The three phases of a stage over the work list, blocks [first, first +
// stride, ...).  Each tile finalises its reductions through the tickets, so
// the phases need only be ordered, by a grid barrier or a kernel boundary.
template <typename Real>
__device__ __forceinline__ void phase_rk(const SolveDev *__restrict__ sv, const WorkItem *__restrict__ work,
                                         int nwork, int stage) {
  const double a = kRK_A[stage], b = kRK_B[stage], c_in = kC_IN[stage];
  const int vi = stage == 0 ? 0 : 2;     // stage input: u_n, then u_s
  // volume + edge fluxes + RK combination; domain means
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const WorkItem it = work[w];
    const SolveDev &S = sv[it.solve];
    if (!S.sc->active) continue;
    const StateDev<Real> v{S.avg[vi], (Real *)S.hi[vi]}, un{S.avg[0], (Real *)S.hi[0]}, uh{S.avg[1], (Real *)S.hi[1]};
    for (int64_t t = it.first_tile; t < it.first_tile + it.ntiles; ++t) {
      if (S.k == 1)
        rk_tile<1, Real>(S.mesh, S.ph, v, un, uh, (const Real *)S.tr, (Real *)S.vd, (Real *)S.hs, S.part_sum, S.sc,
                         a, b, c_in, t);
      else
        rk_tile<2, Real>(S.mesh, S.ph, v, un, uh, (const Real *)S.tr, (Real *)S.vd, (Real *)S.hs, S.part_sum, S.sc,
                         a, b, c_in, t);
      finish_means(S.part_sum, S.fin, t, S.ntiles, S.sc);
    }
  }
}

template <typename Real>
__device__ __forceinline__ void phase_stats(const SolveDev *__restrict__ sv, const WorkItem *__restrict__ work,
                                            int nwork, int stage) {
  const double c_out = kC_OUT[stage];
  // sup deviations at the volume points, edge OE records; normalisers
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const WorkItem it = work[w];
    const SolveDev &S = sv[it.solve];
    if (!S.sc->active || !S.oe) continue;
    const StateDev<Real> uh{S.avg[1], (Real *)S.hi[1]};
    for (int64_t t = it.first_tile; t < it.first_tile + it.ntiles; ++t) {
      if (S.k == 1) {
        stats_tile<1, Real>(S.mesh, uh, S.part_dev, S.sc, t);
        edge_tile<1, Real>(S.mesh, S.ph, uh.avg, (const Real *)S.vd, (const Real *)S.hs, (Real *)S.ej, S.sc, c_out,
                           t);
      } else {
        stats_tile<2, Real>(S.mesh, uh, S.part_dev, S.sc, t);
        edge_tile<2, Real>(S.mesh, S.ph, uh.avg, (const Real *)S.vd, (const Real *)S.hs, (Real *)S.ej, S.sc, c_out,
                           t);
      }
      finish_deviations(S.part_dev, S.fin, t, S.ntiles, S.sc, S.oe == 2);
    }
  }
}

template <typename Real>
__device__ __forceinline__ void phase_oe_bp(const SolveDev *__restrict__ sv, const WorkItem *__restrict__ work,
                                            int nwork, int stage) {
  const double c_out = kC_OUT[stage];
  const int oi = stage == 2 ? 0 : 2;     // stage output: u_s, last stage writes u_n
  // RIOE + BP limiter + traces; alpha of the stage result, time update
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const WorkItem it = work[w];
    const SolveDev &S = sv[it.solve];
    if (!S.sc->active) continue;
    const StateDev<Real> uh{S.avg[1], (Real *)S.hi[1]}, out{S.avg[oi], (Real *)S.hi[oi]};
    for (int64_t t = it.first_tile; t < it.first_tile + it.ntiles; ++t) {
      if (S.k == 1)
        oe_bp_tile<1, Real>(S.mesh, S.ph, uh, out, (const Real *)S.ej, (Real *)S.tr, S.part_alpha, S.part_cnt,
                            S.sc, S.oe != 0, S.bp != 0, c_out, stage == 2, t);
      else
        oe_bp_tile<2, Real>(S.mesh, S.ph, uh, out, (const Real *)S.ej, (Real *)S.tr, S.part_alpha, S.part_cnt,
                            S.sc, S.oe != 0, S.bp != 0, c_out, stage == 2, t);
      finish_alpha(S.part_alpha, S.part_cnt, S.fin, t, S.ntiles, S.sc, stage);
    }
  }
}

// Fused form: one cooperative launch per stage runs the three phases with
// grid barriers between them (and the step start before stage 0).
template <typename Real>
__global__ void __launch_bounds__(TPB) k_batch_stage(const SolveDev *__restrict__ sv, int nsv,
                                                     const WorkItem *__restrict__ work, int nwork,
                                                     BarrierState *bar, int stage) {
  const unsigned nb = gridDim.x;
  if (stage == 0) {
    if (threadIdx.x == 0)
      for (int i = blockIdx.x; i < nsv; i += gridDim.x) step_begin_thread(sv[i].sc);
    if (!grid_sync(bar, nb)) return;
  }
  phase_rk<Real>(sv, work, nwork, stage);
  if (!grid_sync(bar, nb)) return;
  phase_stats<Real>(sv, work, nwork, stage);
  if (!grid_sync(bar, nb)) return;
  phase_oe_bp<Real>(sv, work, nwork, stage);
}

// Phased form: one ordinary launch per phase, each with the register budget
// and occupancy of the per-solve kernel of that phase; kernel boundaries
// order the phases, so no block ever waits on another.
__global__ void __launch_bounds__(TPB) k_batch_begin(const SolveDev *__restrict__ sv, int nsv) {
  const int i = blockIdx.x * TPB + threadIdx.x;
  if (i < nsv) step_begin_thread(sv[i].sc);
}

template <typename Real>
__global__ void __launch_bounds__(TPB, sizeof(Real) == 4 ? RK_MINB_F : RK_MINB_D)
    k_batch_rk(const SolveDev *__restrict__ sv, const WorkItem *__restrict__ work, int nwork, int stage) {
  phase_rk<Real>(sv, work, nwork, stage);
}

template <typename Real>
__global__ void __launch_bounds__(TPB, sizeof(Real) == 4 ? STATS_MINB_F : STATS_MINB_D)
    k_batch_stats(const SolveDev *__restrict__ sv, const WorkItem *__restrict__ work, int nwork, int stage) {
  phase_stats<Real>(sv, work, nwork, stage);
}

template <typename Real>
__global__ void __launch_bounds__(TPB, sizeof(Real) == 4 ? OEBP_MINB_F : OEBP_MINB_D)
    k_batch_oe_bp(const SolveDev *__restrict__ sv, const WorkItem *__restrict__ work, int nwork, int stage) {
  phase_oe_bp<Real>(sv, work, nwork, stage);
}

}  // namespace dg

using namespace dg;

namespace dg {

// A set of solves advanced together.  A step is either three cooperative
// launches of the fused stage kernel (form 1) or, per stage, three ordinary
// launches of the phase kernels after one step-start launch (form 3).  The set
// can change between steps (set_solves): the solve descriptors, the work list
// and the step graph are rebuilt.
struct BatchCore {
  int prec = 0;
  cudaStream_t stream = nullptr;
  std::vector<dg_solver *> solves;
  std::vector<SolveDev> host_sv;
  SolveDev *d_sv = nullptr;
  size_t sv_cap = 0;
  WorkItem *d_work = nullptr;
  size_t work_cap = 0;
  BarrierState *d_bar = nullptr;
  unsigned long long bar_timeout_ns = BARRIER_TIMEOUT_NS;
  unsigned bar_extra = 0;
  // the server's core picks the chunk size from the cells in the batch: the
  // largest power of two (up to 8 tiles) that still gives every resident
  // block of the grid two chunks, so a few small solves spread over the GPU
  bool auto_chunk = false;
  int nwork = 0, grid = 0, cpb = 4 * TPB, blocks_per_sm = 0, num_sms = 0, form = 3;
  int occ_fused = 0, occ_phase[3] = {0, 0, 0}, grid_phase[3] = {0, 0, 0};
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;

  ~BatchCore() {
    if (stream) cudaStreamSynchronize(stream);
    if (exec) cudaGraphExecDestroy(exec);
    cudaFree(d_sv);
    cudaFree(d_work);
    cudaFree(d_bar);
  }

  int32_t init(int precision, cudaStream_t s) {
    prec = precision;
    stream = s;
    int dev = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (coop && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_fused, fused_kernel(), TPB, 0) != cudaSuccess))
      return set_error(DG_ECUDA, "occupancy query failed");
    if (!coop) occ_fused = 0;
    for (int p = 0; p < 3; ++p)
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_phase[p], phase_kernel(p), TPB, 0) != cudaSuccess ||
          occ_phase[p] < 1)
        return set_error(DG_ECUDA, "occupancy query failed");
    form = 3;
    blocks_per_sm = max_blocks_per_sm(form);
    if (cudaMalloc(&d_bar, sizeof(BarrierState)) != cudaSuccess) return set_error(DG_ENOMEM, "barrier state");
    return reset_barrier();
  }

  // a fresh barrier (no arrivals, no error) with the configured wait limit
  int32_t reset_barrier() {
    BarrierState z{};
    z.extra = bar_extra;
    z.timeout_ns = bar_timeout_ns;
    if (cudaMemcpy(d_bar, &z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) return set_error(DG_ECUDA, "barrier");
    return DG_OK;
  }

  // resident blocks per SM of the form's kernels (0: form unavailable); the
  // per-solve form (0) runs the solves' own kernels, whose shape is their own
  int max_blocks_per_sm(int f) const {
    return f == 1 ? occ_fused : std::max(occ_phase[0], std::max(occ_phase[1], occ_phase[2]));
  }

  const void *fused_kernel() const {
    return prec == DG_PREC_MIXED ? (const void *)k_batch_stage<float> : (const void *)k_batch_stage<double>;
  }

  const void *phase_kernel(int p) const {
    if (prec == DG_PREC_MIXED)
      return p == 0 ? (const void *)k_batch_rk<float> : p == 1 ? (const void *)k_batch_stats<float>
                                                               : (const void *)k_batch_oe_bp<float>;
    return p == 0 ? (const void *)k_batch_rk<double> : p == 1 ? (const void *)k_batch_stats<double>
                                                              : (const void *)k_batch_oe_bp<double>;
  }

  size_t stack_bytes() const {
    if (form == 0) return 0;   // each solver made room for its own kernels
    if (prec == DG_PREC_MIXED)
      return form == 1 ? kernel_local_bytes(k_batch_stage<float>)
                       : std::max(kernel_local_bytes(k_batch_rk<float>),
                                  std::max(kernel_local_bytes(k_batch_stats<float>),
                                           kernel_local_bytes(k_batch_oe_bp<float>)));
    return form == 1 ? kernel_local_bytes(k_batch_stage<double>)
                     : std::max(kernel_local_bytes(k_batch_rk<double>),
                                std::max(kernel_local_bytes(k_batch_stats<double>),
                                         kernel_local_bytes(k_batch_oe_bp<double>)));
  }

  cudaError_t launch_stage(int stage) {
    int nsv = (int)host_sv.size(), nw = nwork;
    if (form == 1) {
      void *args[] = {&d_sv, &nsv, &d_work, &nw, &d_bar, &stage};
      return cudaLaunchCooperativeKernel(fused_kernel(), dim3(grid), dim3(TPB), args, 0, stream);
    }
    if (stage == 0) k_batch_begin<<<(nsv + TPB - 1) / TPB, TPB, 0, stream>>>(d_sv, nsv);
    void *args[] = {&d_sv, &d_work, &nw, &stage};
    for (int p = 0; p < 3; ++p) {
      cudaError_t e = cudaLaunchKernel(phase_kernel(p), dim3(grid_phase[p]), dim3(TPB), args, 0, stream);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  }

  // the solves to advance (not owned); rebuilds descriptors, work list and graph
  int32_t set_solves(const std::vector<dg_solver *> &list) {
    if (cudaStreamSynchronize(stream) != cudaSuccess) return set_error(DG_ECUDA, "sync");
    solves = list;
    host_sv.clear();
    for (dg_solver *s : solves) {
      SolveDev d{};
      const StageCtx &c = solver_ctx(s);
      d.mesh = c.mesh;
      d.ph = c.phys;
      StateBuf un, uh, us;
      solver_states(s, &un, &uh, &us);
      d.avg[0] = un.avg; d.hi[0] = un.hi;
      d.avg[1] = uh.avg; d.hi[1] = uh.hi;
      d.avg[2] = us.avg; d.hi[2] = us.hi;
      d.tr = c.tr; d.vd = c.vd; d.hs = c.hs; d.ej = c.ej;
      d.part_sum = c.part_sum; d.part_dev = c.part_dev; d.part_alpha = c.part_alpha; d.part_cnt = c.part_cnt;
      d.fin = c.fin;
      d.sc = c.sc;
      d.k = c.k;
      d.oe = c.phys.oe;
      d.bp = c.phys.bp;
      d.ntiles = num_blocks(c.mesh.nt);
      host_sv.push_back(d);
    }
    if (host_sv.size() > sv_cap) {
      cudaFree(d_sv);
      d_sv = nullptr;
      sv_cap = std::max<size_t>(host_sv.size(), 2 * sv_cap);
      if (cudaMalloc(&d_sv, sizeof(SolveDev) * sv_cap) != cudaSuccess) { sv_cap = 0; return set_error(DG_ENOMEM, "solve table"); }
    }
    if (!host_sv.empty() &&
        cudaMemcpy(d_sv, host_sv.data(), sizeof(SolveDev) * host_sv.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return set_error(DG_ECUDA, "solve table upload");
    if (auto_chunk) {
      int64_t tiles = 0;
      for (const SolveDev &d : host_sv) tiles += d.ntiles;
      const int64_t resident = (int64_t)num_sms * std::max(1, max_blocks_per_sm(form));
      int tpw = 1;
      while (tpw < 8 && tiles / (2 * tpw) >= 2 * resident) tpw *= 2;
      cpb = tpw * TPB;
    }
    int32_t rc = set_shape(cpb, blocks_per_sm, form);
    if (rc != DG_OK && form == 0) rc = set_shape(cpb, blocks_per_sm, 3);   // no graph: the phased form
    return rc;
  }

  // work list of chunks of cpb cells (a multiple of TPB), then the step graph
  int32_t set_shape(int cells_per_block, int bpsm, int launch_form) {
    if (launch_form != 0 && launch_form != 1 && launch_form != 3)
      return set_error(DG_EINVAL, "launch form must be 0, 1 or 3");
    if (max_blocks_per_sm(launch_form) < 1)
      return set_error(DG_EINVAL, "the device does not support cooperative launches");
    std::vector<WorkItem> work;
    const int64_t tpw = cells_per_block / TPB;
    for (size_t i = 0; i < host_sv.size(); ++i)
      for (int64_t t = 0; t < host_sv[i].ntiles; t += tpw)
        work.push_back(WorkItem{(int)i, 0, t, std::min<int64_t>(tpw, host_sv[i].ntiles - t)});
    if (work.size() > work_cap) {
      cudaFree(d_work);
      d_work = nullptr;
      work_cap = std::max<size_t>(work.size(), 2 * work_cap);
      if (cudaMalloc(&d_work, sizeof(WorkItem) * work_cap) != cudaSuccess) { work_cap = 0; return set_error(DG_ENOMEM, "work list"); }
    }
    if (!work.empty() &&
        cudaMemcpy(d_work, work.data(), sizeof(WorkItem) * work.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return set_error(DG_ECUDA, "work list upload");
    nwork = (int)work.size();
    cpb = cells_per_block;
    form = launch_form;
    blocks_per_sm = std::max(1, std::min(bpsm, max_blocks_per_sm(form)));
    const int nw = std::max(nwork, 1);
    if (form == 1) {
      grid = std::max(1, std::min(num_sms * blocks_per_sm, nw));
    } else {
      grid = 0;
      for (int p = 0; p < 3; ++p) {
        grid_phase[p] = std::max(1, std::min(num_sms * std::min(blocks_per_sm, occ_phase[p]), nw));
        grid = std::max(grid, grid_phase[p]);
      }
    }
    // one SSP-RK3 step, captured as a graph when supported
    if (exec) { cudaGraphExecDestroy(exec); exec = nullptr; }
    graph_ok = false;
    if (host_sv.empty()) return DG_OK;
    if (form == 0) return build_per_solve_graph();
    int32_t rc = ensure_stack_limit(stack_bytes());
    if (rc != DG_OK) return rc;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaError_t e = cudaSuccess;
      for (int st = 0; st < 3 && e == cudaSuccess; ++st) e = launch_stage(st);
      cudaError_t e2 = cudaStreamEndCapture(stream, &g);
      if (e == cudaSuccess && e2 == cudaSuccess && g && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess)
        graph_ok = true;
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();   // a refused capture leaves an error behind: clear it
    }
    return DG_OK;
  }

  // Form 0: every solve's own step (the kernels of its per-solve graph, with
  // their own registers and occupancy), the solves as independent branches
  // of one graph, so that the small ones run side by side on the device.
  // Needs graph support: without it the form is refused.
  int32_t build_per_solve_graph() {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return set_error(DG_ECUDA, "graph create");
    int32_t rc = DG_OK;
    for (dg_solver *sv_ : solves) {
      cudaGraph_t child = nullptr;
      if ((rc = solver_capture_step(sv_, &child)) != DG_OK) break;
      cudaGraphNode_t node;
      const cudaError_t e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, child);
      cudaGraphDestroy(child);
      if (e != cudaSuccess) { rc = set_error(DG_ECUDA, cudaGetErrorString(e)); break; }
    }
    if (rc == DG_OK && cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
      exec = nullptr;
      rc = set_error(DG_ECUDA, "per-solve batch graph instantiation failed");
    }
    cudaGraphDestroy(g);
    cudaGetLastError();
    if (rc == DG_OK) graph_ok = true;
    return rc;
  }

  int32_t enqueue_steps(int64_t n) {
    if (host_sv.empty()) return DG_OK;
    if (form == 0 && !graph_ok) return set_error(DG_ECUDA, "the per-solve batch graph is missing");
    for (int64_t s = 0; s < n; ++s) {
      if (graph_ok) {
        if (cudaGraphLaunch(exec, stream) != cudaSuccess) return set_error(DG_ECUDA, "batch graph launch");
      } else {
        for (int st = 0; st < 3; ++st) {
          cudaError_t e = launch_stage(st);
          if (e != cudaSuccess) return set_error(DG_ECUDA, cudaGetErrorString(e));
        }
      }
    }
    return DG_OK;
  }

  int32_t check_barrier() {
    BarrierState h{};
    if (cudaMemcpyAsync(&h, d_bar, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return set_error(DG_ECUDA, "batch sync");
    if (h.error) {
      reset_barrier();
      // blocks that left early may hold finalisation tickets: clear them
      for (const SolveDev &d : host_sv)
        cudaMemset(d.fin.tick, 0, 3 * ticket_slots(d.ntiles) * sizeof(unsigned));
      return set_error(DG_ETIMEOUT, "a grid barrier of the batch kernel timed out");
    }
    return DG_OK;
  }
};

}  // namespace dg

struct dg_batch {
  BatchCore core;
  std::vector<dg_solver *> owned;
  bool own_stream = false;
  cudaStream_t stream = nullptr;
  ~dg_batch() {
    if (stream) cudaStreamSynchronize(stream);
    for (auto *s : owned) dg_solver_destroy(s);
    core.~BatchCore();
    new (&core) BatchCore();
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

extern "C" int32_t dg_batch_create(int32_t n, const dg_mesh *const *meshes, const dg_config *cfgs,
                                   const double *const *coeffs, void *cuda_stream, dg_batch **out) {
  if (!out) return set_error(DG_EINVAL, "out is NULL");
  *out = nullptr;
  if (n <= 0 || !meshes || !cfgs || !coeffs) return set_error(DG_EINVAL, "empty batch or NULL arrays");
  for (int i = 0; i < n; ++i)
    if (cfgs[i].precision != cfgs[0].precision) return set_error(DG_EINVAL, "a batch has one precision");
  auto b = new (std::nothrow) dg_batch();
  if (!b) return set_error(DG_ENOMEM, "host allocation failed");
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return set_error(DG_ECUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  int32_t rc = b->core.init(cfgs[0].precision, b->stream);
  for (int i = 0; i < n && rc == DG_OK; ++i) {
    dg_solver *s = nullptr;
    rc = dg_init(meshes[i], &cfgs[i], coeffs[i], b->stream, &s);
    if (rc == DG_OK) b->owned.push_back(s);
  }
  if (rc == DG_OK) rc = b->core.set_solves(b->owned);
  if (rc != DG_OK) { delete b; return rc; }
  *out = b;
  return DG_OK;
}

extern "C" void dg_batch_destroy(dg_batch *b) { delete b; }

extern "C" int32_t dg_batch_set_shape(dg_batch *b, int32_t cells_per_block, int32_t blocks_per_sm,
                                      int32_t launches_per_stage) {
  if (!b || cells_per_block < TPB || cells_per_block % TPB != 0 || blocks_per_sm < 1)
    return set_error(DG_EINVAL, "cells_per_block must be a positive multiple of 128, blocks_per_sm >= 1");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return set_error(DG_ECUDA, "sync");
  return b->core.set_shape(cells_per_block, blocks_per_sm, launches_per_stage);
}

extern "C" int32_t dg_batch_shape(const dg_batch *b, int32_t *cells_per_block, int32_t *blocks_per_sm,
                                  int32_t *launches_per_stage, int32_t *grid, int32_t *graph) {
  if (!b) return set_error(DG_EINVAL, "batch is NULL");
  if (cells_per_block) *cells_per_block = b->core.cpb;
  if (blocks_per_sm) *blocks_per_sm = b->core.blocks_per_sm;
  if (launches_per_stage) *launches_per_stage = b->core.form;
  if (grid) *grid = b->core.grid;
  if (graph) *graph = b->core.graph_ok ? 1 : 0;
  return DG_OK;
}

extern "C" int32_t dg_batch_set_barrier(dg_batch *b, int64_t timeout_ns, int32_t extra_arrivals) {
  if (!b || timeout_ns <= 0 || extra_arrivals < 0) return set_error(DG_EINVAL, "bad argument");
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return set_error(DG_ECUDA, "sync");
  b->core.bar_timeout_ns = (unsigned long long)timeout_ns;
  b->core.bar_extra = (unsigned)extra_arrivals;
  return b->core.reset_barrier();
}

extern "C" int32_t dg_batch_advance_async(dg_batch *b, int64_t nsteps) {
  if (!b || nsteps < 0) return set_error(DG_EINVAL, "bad argument");
  return b->core.enqueue_steps(nsteps);
}

namespace dg {
// advance the solves of a batch core until every one reached its t_end (or max_steps)
int32_t batch_advance(BatchCore &core, const double *t_end, int64_t max_steps, dg_stats *stats) {
  const size_t n = core.solves.size();
  std::vector<Scalars> h(n), start(n);
  for (size_t i = 0; i < n; ++i) {
    if (cudaMemcpyAsync(&h[i], core.host_sv[i].sc, sizeof(Scalars), cudaMemcpyDeviceToHost, core.stream) != cudaSuccess)
      return set_error(DG_ECUDA, "scalars");
  }
  if (cudaStreamSynchronize(core.stream) != cudaSuccess) return set_error(DG_ECUDA, "sync");
  start = h;
  for (size_t i = 0; i < n; ++i) {
    h[i].t_end = t_end ? t_end[i] : INFINITY;
    if (cudaMemcpyAsync(&core.host_sv[i].sc->t_end, &h[i].t_end, sizeof(double), cudaMemcpyHostToDevice,
                        core.stream) != cudaSuccess)
      return set_error(DG_ECUDA, "t_end");
  }
  int64_t done = 0;
  auto unfinished = [&]() {
    for (size_t i = 0; i < n; ++i)
      if (h[i].t < h[i].t_end && std::isfinite(h[i].alpha) && h[i].alpha > 0.0) return true;
    return false;
  };
  while (done < max_steps && unfinished()) {
    const int64_t chunk = std::min<int64_t>(max_steps - done, 32);
    int32_t rc = core.enqueue_steps(chunk);
    if (rc != DG_OK) return rc;
    done += chunk;
    if ((rc = core.check_barrier()) != DG_OK) return rc;
    for (size_t i = 0; i < n; ++i)
      cudaMemcpyAsync(&h[i], core.host_sv[i].sc, sizeof(Scalars), cudaMemcpyDeviceToHost, core.stream);
    if (cudaStreamSynchronize(core.stream) != cudaSuccess) return set_error(DG_ECUDA, "sync");
  }
  int64_t bad = 0;
  for (size_t i = 0; i < n; ++i) {
    if (stats) {
      stats[i].steps = h[i].steps - start[i].steps;
      stats[i].limited_cells = h[i].limited - start[i].limited;
      stats[i].nonphysical = h[i].nonphys - start[i].nonphys;
      stats[i].cfl_breaches = h[i].breaches - start[i].breaches;
      stats[i].t = h[i].t;
      stats[i].dt_last = h[i].dt;
      stats[i].alpha = h[i].alpha;
    }
    bad += h[i].nonphys - start[i].nonphys;
  }
  if (bad > 0) return set_error(DG_ENONPHYS, "cell averages left the admissible set in the batch");
  return DG_OK;
}
}  // namespace dg

extern "C" int32_t dg_batch_advance(dg_batch *b, const double *t_end, int64_t max_steps, dg_stats *stats) {
  if (!b || max_steps < 0) return set_error(DG_EINVAL, "bad argument");
  return batch_advance(b->core, t_end, max_steps, stats);
}

extern "C" int32_t dg_batch_sync(dg_batch *b) {
  if (!b) return set_error(DG_EINVAL, "batch is NULL");
  return b->core.check_barrier();
}

extern "C" int32_t dg_batch_solver(dg_batch *b, int32_t i, dg_solver **out) {
  if (!b || !out || i < 0 || i >= (int32_t)b->owned.size()) return set_error(DG_EINVAL, "bad index");
  *out = b->owned[i];
  return DG_OK;
}

extern "C" int32_t dg_batch_autotune(dg_batch *b, int32_t steps, int32_t *best_cpb, int32_t *best_bpsm,
                                     int32_t *best_launches, double *best_ms) {
  if (!b || steps < 1) return set_error(DG_EINVAL, "bad argument");
  BatchCore &core = b->core;
  const int n = (int)core.solves.size();
  // snapshot every solve's device state (averages, modes, traces of u_n and
  // scalars); restoring these bytes undoes the tuning steps exactly
  struct Snap { void *avg, *hi, *tr; size_t navg, nhi, ntr; Scalars sc; };
  std::vector<Snap> snaps(n);
  const size_t rs = core.prec == DG_PREC_MIXED ? sizeof(float) : sizeof(double);
  auto free_snaps = [&]() { for (auto &q : snaps) { cudaFree(q.avg); cudaFree(q.hi); cudaFree(q.tr); } };
  for (int i = 0; i < n; ++i) {
    dg_solver *s = core.solves[i];
    const int64_t nt = solver_ctx(s).mesh.nt;
    const int nb = solver_nb(s), nq = nb == 3 ? 2 : 3;
    StateBuf un, uh, us;
    solver_states(s, &un, &uh, &us);
    Snap &q = snaps[i];
    const size_t ntr = uses_exchange(core.prec) ? rs * nt * 3 * nq * trace_stride(core.prec) : 0;
    q = Snap{nullptr, nullptr, nullptr, sizeof(double) * 4 * nt, rs * 4 * (nb - 1) * nt, ntr, {}};
    if (cudaMalloc(&q.avg, q.navg) != cudaSuccess || cudaMalloc(&q.hi, q.nhi) != cudaSuccess ||
        (q.ntr && cudaMalloc(&q.tr, q.ntr) != cudaSuccess)) {
      free_snaps();
      return set_error(DG_ENOMEM, "autotune snapshot");
    }
    cudaMemcpyAsync(q.avg, un.avg, q.navg, cudaMemcpyDeviceToDevice, core.stream);
    cudaMemcpyAsync(q.hi, un.hi, q.nhi, cudaMemcpyDeviceToDevice, core.stream);
    if (q.ntr) cudaMemcpyAsync(q.tr, solver_ctx(s).tr, q.ntr, cudaMemcpyDeviceToDevice, core.stream);
    if (solver_read_scalars(s, &q.sc) != DG_OK) { free_snaps(); return DG_ECUDA; }
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = INFINITY;
  int bc = core.cpb, bb = core.blocks_per_sm, bf = core.form;
  const int cpbs[4] = {TPB, 2 * TPB, 4 * TPB, 8 * TPB};
  // form 0 (per-solve graphs) has no shape of its own: one timing
  const int forms[3] = {0, 3, 1};
  for (int fi = 0; fi < 3; ++fi)
    for (int ci = 0; ci < (forms[fi] == 0 ? 1 : 4); ++ci)
      for (int bpsm = 1; bpsm <= (forms[fi] == 0 ? 1 : core.max_blocks_per_sm(forms[fi])); ++bpsm) {
        const int cpb_try = forms[fi] == 0 ? core.cpb : cpbs[ci];
        const int bpsm_try = forms[fi] == 0 ? core.blocks_per_sm : bpsm;
        int32_t rc = core.set_shape(cpb_try, bpsm_try, forms[fi]);
        if (rc != DG_OK && forms[fi] == 0) continue;   // no graph support: the form is unavailable
        if (rc == DG_OK) rc = core.enqueue_steps(1);   // warm-up
        cudaEventRecord(e0, core.stream);
        if (rc == DG_OK) rc = core.enqueue_steps(steps);
        cudaEventRecord(e1, core.stream);
        if (rc == DG_OK) rc = core.check_barrier();
        if (rc != DG_OK) { free_snaps(); return rc; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; bc = cpb_try; bb = bpsm_try; bf = forms[fi]; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < n; ++i) {
    dg_solver *s = core.solves[i];
    StateBuf un, uh, us;
    solver_states(s, &un, &uh, &us);
    const Snap &q = snaps[i];
    cudaMemcpyAsync(un.avg, q.avg, q.navg, cudaMemcpyDeviceToDevice, core.stream);
    cudaMemcpyAsync(un.hi, q.hi, q.nhi, cudaMemcpyDeviceToDevice, core.stream);
    if (q.ntr) cudaMemcpyAsync(solver_ctx(s).tr, q.tr, q.ntr, cudaMemcpyDeviceToDevice, core.stream);
    if (solver_write_scalars(s, &q.sc) != DG_OK) { free_snaps(); return DG_ECUDA; }
  }
  free_snaps();
  int32_t rc = core.set_shape(bc, bb, bf);
  if (rc != DG_OK) return rc;
  if (best_cpb) *best_cpb = bc;
  if (best_bpsm) *best_bpsm = bb;
  if (best_launches) *best_launches = bf;
  if (best_ms) *best_ms = best / steps;
  return DG_OK;
}

// ============================================================================
// Batch core for the server (dg_serve.cu)
// ============================================================================
namespace dg {
int32_t batch_core_new(int precision, cudaStream_t stream, BatchCore **out) {
  auto c = new (std::nothrow) BatchCore();
  if (!c) return set_error(DG_ENOMEM, "host allocation failed");
  int32_t rc = c->init(precision, stream);
  if (rc != DG_OK) { delete c; return rc; }
  c->auto_chunk = true;
  // the server's solves run their own step kernels side by side (form 0):
  // requests of very different sizes keep their own launch shapes, and the
  // graph is rebuilt only when the set of running solves changes
  c->form = 0;
  *out = c;
  return DG_OK;
}
void batch_core_delete(BatchCore *core) { delete core; }
int32_t batch_core_set_solves(BatchCore *core, const std::vector<dg_solver *> &list) {
  return core->set_solves(list);
}
int32_t batch_core_enqueue(BatchCore *core, int64_t nsteps) { return core->enqueue_steps(nsteps); }
int32_t batch_core_check(BatchCore *core) { return core->check_barrier(); }
}  // namespace dg

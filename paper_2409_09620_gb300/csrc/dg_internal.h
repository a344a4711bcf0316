// dg_internal.h -- host-side interface between the C ABI (dg_api.cu) and the
// kernel launch wrappers (dg_kernels.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/dg.h"
#include "dg_common.cuh"

namespace dg {

struct GeomPtrs {
  double *area, *jinv, *nrm, *len, *hgeo, *node, *c_area;
  int8_t *limv;
  float *jinv_f, *nrm_f, *len_f, *hgeo_f;
  double *iarea;
  float *node_f;
  double *psi_node;
};

// a modal state: FP64 averages [4][nt] + higher modes [4][nb-1][nt] (double or float)
struct StateBuf {
  double *avg;
  void *hi;
};

// everything a stage launch needs
struct StageCtx {
  cudaStream_t stream;
  int k, prec;
  MeshDev mesh;
  Phys phys;
  void *tr, *vd, *hs, *ej;
  double *part_sum, *part_dev, *part_alpha;
  long long *part_cnt;
  FinBufs fin;   // scratch and ticket counters of the in-kernel finalisation
  Scalars *sc;
};

void launch_geometry(cudaStream_t s, int64_t nt, const double *vxy, const GeomPtrs &g, double *part_min,
                     double *out_min4);
void launch_rk(const StageCtx &c, const StateBuf &v, const StateBuf &un, const StateBuf &uh, double a, double b,
               double c_in);
void launch_rk_only(const StageCtx &c, const StateBuf &v, const StateBuf &un, const StateBuf &uh, double a,
                    double b, double c_in);
void launch_fin_mean(const StageCtx &c);
void launch_stats(const StageCtx &c, const StateBuf &uh, double c_out);
void launch_stats_only(const StageCtx &c, const StateBuf &uh, double c_out);
void launch_fin_dev(const StageCtx &c);
void launch_oe_bp(const StageCtx &c, const StateBuf &uh, const StateBuf &out, int do_oe, int do_bp, double c_out,
                  int stage);
void launch_oe_bp_only(const StageCtx &c, const StateBuf &uh, const StateBuf &out, int do_oe, int do_bp,
                       double c_out, int end_of_step);
void launch_fin_alpha(const StageCtx &c, int stage);
void launch_step_begin(const StageCtx &c);
void launch_set_active(const StageCtx &c, int active);
void launch_set_inv_normalisers(const StageCtx &c);
int64_t num_blocks(int64_t nt);

// access to a solver's launch context and buffers (dg_api.cu)
const StageCtx &solver_ctx(const dg_solver *s);
void solver_states(const dg_solver *s, StateBuf *un, StateBuf *uh, StateBuf *us);
int solver_nb(const dg_solver *s);
int32_t solver_read_scalars(const dg_solver *s, Scalars *h);
int32_t solver_write_scalars(dg_solver *s, const Scalars *h);
// one SSP-RK3 step of the solver (the kernels of its own step graph) captured
// into a new graph, which the caller destroys
int32_t solver_capture_step(dg_solver *s, cudaGraph_t *graph);

// the mesh's device arrays as the kernels see them; boundary tags usable by
// the scalar solver (dg_api.cu)
MeshDev mesh_device_view(const dg_mesh *m);
bool mesh_boundary_tags_ok(const dg_mesh *m, int scalar);

// Raise the context's per-thread stack limit to at least `bytes` (it is never
// lowered).  The driver grows the stack for a plain kernel launch on its own;
// this makes sure kernels replayed from a CUDA graph find the same room
// (dg_api.cu).
int32_t ensure_stack_limit(size_t bytes);
// local (stack) bytes per thread a kernel needs, 0 if it cannot be queried
template <typename F>
size_t kernel_local_bytes(F *fn) {
  cudaFuncAttributes a{};
  return cudaFuncGetAttributes(&a, reinterpret_cast<const void *>(fn)) == cudaSuccess ? a.localSizeBytes : 0;
}
// the largest of the per-stage kernels of the given degree and precision (dg_kernels.cu)
size_t stage_kernels_local_bytes(int k, int prec);

// mesh size, device cell areas and their host-summed total (dg_api.cu)
void mesh_view(const dg_mesh *mesh, int64_t *nt, const double **area, double *area_total);
// the CUDA device that was current when the mesh was created (dg_api.cu)
int mesh_device(const dg_mesh *mesh);
// record a message for dg_last_error and return code (dg_api.cu)
int32_t set_error(int32_t code, const char *msg);

}  // namespace dg

// dg_serve.cu -- continuous-batching server of independent solves.
//
// Requests (host mesh arrays, configuration, initial coefficients, end time)
// wait in a FIFO queue.  Each tick: the steps launched by the previous tick
// are finished; solves that reached their end time are retired (result copied
// to the host, device memory freed); queued requests are admitted, in order,
// while their device memory fits in the HBM budget; the batch of running
// solves is rebuilt when it changed; and the next steps are enqueued without
// waiting, so the GPU works while the caller submits new requests.  All
// running solves advance together in the persistent batch kernel, each with
// its own time step, so a result does not depend on which other solves ran
// beside it.  The queue, the budget and the retirement rules are the plain
// C++ ServeScheduler (dg_serve_sched.cpp); this file is its device engine.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"
#include "dg_serve_sched.h"

namespace dg {
struct BatchCore;
int32_t batch_core_new(int precision, cudaStream_t stream, BatchCore **out);
void batch_core_delete(BatchCore *core);
int32_t batch_core_set_solves(BatchCore *core, const std::vector<dg_solver *> &list);
int32_t batch_core_enqueue(BatchCore *core, int64_t nsteps);
int32_t batch_core_check(BatchCore *core);
}  // namespace dg

using namespace dg;

namespace {

// what the device side keeps of a request: its inputs until it starts, its
// mesh and solver while it runs, its result once done
struct Payload {
  std::vector<double> xy;
  std::vector<int32_t> tri, canon;
  std::vector<int8_t> bc;
  dg_config cfg{};
  std::vector<double> coeffs, result;
  double t_end = 0.0;
  int64_t nv = 0, nt = 0;
  dg_mesh *mesh = nullptr;
  dg_solver *solver = nullptr;
};

// device bytes of one solve: mesh geometry and connectivity + solver buffers
size_t solve_bytes(int64_t nt, int k, int prec) {
  const size_t rs = prec == DG_PREC_MIXED ? 4 : 8;
  const size_t nb = k == 1 ? 3 : 6, nq = k == 1 ? 2 : 3;
  const size_t mesh = 45 * 8 + 23 * 4 + 2 + 12 + 4 * 3 + 4 * 2;   // geometry (FP64 + FP32 copies), connectivity, edges
  const size_t state = 3 * (4 * 8 + rs * 4 * (nb - 1));
  // traces, vertex records, Hessians, ~1.5 edge records (FP64 form only)
  const size_t exch = uses_exchange(prec) ? rs * (3 * nq * trace_stride(prec) + 48 + 12 + 2 * 16) : 0;
  const size_t part = 10 * 8 + 16;   // per 128-cell block, rounded up per cell below
  return (size_t)nt * (mesh + state + exch) + ((size_t)nt / 128 + 1) * part + 4096;
}

void free_payload_device(Payload &p) {
  if (p.solver) dg_solver_destroy(p.solver);
  if (p.mesh) dg_mesh_destroy(p.mesh);
  p.solver = nullptr;
  p.mesh = nullptr;
}

// the device side: one mesh and solver per running request, all advanced by
// the persistent batch kernel on the server's stream
struct DeviceEngine final : ServeEngine {
  cudaStream_t stream = nullptr;
  BatchCore *core = nullptr;
  std::map<int64_t, Payload> pay;

  int32_t finish_tick() override { return batch_core_check(core); }
  int32_t start(int64_t id) override {
    Payload &p = pay[id];
    int32_t rc = dg_mesh_create(p.nv, p.xy.data(), p.nt, p.tri.data(), p.canon.empty() ? nullptr : p.canon.data(),
                                p.bc.empty() ? nullptr : p.bc.data(), &p.mesh);
    if (rc == DG_OK) rc = dg_init(p.mesh, &p.cfg, p.coeffs.data(), stream, &p.solver);
    Scalars h{};
    if (rc == DG_OK) rc = solver_read_scalars(p.solver, &h);
    if (rc == DG_OK) {
      h.t_end = p.t_end;
      rc = solver_write_scalars(p.solver, &h);
    }
    if (rc != DG_OK) {
      free_payload_device(p);
      return rc;
    }
    p.xy.clear(); p.xy.shrink_to_fit();
    p.tri.clear(); p.tri.shrink_to_fit();
    return DG_OK;
  }
  int32_t poll(int64_t id, double *t, int64_t *steps, bool *bad) override {
    Payload &p = pay[id];
    Scalars h{};
    const int32_t rc = solver_read_scalars(p.solver, &h);
    if (rc != DG_OK) return rc;
    *t = h.t;
    *steps = h.steps;
    *bad = h.nonphys > 0 || !std::isfinite(h.alpha);
    return DG_OK;
  }
  int32_t retire(int64_t id, bool keep_result) override {
    Payload &p = pay[id];
    int32_t rc = DG_OK;
    if (p.solver && keep_result) {
      p.result.resize(p.coeffs.size());
      double t = 0.0;
      rc = dg_get_state(p.solver, p.result.data(), p.result.size(), &t);
    }
    free_payload_device(p);
    p.xy.clear(); p.xy.shrink_to_fit();
    p.tri.clear(); p.tri.shrink_to_fit();
    p.coeffs.clear(); p.coeffs.shrink_to_fit();
    return rc;
  }
  int32_t set_batch(const std::vector<int64_t> &running) override {
    std::vector<dg_solver *> list;
    for (int64_t id : running) list.push_back(pay[id].solver);
    return batch_core_set_solves(core, list);
  }
  int32_t enqueue(int64_t nsteps) override { return batch_core_enqueue(core, nsteps); }
};

}  // namespace

struct dg_server {
  int prec = 0;
  bool own_stream = false;
  ServeScheduler sched;
  DeviceEngine eng;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  dg_server(size_t budget, int steps_per_tick) : sched(budget, steps_per_tick) {}
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  ~dg_server() {
    if (eng.stream) cudaStreamSynchronize(eng.stream);
    batch_core_delete(eng.core);
    for (auto &kv : eng.pay) free_payload_device(kv.second);
    if (own_stream && eng.stream) cudaStreamDestroy(eng.stream);
  }
};

extern "C" int32_t dg_server_create(int32_t precision, size_t hbm_budget_bytes, int32_t steps_per_tick,
                                    void *cuda_stream, dg_server **out) {
  if (!out) return set_error(DG_EINVAL, "out is NULL");
  *out = nullptr;
  if ((precision != DG_PREC_FP64 && precision != DG_PREC_MIXED) || hbm_budget_bytes == 0 || steps_per_tick < 1)
    return set_error(DG_EINVAL, "bad precision, budget or steps per tick");
  auto s = new (std::nothrow) dg_server(hbm_budget_bytes, steps_per_tick);
  if (!s) return set_error(DG_ENOMEM, "host allocation failed");
  s->prec = precision;
  if (cuda_stream) {
    s->eng.stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->eng.stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return set_error(DG_ECUDA, "stream creation failed");
    }
    s->own_stream = true;
  }
  int32_t rc = batch_core_new(precision, s->eng.stream, &s->eng.core);
  if (rc != DG_OK) { delete s; return rc; }
  *out = s;
  return DG_OK;
}

extern "C" void dg_server_destroy(dg_server *s) { delete s; }

extern "C" int32_t dg_server_submit(dg_server *s, int64_t nv, const double *xy, int64_t nt, const int32_t *tri,
                                    const int32_t *canon, const int8_t *bc, const dg_config *cfg,
                                    const double *coeffs, double t_end, int64_t *id) {
  if (!s || !xy || !tri || !cfg || !coeffs || !id || nv <= 0 || nt <= 0)
    return set_error(DG_EINVAL, "bad request");
  if (cfg->precision != s->prec) return set_error(DG_EINVAL, "request precision differs from the server's");
  if (cfg->k != 1 && cfg->k != 2) return set_error(DG_EINVAL, "k must be 1 or 2");
  Payload p;
  p.nv = nv;
  p.nt = nt;
  p.xy.assign(xy, xy + 2 * nv);
  p.tri.assign(tri, tri + 3 * nt);
  if (canon) p.canon.assign(canon, canon + nv);
  if (bc) p.bc.assign(bc, bc + 3 * nt);
  p.cfg = *cfg;
  const int nb = cfg->k == 1 ? 3 : 6;
  p.coeffs.assign(coeffs, coeffs + 4 * nb * nt);
  p.t_end = t_end;
  *id = s->sched.submit(nt, solve_bytes(nt, cfg->k, s->prec), t_end, s->now());
  s->eng.pay.emplace(*id, std::move(p));
  return DG_OK;
}

extern "C" int32_t dg_server_tick(dg_server *s, int32_t *n_running, int32_t *n_queued) {
  if (!s) return set_error(DG_EINVAL, "server is NULL");
  return s->sched.tick(s->eng, s->now(), n_running, n_queued);
}

extern "C" int32_t dg_server_request(const dg_server *s, int64_t id, dg_request_info *info) {
  if (!s || !info) return set_error(DG_EINVAL, "NULL argument");
  const SchedRequest *rp = s->sched.find(id);
  if (!rp) return set_error(DG_EINVAL, "unknown request id");
  const SchedRequest &r = *rp;
  info->state = r.state;
  info->error = r.error;
  info->cells = r.cells;
  info->steps = r.steps;
  info->t = r.t;
  info->t_end = r.t_end;
  info->submit_s = r.submit_s;
  info->start_s = r.start_s;
  info->done_s = r.done_s;
  info->device_bytes = (int64_t)r.bytes;
  return DG_OK;
}

extern "C" int32_t dg_server_result(dg_server *s, int64_t id, double *coeffs, size_t len) {
  if (!s || !coeffs) return set_error(DG_EINVAL, "NULL argument");
  const SchedRequest *r = s->sched.find(id);
  if (!r) return set_error(DG_EINVAL, "unknown request id");
  if (r->state != DG_REQ_DONE) return set_error(DG_EBUSY, "request not done");
  const std::vector<double> &res = s->eng.pay[id].result;
  if (len < res.size()) return set_error(DG_EINVAL, "output too small");
  std::copy(res.begin(), res.end(), coeffs);
  return DG_OK;
}

extern "C" int32_t dg_server_stats(const dg_server *s, int64_t *bytes_in_use, int64_t *cell_stages_done) {
  if (!s) return set_error(DG_EINVAL, "server is NULL");
  if (bytes_in_use) *bytes_in_use = (int64_t)s->sched.used();
  if (cell_stages_done) *cell_stages_done = s->sched.cell_stages();
  return DG_OK;
}

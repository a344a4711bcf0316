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
// beside it.
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <vector>

#include "../../include/dg.h"
#include "dg_internal.h"

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

struct Request {
  int64_t id = 0;
  std::vector<double> xy;
  std::vector<int32_t> tri, canon;
  std::vector<int8_t> bc;
  dg_config cfg{};
  std::vector<double> coeffs, result;
  double t_end = 0.0;
  int64_t nv = 0, nt = 0;
  size_t bytes = 0;
  int32_t state = DG_REQ_QUEUED, error = DG_OK;
  dg_mesh *mesh = nullptr;
  dg_solver *solver = nullptr;
  double submit_s = 0.0, start_s = 0.0, done_s = 0.0, t = 0.0;
  int64_t steps = 0;
};

// device bytes of one solve: mesh geometry and connectivity + solver buffers
size_t solve_bytes(int64_t nt, int k, int prec) {
  const size_t rs = prec == DG_PREC_MIXED ? 4 : 8;
  const size_t nb = k == 1 ? 3 : 6, nq = k == 1 ? 2 : 3;
  const size_t mesh = 45 * 8 + 23 * 4 + 2 + 12 + 4 * 3 + 4 * 2;   // geometry (FP64 + FP32 copies), connectivity, edges
  const size_t state = 3 * (4 * 8 + rs * 4 * (nb - 1));
  const size_t exch = rs * (3 * nq * trace_stride(prec) + 48 + 12 + 2 * 16);   // traces, vertex records, Hessians, ~1.5 edge records
  const size_t part = 10 * 8 + 16;   // per 128-cell block, rounded up per cell below
  return (size_t)nt * (mesh + state + exch) + ((size_t)nt / 128 + 1) * part + 4096;
}

}  // namespace

struct dg_server {
  int prec = 0;
  size_t budget = 0, used = 0;
  int steps_per_tick = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  BatchCore *core = nullptr;
  std::deque<int64_t> queue;
  std::map<int64_t, Request> reqs;
  std::vector<int64_t> running;
  int64_t next_id = 1;
  int64_t cell_stages = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  ~dg_server() {
    if (stream) cudaStreamSynchronize(stream);
    batch_core_delete(core);
    for (auto &kv : reqs) {
      if (kv.second.solver) dg_solver_destroy(kv.second.solver);
      if (kv.second.mesh) dg_mesh_destroy(kv.second.mesh);
    }
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

extern "C" int32_t dg_server_create(int32_t precision, size_t hbm_budget_bytes, int32_t steps_per_tick,
                                    void *cuda_stream, dg_server **out) {
  if (!out) return set_error(DG_EINVAL, "out is NULL");
  *out = nullptr;
  if ((precision != DG_PREC_FP64 && precision != DG_PREC_MIXED) || hbm_budget_bytes == 0 || steps_per_tick < 1)
    return set_error(DG_EINVAL, "bad precision, budget or steps per tick");
  auto s = new (std::nothrow) dg_server();
  if (!s) return set_error(DG_ENOMEM, "host allocation failed");
  s->prec = precision;
  s->budget = hbm_budget_bytes;
  s->steps_per_tick = steps_per_tick;
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return set_error(DG_ECUDA, "stream creation failed");
    }
    s->own_stream = true;
  }
  int32_t rc = batch_core_new(precision, s->stream, &s->core);
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
  Request r;
  r.id = s->next_id++;
  r.nv = nv;
  r.nt = nt;
  r.xy.assign(xy, xy + 2 * nv);
  r.tri.assign(tri, tri + 3 * nt);
  if (canon) r.canon.assign(canon, canon + nv);
  if (bc) r.bc.assign(bc, bc + 3 * nt);
  r.cfg = *cfg;
  const int nb = cfg->k == 1 ? 3 : 6;
  r.coeffs.assign(coeffs, coeffs + 4 * nb * nt);
  r.t_end = t_end;
  r.bytes = solve_bytes(nt, cfg->k, s->prec);
  r.submit_s = s->now();
  *id = r.id;
  s->queue.push_back(r.id);
  s->reqs.emplace(r.id, std::move(r));
  return DG_OK;
}

static void retire(dg_server *s, Request &r, int32_t state, int32_t error) {
  r.state = state;
  r.error = error;
  r.done_s = s->now();
  if (r.solver) {
    if (state == DG_REQ_DONE) {
      r.result.resize(r.coeffs.size());
      double t = 0.0;
      if (dg_get_state(r.solver, r.result.data(), r.result.size(), &t) != DG_OK) {
        r.state = DG_REQ_FAILED;
        r.error = DG_ECUDA;
      }
      r.t = t;
    }
    dg_solver_destroy(r.solver);
    r.solver = nullptr;
  }
  if (r.mesh) {
    dg_mesh_destroy(r.mesh);
    r.mesh = nullptr;
  }
  s->used -= std::min(s->used, r.bytes);
  r.coeffs.clear();
  r.coeffs.shrink_to_fit();
}

extern "C" int32_t dg_server_tick(dg_server *s, int32_t *n_running, int32_t *n_queued) {
  if (!s) return set_error(DG_EINVAL, "server is NULL");
  // 1. finish the steps of the previous tick
  int32_t rc = batch_core_check(s->core);
  if (rc != DG_OK) return rc;
  // 2. retire finished solves
  bool changed = false;
  std::vector<int64_t> still;
  for (int64_t id : s->running) {
    Request &r = s->reqs[id];
    Scalars h{};
    if ((rc = solver_read_scalars(r.solver, &h)) != DG_OK) return rc;
    r.t = h.t;
    r.steps = h.steps;
    const bool bad = h.nonphys > 0 || !std::isfinite(h.alpha);
    if (h.t >= r.t_end || bad) {
      s->cell_stages += r.nt * 3 * h.steps;
      retire(s, r, bad ? DG_REQ_FAILED : DG_REQ_DONE, bad ? DG_ENONPHYS : DG_OK);
      changed = true;
    } else {
      still.push_back(id);
    }
  }
  s->running.swap(still);
  // 3. admit queued requests in order while their memory fits in the budget
  while (!s->queue.empty()) {
    Request &r = s->reqs[s->queue.front()];
    if (r.bytes > s->budget) {   // can never fit
      s->queue.pop_front();
      retire(s, r, DG_REQ_FAILED, DG_ENOMEM);
      continue;
    }
    if (s->used + r.bytes > s->budget) break;
    s->queue.pop_front();
    rc = dg_mesh_create(r.nv, r.xy.data(), r.nt, r.tri.data(), r.canon.empty() ? nullptr : r.canon.data(),
                        r.bc.empty() ? nullptr : r.bc.data(), &r.mesh);
    if (rc == DG_OK) rc = dg_init(r.mesh, &r.cfg, r.coeffs.data(), s->stream, &r.solver);
    Scalars h{};
    if (rc == DG_OK) rc = solver_read_scalars(r.solver, &h);
    if (rc == DG_OK) {
      h.t_end = r.t_end;
      rc = solver_write_scalars(r.solver, &h);
    }
    if (rc != DG_OK) {
      retire(s, r, DG_REQ_FAILED, rc);
      continue;
    }
    r.xy.clear(); r.xy.shrink_to_fit();
    r.tri.clear(); r.tri.shrink_to_fit();
    r.state = DG_REQ_RUNNING;
    r.start_s = s->now();
    s->used += r.bytes;
    s->running.push_back(r.id);
    changed = true;
  }
  // 4. rebuild the batch when its membership changed, 5. enqueue the next steps
  if (changed) {
    std::vector<dg_solver *> list;
    for (int64_t id : s->running) list.push_back(s->reqs[id].solver);
    if ((rc = batch_core_set_solves(s->core, list)) != DG_OK) return rc;
  }
  if (!s->running.empty() && (rc = batch_core_enqueue(s->core, s->steps_per_tick)) != DG_OK) return rc;
  if (n_running) *n_running = (int32_t)s->running.size();
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  return DG_OK;
}

extern "C" int32_t dg_server_request(const dg_server *s, int64_t id, dg_request_info *info) {
  if (!s || !info) return set_error(DG_EINVAL, "NULL argument");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(DG_EINVAL, "unknown request id");
  const Request &r = it->second;
  info->state = r.state;
  info->error = r.error;
  info->cells = r.nt;
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
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return set_error(DG_EINVAL, "unknown request id");
  Request &r = it->second;
  if (r.state != DG_REQ_DONE) return set_error(DG_EBUSY, "request not done");
  if (len < r.result.size()) return set_error(DG_EINVAL, "output too small");
  std::copy(r.result.begin(), r.result.end(), coeffs);
  return DG_OK;
}

extern "C" int32_t dg_server_stats(const dg_server *s, int64_t *bytes_in_use, int64_t *cell_stages_done) {
  if (!s) return set_error(DG_EINVAL, "server is NULL");
  if (bytes_in_use) *bytes_in_use = (int64_t)s->used;
  if (cell_stages_done) *cell_stages_done = s->cell_stages;
  return DG_OK;
}

// dg_serve_sched.h -- the host-side scheduler of the continuous-batching
// server: FIFO queue, admission by device-memory budget, retirement and the
// accounting of bytes and cell-stages.  The device work (mesh and solver
// creation, the batch kernel, results) sits behind ServeEngine, so the
// scheduler is plain C++ that also runs, against a fake engine, without a GPU.
#pragma once
#include <cstddef>
#include <cstdint>
#include <deque>
#include <map>
#include <vector>

namespace dg {

// The device side of the server.  Every call returns DG_OK or an error code.
struct ServeEngine {
  virtual ~ServeEngine() = default;
  // wait for the steps enqueued by the previous tick
  virtual int32_t finish_tick() = 0;
  // create the device state of a queued request; all or nothing
  virtual int32_t start(int64_t id) = 0;
  // time, steps taken and failure flag (non-admissible state or non-finite
  // wave speed) of a running request
  virtual int32_t poll(int64_t id, double *t, int64_t *steps, bool *bad) = 0;
  // free everything the request holds (device state and inputs), first
  // copying its result to the host when keep_result is set; an error means
  // the copy failed
  virtual int32_t retire(int64_t id, bool keep_result) = 0;
  // the running requests, in order, form the next batch
  virtual int32_t set_batch(const std::vector<int64_t> &running) = 0;
  // enqueue nsteps steps of the batch without waiting
  virtual int32_t enqueue(int64_t nsteps) = 0;
};

struct SchedRequest {
  int64_t id = 0, cells = 0, steps = 0;
  size_t bytes = 0;
  double t_end = 0.0, t = 0.0;
  int32_t state = 0, error = 0;   // DG_REQ_* and the DG_* status of a failed request
  double submit_s = 0.0, start_s = 0.0, done_s = 0.0;
};

class ServeScheduler {
 public:
  ServeScheduler(size_t budget, int64_t steps_per_tick) : budget_(budget), steps_per_tick_(steps_per_tick) {}
  // queue a request of `cells` cells needing `bytes` of device memory
  int64_t submit(int64_t cells, size_t bytes, double t_end, double now);
  // one tick at time `now`: finish the previous steps, retire finished
  // solves, admit queued requests in order while they fit in the budget
  // (a request larger than the whole budget fails with DG_ENOMEM; one whose
  // start fails fails with that status), rebuild the batch if its membership
  // changed and enqueue the next steps
  int32_t tick(ServeEngine &eng, double now, int32_t *n_running, int32_t *n_queued);
  const SchedRequest *find(int64_t id) const;
  size_t used() const { return used_; }
  size_t budget() const { return budget_; }
  int64_t cell_stages() const { return cell_stages_; }
  const std::vector<int64_t> &running() const { return running_; }
  const std::map<int64_t, SchedRequest> &requests() const { return reqs_; }

 private:
  void finish(ServeEngine &eng, SchedRequest &r, int32_t state, int32_t error, double now);
  size_t budget_, used_ = 0;
  int64_t steps_per_tick_;
  int64_t next_id_ = 1, cell_stages_ = 0;
  std::deque<int64_t> queue_;
  std::map<int64_t, SchedRequest> reqs_;
  std::vector<int64_t> running_;
  bool stale_batch_ = false;   // the engine's batch may name retired solves
};

}  // namespace dg

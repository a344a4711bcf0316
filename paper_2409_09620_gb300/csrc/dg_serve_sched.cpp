// dg_serve_sched.cpp -- host-side scheduler of the server (see dg_serve_sched.h).
#include "dg_serve_sched.h"

#include "../../include/dg.h"

namespace dg {

int64_t ServeScheduler::submit(int64_t cells, size_t bytes, double t_end, double now) {
  SchedRequest r;
  r.id = next_id_++;
  r.cells = cells;
  r.bytes = bytes;
  r.t_end = t_end;
  r.state = DG_REQ_QUEUED;
  r.error = DG_OK;
  r.submit_s = now;
  queue_.push_back(r.id);
  reqs_.emplace(r.id, r);
  return r.id;
}

const SchedRequest *ServeScheduler::find(int64_t id) const {
  auto it = reqs_.find(id);
  return it == reqs_.end() ? nullptr : &it->second;
}

// End a request.  Only a running request holds device memory, so only its
// bytes return to the budget.
void ServeScheduler::finish(ServeEngine &eng, SchedRequest &r, int32_t state, int32_t error, double now) {
  const bool held = r.state == DG_REQ_RUNNING;
  r.state = state;
  r.error = error;
  r.done_s = now;
  if (eng.retire(r.id, state == DG_REQ_DONE) != DG_OK && state == DG_REQ_DONE) {
    r.state = DG_REQ_FAILED;
    r.error = DG_ECUDA;
  }
  if (held) used_ -= r.bytes;
}

int32_t ServeScheduler::tick(ServeEngine &eng, double now, int32_t *n_running, int32_t *n_queued) {
  // 1. finish the steps of the previous tick
  int32_t rc = eng.finish_tick();
  if (rc != DG_OK) return rc;
  // 2. retire finished solves (a batch left stale by an earlier error is
  // rebuilt below whatever happens here)
  bool changed = stale_batch_;
  std::vector<int64_t> still;
  for (size_t i = 0; i < running_.size(); ++i) {
    SchedRequest &r = reqs_[running_[i]];
    double t = 0.0;
    int64_t steps = 0;
    bool bad = false;
    if ((rc = eng.poll(r.id, &t, &steps, &bad)) != DG_OK) {
      // keep the unretired solves; the batch still names the retired ones
      still.insert(still.end(), running_.begin() + (std::ptrdiff_t)i, running_.end());
      running_.swap(still);
      stale_batch_ = changed;
      return rc;
    }
    r.t = t;
    r.steps = steps;
    if (t >= r.t_end || bad) {
      cell_stages_ += r.cells * 3 * steps;
      finish(eng, r, bad ? DG_REQ_FAILED : DG_REQ_DONE, bad ? DG_ENONPHYS : DG_OK, now);
      changed = true;
    } else {
      still.push_back(r.id);
    }
  }
  running_.swap(still);
  // 3. admit queued requests in order while their memory fits in the budget
  while (!queue_.empty()) {
    SchedRequest &r = reqs_[queue_.front()];
    if (r.bytes > budget_) {   // can never fit
      queue_.pop_front();
      finish(eng, r, DG_REQ_FAILED, DG_ENOMEM, now);
      continue;
    }
    if (used_ + r.bytes > budget_) break;
    queue_.pop_front();
    if ((rc = eng.start(r.id)) != DG_OK) {
      finish(eng, r, DG_REQ_FAILED, rc, now);
      continue;
    }
    r.state = DG_REQ_RUNNING;
    r.start_s = now;
    used_ += r.bytes;
    running_.push_back(r.id);
    changed = true;
  }
  // 4. rebuild the batch when its membership changed, 5. enqueue the next steps
  if (changed) {
    stale_batch_ = true;
    if ((rc = eng.set_batch(running_)) != DG_OK) return rc;
    stale_batch_ = false;
  }
  if (!running_.empty() && (rc = eng.enqueue(steps_per_tick_)) != DG_OK) return rc;
  if (n_running) *n_running = (int32_t)running_.size();
  if (n_queued) *n_queued = (int32_t)queue_.size();
  return DG_OK;
}

}  // namespace dg

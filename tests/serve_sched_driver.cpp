// serve_sched_driver.cpp -- the server's scheduler (dg_serve_sched.cpp) against
// a fake device engine, on the CPU, for a build under AddressSanitizer and
// UndefinedBehaviorSanitizer (tests/test_serve_sched.py).  Test infrastructure.
//
// The fake engine advances every running solve by a fixed time step per
// enqueued step and can be told to fail a start, a poll, a result copy or the
// end of a tick, or to mark a solve non-admissible after some steps.  Each
// scenario checks the scheduler's states, error codes, budget accounting and
// calls into the engine; the program prints the first failed check and exits
// non-zero, or prints "ok".
#include <cstdio>
#include <cstdlib>
#include <map>
#include <set>
#include <vector>

#include "../include/dg.h"
#include "dg_serve_sched.h"

using dg::SchedRequest;
using dg::ServeScheduler;

static int g_failures = 0;
#define EXPECT(cond)                                                                 \
  do {                                                                               \
    if (!(cond)) {                                                                   \
      fprintf(stderr, "%s: check failed at line %d: %s\n", g_scenario, __LINE__, #cond); \
      ++g_failures;                                                                  \
    }                                                                                \
  } while (0)
static const char *g_scenario = "";

struct Fake final : dg::ServeEngine {
  double dt = 0.1;
  struct Solve {
    double t = 0.0;
    int64_t steps = 0;
    bool live = false, inputs = true;
    int retires = 0;
  };
  std::map<int64_t, Solve> solves;
  std::vector<int64_t> batch;
  std::map<int64_t, int32_t> fail_start, fail_poll;
  std::set<int64_t> fail_copy;
  std::map<int64_t, int64_t> bad_after;   // id -> steps after which the solve is non-admissible
  int32_t fail_finish = DG_OK;
  int set_batch_calls = 0, enqueue_calls = 0, retired_with_result = 0;
  int64_t enqueued_steps = 0;

  int32_t finish_tick() override { return fail_finish; }
  int32_t start(int64_t id) override {
    auto f = fail_start.find(id);
    if (f != fail_start.end()) return f->second;
    Solve &s = solves[id];
    if (s.live) return DG_EINVAL;   // started twice
    s.live = true;
    return DG_OK;
  }
  int32_t poll(int64_t id, double *t, int64_t *steps, bool *bad) override {
    auto f = fail_poll.find(id);
    if (f != fail_poll.end()) return f->second;
    Solve &s = solves[id];
    if (!s.live) return DG_EINVAL;   // polled while not running
    *t = s.t;
    *steps = s.steps;
    auto b = bad_after.find(id);
    *bad = b != bad_after.end() && s.steps >= b->second;
    return DG_OK;
  }
  int32_t retire(int64_t id, bool keep_result) override {
    Solve &s = solves[id];
    ++s.retires;
    if (!s.inputs) return DG_EINVAL;   // retired twice
    s.inputs = false;
    s.live = false;
    if (keep_result) {
      ++retired_with_result;
      if (fail_copy.count(id)) return DG_ECUDA;
    }
    return DG_OK;
  }
  int32_t set_batch(const std::vector<int64_t> &running) override {
    ++set_batch_calls;
    for (int64_t id : running)
      if (!solves[id].live) return DG_EINVAL;
    batch = running;
    return DG_OK;
  }
  int32_t enqueue(int64_t nsteps) override {
    ++enqueue_calls;
    enqueued_steps += nsteps;
    for (int64_t id : batch)
      if (!solves[id].live) return DG_EINVAL;   // the batch names a retired solve
    for (int64_t id : batch) {
      Solve &s = solves[id];
      s.t += dt * (double)nsteps;
      s.steps += nsteps;
    }
    return DG_OK;
  }
};

static int32_t state(const ServeScheduler &s, int64_t id) { return s.find(id)->state; }
static int32_t error(const ServeScheduler &s, int64_t id) { return s.find(id)->error; }

// run ticks until nothing runs or queues (at most `max` ticks)
static int drain(ServeScheduler &s, Fake &e, int max = 100) {
  int n = 0;
  for (; n < max; ++n) {
    int32_t r = -1, q = -1;
    if (s.tick(e, (double)n, &r, &q) != DG_OK) return -1;
    if (s.used() > s.budget()) return -2;
    if (r == 0 && q == 0) break;
  }
  return n;
}

static void fifo_and_budget() {
  g_scenario = "fifo_and_budget";
  ServeScheduler s(100, 1);
  Fake e;
  const int64_t a = s.submit(10, 40, 0.25, 0.0), b = s.submit(10, 40, 0.25, 0.0);
  const int64_t c = s.submit(10, 40, 0.25, 0.0), d = s.submit(10, 10, 0.25, 0.0);
  int32_t r = -1, q = -1;
  EXPECT(s.tick(e, 0.0, &r, &q) == DG_OK);
  // a and b fit (80); c does not, and d waits behind it (first come, first served)
  EXPECT(r == 2 && q == 2 && s.used() == 80);
  EXPECT(state(s, a) == DG_REQ_RUNNING && state(s, b) == DG_REQ_RUNNING);
  EXPECT(state(s, c) == DG_REQ_QUEUED && state(s, d) == DG_REQ_QUEUED);
  EXPECT(e.set_batch_calls == 1 && e.enqueue_calls == 1);
  EXPECT(s.tick(e, 1.0, &r, &q) == DG_OK);   // t = 0.1: no change
  EXPECT(r == 2 && q == 2 && e.set_batch_calls == 1 && e.enqueue_calls == 2);
  EXPECT(s.tick(e, 2.0, &r, &q) == DG_OK);   // t = 0.2
  EXPECT(s.tick(e, 3.0, &r, &q) == DG_OK);   // t = 0.3 >= 0.25: a, b done; c, d admitted
  EXPECT(state(s, a) == DG_REQ_DONE && state(s, b) == DG_REQ_DONE);
  EXPECT(r == 2 && q == 0 && s.used() == 50);
  EXPECT(s.find(a)->steps == 3 && s.find(a)->done_s == 3.0 && s.find(c)->start_s == 3.0);
  EXPECT(drain(s, e) >= 0);
  EXPECT(state(s, c) == DG_REQ_DONE && state(s, d) == DG_REQ_DONE && s.used() == 0);
  EXPECT(s.cell_stages() == 4 * 10 * 3 * 3);
  EXPECT(e.retired_with_result == 4);
}

static void oversized_request_keeps_the_accounting() {
  g_scenario = "oversized_request_keeps_the_accounting";
  ServeScheduler s(100, 1);
  Fake e;
  const int64_t a = s.submit(10, 60, 0.55, 0.0);
  int32_t r = -1, q = -1;
  EXPECT(s.tick(e, 0.0, &r, &q) == DG_OK && s.used() == 60);
  const int64_t big = s.submit(10, 150, 1.0, 1.0);   // larger than the whole budget
  const int64_t c = s.submit(10, 50, 0.15, 1.0);     // does not fit beside a
  EXPECT(s.tick(e, 1.0, &r, &q) == DG_OK);
  EXPECT(state(s, big) == DG_REQ_FAILED && error(s, big) == DG_ENOMEM);
  // the rejected request never held memory: a's 60 bytes are still counted,
  // so c (50) must wait
  EXPECT(s.used() == 60 && state(s, c) == DG_REQ_QUEUED && r == 1 && q == 1);
  EXPECT(drain(s, e) >= 0);
  EXPECT(state(s, a) == DG_REQ_DONE && state(s, c) == DG_REQ_DONE && s.used() == 0);
}

static void failed_start_keeps_the_accounting() {
  g_scenario = "failed_start_keeps_the_accounting";
  ServeScheduler s(100, 2);
  Fake e;
  const int64_t a = s.submit(5, 60, 0.35, 0.0);
  int32_t r = -1, q = -1;
  EXPECT(s.tick(e, 0.0, &r, &q) == DG_OK);
  const int64_t bad = s.submit(5, 30, 1.0, 0.5), c = s.submit(5, 40, 1.0, 0.5), d = s.submit(5, 10, 1.0, 0.5);
  e.fail_start[bad] = DG_ECUDA;
  e.fail_start[c] = DG_ENOMEM;
  EXPECT(s.tick(e, 1.0, &r, &q) == DG_OK);
  EXPECT(state(s, bad) == DG_REQ_FAILED && error(s, bad) == DG_ECUDA);
  EXPECT(state(s, c) == DG_REQ_FAILED && error(s, c) == DG_ENOMEM);
  // neither failed start holds memory; d (10) fits beside a (60)
  EXPECT(state(s, d) == DG_REQ_RUNNING && s.used() == 70 && r == 2 && q == 0);
  EXPECT(!e.solves[bad].inputs && !e.solves[c].inputs);   // their inputs were freed
  EXPECT(drain(s, e) >= 0 && s.used() == 0);
  EXPECT(state(s, a) == DG_REQ_DONE && state(s, d) == DG_REQ_DONE);
  EXPECT(e.enqueued_steps % 2 == 0);
}

static void nonphysical_solve_fails_and_frees() {
  g_scenario = "nonphysical_solve_fails_and_frees";
  ServeScheduler s(100, 1);
  Fake e;
  const int64_t a = s.submit(7, 50, 10.0, 0.0), b = s.submit(7, 50, 0.45, 0.0), c = s.submit(7, 50, 0.15, 0.0);
  e.bad_after[a] = 2;
  int32_t r = -1, q = -1;
  EXPECT(s.tick(e, 0.0, &r, &q) == DG_OK && r == 2 && q == 1);
  EXPECT(s.tick(e, 1.0, &r, &q) == DG_OK && r == 2);
  EXPECT(s.tick(e, 2.0, &r, &q) == DG_OK);   // a non-admissible after 2 steps; c admitted
  EXPECT(state(s, a) == DG_REQ_FAILED && error(s, a) == DG_ENONPHYS);
  EXPECT(state(s, c) == DG_REQ_RUNNING && s.used() == 100 && r == 2 && q == 0);
  EXPECT(drain(s, e) >= 0 && s.used() == 0);
  EXPECT(state(s, b) == DG_REQ_DONE && state(s, c) == DG_REQ_DONE);
  EXPECT(s.cell_stages() == 7 * 3 * (2 + 5 + 2));
}

static void failed_result_copy() {
  g_scenario = "failed_result_copy";
  ServeScheduler s(100, 1);
  Fake e;
  const int64_t a = s.submit(3, 10, 0.05, 0.0), b = s.submit(3, 10, 0.05, 0.0);
  e.fail_copy.insert(a);
  EXPECT(drain(s, e) >= 0);
  EXPECT(state(s, a) == DG_REQ_FAILED && error(s, a) == DG_ECUDA);
  EXPECT(state(s, b) == DG_REQ_DONE && error(s, b) == DG_OK && s.used() == 0);
}

static void engine_errors_propagate() {
  g_scenario = "engine_errors_propagate";
  ServeScheduler s(100, 1);
  Fake e;
  const int64_t a = s.submit(3, 10, 1.0, 0.0), b = s.submit(3, 10, 1.0, 0.0), c = s.submit(3, 10, 1.0, 0.0);
  int32_t r = -1, q = -1;
  EXPECT(s.tick(e, 0.0, &r, &q) == DG_OK && r == 3);
  e.fail_finish = DG_ETIMEOUT;   // e.g. a bounded wait in the batch kernel gave up
  EXPECT(s.tick(e, 1.0, &r, &q) == DG_ETIMEOUT);
  e.fail_finish = DG_OK;
  e.fail_poll[b] = DG_ECUDA;
  EXPECT(s.tick(e, 2.0, &r, &q) == DG_ECUDA);
  // the running list is intact: nothing was retired
  EXPECT(s.running().size() == 3 && state(s, a) == DG_REQ_RUNNING && state(s, c) == DG_REQ_RUNNING);
  e.fail_poll.clear();
  EXPECT(drain(s, e) >= 0 && s.used() == 0);
  EXPECT(state(s, a) == DG_REQ_DONE && state(s, b) == DG_REQ_DONE && state(s, c) == DG_REQ_DONE);
}

static void poll_error_after_a_retirement() {
  g_scenario = "poll_error_after_a_retirement";
  ServeScheduler s(100, 1);
  Fake e;
  const int64_t a = s.submit(3, 10, 0.05, 0.0), b = s.submit(3, 10, 1.0, 0.0);
  int32_t r = -1, q = -1;
  EXPECT(s.tick(e, 0.0, &r, &q) == DG_OK && r == 2);
  e.fail_poll[b] = DG_ECUDA;
  // a finishes in this tick before b's poll fails: a is retired once and
  // leaves the running list, b stays
  EXPECT(s.tick(e, 1.0, &r, &q) == DG_ECUDA);
  EXPECT(state(s, a) == DG_REQ_DONE && s.running().size() == 1 && s.running()[0] == b && s.used() == 10);
  e.fail_poll.clear();
  EXPECT(drain(s, e) >= 0 && state(s, b) == DG_REQ_DONE && s.used() == 0);
}

static void random_traffic() {
  g_scenario = "random_traffic";
  ServeScheduler s(1000, 3);
  Fake e;
  uint64_t x = 0x9E3779B97F4A7C15ull;
  auto rnd = [&]() { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return x; };
  std::vector<int64_t> ids;
  for (int tick = 0; tick < 400; ++tick) {
    for (int k = (int)(rnd() % 3); k > 0; --k) {
      const size_t bytes = 1 + rnd() % 1200;   // some never fit
      const int64_t id = s.submit(1 + (int64_t)(rnd() % 50), bytes, 0.05 + 0.01 * (double)(rnd() % 100), tick);
      if (rnd() % 17 == 0) e.fail_start[id] = DG_ECUDA;
      if (rnd() % 19 == 0) e.bad_after[id] = 1 + (int64_t)(rnd() % 5);
      ids.push_back(id);
    }
    int32_t r = -1, q = -1;
    EXPECT(s.tick(e, tick, &r, &q) == DG_OK);
    size_t held = 0;
    for (int64_t id : s.running()) held += s.find(id)->bytes;
    EXPECT(held == s.used() && s.used() <= s.budget());
  }
  EXPECT(drain(s, e, 10000) >= 0 && s.used() == 0);
  for (int64_t id : ids) {
    const SchedRequest *r = s.find(id);
    EXPECT(r->state == DG_REQ_DONE || r->state == DG_REQ_FAILED);
    if (r->bytes > s.budget()) EXPECT(r->error == DG_ENOMEM);
    EXPECT(!e.solves[id].inputs && e.solves[id].retires == 1);   // freed exactly once
  }
}

int main() {
  fifo_and_budget();
  oversized_request_keeps_the_accounting();
  failed_start_keeps_the_accounting();
  nonphysical_solve_fails_and_frees();
  failed_result_copy();
  engine_errors_propagate();
  poll_error_after_a_retirement();
  random_traffic();
  if (g_failures) return 1;
  printf("ok\n");
  return 0;
}

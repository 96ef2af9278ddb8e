// Serving loop: continuous batching of PCP solves.
//
// Requests (any m, n, r) are submitted without blocking.  A scheduler
// thread admits queued requests in arrival order while the device-memory
// budget and the slot count allow, launches each admitted group as one
// batched solve (batch.cu) on its own stream from a small pool, and keeps
// admitting while earlier groups are still on the GPU, so their work
// overlaps on the device.  Completion is detected with events; the host
// control path crosses the device boundary only at admission and
// completion.  Every request's result depends on that request alone (the
// seed of each instance is solved by its own CTA, and each filter tile's
// arithmetic is fixed by its own problem sizes), so a request gives the
// same result alone and in any mix.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"
#include "common.cuh"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(
             steady_clock::now().time_since_epoch())
      .count();
}

enum ReqState { kQueued, kRunning, kDone };

struct Request {
  pcp_problem prob;
  std::vector<int64_t> rows, cols;      // copies of the optional seed sets
  std::vector<int64_t> rorder, corder;  // and sampling orders
  size_t bytes = 0;
  ReqState state = kQueued;
  pcp_status status = PCP_OK;
  pcp_info info;
  double t_submit = 0, t_done = 0;
  // the filters of a seed that fails Eq. rank_test may be skipped on the
  // device (it grows and comes back); a skipped request that is not
  // requeued runs once more with this set, filters included
  bool no_gate = false;
};

struct Flight {
  pcp::BatchHandle h;
  int stream_slot = -1;
  cudaEvent_t start = nullptr, done = nullptr;
  std::vector<uint64_t> tickets;
  std::vector<unsigned char> gate;  // per request: growth follows a failure
  size_t bytes = 0;
};

}  // namespace

struct pcp_server {
  size_t budget = 0;
  int max_slots = 0;
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::vector<char> stream_busy;
  std::mutex mu;
  std::condition_variable cv;       // wakes the scheduler
  std::condition_variable done_cv;  // wakes waiters
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<Flight*> flights;
  size_t used_bytes = 0;
  int used_slots = 0;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::thread worker;
};

namespace {

// Launch one admitted group (called without the lock held).
void launch_group(pcp_server* S, Flight* f, std::vector<pcp_problem>& probs) {
  cudaStream_t st = S->streams[f->stream_slot];
  cudaEventCreate(&f->start);
  cudaEventCreate(&f->done);
  cudaEventRecord(f->start, st);
  pcp_status s = pcp::batch_launch((int)probs.size(), probs.data(), st,
                                   &f->h, true, f->gate.data());
  cudaEventRecord(f->done, st);
  if (s != PCP_OK) {
    // mark the whole group failed; the workspace (if any) is released when
    // the group completes
    std::lock_guard<std::mutex> lock(S->mu);
    for (uint64_t t : f->tickets) S->reqs[t].status = s;
  }
}

void finish_group(pcp_server* S, Flight* f) {
  cudaStream_t st = S->streams[f->stream_slot];
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, f->start, f->done);
  std::vector<pcp_info> infos(f->tickets.size());
  pcp_status launch_status = PCP_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    launch_status = S->reqs[f->tickets[0]].status;
  }
  if (launch_status == PCP_OK && f->h.count == (int)f->tickets.size()) {
    const pcp_status fs = pcp::batch_finish(&f->h, infos.data(), st, ms);
    if (f->h.status.size() != f->tickets.size()) {
      // the group failed as a whole (a CUDA error): every request gets it
      launch_status = fs == PCP_OK ? PCP_ERR_CUDA : fs;
      std::lock_guard<std::mutex> lock(S->mu);
      for (uint64_t t : f->tickets) S->reqs[t].status = launch_status;
    }
  } else {
    if (f->h.d_base) cudaFreeAsync(f->h.d_base, st);
    cudaStreamSynchronize(st);
    for (cudaEvent_t e : f->h.ev)
      if (e) cudaEventDestroy(e);
  }
  cudaEventDestroy(f->start);
  cudaEventDestroy(f->done);
  const double t = now_ms();
  std::lock_guard<std::mutex> lock(S->mu);
  std::vector<uint64_t> requeue;
  for (size_t i = 0; i < f->tickets.size(); ++i) {
    Request& r = S->reqs[f->tickets[i]];
    if (launch_status == PCP_OK && i < f->h.status.size()) {
      r.info = infos[i];
      r.status = f->h.status[i];
    } else {
      std::memset(&r.info, 0, sizeof(r.info));
      r.info.status = (int32_t)r.status;
    }
    // Section 3.5: a seed failing Eq. rank_test grows and the request goes
    // back to the head of the queue
    const pcp_params& q = r.prob.params;
    int gm = 0, gn = 0;
    if (q.grow_seed && r.status == PCP_ERR_RANK_TEST &&
        pcp::grown_seed_size(q, r.info, &gm, &gn)) {
      if (r.rorder.empty()) r.rorder = pcp::sample_order(q.m, q.rng_seed);
      if (r.corder.empty())
        r.corder = pcp::sample_order(q.n, q.rng_seed ^ 0xC01C01C0ull);
      pcp_problem grown = r.prob;
      grown.params.seed_m = gm;
      grown.params.seed_n = gn;
      grown.params.row_order = r.rorder.data();
      grown.params.col_order = r.corder.data();
      pcp::BatchInstance bi;
      if (pcp::batch_validate(grown, &bi) == PCP_OK) {
        r.prob = grown;
        r.bytes = pcp::batch_footprint(r.prob, bi);
        r.status = PCP_OK;
        r.state = kQueued;
        requeue.push_back(f->tickets[i]);
        continue;
      }
    }
    if (launch_status == PCP_OK && i < f->h.skipped.size() &&
        f->h.skipped[i] && !r.no_gate) {
      // its filters were skipped but it does not grow: run it again in full
      // (the seed size is unchanged, so the footprint is too)
      r.no_gate = true;
      r.status = PCP_OK;
      r.state = kQueued;
      requeue.push_back(f->tickets[i]);
      continue;
    }
    r.t_done = t;
    r.info.t_total_ms = (float)(t - r.t_submit);
    r.state = kDone;
  }
  for (auto it = requeue.rbegin(); it != requeue.rend(); ++it)
    S->queue.push_front(*it);
  if (!requeue.empty()) S->cv.notify_all();
  S->used_bytes -= f->bytes;
  S->used_slots -= (int)f->tickets.size();
  S->stream_busy[f->stream_slot] = 0;
  S->done_cv.notify_all();
}

void scheduler(pcp_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (true) {
    // admit a group if a stream is free
    int slot = -1;
    for (size_t i = 0; i < S->streams.size(); ++i)
      if (!S->stream_busy[i]) {
        slot = (int)i;
        break;
      }
    Flight* nf = nullptr;
    std::vector<pcp_problem> probs;
    if (slot >= 0 && !S->queue.empty()) {
      nf = new Flight();
      nf->stream_slot = slot;
      while (!S->queue.empty()) {
        const uint64_t ticket = S->queue.front();
        Request& r = S->reqs[ticket];
        const bool fits = S->used_slots + 1 <= S->max_slots &&
                          S->used_bytes + r.bytes <= S->budget;
        if (!fits) {
          if (nf->tickets.empty() && S->flights.empty()) {
            // alone on an idle device and still too big: refuse it
            r.status = PCP_ERR_NOMEM;
            r.info.status = (int32_t)PCP_ERR_NOMEM;
            r.state = kDone;
            r.t_done = now_ms();
            S->queue.pop_front();
            S->done_cv.notify_all();
            continue;
          }
          break;
        }
        S->queue.pop_front();
        r.state = kRunning;
        S->used_bytes += r.bytes;
        S->used_slots += 1;
        nf->bytes += r.bytes;
        nf->tickets.push_back(ticket);
        nf->gate.push_back(r.no_gate ? 0 : 1);
        probs.push_back(r.prob);
      }
      if (probs.empty()) {
        delete nf;
        nf = nullptr;
      }
    }
    if (nf) {
      S->stream_busy[slot] = 1;
      S->flights.push_back(nf);
      lock.unlock();
      launch_group(S, nf, probs);
      lock.lock();
      continue;
    }
    // poll running groups
    bool progressed = false;
    for (size_t i = 0; i < S->flights.size();) {
      Flight* f = S->flights[i];
      lock.unlock();
      // anything but "not ready" ends the group (an error is reported by
      // finish_group through the group's status)
      const bool ready = cudaEventQuery(f->done) != cudaErrorNotReady;
      if (ready) finish_group(S, f);
      lock.lock();
      if (ready) {
        S->flights.erase(S->flights.begin() + i);
        delete f;
        progressed = true;
      } else {
        ++i;
      }
    }
    if (S->stopping && S->queue.empty() && S->flights.empty()) break;
    if (!progressed) {
      S->cv.wait_for(lock, std::chrono::microseconds(
                               S->flights.empty() ? 2000 : 50));
    }
  }
}

}  // namespace

extern "C" pcp_status pcp_serve_create(size_t hbm_budget_bytes,
                                       int32_t max_slots, int32_t streams,
                                       pcp_server** out) {
  PCP_ARG(out, "pcp_serve_create: null pointer");
  *out = nullptr;
  PCP_ARG(hbm_budget_bytes > 0 && max_slots >= 1 && streams >= 1 &&
              streams <= 16,
          "pcp_serve_create: need budget > 0, max_slots >= 1, "
          "1 <= streams <= 16");
  pcp_server* S = new pcp_server();
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  if (cudaGetDevice(&S->device) != cudaSuccess) S->device = 0;
  for (int i = 0; i < streams; ++i) {
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (cudaStream_t s2 : S->streams) cudaStreamDestroy(s2);
      delete S;
      return pcp::cuda_fail(e, "cudaStreamCreate", __FILE__, __LINE__);
    }
    S->streams.push_back(st);
    S->stream_busy.push_back(0);
  }
  S->worker = std::thread(scheduler, S);
  *out = S;
  return PCP_OK;
}

extern "C" pcp_status pcp_serve_submit(pcp_server* S, const pcp_problem* prob,
                                       uint64_t* ticket) {
  PCP_ARG(S && prob && ticket, "pcp_serve_submit: null pointer");
  pcp::BatchInstance bi;
  pcp_status s = pcp::batch_validate(*prob, &bi);
  if (s != PCP_OK) return s;
  std::lock_guard<std::mutex> lock(S->mu);
  if (S->stopping) {
    pcp::set_error("pcp_serve_submit: server is shutting down");
    return PCP_ERR_CANCELLED;
  }
  const uint64_t t = S->next_ticket++;
  Request& r = S->reqs[t];
  r.prob = *prob;
  if (prob->params.seed_rows) {
    r.rows.assign(prob->params.seed_rows, prob->params.seed_rows + bi.mp);
    r.prob.params.seed_rows = r.rows.data();
  }
  if (prob->params.seed_cols) {
    r.cols.assign(prob->params.seed_cols, prob->params.seed_cols + bi.np);
    r.prob.params.seed_cols = r.cols.data();
  }
  if (prob->params.row_order) {
    r.rorder.assign(prob->params.row_order,
                    prob->params.row_order + prob->params.m);
    r.prob.params.row_order = r.rorder.data();
  }
  if (prob->params.col_order) {
    r.corder.assign(prob->params.col_order,
                    prob->params.col_order + prob->params.n);
    r.prob.params.col_order = r.corder.data();
  }
  r.bytes = pcp::batch_footprint(*prob, bi);
  r.t_submit = now_ms();
  std::memset(&r.info, 0, sizeof(r.info));
  S->queue.push_back(t);
  *ticket = t;
  S->cv.notify_all();
  return PCP_OK;
}

static pcp_status take_result(pcp_server* S, uint64_t ticket, pcp_info* info,
                              bool* found) {
  auto it = S->reqs.find(ticket);
  *found = it != S->reqs.end();
  if (!*found) {
    pcp::set_error("pcp_serve: unknown ticket %llu",
                   (unsigned long long)ticket);
    return PCP_ERR_ARG;
  }
  if (it->second.state != kDone) return PCP_ERR_BUSY;
  const pcp_status s = it->second.status;
  if (info) *info = it->second.info;
  S->reqs.erase(it);
  return s;
}

extern "C" pcp_status pcp_serve_poll(pcp_server* S, uint64_t ticket,
                                     pcp_info* info) {
  PCP_ARG(S, "pcp_serve_poll: null server");
  std::lock_guard<std::mutex> lock(S->mu);
  bool found = false;
  return take_result(S, ticket, info, &found);
}

extern "C" pcp_status pcp_serve_wait(pcp_server* S, uint64_t ticket,
                                     pcp_info* info) {
  PCP_ARG(S, "pcp_serve_wait: null server");
  std::unique_lock<std::mutex> lock(S->mu);
  while (true) {
    bool found = false;
    const pcp_status s = take_result(S, ticket, info, &found);
    if (s != PCP_ERR_BUSY || !found) return s;
    S->done_cv.wait_for(lock, std::chrono::milliseconds(10));
  }
}

extern "C" pcp_status pcp_serve_stop(pcp_server* S) {
  PCP_ARG(S, "pcp_serve_stop: null server");
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stopping = true;
    // requests that never reached the GPU are cancelled
    for (uint64_t t : S->queue) {
      Request& r = S->reqs[t];
      r.state = kDone;
      r.status = PCP_ERR_CANCELLED;
      r.info.status = (int32_t)PCP_ERR_CANCELLED;
      r.t_done = now_ms();
    }
    S->queue.clear();
    S->cv.notify_all();
    S->done_cv.notify_all();
  }
  if (S->worker.joinable()) S->worker.join();
  return PCP_OK;
}

extern "C" pcp_status pcp_serve_destroy(pcp_server* S) {
  if (!S) return PCP_OK;
  pcp_serve_stop(S);
  for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
  delete S;
  return PCP_OK;
}

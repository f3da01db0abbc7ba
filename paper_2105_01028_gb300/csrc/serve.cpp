// Serving: a request loop that runs many forward solves at once on one GPU.
//
// Reconstruction needs many forward models, so the server keeps a queue of solve
// requests and admits them into slots while their device-memory footprint fits a
// budget.  Every admitted request gets its own context and CUDA stream; the worker
// thread advances all active slots round-robin in slices of steps replayed from each
// context's captured CUDA graph, so the solves' kernels overlap on the device.  A slot
// that finishes has its detector curves read back, its memory returned, and the next
// waiting request admitted.  All CUDA work happens on the worker thread; the public
// calls only touch the request table under a mutex.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "trinity.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  trinity_grid_desc grid{};
  std::vector<float> mua, mus, n;
  double g = 0.0;
  trinity_source_desc source{};
  std::vector<trinity_detector_desc> dets;
  double bin_ps = 10.0;
  int nbins = 1;
  int nsteps = 0;
  int fresnel = 0;
  size_t footprint = 0;
  Clock::time_point t_submit, t_admit, t_done;
  int state = 0;  // 0 queued, 1 active, 2 done, 3 failed, 4 cancelled
  int status = TRINITY_OK;
  std::string error;
  std::vector<double> detectors;
  // worker-side
  trinity_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  int steps_queued = 0;
  bool cancel = false;
};

}  // namespace

struct trinity_server {
  size_t budget = 0;
  int max_slots = 1;
  int slice = 32;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<Request*> active;
  size_t used = 0;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  bool started = false;
  int device = 0;
  // statistics
  int max_concurrent = 0;
  uint64_t completed = 0, failed = 0;
};

namespace {

void finish(trinity_server* s, Request* r, int status, const std::string& err) {
  if (r->ctx) {
    trinity_destroy(r->ctx);
    r->ctx = nullptr;
  }
  if (r->stream) {
    cudaStreamDestroy(r->stream);
    r->stream = nullptr;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= r->footprint;
  r->t_done = Clock::now();
  r->status = status;
  r->error = err;
  if (r->cancel)
    r->state = 4;
  else
    r->state = (status == TRINITY_OK || status == TRINITY_W_NOT_CONVERGED) ? 2 : 3;
  if (r->state == 2)
    ++s->completed;
  else if (r->state == 3)
    ++s->failed;
  s->active.erase(std::remove(s->active.begin(), s->active.end(), r), s->active.end());
  s->cv_done.notify_all();
}

// Create the context of an admitted request (worker thread).
int start_request(Request* r) {
  if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess) return TRINITY_E_CUDA;
  int rc = trinity_create_grid(&r->grid, r->stream, &r->ctx);
  if (rc != TRINITY_OK) return rc;
  rc = trinity_set_optics(r->ctx, r->mua.data(), r->mus.data(), r->n.data(), r->g, 0);
  if (rc != TRINITY_OK) return rc;
  if (r->fresnel && (rc = trinity_set_fresnel(r->ctx, 1)) != TRINITY_OK) return rc;
  if (r->source.pulse_steps > 0) {
    rc = trinity_set_source(r->ctx, r->source.face, r->source.u_mm, r->source.v_mm, r->source.half_angle_deg,
                            r->source.pulse_steps, r->source.energy);
    if (rc != TRINITY_OK) return rc;
  }
  for (const auto& d : r->dets) {
    int id = 0;
    rc = trinity_add_detector(r->ctx, d.face, d.u_mm, d.v_mm, d.radius_mm, d.half_angle_deg, &id);
    if (rc != TRINITY_OK) return rc;
  }
  return trinity_set_bins(r->ctx, r->bin_ps, r->nbins);
}

void worker_loop(trinity_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::vector<Request*> admit;
    std::vector<Request*> run;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty() || !s->active.empty(); });
      if (s->stop && s->active.empty()) break;
      // admission: FIFO while slots and memory allow (the head blocks the queue, so a
      // large request is not starved by small ones behind it)
      while (!s->stop && !s->queue.empty() && static_cast<int>(s->active.size()) < s->max_slots) {
        Request* r = s->reqs[s->queue.front()].get();
        if (r->cancel) {
          s->queue.pop_front();
          r->state = 4;
          r->t_done = Clock::now();
          s->cv_done.notify_all();
          continue;
        }
        if (s->used + r->footprint > s->budget) break;
        s->queue.pop_front();
        s->used += r->footprint;
        r->state = 1;
        r->t_admit = Clock::now();
        s->active.push_back(r);
        admit.push_back(r);
      }
      s->max_concurrent = std::max(s->max_concurrent, static_cast<int>(s->active.size()));
      run = s->active;
    }
    for (Request* r : admit) {
      const int rc = start_request(r);
      if (rc != TRINITY_OK) {
        const std::string msg = r->ctx ? trinity_last_error(r->ctx) : "context creation failed";
        finish(s, r, rc, msg);
      }
    }
    // advance every active slot by one slice; slots whose previous slice is still running
    // are skipped so the host never blocks on one solve while others could run
    bool any_busy = false;
    for (Request* r : run) {
      if (!r->ctx) continue;
      if (cudaStreamQuery(r->stream) == cudaErrorNotReady) {
        any_busy = true;
        continue;
      }
      if (r->cancel) {
        finish(s, r, TRINITY_E_STATE, "cancelled");
        continue;
      }
      if (r->steps_queued < r->nsteps) {
        const int k = std::min(s->slice, r->nsteps - r->steps_queued);
        const int rc = trinity_run(r->ctx, k);
        if (rc != TRINITY_OK) {
          finish(s, r, rc, trinity_last_error(r->ctx));
          continue;
        }
        r->steps_queued += k;
        any_busy = true;
      } else {
        int rc = trinity_sync(r->ctx);
        std::vector<double> det(r->dets.size() * static_cast<size_t>(r->nbins));
        if (rc == TRINITY_OK || rc == TRINITY_W_NOT_CONVERGED) {
          const int rc2 = trinity_read_detectors(r->ctx, det.data(), det.size());
          if (rc2 != TRINITY_OK) rc = rc2;
        }
        r->detectors = std::move(det);
        finish(s, r, rc, rc == TRINITY_OK ? "" : trinity_last_error(r->ctx));
      }
    }
    if (any_busy) std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

bool request_valid(const trinity_request* q, std::string* why) {
  if (!q) {
    *why = "null request";
    return false;
  }
  if (!q->mua || !q->mus || !q->n) {
    *why = "null optics";
    return false;
  }
  if (q->nsteps < 1 || q->nbins < 1 || !(q->bin_ps > 0.0)) {
    *why = "nsteps and nbins must be >= 1 and bin_ps > 0";
    return false;
  }
  if (q->n_detectors < 0 || (q->n_detectors > 0 && !q->detectors)) {
    *why = "bad detector list";
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

int trinity_serve_create(size_t hbm_budget_bytes, int max_slots, int steps_per_slice, trinity_server** out) {
  if (!out || max_slots < 1 || steps_per_slice < 1 || hbm_budget_bytes == 0) return TRINITY_E_INVALID;
  *out = nullptr;
  trinity_server* s = new (std::nothrow) trinity_server();
  if (!s) return TRINITY_E_OOM;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->slice = steps_per_slice;
  *out = s;
  return TRINITY_OK;
}

int trinity_serve_submit(trinity_server* s, const trinity_request* q, uint64_t* req_id) {
  if (!s || !req_id) return TRINITY_E_INVALID;
  std::string why;
  if (!request_valid(q, &why)) return TRINITY_E_INVALID;
  const size_t fp = trinity_footprint_bytes(&q->grid);
  if (fp == 0) return TRINITY_E_INVALID;
  if (fp > s->budget) return TRINITY_E_OOM;  // could never be admitted
  auto r = std::make_unique<Request>();
  r->grid = q->grid;
  const size_t nv = static_cast<size_t>(q->grid.nx) * q->grid.ny * q->grid.nz;
  r->mua.assign(q->mua, q->mua + nv);
  r->mus.assign(q->mus, q->mus + nv);
  r->n.assign(q->n, q->n + nv);
  r->g = q->g;
  r->source = q->source;
  r->dets.assign(q->detectors, q->detectors + q->n_detectors);
  r->bin_ps = q->bin_ps;
  r->nbins = q->nbins;
  r->nsteps = q->nsteps;
  r->fresnel = q->fresnel;
  r->footprint = fp;
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->started) {
    cudaGetDevice(&s->device);
    s->worker = std::thread(worker_loop, s);
    s->started = true;
  }
  r->id = s->next_id++;
  *req_id = r->id;
  s->queue.push_back(r->id);
  s->reqs[r->id] = std::move(r);
  s->cv_work.notify_all();
  return TRINITY_OK;
}

int trinity_serve_poll(trinity_server* s, uint64_t req, int* state, double* detectors, size_t n,
                       double* latency_ms) {
  if (!s || !state) return TRINITY_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req);
  if (it == s->reqs.end()) return TRINITY_E_INVALID;
  Request* r = it->second.get();
  *state = r->state;
  if (r->state < 2) return TRINITY_OK;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  if (r->state == 2 && detectors) {
    if (n != r->detectors.size()) return TRINITY_E_INVALID;
    std::copy(r->detectors.begin(), r->detectors.end(), detectors);
  }
  return r->state == 2 ? r->status : (r->state == 4 ? TRINITY_E_STATE : r->status);
}

int trinity_serve_wait(trinity_server* s, uint64_t req, double timeout_s) {
  if (!s) return TRINITY_E_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req);
  if (it == s->reqs.end()) return TRINITY_E_INVALID;
  Request* r = it->second.get();
  const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->state >= 2; });
  return ok ? TRINITY_OK : TRINITY_E_TIMEOUT;
}

int trinity_serve_cancel(trinity_server* s, uint64_t req) {
  if (!s) return TRINITY_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req);
  if (it == s->reqs.end()) return TRINITY_E_INVALID;
  it->second->cancel = true;
  s->cv_work.notify_all();
  return TRINITY_OK;
}

int trinity_serve_stats(trinity_server* s, uint64_t* completed, uint64_t* failed, int* max_concurrent,
                        size_t* bytes_in_use) {
  if (!s) return TRINITY_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (completed) *completed = s->completed;
  if (failed) *failed = s->failed;
  if (max_concurrent) *max_concurrent = s->max_concurrent;
  if (bytes_in_use) *bytes_in_use = s->used;
  return TRINITY_OK;
}

void trinity_serve_destroy(trinity_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& kv : s->reqs)
      if (kv.second->state < 2) kv.second->cancel = true;
    s->cv_work.notify_all();
  }
  if (s->started) s->worker.join();
  delete s;
}

}  // extern "C"

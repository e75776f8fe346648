// Serving loop over the C ABI (declared in include/galario_gb300.h): a FIFO
// of chi-square requests, an HBM budget, and a scheduler thread that keeps
// `slots` worker contexts (one CUDA stream each) busy, admitting queued
// requests -- alone or several of one precision as one batch -- whenever a
// slot and the budget allow.  Host code only; every evaluation runs through
// gal_chi2_* / gal_chi2_batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/galario_gb300.h"

namespace {

using Clock = std::chrono::steady_clock;
constexpr size_t kMaxQueue = 65536;

struct Pending {
  uint64_t ticket;
  gal_request req;
  Clock::time_point t0;
  int prec;     // 0 float, 1 double
  size_t need;  // workspace the request may add to its slot
};

struct Result {
  int status = GAL_OK;
  double chi2 = 0.0;
  double latency = 0.0;
  bool done = false;
};

struct Slot {
  gal_ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  double* d_out = nullptr;  // max_batch results (device)
  double* h_out = nullptr;  // the same, pinned host copy
  std::vector<Pending> run;
  bool busy = false;
  size_t base_ws = 0;  // workspace of a fresh context (not releasable)
};

int pow2_side(int n) { return n >= 4 && n <= 8192 && (n & (n - 1)) == 0; }

// a request's workspace: the single call's row output and window buffer
// (three half spectra); a batch needs less per request
size_t need_bytes(const gal_request& r, int real_bytes) {
  const size_t spec = (size_t)r.nxy * (size_t)(r.nxy / 2 + 1) * 2 * (size_t)real_bytes;
  const size_t beam = r.pb_fwhm > 0.0 ? 2 * (size_t)r.nxy * (size_t)real_bytes : 0;
  // the full plane keeps up to nxy columns in the row-pass output
  const size_t full = r.full_plane ? (size_t)r.nxy * (size_t)r.nxy * 2 * (size_t)real_bytes : 0;
  return 3 * spec + beam + full;
}

}  // namespace

struct gal_server {
  int device = 0;
  size_t budget = 0;
  int max_batch = 1;
  gal_ctx* primary = nullptr;  // observations are registered on it
  std::vector<gal_data*> data;
  size_t data_bytes = 0;
  std::vector<Slot> slots;

  std::mutex mu;
  std::condition_variable cv_submit;  // scheduler waits for work
  std::condition_variable cv_done;    // waiters wait for results
  std::deque<Pending> queue;
  std::unordered_map<uint64_t, Result> results;
  uint64_t next_ticket = 1;
  bool stop = false;

  // statistics (scheduler thread writes, under mu)
  uint64_t submitted = 0, completed = 0, launches = 0, max_inflight = 0;
  size_t workspace_bytes = 0, peak_bytes = 0;

  std::thread thread;

  size_t held() const {
    size_t b = 0;
    for (const Slot& s : slots) b += gal_workspace_bytes(s.ctx);
    return b;
  }
  void loop();
  int launch(Slot& s, std::vector<Pending>& grp);
  void finish(std::vector<Pending>& grp, const double* vals, int status, Clock::time_point t);
  int recreate(Slot& s);
};

// A fresh worker context: no launch-shape tuning (its timing runs would
// synchronise the slot's stream in the middle of serving).
static int new_worker(int device, Slot& s) {
  int st = gal_create(&s.ctx, device);
  if (st == GAL_OK) st = gal_set_batch_tuning(s.ctx, 0);
  s.base_ws = gal_workspace_bytes(s.ctx);
  return st;
}

int gal_server::recreate(Slot& s) {
  // release an idle slot's workspace by replacing its context
  gal_destroy(s.ctx);
  s.ctx = nullptr;
  return new_worker(device, s);
}

void gal_server::finish(std::vector<Pending>& grp, const double* vals, int status,
                        Clock::time_point t) {
  {
    std::lock_guard<std::mutex> lk(mu);
    for (size_t k = 0; k < grp.size(); ++k) {
      Result& r = results[grp[k].ticket];
      r.status = status;
      r.chi2 = status == GAL_OK && vals ? vals[k] : 0.0;
      r.latency = std::chrono::duration<double>(t - grp[k].t0).count();
      r.done = true;
      ++completed;
    }
  }
  cv_done.notify_all();
}

int gal_server::launch(Slot& s, std::vector<Pending>& grp) {
  const int n = (int)grp.size();
  int st;
  if (n == 1) {
    const gal_request& r = grp[0].req;
    const gal_opts o{r.pb_fwhm, r.full_plane};  // the request's options
    if (grp[0].prec == 0) {
      st = r.image ? gal_chi2_image_ex_f32(s.ctx, static_cast<const float*>(r.image), r.nxy,
                                           r.dxy, r.dRA, r.dDec, r.PA, &o, r.data, s.d_out, s.st)
                   : gal_chi2_profile_ex_f32(s.ctx, static_cast<const float*>(r.intensity), r.nr,
                                             r.Rmin, r.dR, r.nxy, r.dxy, r.inc, r.dRA, r.dDec,
                                             r.PA, &o, r.data, s.d_out, s.st);
    } else {
      st = r.image ? gal_chi2_image_ex_f64(s.ctx, static_cast<const double*>(r.image), r.nxy,
                                           r.dxy, r.dRA, r.dDec, r.PA, &o, r.data, s.d_out, s.st)
                   : gal_chi2_profile_ex_f64(s.ctx, static_cast<const double*>(r.intensity), r.nr,
                                             r.Rmin, r.dR, r.nxy, r.dxy, r.inc, r.dRA, r.dDec,
                                             r.PA, &o, r.data, s.d_out, s.st);
    }
  } else {
    std::vector<gal_request> rq(n);
    for (int k = 0; k < n; ++k) rq[k] = grp[k].req;
    st = gal_chi2_batch(s.ctx, rq.data(), n, s.d_out, s.st);
  }
  if (st != GAL_OK) return st;
  if (cudaMemcpyAsync(s.h_out, s.d_out, sizeof(double) * n, cudaMemcpyDeviceToHost, s.st) ||
      cudaEventRecord(s.ev, s.st))
    return GAL_E_CUDA;
  return GAL_OK;
}

void gal_server::loop() {
  cudaSetDevice(device);
  uint64_t inflight = 0;
  std::vector<Pending> grp;
  for (;;) {
    bool progress = false;
    // completions
    for (Slot& s : slots) {
      if (!s.busy) continue;
      const cudaError_t q = cudaEventQuery(s.ev);
      if (q == cudaErrorNotReady) continue;
      const auto t = Clock::now();
      finish(s.run, s.h_out, q == cudaSuccess ? GAL_OK : GAL_E_CUDA, t);
      if (q != cudaSuccess) (void)cudaGetLastError();
      inflight -= s.run.size();
      s.run.clear();
      s.busy = false;
      progress = true;
    }
    // admissions: the head of the queue (plus followers of its precision)
    for (Slot& s : slots) {
      if (s.busy) continue;
      enum { kLaunch, kRelease, kFail, kWait, kEmpty } act = kEmpty;
      grp.clear();
      {
        std::lock_guard<std::mutex> lk(mu);
        if (!queue.empty()) {
          const int prec = queue.front().prec;
          size_t need = 0;
          for (size_t k = 0; k < queue.size() && (int)grp.size() < max_batch; ++k) {
            if (queue[k].prec != prec) break;
            grp.push_back(queue[k]);
            need += queue[k].need;
          }
          const size_t base = data_bytes + held();
          while (grp.size() > 1 && base + need > budget) {  // admit fewer
            need -= grp.back().need;
            grp.pop_back();
          }
          if (base + need <= budget) {
            act = kLaunch;
            for (size_t k = 0; k < grp.size(); ++k) queue.pop_front();
            peak_bytes = std::max(peak_bytes, base + need);
          } else {
            bool idle_ws = false;
            for (const Slot& o : slots)
              idle_ws |= !o.busy && gal_workspace_bytes(o.ctx) > o.base_ws;
            if (idle_ws) {
              act = kRelease;
            } else if (inflight == 0) {
              act = kFail;  // does not fit even with no workspace held anywhere
              grp.assign(1, queue.front());
              queue.pop_front();
            } else {
              act = kWait;
            }
          }
        }
      }
      if (act == kEmpty || act == kWait) break;
      progress = true;
      if (act == kRelease) {
        for (Slot& o : slots)
          if (!o.busy && gal_workspace_bytes(o.ctx) > o.base_ws) recreate(o);
        break;
      }
      if (act == kFail) {
        finish(grp, nullptr, GAL_E_NOMEM, Clock::now());
        continue;
      }
      const int st = launch(s, grp);
      if (st != GAL_OK) {
        finish(grp, nullptr, st, Clock::now());
        continue;
      }
      s.run = grp;
      s.busy = true;
      inflight += grp.size();
      {
        std::lock_guard<std::mutex> lk(mu);
        ++launches;
        max_inflight = std::max<uint64_t>(max_inflight, inflight);
        workspace_bytes = held();
        peak_bytes = std::max(peak_bytes, data_bytes + workspace_bytes);
      }
    }
    if (progress) continue;
    if (inflight > 0) {
      std::this_thread::yield();  // results are polled; the GPU is working
      continue;
    }
    std::unique_lock<std::mutex> lk(mu);
    if (stop && queue.empty()) break;
    cv_submit.wait_for(lk, std::chrono::milliseconds(1),
                       [&] { return stop || !queue.empty(); });
  }
}

extern "C" {

int gal_server_create(int device, size_t hbm_budget_bytes, int slots, int max_batch,
                      gal_server** out) {
  if (!out) return GAL_E_INVAL;
  *out = nullptr;
  if (slots < 1 || slots > 256 || max_batch < 1 || hbm_budget_bytes == 0) return GAL_E_INVAL;
  gal_server* s = new (std::nothrow) gal_server;
  if (!s) return GAL_E_NOMEM;
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->max_batch = max_batch;
  int st = gal_create(&s->primary, device);
  s->slots.resize(slots);
  for (Slot& sl : s->slots) {
    if (st != GAL_OK) break;
    st = new_worker(device, sl);
    if (st == GAL_OK &&
        (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) ||
         cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) ||
         cudaMalloc(&sl.d_out, sizeof(double) * max_batch) ||
         cudaMallocHost(&sl.h_out, sizeof(double) * max_batch)))
      st = GAL_E_CUDA;
  }
  if (st != GAL_OK) {
    gal_server_destroy(s);
    return st;
  }
  s->thread = std::thread([s] { s->loop(); });
  *out = s;
  return GAL_OK;
}

static int add_data(gal_server* s, const void* u, const void* v, const void* re, const void* im,
                    const void* w, int64_t M, int rb, bool z_order, gal_data** out) {
  if (!s || !out || M < 0) return GAL_E_INVAL;
  const size_t bytes = 5 * (size_t)M * (size_t)rb;
  {
    // reserve the bytes before registering, so that concurrent add_data
    // calls cannot pass the check together and overrun the budget
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->data_bytes + bytes > s->budget) return GAL_E_NOMEM;
    s->data_bytes += bytes;
  }
  cudaSetDevice(s->device);
  // z_order: the library keeps its own copies (the budget charges the same
  // 5 M values either way)
  auto f32 = z_order ? gal_data_create_sorted_f32 : gal_data_create_f32;
  auto f64 = z_order ? gal_data_create_sorted_f64 : gal_data_create_f64;
  const int st =
      rb == 4 ? f32(s->primary, static_cast<const float*>(u), static_cast<const float*>(v),
                    static_cast<const float*>(re), static_cast<const float*>(im),
                    static_cast<const float*>(w), M, nullptr, out)
              : f64(s->primary, static_cast<const double*>(u), static_cast<const double*>(v),
                    static_cast<const double*>(re), static_cast<const double*>(im),
                    static_cast<const double*>(w), M, nullptr, out);
  std::lock_guard<std::mutex> lk(s->mu);
  if (st != GAL_OK) {
    s->data_bytes -= bytes;  // give the reservation back
    return st;
  }
  s->data.push_back(*out);
  return GAL_OK;
}

int gal_server_add_data_f32(gal_server* s, const float* u, const float* v, const float* re,
                            const float* im, const float* w, int64_t M, gal_data** out) {
  return add_data(s, u, v, re, im, w, M, 4, false, out);
}
int gal_server_add_data_f64(gal_server* s, const double* u, const double* v, const double* re,
                            const double* im, const double* w, int64_t M, gal_data** out) {
  return add_data(s, u, v, re, im, w, M, 8, false, out);
}
int gal_server_add_data_sorted_f32(gal_server* s, const float* u, const float* v, const float* re,
                                   const float* im, const float* w, int64_t M, gal_data** out) {
  return add_data(s, u, v, re, im, w, M, 4, true, out);
}
int gal_server_add_data_sorted_f64(gal_server* s, const double* u, const double* v,
                                   const double* re, const double* im, const double* w, int64_t M,
                                   gal_data** out) {
  return add_data(s, u, v, re, im, w, M, 8, true, out);
}

static int make_pending(const gal_request* req, Pending* p) {
  int64_t M = 0;
  int rb = 0;
  if (gal_data_info(req->data, &M, &rb) != GAL_OK) return GAL_E_INVAL;
  if ((req->image != nullptr) == (req->intensity != nullptr)) return GAL_E_INVAL;
  if (!pow2_side(req->nxy) || !(req->dxy > 0.0)) return GAL_E_INVAL;
  if (!(req->pb_fwhm >= 0.0) || !std::isfinite(req->pb_fwhm)) return GAL_E_INVAL;
  if (req->full_plane != 0 && req->full_plane != 1) return GAL_E_INVAL;
  p->req = *req;
  p->prec = rb == 8 ? 1 : 0;
  p->need = need_bytes(*req, rb);
  return GAL_OK;
}

int gal_server_submit_many(gal_server* s, const gal_request* reqs, int n, uint64_t* tickets) {
  if (!s || n < 0 || (n > 0 && (!reqs || !tickets))) return GAL_E_INVAL;
  std::vector<Pending> ps(n);
  for (int i = 0; i < n; ++i) {
    const int st = make_pending(&reqs[i], &ps[i]);
    if (st != GAL_OK) return st;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return GAL_E_INVAL;
    if (s->queue.size() + (size_t)n > kMaxQueue) return GAL_E_BUSY;
    const auto t0 = Clock::now();
    for (int i = 0; i < n; ++i) {
      ps[i].ticket = s->next_ticket++;
      ps[i].t0 = t0;
      s->results[ps[i].ticket] = Result{};
      s->queue.push_back(ps[i]);
      tickets[i] = ps[i].ticket;
    }
    s->submitted += (uint64_t)n;
  }
  s->cv_submit.notify_one();
  return GAL_OK;
}

int gal_server_submit(gal_server* s, const gal_request* req, uint64_t* ticket) {
  if (!req) return GAL_E_INVAL;
  return gal_server_submit_many(s, req, 1, ticket);
}

int gal_server_wait(gal_server* s, uint64_t ticket, int timeout_ms, double* chi2,
                    double* latency_s) {
  if (!s) return GAL_E_INVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return GAL_E_INVAL;
  auto ready = [&] { return s->results[ticket].done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return GAL_E_TIMEOUT;
  }
  const Result r = s->results[ticket];
  s->results.erase(ticket);
  if (chi2) *chi2 = r.chi2;
  if (latency_s) *latency_s = r.latency;
  return r.status;
}

int gal_server_get_stats(gal_server* s, gal_server_stats* out) {
  if (!s || !out) return GAL_E_INVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->launches = s->launches;
  out->max_inflight = s->max_inflight;
  out->data_bytes = s->data_bytes;
  out->workspace_bytes = s->workspace_bytes;
  out->peak_bytes = s->peak_bytes;
  return GAL_OK;
}

void gal_server_destroy(gal_server* s) {
  if (!s) return;
  if (s->thread.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv_submit.notify_all();
    s->thread.join();
  }
  cudaSetDevice(s->device);
  for (Slot& sl : s->slots) {
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.d_out) cudaFree(sl.d_out);
    if (sl.h_out) cudaFreeHost(sl.h_out);
    gal_destroy(sl.ctx);
  }
  for (gal_data* d : s->data) gal_data_destroy(d);
  gal_destroy(s->primary);
  delete s;
}

}  // extern "C"

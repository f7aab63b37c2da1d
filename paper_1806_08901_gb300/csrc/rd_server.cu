// rd_server.cu -- the serving loop (rd_server_*): per-field selection
// requests (Algorithm 1 lines 2-12 on one field each) arrive at any time and
// are served by a fixed set of slots, each a host thread with its own
// context and CUDA stream, so that the work of requests in different slots
// overlaps on the device.
//
// Continuous admission: a free slot takes the first admissible request
// among the first `window` pending ones.  A request on a HOST field needs
// its field resident in device memory: the admission policy
// (rd_server_policy.h) admits it when its key is resident (a hit) or when
// the HBM budget, after evicting unpinned resident fields least recently
// used first, has room; the slot then copies the field in
// (stream-ordered allocation, no device-wide synchronisation) and the copy
// stays resident for later requests with the same key.  Requests on DEVICE
// fields use the caller's memory and always fit.  Completions carry the
// result and the queueing and service times; rd_server_get_stats reports
// p50 / p99 latency.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rd_server_policy.h"
#include "rdsel.h"

void rdk_set_graph_capture(rd_context* c, bool on);  // rd_api.cu

namespace {

using Clock = std::chrono::steady_clock;

struct ServerRequest {
  uint64_t id = 0, tag = 0, key = 0;
  rd_field field;
  rd_params params;
  size_t bytes = 0;
  bool host = false;
  Clock::time_point t_submit;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct rd_server {
  explicit rd_server(size_t budget) : policy(budget) {}
  int device = 0;
  int window = 8;
  rdk::AdmissionPolicy policy;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServerRequest> pending;
  std::deque<rd_server_completion> done;
  std::unordered_map<uint64_t, float*> resident;  // key -> device copy
  std::vector<std::thread> workers;
  std::vector<double> latencies;  // ms, completed requests
  uint64_t next_id = 1, submitted = 0, completed = 0, rejected = 0, hits = 0;
  int worker_errors = 0;
  int started = 0, ready = 0;  // workers that reported their start-up, and those ready
  bool stop = false;
};

namespace {

void serve(rd_server* s) {
  cudaSetDevice(s->device);
  rd_context* ctx = nullptr;
  cudaStream_t st = nullptr;
  const bool ready = rd_context_create(s->device, 0, &ctx) == RD_OK &&
                     cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  // a graph capture on a key's second request would land in that request's
  // latency; slots launch directly
  if (ctx) rdk_set_graph_capture(ctx, false);
  std::unique_lock<std::mutex> lk(s->mu);
  s->started++;
  if (ready) s->ready++;
  else s->worker_errors++;
  s->cv_done.notify_all();
  if (!ready) {
    // a slot without a context or stream takes no work: it leaves at once
    lk.unlock();
    if (st) cudaStreamDestroy(st);
    if (ctx) rd_context_destroy(ctx);
    return;
  }
  for (;;) {
    // take the first admissible request of the window
    ServerRequest req;
    rdk::AdmissionPolicy::Decision dec;
    bool taken = false;
    while (!taken) {
      if (s->stop && s->pending.empty()) break;
      const size_t lim = std::min(s->pending.size(), (size_t)s->window);
      for (size_t i = 0; i < lim; i++) {
        const ServerRequest& r = s->pending[i];
        if (r.host) {
          dec = s->policy.admit(r.key, r.bytes);
          if (!dec.admitted) continue;
        } else {
          dec = rdk::AdmissionPolicy::Decision();
          dec.admitted = true;
        }
        req = r;
        s->pending.erase(s->pending.begin() + (long)i);
        taken = true;
        break;
      }
      if (!taken) {
        if (s->stop && s->pending.empty()) break;
        s->cv_work.wait(lk);
      }
    }
    if (!taken) break;
    std::vector<float*> freed;
    for (uint64_t k : dec.evicted) {
      auto it = s->resident.find(k);
      if (it != s->resident.end()) {
        freed.push_back(it->second);
        s->resident.erase(it);
      }
    }
    float* dev = nullptr;
    if (req.host && dec.hit) dev = s->resident[req.key];
    lk.unlock();

    const Clock::time_point t_start = Clock::now();
    for (float* p : freed) cudaFreeAsync(p, st);
    int32_t status = RD_OK;
    bool dropped = false;
    rd_field f = req.field;
    if (req.host) {
      if (!dec.hit) {
        cudaError_t e = cudaMallocAsync((void**)&dev, req.bytes, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(dev, req.field.data, req.bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
          cudaGetLastError();
          status = e == cudaErrorMemoryAllocation ? RD_ERR_OOM : RD_ERR_CUDA;
        }
        lk.lock();
        if (req.key != 0) {
          if (status == RD_OK) {
            s->resident[req.key] = dev;
            s->policy.mark_loaded(req.key);
          } else {
            s->policy.drop(req.key);
            dropped = true;
          }
        }
        lk.unlock();
        s->cv_work.notify_all();
      }
      f.data = dev;
      f.location = RD_LOC_DEVICE;
    }
    rd_server_completion c;
    memset(&c, 0, sizeof(c));
    if (status == RD_OK) status = rd_select(ctx, &f, &req.params, &c.result, st);
    if (req.host && req.key == 0 && dev) {
      cudaFreeAsync(dev, st);
      cudaStreamSynchronize(st);
    }
    const Clock::time_point t_done = Clock::now();
    c.request_id = req.id;
    c.tag = req.tag;
    c.status = status;
    c.resident_hit = dec.hit ? 1 : 0;
    c.queue_ms = ms_between(req.t_submit, t_start);
    c.service_ms = ms_between(t_start, t_done);
    c.latency_ms = ms_between(req.t_submit, t_done);

    lk.lock();
    if (req.host && !dropped) s->policy.release(req.key, req.bytes);
    if (dec.hit) s->hits++;
    s->done.push_back(c);
    s->latencies.push_back(c.latency_ms);
    s->completed++;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  lk.unlock();
  if (st) cudaStreamDestroy(st);
  if (ctx) rd_context_destroy(ctx);
}

}  // namespace

extern "C" {

int32_t rd_server_create(const rd_server_config* cfg, rd_server** out) {
  if (!cfg || !out) return RD_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return RD_ERR_CUDA;
  if (cfg->device < 0 || cfg->device >= ndev) return RD_ERR_INVALID_ARG;
  if (cfg->slots < 1 || cfg->slots > 64 || cfg->window < 1) return RD_ERR_INVALID_ARG;
  rd_server* s = new (std::nothrow) rd_server((size_t)cfg->hbm_budget);
  if (!s) return RD_ERR_OOM;
  s->device = cfg->device;
  s->window = cfg->window;
  for (int i = 0; i < cfg->slots; i++) s->workers.emplace_back(serve, s);
  // wait until every slot has reported whether it could start
  int ready = 0;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->started == cfg->slots; });
    ready = s->ready;
  }
  if (ready == 0) {
    rd_server_destroy(s);
    return RD_ERR_CUDA;
  }
  *out = s;
  return RD_OK;
}

int32_t rd_server_submit(rd_server* s, const rd_field* field, const rd_params* params,
                         uint64_t field_key, uint64_t tag, uint64_t* request_id) {
  if (!s || !field || !params || !field->data) return RD_ERR_INVALID_ARG;
  if (field->ndim < 1 || field->ndim > 3) return RD_ERR_INVALID_ARG;
  if (field->location != RD_LOC_DEVICE && field->location != RD_LOC_HOST) return RD_ERR_INVALID_ARG;
  long long n = 1;
  for (int k = 0; k < field->ndim; k++) {
    if (field->shape[k] < 1 || field->shape[k] > 2147483647LL) return RD_ERR_INVALID_ARG;
    n *= field->shape[k];
    if (n > 2147483647LL) return RD_ERR_INVALID_ARG;
  }
  ServerRequest r;
  r.tag = tag;
  r.key = field_key;
  r.field = *field;
  r.params = *params;
  r.bytes = (size_t)n * sizeof(float);
  r.host = field->location == RD_LOC_HOST;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return RD_ERR_INVALID_ARG;
    if (r.host && !s->policy.fits_at_all(r.bytes)) {
      s->rejected++;
      return RD_ERR_BUDGET;
    }
    r.id = s->next_id++;
    r.t_submit = Clock::now();
    s->pending.push_back(r);
    s->submitted++;
  }
  s->cv_work.notify_one();
  if (request_id) *request_id = r.id;
  return RD_OK;
}

int32_t rd_server_poll(rd_server* s, rd_server_completion* out, int32_t max, int32_t wait_ms,
                       int32_t* n) {
  if (!s || !n || max < 0 || (max > 0 && !out)) return RD_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  int32_t k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  return s->worker_errors ? RD_ERR_CUDA : RD_OK;
}

int32_t rd_server_get_stats(rd_server* s, rd_server_stats* out) {
  if (!s || !out) return RD_ERR_INVALID_ARG;
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->resident_hits = s->hits;
    out->evictions = s->policy.evictions();
    out->resident_fields = s->policy.resident_count();
    out->resident_bytes = s->policy.used();
    out->pending = s->pending.size();
    lat = s->latencies;
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto q = [&](double p) {
      // nearest-rank percentile
      size_t r = (size_t)(p * (double)lat.size() + 0.999999);
      if (r < 1) r = 1;
      if (r > lat.size()) r = lat.size();
      return lat[r - 1];
    };
    double sum = 0.0;
    for (double v : lat) sum += v;
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
    out->mean_ms = sum / (double)lat.size();
    out->max_ms = lat.back();
  }
  return RD_OK;
}

int32_t rd_server_reset_stats(rd_server* s) {
  if (!s) return RD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies.clear();
  return RD_OK;
}

int32_t rd_server_destroy(rd_server* s) {
  if (!s) return RD_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (std::thread& t : s->workers) t.join();
  cudaSetDevice(s->device);
  for (auto& kv : s->resident) cudaFreeAsync(kv.second, 0);
  cudaStreamSynchronize(0);
  delete s;
  return RD_OK;
}

}  // extern "C"

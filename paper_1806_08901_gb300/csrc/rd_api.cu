// rd_api.cu -- host side of the C ABI declared in include/rdsel.h: context
// and workspace, argument checks, the block-sampling lattice, and the launch
// sequence of each entry point.  Every arithmetic step of the path runs in
// the kernels; the host only sizes grids and copies the final record back.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "rd_internal.cuh"

using namespace rdk;

namespace {

const char* kKernelNames[K_COUNT] = {
    "reset", "range", "prepare", "zfp_pass", "delta", "sz_est", "sz_pass",
    "code_prep", "huffman", "finish", "zfp_inspect", "sz_inspect"};

struct KStat {
  double ms;
  long long launches;
};

struct Pending {
  int kid;
  cudaEvent_t a, b;
};

struct HostOut {
  rd_result res;
  rd_truth truth;
  int32_t status;
};

// Everything a call's launch sequence depends on.  Two calls with equal keys
// issue identical work, so the second replays the first one's CUDA graph.
struct CallKey {
  FieldDev f;
  ParamsDev p;
  int passes;
  int delta_mode;
  double delta_arg;
  int profiling;
  int pad;
};

struct GraphEntry {
  CallKey key;
  cudaGraphExec_t exec;
  std::vector<Pending> events;  // per-kernel event pairs recorded inside the graph
  long long kernels;
  unsigned long long last_use;
};

constexpr size_t kMaxGraphs = 16;
constexpr size_t kMaxSeen = 32;

}  // namespace

struct rd_context {
  int device = 0;
  size_t budget = 0;
  size_t held = 0;
  Workspace* ws = nullptr;
  HostOut* out = nullptr;  // pinned
  float* staging = nullptr;
  size_t staging_bytes = 0;
  int num_sms = 0;
  int range_ctas = 0;
  int zfp_ctas[4] = {0, 0, 0, 0};
  int sz_ctas[4] = {0, 0, 0, 0};
  bool profiling = false;
  KStat stats[K_COUNT];
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  long long launches = 0;
  // CUDA graphs of repeated calls
  cudaStream_t cap = nullptr;  // capture stream (the legacy stream cannot capture)
  std::vector<GraphEntry> graphs;
  std::vector<CallKey> seen;
  unsigned long long tick = 0;
  bool capturing = false;
  std::vector<Pending>* sink = nullptr;
  long long cap_kernels = 0;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RD_OK;
  if (e == cudaErrorMemoryAllocation) return RD_ERR_OOM;
  return RD_ERR_CUDA;
}

cudaEvent_t take_event(rd_context* c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch one kernel (through fn), bracketed by timing events when profiling.
// While a graph is being captured the events belong to the graph entry.
template <typename F>
int launch(rd_context* c, int kid, cudaStream_t s, F&& fn) {
  Pending p{kid, nullptr, nullptr};
  // inside a capture an event record must be an external record node (a
  // timestamp on every replay), not an internal dependency marker
  const unsigned rec = c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  if (c->profiling) {
    if (c->capturing) {
      cudaEventCreate(&p.a);
      cudaEventCreate(&p.b);
    } else {
      p.a = take_event(c);
      p.b = take_event(c);
    }
    cudaEventRecordWithFlags(p.a, s, rec);
  }
  cudaError_t e = fn();
  if (c->profiling) {
    cudaEventRecordWithFlags(p.b, s, rec);
    (c->capturing ? *c->sink : c->pending).push_back(p);
  }
  if (c->capturing)
    c->cap_kernels++;
  else
    c->launches++;
  return cuda_status(e);
}

void add_times(rd_context* c, const std::vector<Pending>& evs) {
  for (const Pending& p : evs) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->stats[p.kid].ms += ms;
      c->stats[p.kid].launches += 1;
    } else {
      cudaGetLastError();  // a missing timing is not the caller's error
    }
  }
}

void drop_entry(GraphEntry& g) {
  cudaGraphExecDestroy(g.exec);
  for (const Pending& p : g.events) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
}

void collect_profile(rd_context* c) {
  for (const Pending& p : c->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->stats[p.kid].ms += ms;
      c->stats[p.kid].launches += 1;
    } else {
      cudaGetLastError();
    }
    c->pool.push_back(p.a);
    c->pool.push_back(p.b);
  }
  c->pending.clear();
}

struct CallGuard {
  int prev = -1;
  explicit CallGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
};

int check_params(const rd_params* p) {
  if (!p) return RD_ERR_INVALID_ARG;
  if (!(p->eb > 0.0) || !isfinite(p->eb)) return RD_ERR_INVALID_ARG;
  if (p->eb_mode != RD_EB_REL && p->eb_mode != RD_EB_ABS) return RD_ERR_INVALID_ARG;
  if (p->ec_mode != RD_EC_PAPER && p->ec_mode != RD_EC_ALL) return RD_ERR_INVALID_ARG;
  if (!(p->r_sp >= 1e-6 && p->r_sp <= 1.0)) return RD_ERR_INVALID_ARG;
  if (p->quant_radius < 1 || p->quant_radius > 32768) return RD_ERR_INVALID_ARG;
  if (p->sel_rule != RD_SEL_PAPER && p->sel_rule != RD_SEL_HUFFMAN) return RD_ERR_INVALID_ARG;
  if (!isfinite(p->sz_offset)) return RD_ERR_INVALID_ARG;
  return RD_OK;
}

ParamsDev to_dev(const rd_params* p) {
  ParamsDev d;
  d.eb = p->eb;
  d.eb_mode = p->eb_mode;
  d.ec_mode = p->ec_mode;
  d.R = p->quant_radius;
  d.sel_rule = p->sel_rule;
  d.sz_offset = p->sz_offset;
  return d;
}

// Block sampling lattice (Section "Data Sampling"): S = round(1/r_sp) is
// factored into primes; each prime, largest first, multiplies the stride of
// the axis with the smallest stride so far (ties: the faster axis).
void sampling_strides(int d, double r_sp, int* s) {
  long long S = (long long)floor(1.0 / r_sp + 0.5);
  if (S < 1) S = 1;
  long long f[64];
  int nf = 0;
  long long m = S;
  for (long long q = 2; q * q <= m; q++)
    while (m % q == 0) {
      f[nf++] = q;
      m /= q;
    }
  if (m > 1) f[nf++] = m;
  for (int k = 0; k < 3; k++) s[k] = 1;
  for (int i = nf - 1; i >= 0; i--) {
    int a = d - 1;
    for (int k = d - 2; k >= 0; k--)
      if (s[k] < s[a]) a = k;
    s[a] = (int)(s[a] * f[i]);
  }
}

struct Geometry {
  FieldDev f;
  unsigned long long npoints_sampled;  // valid points of sampled blocks
  int partial;
};

int make_geometry(rd_context* c, const rd_field* fld, const int* strides_or_null, double r_sp,
                  cudaStream_t s, Geometry* g) {
  if (!fld || fld->ndim < 1 || fld->ndim > 3 || !fld->data) return RD_ERR_INVALID_ARG;
  if (fld->location != RD_LOC_DEVICE && fld->location != RD_LOC_HOST) return RD_ERR_INVALID_ARG;
  FieldDev& f = g->f;
  memset(&f, 0, sizeof(f));
  f.d = fld->ndim;
  long long N = 1;
  for (int k = 0; k < 3; k++) f.n[k] = 1;
  for (int k = 0; k < f.d; k++) {
    if (fld->shape[k] < 1 || fld->shape[k] > 2147483647LL) return RD_ERR_INVALID_ARG;
    f.n[k] = (int)fld->shape[k];
    N *= fld->shape[k];
    if (N > 2147483647LL) return RD_ERR_INVALID_ARG;
  }
  f.N = N;
  const float* x = fld->data;
  if (fld->location == RD_LOC_HOST) {
    size_t bytes = (size_t)N * sizeof(float);
    if (bytes > c->staging_bytes) {
      size_t grow = bytes - c->staging_bytes;
      if (c->budget && c->held + grow > c->budget) return RD_ERR_BUDGET;
      if (c->staging) cudaFree(c->staging);
      c->held -= c->staging_bytes;
      c->staging = nullptr;
      c->staging_bytes = 0;
      if (cudaMalloc(&c->staging, bytes) != cudaSuccess) return RD_ERR_OOM;
      c->staging_bytes = bytes;
      c->held += bytes;
    }
    cudaError_t e = cudaMemcpyAsync(c->staging, x, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return RD_ERR_CUDA;
    x = c->staging;
  }
  f.x = x;
  f.vec_ok = (((uintptr_t)x & 15u) == 0) && (f.n[f.d - 1] % 4 == 0);
  int st[3] = {1, 1, 1};
  if (strides_or_null) {
    for (int k = 0; k < f.d; k++) {
      if (strides_or_null[k] < 1) return RD_ERR_INVALID_ARG;
      st[k] = strides_or_null[k];
    }
  } else {
    sampling_strides(f.d, r_sp, st);
  }
  f.nblocks = 1;
  f.nsampled = 1;
  g->npoints_sampled = 1;
  g->partial = 0;
  for (int k = 0; k < f.d; k++) {
    f.B[k] = (f.n[k] + 3) / 4;
    f.s[k] = st[k];
    f.L[k] = (f.B[k] + st[k] - 1) / st[k];
    f.nblocks *= f.B[k];
    f.nsampled *= f.L[k];
    unsigned long long pts = 0;
    for (int b = 0; b < f.B[k]; b += st[k]) pts += (unsigned long long)(f.n[k] - 4 * b < 4 ? f.n[k] - 4 * b : 4);
    g->npoints_sampled *= pts;
    if (f.n[k] % 4) g->partial = 1;
  }
  return RD_OK;
}

int ec_count(int d, int ec_mode) {
  if (ec_mode == RD_EC_ALL) return 1 << (2 * d);
  return d == 1 ? 3 : d == 2 ? 9 : 16;
}

// Issue the launch sequence of one call and the copy of its result records
// into pinned host memory, on stream s (which may be capturing).
int issue(rd_context* c, const CallKey& k, const Geometry& g, cudaStream_t s) {
  const FieldDev& f = k.f;
  const ParamsDev& p = k.p;
  const int passes = k.passes;
  const int delta_mode = k.delta_mode;
  const double delta_arg = k.delta_arg;
  Workspace* ws = c->ws;
  const int d = f.d;
  const bool need_gt = passes & P_SZ_GT;
  const bool need_quant = passes & (P_SZ_EST | P_SZ_GT);
  const unsigned long long ncoeff = (unsigned long long)f.nsampled * ec_count(d, p.ec_mode);
  int zfp_parts = 0, sz_parts = 0;
  int rc;

  if ((rc = launch(c, K_RESET, s, [&] { return launch_reset(ws, s); }))) return rc;
  if ((rc = launch(c, K_RANGE, s, [&] { return launch_range(f, ws, c->range_ctas, s); }))) return rc;
  if ((rc = launch(c, K_PREPARE, s, [&] { return launch_prepare(p, ws, s); }))) return rc;
  if (passes & (P_ZFP_EST | P_ZFP_GT)) {
    int zp = passes & (P_ZFP_EST | P_ZFP_GT);
    if ((rc = launch(c, K_ZFP, s, [&] { return launch_zfp(f, p, zp, ws, c->zfp_ctas[d], s, &zfp_parts); })))
      return rc;
  }
  if (need_quant || (passes & P_ZFP_EST)) {
    if ((rc = launch(c, K_DELTA, s, [&] {
           return launch_delta(p, ws, delta_mode, delta_arg, need_quant ? 1 : 0, need_gt ? 1 : 0,
                               ncoeff, g.npoints_sampled, s);
         })))
      return rc;
  }
  if (passes & P_SZ_GT) {
    int with_est = (passes & P_SZ_EST) ? 1 : 0;
    if ((rc = launch(c, K_SZ_GT, s, [&] {
           if (sz_march_supported(f))
             return launch_sz_march(f, p, with_est, ws, c->num_sms, s, &sz_parts);
           return launch_sz_gt(f, p, with_est, ws, c->sz_ctas[d], s, &sz_parts);
         })))
      return rc;
  } else if (passes & P_SZ_EST) {
    if ((rc = launch(c, K_SZ_EST, s, [&] { return launch_sz_est(f, p, ws, c->sz_ctas[d], s); })))
      return rc;
  }
  int hist_mask = ((passes & P_SZ_EST) ? 1 : 0) | ((passes & P_SZ_GT) ? 2 : 0);
  if (hist_mask) {
    if ((rc = launch(c, K_CODE_PREP, s, [&] { return launch_code_prep(ws, hist_mask, s); }))) return rc;
    if ((rc = launch(c, K_HUFFMAN, s, [&] { return launch_huffman(ws, hist_mask, s); }))) return rc;
  }
  if ((rc = launch(c, K_FINISH, s, [&] {
         return launch_finish(p, ws, passes, zfp_parts, sz_parts, f.N, g.npoints_sampled, s);
       })))
    return rc;
  // one copy of the result records and the device status
  cudaError_t e = cudaMemcpyAsync(&c->out->res, &ws->res, sizeof(rd_result), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&c->out->truth, &ws->truth, sizeof(rd_truth), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&c->out->status, &ws->sc.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  return cuda_status(e);
}

GraphEntry* find_graph(rd_context* c, const CallKey& k) {
  for (GraphEntry& g : c->graphs)
    if (memcmp(&g.key, &k, sizeof(CallKey)) == 0) return &g;
  return nullptr;
}

// Capture the call's launch sequence into a graph (on the context's capture
// stream) and cache it; evicts the least recently used graph when full.
GraphEntry* capture_graph(rd_context* c, const CallKey& k, const Geometry& g) {
  if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
  GraphEntry ent;
  ent.key = k;
  ent.exec = nullptr;
  ent.kernels = 0;
  ent.last_use = 0;
  if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return nullptr;
  c->capturing = true;
  c->sink = &ent.events;
  c->cap_kernels = 0;
  int rc = issue(c, k, g, c->cap);
  c->capturing = false;
  c->sink = nullptr;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap, &graph);
  if (rc == RD_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ent.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (rc != RD_OK || e != cudaSuccess || !ent.exec) {
    cudaGetLastError();
    for (const Pending& p : ent.events) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    return nullptr;
  }
  ent.kernels = c->cap_kernels;
  if (c->graphs.size() >= kMaxGraphs) {
    size_t lru = 0;
    for (size_t i = 1; i < c->graphs.size(); i++)
      if (c->graphs[i].last_use < c->graphs[lru].last_use) lru = i;
    drop_entry(c->graphs[lru]);
    c->graphs.erase(c->graphs.begin() + lru);
  }
  c->graphs.push_back(ent);
  return &c->graphs.back();
}

// Run the passes of one call; est/truth may be NULL.  The first call with a
// given key launches directly; a repeat is captured once into a CUDA graph
// and every later repeat replays it with a single launch.
int run(rd_context* c, const rd_field* fld, const rd_params* prm, int passes, int delta_mode,
        double delta_arg, rd_result* est, rd_truth* truth, void* stream) {
  if (!c) return RD_ERR_INVALID_ARG;
  int rc = check_params(prm);
  if (rc) return rc;
  CallGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  Geometry g;
  rc = make_geometry(c, fld, nullptr, prm->r_sp, s, &g);
  if (rc) return rc;
  CallKey k;
  memset(&k, 0, sizeof(k));
  k.f = g.f;
  k.p = to_dev(prm);
  k.passes = passes;
  k.delta_mode = delta_mode;
  k.delta_arg = delta_arg;
  k.profiling = c->profiling ? 1 : 0;
  const FieldDev& f = g.f;
  const int d = f.d;
  const unsigned long long ncoeff = (unsigned long long)f.nsampled * ec_count(d, prm->ec_mode);

  GraphEntry* ent = find_graph(c, k);
  if (!ent) {
    bool repeat = false;
    for (const CallKey& q : c->seen)
      if (memcmp(&q, &k, sizeof(CallKey)) == 0) repeat = true;
    if (repeat) {
      ent = capture_graph(c, k, g);
    } else {
      if (c->seen.size() >= kMaxSeen) c->seen.erase(c->seen.begin());
      c->seen.push_back(k);
    }
  }
  cudaError_t e;
  if (ent) {
    ent->last_use = ++c->tick;
    e = cudaGraphLaunch(ent->exec, s);
    c->launches += ent->kernels;
    rc = cuda_status(e);
  } else {
    rc = issue(c, k, g, s);
  }
  e = cudaStreamSynchronize(s);
  if (c->profiling) {
    if (ent)
      add_times(c, ent->events);
    else
      collect_profile(c);
  }
  if (rc != RD_OK) return rc;
  if (e != cudaSuccess) return cuda_status(e);
  int status = c->out->status;
  if (status != RD_OK) {
    if (est) memset(est, 0, sizeof(*est));
    if (truth) memset(truth, 0, sizeof(*truth));
    return status;
  }
  rd_result r = c->out->res;
  rd_truth t = c->out->truth;
  for (int k = 0; k < d; k++) r.strides[k] = f.s[k];
  for (int k = d; k < 3; k++) r.strides[k] = 0;
  r.n_blocks = (uint64_t)f.nblocks;
  if (!(r.flags & RD_F_CONSTANT)) {
    r.n_sampled_blocks = (uint64_t)f.nsampled;
    r.r_sp_eff = (double)f.nsampled / (double)f.nblocks;
    r.zfp_npoints = g.npoints_sampled;
    if (passes & P_ZFP_EST) r.zfp_ncoeff = ncoeff;
  }
  if (g.partial) r.flags |= RD_F_PARTIAL_BLOCKS;
  if (est) *est = r;
  if (truth) *truth = t;
  return RD_OK;
}

}  // namespace

extern "C" {

int32_t rd_context_create(int32_t device, size_t hbm_budget, rd_context** out) {
  if (!out) return RD_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) return RD_ERR_CUDA;
  if (device < 0 || device >= ndev) return RD_ERR_INVALID_ARG;
  if (hbm_budget && hbm_budget < sizeof(Workspace)) return RD_ERR_BUDGET;
  CallGuard guard(device);
  rd_context* c = new (std::nothrow) rd_context();
  if (!c) return RD_ERR_OOM;
  c->device = device;
  c->budget = hbm_budget;
  for (int i = 0; i < K_COUNT; i++) c->stats[i] = KStat{0.0, 0};
  if (cudaMalloc(&c->ws, sizeof(Workspace)) != cudaSuccess) {
    delete c;
    return RD_ERR_OOM;
  }
  c->held = sizeof(Workspace);
  if (cudaMallocHost(&c->out, sizeof(HostOut)) != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return RD_ERR_OOM;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (prepare_code_stats() != cudaSuccess || prepare_sz_march() != cudaSuccess ||
      launch_init_tables(c->ws, 0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) {
    cudaFreeHost(c->out);
    cudaFree(c->ws);
    delete c;
    return RD_ERR_CUDA;
  }
  c->range_ctas = c->num_sms * 4;
  for (int d = 1; d <= 3; d++) {
    c->zfp_ctas[d] = zfp_occupancy(d, c->num_sms);
    c->sz_ctas[d] = sz_occupancy(d, c->num_sms);
  }
  *out = c;
  return RD_OK;
}

int32_t rd_context_destroy(rd_context* c) {
  if (!c) return RD_ERR_INVALID_ARG;
  CallGuard guard(c->device);
  cudaDeviceSynchronize();
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  for (const Pending& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (GraphEntry& g : c->graphs) drop_entry(g);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->staging) cudaFree(c->staging);
  if (c->ws) cudaFree(c->ws);
  if (c->out) cudaFreeHost(c->out);
  delete c;
  return RD_OK;
}

int32_t rd_estimate_zfp(rd_context* c, const rd_field* f, const rd_params* p, rd_result* out,
                        void* stream) {
  if (!out) return RD_ERR_INVALID_ARG;
  return run(c, f, p, P_ZFP_EST, DELTA_FROM_MSE, 0.0, out, nullptr, stream);
}

int32_t rd_estimate_sz(rd_context* c, const rd_field* f, const rd_params* p, double delta,
                       rd_result* out, void* stream) {
  if (!out || isnan(delta)) return RD_ERR_INVALID_ARG;
  return run(c, f, p, P_SZ_EST, DELTA_EXPLICIT, delta, out, nullptr, stream);
}

int32_t rd_select(rd_context* c, const rd_field* f, const rd_params* p, rd_result* out,
                  void* stream) {
  if (!out) return RD_ERR_INVALID_ARG;
  return run(c, f, p, P_ZFP_EST | P_SZ_EST, DELTA_FROM_MSE, 0.0, out, nullptr, stream);
}

int32_t rd_ground_truth(rd_context* c, const rd_field* f, const rd_params* p, double eb_sz,
                        rd_truth* out, void* stream) {
  if (!out || isnan(eb_sz)) return RD_ERR_INVALID_ARG;
  if (eb_sz > 0.0)
    return run(c, f, p, P_ZFP_GT | P_SZ_GT, DELTA_FROM_EB_SZ, eb_sz, nullptr, out, stream);
  return run(c, f, p, P_ZFP_GT | P_ZFP_EST | P_SZ_GT, DELTA_FROM_MSE, 0.0, nullptr, out, stream);
}

int32_t rd_evaluate(rd_context* c, const rd_field* f, const rd_params* p, rd_result* est,
                    rd_truth* truth, void* stream) {
  return run(c, f, p, P_ZFP_EST | P_ZFP_GT | P_SZ_EST | P_SZ_GT, DELTA_FROM_MSE, 0.0, est, truth,
             stream);
}

int32_t rd_copy_histograms(rd_context* c, uint32_t* est_hist, uint32_t* gt_hist) {
  if (!c) return RD_ERR_INVALID_ARG;
  CallGuard guard(c->device);
  cudaError_t e = cudaSuccess;
  if (est_hist) e = cudaMemcpy(est_hist, c->ws->hist[0], sizeof(uint32_t) * kNsym, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && gt_hist)
    e = cudaMemcpy(gt_hist, c->ws->hist[1], sizeof(uint32_t) * kNsym, cudaMemcpyDeviceToHost);
  return cuda_status(e);
}

int32_t rd_zfp_blocks(rd_context* c, const rd_field* fld, double eb_abs, int32_t* emax,
                      int32_t* prec, uint64_t* bits, uint32_t* coeffs, void* stream) {
  if (!c || !(eb_abs > 0.0) || !isfinite(eb_abs)) return RD_ERR_INVALID_ARG;
  CallGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  Geometry g;
  int rc = make_geometry(c, fld, nullptr, 1.0, s, &g);
  if (rc) return rc;
  rc = launch(c, K_ZFP_INSPECT, s, [&] {
    return launch_zfp_inspect(g.f, eb_abs, emax, prec, bits, coeffs, s);
  });
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(s);
  if (c->profiling) collect_profile(c);
  return cuda_status(e);
}

int32_t rd_sz_symbols(rd_context* c, const rd_field* fld, double delta, int32_t quant_radius,
                      const int32_t* strides, int32_t* est_sym, int32_t* gt_sym, float* recon,
                      void* stream) {
  if (!c || !(delta > 0.0) || !isfinite(delta)) return RD_ERR_INVALID_ARG;
  if (quant_radius < 1 || quant_radius > 32768) return RD_ERR_INVALID_ARG;
  CallGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  Geometry g;
  int rc = make_geometry(c, fld, strides, 1.0, s, &g);
  if (rc) return rc;
  // the same float quantiser as the passes: w, 1/w and the escape threshold
  // tau = the largest float not above (delta/2)(1 - 2^-23)
  float w = (float)delta;
  if (!(w >= 1.17549435e-38f) || isinf(w)) return RD_ERR_RANGE;
  volatile float one = 1.0f;
  float inv = one / w;
  if (isinf(inv) || !(inv >= 1.17549435e-38f)) return RD_ERR_RANGE;
  double t = (delta / 2.0) * (1.0 - 1.1920928955078125e-07);
  float tau = (float)t;
  if ((double)tau > t) tau = nextafterf(tau, 0.0f);
  rc = launch(c, K_SZ_INSPECT, s, [&] {
    return launch_sz_inspect_q(g.f, w, inv, tau, quant_radius, est_sym, gt_sym, recon,
                               strides != nullptr, s);
  });
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(s);
  if (c->profiling) collect_profile(c);
  return cuda_status(e);
}

int32_t rd_set_profiling(rd_context* c, int32_t on) {
  if (!c) return RD_ERR_INVALID_ARG;
  c->profiling = on != 0;
  return RD_OK;
}

int32_t rd_reset_profile(rd_context* c) {
  if (!c) return RD_ERR_INVALID_ARG;
  for (int i = 0; i < K_COUNT; i++) c->stats[i] = KStat{0.0, 0};
  return RD_OK;
}

int32_t rd_kernel_stat(rd_context* c, int32_t i, const char** name, double* total_ms,
                       int64_t* launches) {
  if (!c || i < 0 || i >= K_COUNT) return RD_ERR_INVALID_ARG;
  if (name) *name = kKernelNames[i];
  if (total_ms) *total_ms = c->stats[i].ms;
  if (launches) *launches = c->stats[i].launches;
  return RD_OK;
}

int64_t rd_launch_count(rd_context* c) { return c ? c->launches : -1; }

const char* rd_status_string(int32_t status) {
  switch (status) {
    case RD_OK: return "ok";
    case RD_ERR_INVALID_ARG: return "invalid argument";
    case RD_ERR_NONFINITE: return "field holds NaN or infinity";
    case RD_ERR_OOM: return "out of memory";
    case RD_ERR_BUDGET: return "HBM budget exceeded";
    case RD_ERR_CUDA: return "CUDA runtime error";
    case RD_ERR_TIMEOUT: return "bounded device wait ran out";
    case RD_ERR_RANGE: return "bin width not representable or codes would overflow";
    default: return "unknown status";
  }
}

}  // extern "C"

// rd_api.cu -- host side of the C ABI declared in include/rdsel.h: context
// and workspace, argument checks, the block-sampling lattice, and the launch
// sequence of each entry point.  Every arithmetic step of the path runs in
// the kernels; the host only sizes grids and copies the final record back.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <new>
#include <utility>
#include <vector>

#include "rd_internal.cuh"
#include "rd_sz_stream.cuh"
#include "rdsel_stream.h"

using namespace rdk;

namespace {

const char* kKernelNames[K_COUNT] = {
    "reset", "range", "zfp_pass", "delta", "sz_est", "sz_pass",
    "code_prep", "huffman", "finish", "zfp_inspect", "sz_inspect",
    "batch_reset", "batch_range", "batch_blocks", "batch_sz_hist", "batch_code_prep",
    "batch_final", "batch_truth", "sz_classic", "sz_classic_err", "sz_log", "zfp_est"};

struct KStat {
  double ms;
  long long launches;
};

struct Pending {
  int kid;
  cudaEvent_t a, b;
};

using HostOut = OutRecords;

// What the log-scale estimate reads back: the range pass's scalars, the
// largest residual, and at the end the record.
struct LogHost {
  int32_t status, constant;
  uint32_t maxabs_bits, flags;
  double vr, eb_abs;
  rd_log_result res;
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
  const void* aux;  // the reconstruction buffer of a classic SZ truth, else NULL
  const float* host_src;  // a pinned host field the range pass stages, else NULL
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

using Geometry = FieldGeom;

// A batch of fields as planned once: device tables of fields and work items
// for one work split, and the CUDA graph of its launches once captured.
struct BatchPlan {
  std::vector<unsigned char> key;  // n, truth flag, split mode, fields and parameters
  int n = 0;
  int need_gt = 0;
  rd_batch_config cfg;
  std::vector<BatchField> hbf;
  std::vector<Geometry> geo;
  BatchField* dbf = nullptr;
  // range items, sampled-block items (grouped by dimensionality), SZ items
  BatchItem* ditems = nullptr;
  float* dres = nullptr;        // SZ residual keys of every field's sampled blocks
  size_t res_bytes = 0;
  int n_range = 0, n_blk = 0, n_sz = 0;
  int blk_first[4] = {0, 0, 0, 0};  // sampled-block items of d-dimensional fields: [blk_first[d-1], blk_first[d])

  cudaGraphExec_t exec = nullptr;
  std::vector<Pending> events;
  long long kernels = 0;
  int uses = 0;
  unsigned long long last_use = 0;
};

constexpr size_t kMaxPlans = 8;

// Candidate work splits of the autotuner (small, middle, large).
constexpr long long kRangeValues[3] = {1ll << 16, 1ll << 18, 1ll << 20};
constexpr int kZfpBlocks[3] = {256, 1024, 4096};
constexpr int kSzBlocks[3] = {256, 1024, 4096};

}  // namespace

struct rd_context {
  int device = 0;
  size_t budget = 0;
  size_t held = 0;
  Workspace* ws = nullptr;
  double* xlogx = nullptr;  // v log2 v table of the entropy sums
  HostOut* out = nullptr;      // pinned
  HostOut* out_dev = nullptr;  // the same memory as the device addresses it
  float* staging = nullptr;
  size_t staging_bytes = 0;
  float* xhat = nullptr;  // reconstruction of the classic SZ truth
  size_t xhat_bytes = 0;
  void* enc = nullptr;  // SZ stream encoder: symbols, code table, per-CTA offsets
  size_t enc_bytes = 0;
  // log-scale estimate: float64 edges A[0..n], float edges F[0..n-2], record
  double* log_a = nullptr;
  float* log_f = nullptr;
  rd_log_result* log_dev = nullptr;
  LogHost* log_host = nullptr;  // pinned
  int num_sms = 0;
  int range_ctas = 0;
  int zfp_ctas[4] = {0, 0, 0, 0};
  int sz_ctas[4] = {0, 0, 0, 0};
  int sz_est_ctas[4] = {0, 0, 0, 0};
  int b_range_ctas = 0, b_sz_ctas = 0;                   // resident CTAs of the batched passes
  int b_blocks_ctas[3] = {0, 0, 0};                       // sampled-blocks pass, per dimensionality
  bool profiling = false;
  KStat stats[K_COUNT];
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  long long launches = 0;
  // CUDA graphs of repeated calls
  cudaStream_t cap = nullptr;  // capture stream (the legacy stream cannot capture)
  bool capture_repeats = true;  // capture repeated calls into CUDA graphs
  std::vector<GraphEntry> graphs;
  std::vector<CallKey> seen;
  unsigned long long tick = 0;
  bool capturing = false;
  std::vector<Pending>* sink = nullptr;
  long long cap_kernels = 0;
  // batches: one workspace per field, gathered records, cached plans
  Workspace* bws = nullptr;
  int bws_n = 0;
  rd_result* d_bres = nullptr;
  rd_truth* d_btruth = nullptr;
  int32_t* d_bstatus = nullptr;
  rd_result* h_bres = nullptr;  // pinned
  rd_truth* h_btruth = nullptr;
  int32_t* h_bstatus = nullptr;
  std::vector<BatchPlan*> plans;
  bool batch_forced = false;
  rd_batch_config batch_force;
  rd_batch_config batch_last;
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

// Kernels launched by one launch() call beyond the first.
void count_extra(rd_context* c, long long n) {
  if (c->capturing)
    c->cap_kernels += n;
  else
    c->launches += n;
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

// A host field is staged into the context's buffer: by a copy, or, with
// stage_src given and the field in pinned host memory (16-byte aligned), by
// the range pass itself (*stage_src = the device's address of the field).
int make_geometry(rd_context* c, const rd_field* fld, const int* strides_or_null, double r_sp,
                  cudaStream_t s, Geometry* g, const float** stage_src = nullptr) {
  if (stage_src) *stage_src = nullptr;
  if (!fld || !fld->data) return RD_ERR_INVALID_ARG;
  if (fld->location != RD_LOC_DEVICE && fld->location != RD_LOC_HOST) return RD_ERR_INVALID_ARG;
  int rc = field_geometry(fld, fld->data, strides_or_null, r_sp, g);
  if (rc) return rc;
  if (fld->location == RD_LOC_HOST) {
    size_t bytes = (size_t)g->f.N * sizeof(float);
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
    cudaPointerAttributes at;
    const bool pinned = cudaPointerGetAttributes(&at, fld->data) == cudaSuccess &&
                        at.type == cudaMemoryTypeHost && at.devicePointer != nullptr &&
                        ((uintptr_t)at.devicePointer & 15u) == 0;
    cudaGetLastError();
    if (stage_src && pinned) {
      *stage_src = static_cast<const float*>(at.devicePointer);
    } else {
      cudaError_t e = cudaMemcpyAsync(c->staging, fld->data, bytes, cudaMemcpyHostToDevice, s);
      if (e != cudaSuccess) return RD_ERR_CUDA;
    }
    // the device copy: the same geometry at the staging buffer's address
    rc = field_geometry(fld, c->staging, strides_or_null, r_sp, g);
    if (rc) return rc;
  }
  return RD_OK;
}

// The evaluate step of a 3D field (both estimates and both truths): the
// truth's ZFP pass needs nothing the SZ side computes, so the ZFP estimate
// runs first (for delta), then the SZ pass, the code prep and the Huffman
// launch, and the truth's ZFP pass is launched as the Huffman launch's
// programmatic dependent: it starts once the Huffman CTAs run (they take two
// SMs; the pass is sized to the rest) and its last CTA, after the Huffman
// launch has completed, finishes the ZFP truth and writes the records.
int issue_overlapped(rd_context* c, const CallKey& k, const Geometry& g, cudaStream_t s) {
  const FieldDev& f = k.f;
  const ParamsDev& p = k.p;
  const int passes = k.passes;
  Workspace* ws = c->ws;
  const int d = f.d;
  const unsigned long long ncoeff = (unsigned long long)f.nsampled * ec_count(d, p.ec_mode);
  int zfp_parts = 0, sz_parts = 0, est_parts = 0;
  int rc;
  if ((rc = launch(c, K_RESET, s, [&] { return launch_reset(ws, s); }))) return rc;
  if ((rc = launch(c, K_RANGE, s, [&] { return launch_range(f, p, ws, c->range_ctas, s, k.host_src); })))
    return rc;
  const DeltaArgs da{1, k.delta_mode, k.delta_arg, 1, 1, ncoeff, g.npoints_sampled};
  if ((rc = launch(c, K_ZFP_EST, s, [&] {
         return launch_zfp(f, p, P_ZFP_EST, da, ws, c->zfp_ctas[d], s, &est_parts);
       })))
    return rc;
  if ((rc = launch(c, K_SZ_GT, s, [&] {
         if (sz_march_supported(f)) return launch_sz_march(f, p, 1, ws, c->num_sms, s, &sz_parts);
         return launch_sz_gt(f, p, 1, ws, c->sz_ctas[d], s, &sz_parts);
       })))
    return rc;
  if ((rc = launch(c, K_CODE_PREP, s, [&] { return launch_code_prep(ws, 3, c->xlogx, s); }))) return rc;
  const FinishArgs fa{p, passes, 0, sz_parts, f.N, g.npoints_sampled, c->out_dev, 1};
  if ((rc = launch(c, K_HUFFMAN, s, [&] { return launch_huffman_finish(ws, 3, fa, s); }))) return rc;
  const int per = c->zfp_ctas[d] / (c->num_sms > 0 ? c->num_sms : 1);
  const int zctas = per > 0 && c->num_sms > 4 ? per * (c->num_sms - 2) : c->zfp_ctas[d];
  return launch(c, K_ZFP, s, [&] { return launch_zfp3_after_huffman(f, p, ws, zctas, fa, s, &zfp_parts); });
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
  const bool classic = passes & P_SZ_CLASSIC;
  const bool need_quant = passes & (P_SZ_EST | P_SZ_GT | P_SZ_CLASSIC);
  const unsigned long long ncoeff = (unsigned long long)f.nsampled * ec_count(d, p.ec_mode);
  int zfp_parts = 0, sz_parts = 0;
  int rc;

  // the evaluate step of a 3D field: the truth's ZFP pass beside the Huffman launch
  if (d == 3 && (passes & P_ZFP_EST) && (passes & P_ZFP_GT) && (passes & P_SZ_GT) && (passes & P_SZ_EST) &&
      !classic)
    return issue_overlapped(c, k, g, s);
  if ((rc = launch(c, K_RESET, s, [&] { return launch_reset(ws, s); }))) return rc;
  if ((rc = launch(c, K_RANGE, s, [&] { return launch_range(f, p, ws, c->range_ctas, s, k.host_src); })))
    return rc;
  // delta: by the last CTA of the ZFP pass when there is one, else its own launch
  const bool need_delta = need_quant || (passes & P_ZFP_EST);
  const DeltaArgs da{need_delta ? 1 : 0, delta_mode, delta_arg, need_quant ? 1 : 0, need_gt ? 1 : 0,
                     ncoeff, g.npoints_sampled};
  const bool zfp = passes & (P_ZFP_EST | P_ZFP_GT);
  if (zfp) {
    int zp = passes & (P_ZFP_EST | P_ZFP_GT);
    if ((rc = launch(c, K_ZFP, s, [&] { return launch_zfp(f, p, zp, da, ws, c->zfp_ctas[d], s, &zfp_parts); })))
      return rc;
  }
  if (need_delta && !zfp) {
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
    if ((rc = launch(c, K_SZ_EST, s, [&] { return launch_sz_est(f, p, ws, c->sz_est_ctas[d], s); })))
      return rc;
  }
  if (classic) {
    // the classic truth shares the truth histogram and the SSE partials
    float* xh = static_cast<float*>(const_cast<void*>(k.aux));
    if ((rc = launch(c, K_SZ_CLASSIC, s, [&] { return launch_classic_waves(f, p, xh, ws, s); })))
      return rc;
    count_extra(c, classic_launches(f) - 1);
    if ((rc = launch(c, K_SZ_CLASSIC_ERR, s, [&] {
           return launch_classic_err(f, xh, ws, c->num_sms * 8, s, &sz_parts);
         })))
      return rc;
  }
  int hist_mask = ((passes & P_SZ_EST) ? 1 : 0) | ((passes & (P_SZ_GT | P_SZ_CLASSIC)) ? 2 : 0);
  const int fin_passes = classic ? (passes | P_SZ_GT) : passes;
  // the finish step writes the records and the status into the pinned host
  // block itself (no copy nodes after it); with histograms it is fused into
  // the Huffman launch, run by the CTA that ends last
  const FinishArgs fa{p, fin_passes, zfp_parts, sz_parts, f.N, g.npoints_sampled, c->out_dev};
  if (hist_mask) {
    if ((rc = launch(c, K_CODE_PREP, s, [&] { return launch_code_prep(ws, hist_mask, c->xlogx, s); }))) return rc;
    if ((rc = launch(c, K_HUFFMAN, s, [&] { return launch_huffman_finish(ws, hist_mask, fa, s); })))
      return rc;
  } else if ((rc = launch(c, K_FINISH, s, [&] {
                return launch_finish(p, ws, fin_passes, zfp_parts, sz_parts, f.N, g.npoints_sampled,
                                     c->out_dev, s);
              }))) {
    return rc;
  }
  return RD_OK;
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
  const float* stage_src = nullptr;
  rc = make_geometry(c, fld, nullptr, prm->r_sp, s, &g, &stage_src);
  if (rc) return rc;
  CallKey k;
  memset(&k, 0, sizeof(k));
  k.f = g.f;
  k.host_src = stage_src;
  k.p = params_dev(prm);
  k.passes = passes;
  k.delta_mode = delta_mode;
  k.delta_arg = delta_arg;
  k.profiling = c->profiling ? 1 : 0;
  if (passes & P_SZ_CLASSIC) {
    // the reconstruction buffer, grown to the field
    const size_t bytes = (size_t)g.f.N * sizeof(float);
    if (bytes > c->xhat_bytes) {
      if (c->budget && c->held + (bytes - c->xhat_bytes) > c->budget) return RD_ERR_BUDGET;
      if (c->xhat) cudaFree(c->xhat);
      c->held -= c->xhat_bytes;
      c->xhat = nullptr;
      c->xhat_bytes = 0;
      if (cudaMalloc(&c->xhat, bytes) != cudaSuccess) return RD_ERR_OOM;
      c->xhat_bytes = bytes;
      c->held += bytes;
    }
    k.aux = c->xhat;
  }
  const FieldDev& f = g.f;
  const int d = f.d;
  const unsigned long long ncoeff = (unsigned long long)f.nsampled * ec_count(d, prm->ec_mode);

  GraphEntry* ent = find_graph(c, k);
  if (!ent) {
    bool repeat = false;
    for (const CallKey& q : c->seen)
      if (memcmp(&q, &k, sizeof(CallKey)) == 0) repeat = true;
    if (repeat && c->capture_repeats) {
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
  record_geometry(&r, g, (passes & P_ZFP_EST) != 0, prm->ec_mode);
  if (est) *est = r;
  if (truth) *truth = t;
  return RD_OK;
}

// ---------------------------------------------------------------------------
// Batches (rd_select_batch)
// ---------------------------------------------------------------------------
void free_plan(BatchPlan* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (const Pending& p : b->events) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  if (b->dbf) cudaFree(b->dbf);
  if (b->ditems) cudaFree(b->ditems);
  if (b->dres) cudaFree(b->dres);
  delete b;
}

void drop_plans(rd_context* c) {
  for (BatchPlan* b : c->plans) {
    c->held -= b->res_bytes;
    free_plan(b);
  }
  c->plans.clear();
}

void free_batch_buffers(rd_context* c) {
  drop_plans(c);
  if (c->bws) cudaFree(c->bws);
  if (c->d_bres) cudaFree(c->d_bres);
  if (c->d_btruth) cudaFree(c->d_btruth);
  if (c->d_bstatus) cudaFree(c->d_bstatus);
  if (c->h_bres) cudaFreeHost(c->h_bres);
  if (c->h_btruth) cudaFreeHost(c->h_btruth);
  if (c->h_bstatus) cudaFreeHost(c->h_bstatus);
  c->bws = nullptr;
  c->d_bres = nullptr;
  c->d_btruth = nullptr;
  c->d_bstatus = nullptr;
  c->h_bres = nullptr;
  c->h_btruth = nullptr;
  c->h_bstatus = nullptr;
}

size_t batch_device_bytes(int n) {
  return (size_t)n * (sizeof(Workspace) + sizeof(rd_result) + sizeof(rd_truth) + sizeof(int32_t));
}

// One workspace per field and the gathered records, grown to n fields (the
// cached plans point into them, so growing drops the plans).
int ensure_batch_capacity(rd_context* c, int n) {
  if (c->bws_n >= n) return RD_OK;
  const size_t old = c->bws_n ? batch_device_bytes(c->bws_n) : 0;
  free_batch_buffers(c);
  c->held -= old;
  c->bws_n = 0;
  const size_t bytes = batch_device_bytes(n);
  if (c->budget && c->held + bytes > c->budget) return RD_ERR_BUDGET;
  bool ok = cudaMalloc(&c->bws, (size_t)n * sizeof(Workspace)) == cudaSuccess &&
            cudaMalloc(&c->d_bres, (size_t)n * sizeof(rd_result)) == cudaSuccess &&
            cudaMalloc(&c->d_btruth, (size_t)n * sizeof(rd_truth)) == cudaSuccess &&
            cudaMalloc(&c->d_bstatus, (size_t)n * sizeof(int32_t)) == cudaSuccess &&
            cudaMallocHost(&c->h_bres, (size_t)n * sizeof(rd_result)) == cudaSuccess &&
            cudaMallocHost(&c->h_btruth, (size_t)n * sizeof(rd_truth)) == cudaSuccess &&
            cudaMallocHost(&c->h_bstatus, (size_t)n * sizeof(int32_t)) == cudaSuccess;
  // zeroed once: every table clean (the batched passes keep them so)
  if (ok) ok = cudaMemset(c->bws, 0, (size_t)n * sizeof(Workspace)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_batch_buffers(c);
    return RD_ERR_OOM;
  }
  c->bws_n = n;
  c->held += bytes;
  return RD_OK;
}

// Work items of the passes for one split: range items (runs of
// range_values values); sampled-block items grouped by dimensionality and SZ
// items (runs of zfp_blocks / sz_blocks sampled blocks of a 3D field;
// 4^(3-d) times as many of a d-dimensional one, so that every item holds
// about as many points); each list otherwise in field order.  Per-field item
// counts go into the field table.
void build_items(BatchPlan* b, const rd_batch_config& cfg, std::vector<BatchItem>& items) {
  auto per_item = [](long long blocks3d, int d) { return blocks3d << (2 * (3 - d)); };
  items.clear();
  auto split = [&](int i, long long units, long long per) {
    const long long cnt = units > 0 ? (units + per - 1) / per : 0;
    for (long long k = 0; k < cnt; k++) {
      BatchItem it;
      it.field = i;
      it.pad = 0;
      it.begin = k * per;
      it.end = (k + 1) * per < units ? (k + 1) * per : units;
      items.push_back(it);
    }
    return (uint32_t)cnt;
  };
  const int n = b->n;
  for (int i = 0; i < n; i++) b->hbf[i].items_range = split(i, b->hbf[i].f.N, cfg.range_values);
  b->n_range = (int)items.size();
  size_t base = items.size();
  b->blk_first[0] = 0;
  for (int d = 1; d <= 3; d++) {
    for (int i = 0; i < n; i++)
      if (b->hbf[i].f.d == d)
        b->hbf[i].items_zfp = split(i, b->hbf[i].f.nsampled, per_item(cfg.zfp_blocks, d));
    b->blk_first[d] = (int)(items.size() - base);
  }
  b->n_blk = (int)(items.size() - base);
  base = items.size();
  for (int i = 0; i < n; i++) split(i, b->hbf[i].f.nsampled, per_item(cfg.sz_blocks, b->hbf[i].f.d));
  b->n_sz = (int)(items.size() - base);
}

// Upload the tables of a split (the item buffer holds the largest count,
// that of the smallest candidate work items).
int upload_plan(BatchPlan* b, const rd_batch_config& cfg) {
  std::vector<BatchItem> items;
  if (!b->dbf && cudaMalloc(&b->dbf, b->hbf.size() * sizeof(BatchField)) != cudaSuccess) return RD_ERR_OOM;
  if (!b->ditems) {
    rd_batch_config small = cfg;
    small.range_values = kRangeValues[0] < cfg.range_values ? kRangeValues[0] : cfg.range_values;
    small.zfp_blocks = kZfpBlocks[0] < cfg.zfp_blocks ? kZfpBlocks[0] : cfg.zfp_blocks;
    small.sz_blocks = kSzBlocks[0] < cfg.sz_blocks ? kSzBlocks[0] : cfg.sz_blocks;
    build_items(b, small, items);
    if (cudaMalloc(&b->ditems, items.size() * sizeof(BatchItem)) != cudaSuccess) return RD_ERR_OOM;
  }
  build_items(b, cfg, items);
  if (cudaMemcpy(b->dbf, b->hbf.data(), b->hbf.size() * sizeof(BatchField), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(b->ditems, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice) !=
          cudaSuccess)
    return RD_ERR_CUDA;
  b->cfg = cfg;
  return RD_OK;
}

// A forced grid caps every pass's grid; 0 keeps each pass's resident count.
rd_batch_config resolve_ctas(const rd_context* c, rd_batch_config cfg) {
  (void)c;
  if (cfg.ctas < 0) cfg.ctas = 0;
  return cfg;
}

int pass_ctas(int resident, int cap) { return cap > 0 && cap < resident ? cap : resident; }

rd_batch_config split_level(const rd_context* c, int level, int ctas) {
  rd_batch_config cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.range_values = kRangeValues[level];
  cfg.zfp_blocks = kZfpBlocks[level];
  cfg.sz_blocks = kSzBlocks[level];
  cfg.ctas = ctas;
  return resolve_ctas(c, cfg);
}

// The estimate launches of a batch (reset .. final), optionally with an
// event pair around the item-based passes (the autotuner's timing).  The
// passes are stream-ordered: running the compute-bound passes of some fields
// beside the bandwidth-bound range pass of others, on a second stream,
// slowed both more than it overlapped.
int issue_batch_estimate(rd_context* c, BatchPlan* b, cudaStream_t s, cudaEvent_t* ev) {
  const int n = b->n;
  const int cap = b->cfg.ctas;
  const BatchItem* rit = b->ditems;
  const BatchItem* bit = rit + b->n_range;
  const BatchItem* sit = bit + b->n_blk;
  int rc;
  if ((rc = launch(c, K_B_RESET, s, [&] { return launch_batch_reset(b->dbf, n, b->need_gt, s); })))
    return rc;
  if (ev) cudaEventRecord(ev[0], s);
  if ((rc = launch(c, K_B_RANGE, s, [&] {
         return launch_batch_range(b->dbf, rit, b->n_range, pass_ctas(c->b_range_ctas, cap), s);
       })))
    return rc;
  for (int d = 1; d <= 3; d++) {
    const int cnt = b->blk_first[d] - b->blk_first[d - 1];
    if (cnt == 0) continue;
    if ((rc = launch(c, K_B_ZFP, s, [&] {
           return launch_batch_blocks(b->dbf, bit + b->blk_first[d - 1], cnt, d,
                                      pass_ctas(c->b_blocks_ctas[d - 1], cap), s);
         })))
      return rc;
  }
  if ((rc = launch(c, K_B_SZ, s, [&] {
         return launch_batch_sz_hist(b->dbf, sit, b->n_sz, pass_ctas(c->b_sz_ctas, cap), s);
       })))
    return rc;
  if (ev) cudaEventRecord(ev[1], s);
  if ((rc = launch(c, K_B_PREP, s, [&] { return launch_batch_code_prep(b->dbf, n, c->xlogx, s); }))) return rc;
  return launch(c, K_B_FINAL, s, [&] {
    return launch_batch_final(b->dbf, n, c->d_bres, c->d_bstatus, s);
  });
}

// The whole launch sequence of a batch call and the copies of its records.
int issue_batch(rd_context* c, BatchPlan* b, cudaStream_t s) {
  int rc = issue_batch_estimate(c, b, s, nullptr);
  if (rc) return rc;
  const int n = b->n;
  if (b->need_gt) {
    // the truth of each field, by the per-field passes on its workspace
    for (int i = 0; i < n; i++) {
      const FieldDev& f = b->hbf[i].f;
      const ParamsDev& p = b->hbf[i].p;
      Workspace* ws = b->hbf[i].ws;
      const unsigned long long npts = b->hbf[i].npoints;
      const int d = f.d;
      int zparts = 0, sparts = 0;
      if ((rc = launch(c, K_ZFP, s, [&] {
             return launch_zfp(f, p, P_ZFP_GT, DeltaArgs{}, ws, c->zfp_ctas[d], s, &zparts);
           })))
        return rc;
      if ((rc = launch(c, K_SZ_GT, s, [&] {
             if (sz_march_supported(f)) return launch_sz_march(f, p, 0, ws, c->num_sms, s, &sparts);
             return launch_sz_gt(f, p, 0, ws, c->sz_ctas[d], s, &sparts);
           })))
        return rc;
      if ((rc = launch(c, K_CODE_PREP, s, [&] { return launch_code_prep(ws, 2, c->xlogx, s); }))) return rc;
      if ((rc = launch(c, K_HUFFMAN, s, [&] { return launch_huffman(ws, 2, s); }))) return rc;
      if ((rc = launch(c, K_FINISH, s, [&] {
             return launch_finish(p, ws, P_ZFP_GT | P_SZ_GT, zparts, sparts, f.N, npts, nullptr, s);
           })))
        return rc;
    }
    if ((rc = launch(c, K_B_TRUTH, s, [&] {
           return launch_batch_truth(b->dbf, n, c->d_btruth, c->d_bstatus, s);
         })))
      return rc;
  }
  cudaError_t e = cudaMemcpyAsync(c->h_bres, c->d_bres, n * sizeof(rd_result), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->h_bstatus, c->d_bstatus, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && b->need_gt)
    e = cudaMemcpyAsync(c->h_btruth, c->d_btruth, n * sizeof(rd_truth), cudaMemcpyDeviceToHost, s);
  return cuda_status(e);
}

// Autotuner: run the estimate with the small, middle and large work items
// of every pass, twice each, time the item-based passes together with
// events, and keep the fastest.  The results do not depend on the split (integer sums,
// fixed-order floating point), so these are ordinary runs.
int autotune_plan(rd_context* c, BatchPlan* b, cudaStream_t s) {
  cudaEvent_t ev[2];
  for (int i = 0; i < 2; i++)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) return RD_ERR_CUDA;
  float best = 1e30f;
  rd_batch_config pick = split_level(c, 1, 0);
  int rc = RD_OK;
  const bool prof = c->profiling;
  c->profiling = false;
  for (int l = 0; l < 3 && rc == RD_OK; l++) {
    const rd_batch_config cfg = split_level(c, l, 0);
    rc = upload_plan(b, cfg);
    // each split twice, the faster run kept (the first may pay cold caches)
    for (int rep = 0; rep < 2 && rc == RD_OK; rep++) {
      rc = issue_batch_estimate(c, b, s, ev);
      if (rc == RD_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = RD_ERR_CUDA;
      float ms = 0.0f;
      if (rc == RD_OK && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess && ms < best) {
        best = ms;
        pick = cfg;
      }
    }
  }
  c->profiling = prof;
  for (int i = 0; i < 2; i++) cudaEventDestroy(ev[i]);
  if (rc) return rc;
  pick.tuned = 1;
  return upload_plan(b, pick);
}

BatchPlan* find_plan(rd_context* c, const std::vector<unsigned char>& key) {
  for (BatchPlan* b : c->plans)
    if (b->key == key) return b;
  return nullptr;
}

// Returns a call-level error (no record written) or, once the records are
// written (*written set), the status of the first failing field.
int batch_call(rd_context* c, const rd_field* fields, const rd_params* params, int n,
               rd_result* results, rd_truth* truths, int32_t* status, cudaStream_t s,
               bool* written) {
  const int need_gt = truths ? 1 : 0;
  std::vector<Geometry> geo((size_t)n);
  for (int i = 0; i < n; i++) {
    int rc = check_params(&params[i]);
    if (rc) return rc;
    if (fields[i].location != RD_LOC_DEVICE) return RD_ERR_INVALID_ARG;
    rc = make_geometry(c, &fields[i], nullptr, params[i].r_sp, s, &geo[i]);
    if (rc) return rc;
  }
  int rc = ensure_batch_capacity(c, n);
  if (rc) return rc;
  // the plan key: everything the launch sequence depends on
  std::vector<unsigned char> key;
  auto put = [&](const void* p, size_t bytes) {
    const unsigned char* q = static_cast<const unsigned char*>(p);
    key.insert(key.end(), q, q + bytes);
  };
  const int forced = c->batch_forced ? 1 : 0;
  const int prof = c->profiling ? 1 : 0;  // a plan's graph records events only if captured so
  put(&n, sizeof(n));
  put(&need_gt, sizeof(need_gt));
  put(&prof, sizeof(prof));
  put(&forced, sizeof(forced));
  if (forced) put(&c->batch_force, sizeof(rd_batch_config));
  std::vector<ParamsDev> pdev((size_t)n);
  for (int i = 0; i < n; i++) {
    pdev[i] = params_dev(&params[i]);
    put(&geo[i].f, sizeof(FieldDev));
    put(&pdev[i], sizeof(ParamsDev));
  }
  BatchPlan* b = find_plan(c, key);
  if (!b) {
    if (c->plans.size() >= kMaxPlans) {
      size_t lru = 0;
      for (size_t i = 1; i < c->plans.size(); i++)
        if (c->plans[i]->last_use < c->plans[lru]->last_use) lru = i;
      c->held -= c->plans[lru]->res_bytes;
      free_plan(c->plans[lru]);
      c->plans.erase(c->plans.begin() + lru);
    }
    b = new (std::nothrow) BatchPlan();
    if (!b) return RD_ERR_OOM;
    b->key = key;
    b->n = n;
    b->need_gt = need_gt;
    b->geo = geo;
    b->hbf.resize((size_t)n);
    // the SZ residuals of every field's sampled blocks (4^d keys each)
    size_t res_floats = 0;
    for (int i = 0; i < n; i++) res_floats += (size_t)geo[i].f.nsampled << (2 * geo[i].f.d);
    b->res_bytes = res_floats * sizeof(float);
    if (c->budget && c->held + b->res_bytes > c->budget) {
      delete b;
      return RD_ERR_BUDGET;
    }
    if (cudaMalloc(&b->dres, b->res_bytes) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return RD_ERR_OOM;
    }
    c->held += b->res_bytes;
    size_t roff = 0;
    for (int i = 0; i < n; i++) {
      BatchField& F = b->hbf[i];
      memset(&F, 0, sizeof(F));
      F.f = geo[i].f;
      F.p = pdev[i];
      F.ws = c->bws + i;
      F.ncoeff = (unsigned long long)F.f.nsampled * ec_count(F.f.d, params[i].ec_mode);
      F.npoints = geo[i].npoints_sampled;
      F.need_gt = need_gt;
      F.res = b->dres + roff;
      roff += (size_t)F.f.nsampled << (2 * F.f.d);
    }
    if (forced) {
      rd_batch_config cfg = c->batch_force;
      if (cfg.range_values <= 0) cfg.range_values = kRangeValues[1];
      if (cfg.zfp_blocks <= 0) cfg.zfp_blocks = kZfpBlocks[1];
      if (cfg.sz_blocks <= 0) cfg.sz_blocks = kSzBlocks[1];
      cfg.range_values = (cfg.range_values + 3) / 4 * 4;
      cfg.tuned = 0;
      rc = upload_plan(b, resolve_ctas(c, cfg));
    } else {
      rc = autotune_plan(c, b, s);
    }
    if (rc) {
      c->held -= b->res_bytes;
      free_plan(b);
      return rc;
    }
    c->plans.push_back(b);
  }
  b->last_use = ++c->tick;
  cudaError_t e = cudaSuccess;
  if (!b->exec && b->uses >= 1) {
    // capture the repeat into a graph
    if (c->cap || cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) == cudaSuccess) {
      if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        c->capturing = true;
        c->sink = &b->events;
        c->cap_kernels = 0;
        int crc = issue_batch(c, b, c->cap);
        c->capturing = false;
        c->sink = nullptr;
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(c->cap, &graph);
        if (crc == RD_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(&b->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (crc != RD_OK || ce != cudaSuccess) {
          cudaGetLastError();
          b->exec = nullptr;
          for (const Pending& p : b->events) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
          }
          b->events.clear();
        } else {
          b->kernels = c->cap_kernels;
        }
      }
    }
  }
  b->uses++;
  if (b->exec) {
    e = cudaGraphLaunch(b->exec, s);
    c->launches += b->kernels;
    rc = cuda_status(e);
  } else {
    rc = issue_batch(c, b, s);
  }
  e = cudaStreamSynchronize(s);
  if (c->profiling) {
    if (b->exec)
      add_times(c, b->events);
    else
      collect_profile(c);
  }
  if (rc != RD_OK) return rc;
  if (e != cudaSuccess) return cuda_status(e);
  c->batch_last = b->cfg;
  *written = true;
  int first = RD_OK;
  for (int i = 0; i < n; i++) {
    const int st = c->h_bstatus[i];
    if (status) status[i] = st;
    if (st != RD_OK) {
      memset(&results[i], 0, sizeof(rd_result));
      if (truths) memset(&truths[i], 0, sizeof(rd_truth));
      if (first == RD_OK) first = st;
      continue;
    }
    rd_result r = c->h_bres[i];
    record_geometry(&r, b->geo[i], true, b->hbf[i].p.ec_mode);
    results[i] = r;
    if (truths) truths[i] = c->h_btruth[i];
  }
  return first;
}

// ---------------------------------------------------------------------------
// Log-scale quantisation estimate (rd_estimate_sz_log)
// ---------------------------------------------------------------------------
// The base of the log scale: the smallest double b >= 1 whose edge
// u * pow(b, n) lies above M, found from the n-th root and stepped by one
// double at a time to the boundary.
double log_scale_base(double u, double M, int n) {
  auto edge = [&](double b) { return u * pow(b, (double)n); };
  double b = 1.0;
  if (M >= u) {
    b = pow(M / u, 1.0 / (double)n);
    if (!(b >= 1.0)) b = 1.0;
  }
  while (!(edge(b) > M)) b = nextafter(b, INFINITY);
  while (b > 1.0 && edge(nextafter(b, 0.0)) > M) b = nextafter(b, 0.0);
  return b;
}

int estimate_sz_log(rd_context* c, const rd_field* fld, const rd_params* prm, rd_log_result* out,
                    void* stream) {
  if (!c || !out) return RD_ERR_INVALID_ARG;
  int rc = check_params(prm);
  if (rc) return rc;
  CallGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  Geometry g;
  if ((rc = make_geometry(c, fld, nullptr, prm->r_sp, s, &g))) return rc;
  const int n = prm->quant_radius;
  if (!c->log_a) {  // tables for the largest n, once per context
    const size_t bytes =
        (kCenter + 1) * sizeof(double) + kCenter * sizeof(float) + sizeof(rd_log_result);
    if (c->budget && c->held + bytes > c->budget) return RD_ERR_BUDGET;
    if (cudaMalloc(&c->log_a, (kCenter + 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&c->log_f, kCenter * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&c->log_dev, sizeof(rd_log_result)) != cudaSuccess ||
        cudaMallocHost(&c->log_host, sizeof(LogHost)) != cudaSuccess) {
      cudaGetLastError();
      if (c->log_a) cudaFree(c->log_a);
      if (c->log_f) cudaFree(c->log_f);
      if (c->log_dev) cudaFree(c->log_dev);
      c->log_a = nullptr;
      c->log_f = nullptr;
      c->log_dev = nullptr;
      c->log_host = nullptr;
      return RD_ERR_OOM;
    }
    c->held += bytes;
  }
  const FieldDev& f = g.f;
  const ParamsDev p = params_dev(prm);
  Workspace* ws = c->ws;
  LogHost* hb = c->log_host;
  const int ctas = c->num_sms * 8;
  // range and the largest residual, then their scalars to the host
  if ((rc = launch(c, K_RESET, s, [&] { return launch_reset(ws, s); }))) return rc;
  if ((rc = launch(c, K_RANGE, s, [&] { return launch_range(f, p, ws, c->range_ctas, s); })))
    return rc;
  if ((rc = launch(c, K_SZ_LOG, s, [&] { return launch_sz_log_max(f, ws, ctas, s); }))) return rc;
  const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
  cudaError_t e = cudaMemcpyAsync(&hb->status, &ws->sc.status, sizeof(int32_t), d2h, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb->constant, &ws->sc.constant, sizeof(int32_t), d2h, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb->maxabs_bits, &ws->sc.log_maxabs, sizeof(uint32_t), d2h, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb->flags, &ws->sc.flags, sizeof(uint32_t), d2h, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb->vr, &ws->sc.vr, sizeof(double), d2h, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb->eb_abs, &ws->sc.eb_abs, sizeof(double), d2h, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (c->profiling) collect_profile(c);
  if (e != cudaSuccess) return cuda_status(e);
  memset(out, 0, sizeof(*out));
  if (hb->status != RD_OK) return hb->status;
  const uint32_t partial = g.partial ? RD_F_PARTIAL_BLOCKS : 0u;
  if (hb->constant) {
    out->vr = hb->vr;
    out->eb_abs = hb->eb_abs;
    out->flags = hb->flags | partial | RD_F_CONSTANT;
    out->psnr_log = INFINITY;
    return RD_OK;
  }
  // the edge tables: float64 edges, and the smallest float at or above each
  float mf;
  memcpy(&mf, &hb->maxabs_bits, sizeof(mf));
  const double M = (double)mf;
  const double u = hb->eb_abs;
  if (!(u > 0.0) || !isfinite(u)) return RD_ERR_INVALID_ARG;
  const double b = log_scale_base(u, M, n);
  std::vector<double> A((size_t)n + 1);
  std::vector<float> F((size_t)(n > 1 ? n - 1 : 1), 0.0f);
  A[0] = u;
  for (int k = 1; k <= n; k++) A[k] = u * pow(b, (double)k);
  for (int k = 2; k <= n; k++)
    if (A[k] < A[k - 1]) return RD_ERR_RANGE;  // a table the binary search cannot use
  for (int k = 1; k < n; k++) {
    float v = (float)A[k];
    if ((double)v < A[k]) v = nextafterf(v, INFINITY);
    F[k - 1] = v;
  }
  e = cudaMemcpyAsync(c->log_a, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->log_f, F.data(), F.size() * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_status(e);
  if ((rc = launch(c, K_SZ_LOG, s, [&] { return launch_sz_log_hist(f, n, c->log_f, ws, ctas, s); })))
    return rc;
  if ((rc = launch(c, K_CODE_PREP, s, [&] { return launch_code_prep(ws, 1, c->xlogx, s); }))) return rc;
  if ((rc = launch(c, K_HUFFMAN, s, [&] { return launch_huffman(ws, 1, s); }))) return rc;
  if ((rc = launch(c, K_FINISH, s,
                   [&] { return launch_sz_log_finish(p, c->log_a, ws, c->log_dev, s); })))
    return rc;
  e = cudaMemcpyAsync(&hb->res, c->log_dev, sizeof(rd_log_result), d2h, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hb->status, &ws->sc.status, sizeof(int32_t), d2h, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host tables live until here
  if (c->profiling) collect_profile(c);
  if (e != cudaSuccess) return cuda_status(e);
  if (hb->status != RD_OK) return hb->status;
  rd_log_result r = hb->res;
  r.unit = u;
  r.max_abs = M;
  r.base = b;
  r.flags |= partial;
  *out = r;
  return RD_OK;
}

}  // namespace

// Off: every per-field call launches its kernels directly (the serving
// slots, whose requests rarely repeat a key often enough to repay a graph
// capture, which would land in one request's latency).
void rdk_set_graph_capture(rd_context* c, bool on) { c->capture_repeats = on; }

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
  if (cudaMalloc(&c->xlogx, kNsym * sizeof(double)) != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return RD_ERR_OOM;
  }
  c->held = sizeof(Workspace) + kNsym * sizeof(double);
  if (cudaMallocHost(&c->out, sizeof(HostOut)) != cudaSuccess) {
    cudaFree(c->xlogx);
    cudaFree(c->ws);
    delete c;
    return RD_ERR_OOM;
  }
  memset(c->out, 0, sizeof(HostOut));
  if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->out_dev), c->out, 0) != cudaSuccess) {
    cudaFreeHost(c->out);
    cudaFree(c->xlogx);
    cudaFree(c->ws);
    delete c;
    return RD_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (prepare_code_stats() != cudaSuccess || prepare_sz_march() != cudaSuccess ||
      prepare_sz_code_table() != cudaSuccess ||
      prepare_sz_est() != cudaSuccess ||
      launch_init_tables(c->xlogx, 0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) {
    cudaFreeHost(c->out);
    cudaFree(c->xlogx);
    cudaFree(c->ws);
    delete c;
    return RD_ERR_CUDA;
  }
  c->range_ctas = c->num_sms * 4;
  for (int d = 1; d <= 3; d++) {
    c->zfp_ctas[d] = zfp_occupancy(d, c->num_sms);
    c->sz_ctas[d] = sz_occupancy(d, c->num_sms);
    c->sz_est_ctas[d] = sz_est_occupancy(d, c->num_sms);
  }
  batch_occupancy(c->num_sms, &c->b_range_ctas, c->b_blocks_ctas, &c->b_sz_ctas);
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
  free_batch_buffers(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  if (c->staging) cudaFree(c->staging);
  if (c->xhat) cudaFree(c->xhat);
  if (c->enc) cudaFree(c->enc);
  if (c->log_a) cudaFree(c->log_a);
  if (c->log_f) cudaFree(c->log_f);
  if (c->log_dev) cudaFree(c->log_dev);
  if (c->log_host) cudaFreeHost(c->log_host);
  if (c->ws) cudaFree(c->ws);
  if (c->xlogx) cudaFree(c->xlogx);
  if (c->out) cudaFreeHost(c->out);
  delete c;
  return RD_OK;
}

int32_t rd_estimate_zfp(rd_context* c, const rd_field* f, const rd_params* p, rd_result* out,
                        void* stream) {
  if (!out) return RD_ERR_INVALID_ARG;
  return run(c, f, p, P_ZFP_EST, DELTA_FROM_MSE, 0.0, out, nullptr, stream);
}

int32_t rd_estimate_sz_log(rd_context* c, const rd_field* f, const rd_params* p,
                           rd_log_result* out, void* stream) {
  return estimate_sz_log(c, f, p, out, stream);
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

int32_t rd_ground_truth_classic(rd_context* c, const rd_field* f, const rd_params* p, double eb_sz,
                                rd_truth* out, float* recon, void* stream) {
  if (!out || !(eb_sz > 0.0) || !isfinite(eb_sz)) return RD_ERR_INVALID_ARG;
  int rc = run(c, f, p, P_SZ_CLASSIC, DELTA_FROM_EB_SZ, eb_sz, nullptr, out, stream);
  if (rc || !recon) return rc;
  CallGuard guard(c->device);
  size_t n = 1;
  for (int k = 0; k < f->ndim; k++) n *= (size_t)f->shape[k];
  const bool constant = out->flags & RD_F_CONSTANT;
  const void* src = constant ? (const void*)f->data : (const void*)c->xhat;
  const cudaMemcpyKind kind =
      constant && f->location == RD_LOC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(recon, src, n * sizeof(float), kind, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_status(e);
}

int32_t rd_sz_compress(rd_context* c, const rd_field* fld, const rd_params* prm, double eb_sz, void* out,
                       uint64_t cap_bytes, uint64_t* nbits, void* stream) {
  if (!c || !nbits || !(eb_sz > 0.0) || !isfinite(eb_sz)) return RD_ERR_INVALID_ARG;
  if (out && ((uintptr_t)out & 7u)) return RD_ERR_INVALID_ARG;
  // the prequantised truth: status checks, histogram, quantiser, bit count
  rd_truth t;
  int rc = run(c, fld, prm, P_SZ_GT, DELTA_FROM_EB_SZ, eb_sz, nullptr, &t, stream);
  if (rc) return rc;
  if (t.flags & RD_F_CONSTANT) return RD_ERR_INVALID_ARG;  // nothing to quantise
  *nbits = t.sz_bits_gt;
  if (!out) return RD_OK;
  const unsigned long long words = (t.sz_bits_gt + 63ull) / 64ull;
  if (cap_bytes < words * 8ull) return RD_ERR_RANGE;
  CallGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  Geometry g;
  if ((rc = make_geometry(c, fld, nullptr, prm->r_sp, s, &g))) return rc;
  const long long n = g.f.N;
  // the code table, the symbols, the offsets and the stream, all on the
  // device: the truth's histogram and quantiser are still in the workspace
  const unsigned long long payload_base = 64ull + 22ull * t.sz_nsym_gt;
  const int nctas = stream_ctas(n);
  const size_t off_len = (size_t)n * sizeof(int32_t);
  const size_t off_code = (off_len + kNsym + 15) / 16 * 16;
  const size_t off_cb = off_code + sizeof(unsigned long long) * kNsym;
  const size_t off_ce = off_cb + sizeof(unsigned long long) * (size_t)nctas;
  const size_t off_tot = (off_ce + sizeof(unsigned) * (size_t)nctas + 15) / 16 * 16;
  const size_t off_cs = off_tot + 2 * sizeof(unsigned long long);
  const size_t off_st = off_cs + sizeof(uint32_t) * (size_t)kCodeScratchWords;
  const size_t bytes = off_st + 16;
  if (bytes > c->enc_bytes) {
    if (c->budget && c->held + (bytes - c->enc_bytes) > c->budget) return RD_ERR_BUDGET;
    if (c->enc) cudaFree(c->enc);
    c->held -= c->enc_bytes;
    c->enc = nullptr;
    c->enc_bytes = 0;
    if (cudaMalloc(&c->enc, bytes) != cudaSuccess) return RD_ERR_OOM;
    c->enc_bytes = bytes;
    c->held += bytes;
  }
  unsigned char* base = static_cast<unsigned char*>(c->enc);
  int32_t* dsym = reinterpret_cast<int32_t*>(base);
  uint8_t* dlen = base + off_len;
  unsigned long long* dcode = reinterpret_cast<unsigned long long*>(base + off_code);
  unsigned long long* dcb = reinterpret_cast<unsigned long long*>(base + off_cb);
  unsigned* dce = reinterpret_cast<unsigned*>(base + off_ce);
  unsigned long long* dtot = reinterpret_cast<unsigned long long*>(base + off_tot);
  uint32_t* cw = reinterpret_cast<uint32_t*>(base + off_cs);
  const CodeScratch cs{cw, cw + kNsym, cw + 2 * kNsym, cw + 3 * kNsym, cw + 4 * kNsym,
                       cw + 5 * kNsym, cw + 6 * kNsym, cw + 7 * kNsym, cw + 8 * kNsym};
  int32_t* dst = reinterpret_cast<int32_t*>(base + off_st);
  unsigned long long* dout = static_cast<unsigned long long*>(out);
  cudaError_t e = cudaMemsetAsync(out, 0, words * 8ull, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dst, 0, sizeof(int32_t), s);
  if (e == cudaSuccess) e = launch_sz_code_table(c->ws->hist[1], cs, dlen, dcode, dout, dst, s);
  if (e == cudaSuccess)
    e = launch_sz_inspect_q(g.f, 0.0f, 0.0f, 0.0f, prm->quant_radius, nullptr, dsym, nullptr, 0, s, c->ws);
  if (e == cudaSuccess) e = launch_stream_count(dsym, n, dlen, dcb, dce, s);
  if (e == cudaSuccess) e = launch_stream_scan(dcb, dce, nctas, dtot, s);
  if (e == cudaSuccess)
    e = launch_stream_pack(dsym, g.f.x, n, dlen, dcode, dcb, dce, dtot, payload_base, dout, s);
  // one read-back, after the last kernel: the totals and the table status
  unsigned long long tot[2] = {0ull, 0ull};
  int32_t st = RD_OK;
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot, dtot, sizeof(tot), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, dst, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  c->launches += 5;
  if (st != RD_OK) return st;
  // an optimal code's payload is the Huffman cost the truth reported, and
  // the symbols are the truth's
  if (tot[0] != t.sz_huff_gt || tot[1] != t.sz_nesc_gt) return RD_ERR_CUDA;
  return RD_OK;
}

int32_t rd_zfp_compress(rd_context* c, const rd_field* fld, const rd_params* prm, void* out,
                        uint64_t cap_bytes, uint64_t* nbits, void* stream) {
  if (!c || !nbits) return RD_ERR_INVALID_ARG;
  if (out && ((uintptr_t)out & 7u)) return RD_ERR_INVALID_ARG;
  // the ZFP truth: status checks, eb_abs and its exponent, the bit count
  rd_result r;
  rd_truth t;
  int rc = run(c, fld, prm, P_ZFP_GT, DELTA_FROM_MSE, 0.0, &r, &t, stream);
  if (rc) return rc;
  if (r.flags & RD_F_CONSTANT) return RD_ERR_INVALID_ARG;  // no bound to code at
  *nbits = t.zfp_bits_gt;
  if (!out) return RD_OK;
  const unsigned long long words = (t.zfp_bits_gt + 63ull) / 64ull;
  if (cap_bytes < words * 8ull) return RD_ERR_RANGE;
  CallGuard guard(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  Geometry g;
  if ((rc = make_geometry(c, fld, nullptr, prm->r_sp, s, &g))) return rc;
  // device scratch: per-block bits, per-chunk sums, the total
  const int nch = zfp_stream_chunks(g.f.nblocks);
  const size_t off_cs = ((size_t)g.f.nblocks * sizeof(uint32_t) + 15) / 16 * 16;
  const size_t off_tot = off_cs + sizeof(unsigned long long) * (size_t)nch;
  const size_t bytes = off_tot + 2 * sizeof(unsigned long long);
  if (bytes > c->enc_bytes) {
    if (c->budget && c->held + (bytes - c->enc_bytes) > c->budget) return RD_ERR_BUDGET;
    if (c->enc) cudaFree(c->enc);
    c->held -= c->enc_bytes;
    c->enc = nullptr;
    c->enc_bytes = 0;
    if (cudaMalloc(&c->enc, bytes) != cudaSuccess) return RD_ERR_OOM;
    c->enc_bytes = bytes;
    c->held += bytes;
  }
  unsigned char* base = static_cast<unsigned char*>(c->enc);
  uint32_t* dbits = reinterpret_cast<uint32_t*>(base);
  unsigned long long* dcs = reinterpret_cast<unsigned long long*>(base + off_cs);
  unsigned long long* dtot = reinterpret_cast<unsigned long long*>(base + off_tot);
  cudaError_t e = cudaMemsetAsync(out, 0, words * 8ull, s);
  if (e == cudaSuccess)
    e = launch_zfp_stream(g.f, r.minexp, dbits, dcs, dtot, static_cast<unsigned long long*>(out), s);
  unsigned long long* ht = reinterpret_cast<unsigned long long*>(&c->out->truth.zfp_bits_gt);  // pinned
  if (e == cudaSuccess) e = cudaMemcpyAsync(ht, dtot, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  c->launches += 3;
  if (e != cudaSuccess) return cuda_status(e);
  return *ht == t.zfp_bits_gt ? RD_OK : RD_ERR_CUDA;  // the blocks' bits add up to the truth's
}

int32_t rd_compress(rd_context* c, const rd_field* fld, const rd_params* prm, void* out,
                    uint64_t cap_bytes, uint64_t* nbits, int32_t* selection, rd_result* est,
                    void* stream) {
  if (!c || !nbits || !selection) return RD_ERR_INVALID_ARG;
  rd_result r;
  int rc = rd_select(c, fld, prm, &r, stream);
  if (rc) return rc;
  if (est) *est = r;
  if (r.flags & RD_F_CONSTANT) return RD_ERR_INVALID_ARG;
  *selection = r.selection;
  if (r.selection == 0) return rd_sz_compress(c, fld, prm, r.delta / 2.0, out, cap_bytes, nbits, stream);
  return rd_zfp_compress(c, fld, prm, out, cap_bytes, nbits, stream);
}

int32_t rd_evaluate(rd_context* c, const rd_field* f, const rd_params* p, rd_result* est,
                    rd_truth* truth, void* stream) {
  return run(c, f, p, P_ZFP_EST | P_ZFP_GT | P_SZ_EST | P_SZ_GT, DELTA_FROM_MSE, 0.0, est, truth,
             stream);
}

int32_t rd_rd_curve(rd_context* c, const rd_field* f, const rd_params* p, const double* eb, int32_t n,
                    rd_rd_point* out, void* stream) {
  if (!c || !f || !p || !eb || !out || n < 1) return RD_ERR_INVALID_ARG;
  memset(out, 0, sizeof(rd_rd_point) * (size_t)n);
  for (int32_t i = 0; i < n; i++) {
    rd_rd_point& pt = out[i];
    pt.eb = eb[i];
    rd_params q = *p;
    q.eb = eb[i];
    int32_t rc = rd_evaluate(c, f, &q, &pt.est, &pt.truth, stream);
    if (rc == RD_OK) rc = rd_estimate_sz(c, f, &q, 0.0, &pt.est_eb, stream);
    if (rc == RD_OK && pt.est.eb_abs > 0.0)
      rc = rd_ground_truth(c, f, &q, pt.est.eb_abs, &pt.truth_eb, stream);
    if (rc != RD_OK) {
      memset(&out[i], 0, sizeof(rd_rd_point) * (size_t)(n - i));
      return rc;
    }
    // same maximum error: SZ (bin 2 eb_abs) against ZFP (fixed accuracy at
    // eb_abs); SZ iff its bit-rate is lower (ties go to ZFP, as in rd_select)
    const double br_sz = q.sel_rule == RD_SEL_HUFFMAN ? pt.est_eb.br_sz_huff : pt.est_eb.br_sz;
    pt.selection_eb = br_sz < pt.est.br_zfp ? 0 : 1;
    pt.best_eb_gt = pt.truth_eb.best_gt;
  }
  return RD_OK;
}

int32_t rd_select_batch(rd_context* c, const rd_field* fields, const rd_params* params, int32_t n,
                        rd_result* results, rd_truth* truths, int32_t* status, void* stream) {
  if (!c || !fields || !params || !results || n < 1) return RD_ERR_INVALID_ARG;
  CallGuard guard(c->device);
  bool written = false;
  int rc = batch_call(c, fields, params, n, results, truths, status, (cudaStream_t)stream, &written);
  if (!written) {
    memset(results, 0, sizeof(rd_result) * (size_t)n);
    if (truths) memset(truths, 0, sizeof(rd_truth) * (size_t)n);
    if (status)
      for (int i = 0; i < n; i++) status[i] = rc;
  }
  return rc;
}

int32_t rd_batch_set_config(rd_context* c, const rd_batch_config* cfg) {
  if (!c) return RD_ERR_INVALID_ARG;
  if (!cfg) {
    c->batch_forced = false;
    return RD_OK;
  }
  if (cfg->range_values < 0 || cfg->zfp_blocks < 0 || cfg->sz_blocks < 0 || cfg->ctas < 0)
    return RD_ERR_INVALID_ARG;
  c->batch_forced = true;
  c->batch_force = *cfg;
  c->batch_force.tuned = 0;  // output
  return RD_OK;
}

int32_t rd_batch_get_config(rd_context* c, rd_batch_config* out) {
  if (!c || !out) return RD_ERR_INVALID_ARG;
  *out = c->batch_last;
  return RD_OK;
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

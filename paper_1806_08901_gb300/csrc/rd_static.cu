// rd_static.cu -- rd_select_static: the estimate of rd_select for callers
// that may not allocate memory, with its scratch in a fixed device array
// inside this library instead of a context's cudaMalloc'd workspace.
//
// Who needs it: code that runs under a device-memory budget it does not own
// (an in-situ simulation that has reserved the GPU's memory for itself, a
// framework whose allocator must serve every allocation), and callers that
// cannot afford the device-wide synchronisation cudaMalloc / cudaFree may
// imply.  Such callers hand in the field and receive the result record; this
// entry point calls no cudaMalloc, cudaFree, cudaMallocHost or any other
// allocating routine.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; each call clears what must start at zero before its
// passes run.  Calls whose work overlaps on the GPU (different streams or
// host threads) race on it and must be serialised by the caller.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "rd_internal.cuh"

using namespace rdk;

namespace {

// Stated maximum of the fixed scratch: 2.75 MiB per device (plus the 0.5 MiB
// entropy table), held for the life of the process by every GPU that loads
// the library.
constexpr size_t kStaticScratchBytes = 2883584;
static_assert(sizeof(Workspace) <= kStaticScratchBytes, "workspace exceeds the static scratch");

static __device__ __align__(256) unsigned char g_select_scratch[kStaticScratchBytes];
static __device__ double g_xlogx[kNsym];  // v log2 v table of the entropy sums

constexpr int kMaxDevices = 64;

struct DeviceSlot {
  bool ready;
  unsigned long long ctx_id;  // the CUDA context the set-up was done in
  Workspace* ws;  // device address of g_select_scratch on that device
  double* xlogx;  // device address of g_xlogx
  int range_ctas;
  int zfp_ctas[4];
  int sz_ctas[4];
  int sz_est_ctas[4];
};

std::mutex g_mu;
DeviceSlot g_slots[kMaxDevices];

// The unique ID of the calling thread's current CUDA context (0 when it
// cannot be read).  A context destroyed and created again (cudaDeviceReset,
// then a new call) gets a new ID: the module is loaded afresh, so the
// array's address, the filled table and the kernels' shared-memory
// attributes must be set up again.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// With the device current: resolve the array's device address (host code
// sees only a host-side stand-in for the symbol), fill the entropy table and
// size the grids from the occupancy calculator.  Done on the first call on
// the device, and again on the first call in a new context of the device.
int setup_device(int dev, DeviceSlot** out) {
  if (dev < 0 || dev >= kMaxDevices) return RD_ERR_INVALID_ARG;
  // any runtime call first makes the device's primary context current
  void* p0 = nullptr;
  if (cudaGetSymbolAddress(&p0, g_select_scratch) != cudaSuccess || !p0) return RD_ERR_CUDA;
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSlot& s = g_slots[dev];
  if (s.ready && (id == 0 || id != s.ctx_id || p0 != (void*)s.ws)) s.ready = false;
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_select_scratch) != cudaSuccess || !p) return RD_ERR_CUDA;
    void* tx = nullptr;
    if (cudaGetSymbolAddress(&tx, g_xlogx) != cudaSuccess || !tx) return RD_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RD_ERR_CUDA;
    if (prepare_code_stats() != cudaSuccess || prepare_sz_est() != cudaSuccess) return RD_ERR_CUDA;
    s.ws = static_cast<Workspace*>(p);
    s.xlogx = static_cast<double*>(tx);
    if (launch_init_tables(s.xlogx, 0) != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess)
      return RD_ERR_CUDA;
    s.range_ctas = sms * 4;
    for (int d = 1; d <= 3; d++) {
      s.zfp_ctas[d] = zfp_occupancy(d, sms);
      s.sz_ctas[d] = sz_occupancy(d, sms);
      s.sz_est_ctas[d] = sz_est_occupancy(d, sms);
    }
    s.ctx_id = id;
    s.ready = true;
  }
  *out = &s;
  return RD_OK;
}

}  // namespace

extern "C" int32_t rd_select_static(const rd_field* fld, const rd_params* prm, rd_result* out,
                                    void* stream) {
  if (!out || !fld || !fld->data) return RD_ERR_INVALID_ARG;
  if (fld->location != RD_LOC_DEVICE) return RD_ERR_INVALID_ARG;  // no staging copy
  int rc = check_params(prm);
  if (rc) return rc;
  // the largest field: 2^31 - 1 points (the scratch itself does not grow
  // with the field: fixed alphabet, fixed exponent bins)
  FieldGeom g;
  if ((rc = field_geometry(fld, fld->data, nullptr, prm->r_sp, &g))) return rc;
  const FieldDev& f = g.f;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RD_ERR_CUDA;
  DeviceSlot* slot = nullptr;
  if ((rc = setup_device(dev, &slot))) return rc;
  Workspace* ws = slot->ws;
  cudaStream_t s = (cudaStream_t)stream;

  const ParamsDev p = params_dev(prm);
  const int d = f.d;
  const unsigned long long ncoeff = (unsigned long long)f.nsampled * ec_count(d, prm->ec_mode);
  const int passes = P_ZFP_EST | P_SZ_EST;
  int zparts = 0;

  // the same launch sequence as rd_select, on the static scratch; the reset
  // kernel clears accumulators, histograms and result records first
  cudaError_t e = launch_reset(ws, s);
  const DeltaArgs da{1, DELTA_FROM_MSE, 0.0, 1, 0, ncoeff, g.npoints_sampled};
  if (e == cudaSuccess) e = launch_range(f, p, ws, slot->range_ctas, s);
  if (e == cudaSuccess) e = launch_zfp(f, p, P_ZFP_EST, da, ws, slot->zfp_ctas[d], s, &zparts);
  if (e == cudaSuccess) e = launch_sz_est(f, p, ws, slot->sz_est_ctas[d], s);
  if (e == cudaSuccess) e = launch_code_stats(ws, 1, slot->xlogx, s);
  if (e == cudaSuccess) e = launch_finish(p, ws, passes, zparts, 0, f.N, g.npoints_sampled, nullptr, s);
  rd_result r;
  int32_t status = RD_OK;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, &ws->res, sizeof(rd_result), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &ws->sc.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? RD_ERR_OOM : RD_ERR_CUDA;
  if (status != RD_OK) {
    memset(out, 0, sizeof(*out));
    return status;
  }
  record_geometry(&r, g, true, prm->ec_mode);
  *out = r;
  return RD_OK;
}

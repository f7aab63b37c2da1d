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
  Workspace* ws;  // device address of g_select_scratch on that device
  double* xlogx;  // device address of g_xlogx
  int range_ctas;
  int zfp_ctas[4];
  int sz_ctas[4];
  int sz_est_ctas[4];
};

std::mutex g_mu;
DeviceSlot g_slots[kMaxDevices];

// Once per device, with that device current: resolve the array's device
// address (host code sees only a host-side stand-in for the symbol) and size
// the grids from the occupancy calculator.
int setup_device(int dev, DeviceSlot** out) {
  if (dev < 0 || dev >= kMaxDevices) return RD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSlot& s = g_slots[dev];
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
    s.ready = true;
  }
  *out = &s;
  return RD_OK;
}

int check(const rd_field* fld, const rd_params* p) {
  if (!fld || !p || !fld->data) return RD_ERR_INVALID_ARG;
  if (fld->location != RD_LOC_DEVICE) return RD_ERR_INVALID_ARG;  // no staging copy
  if (fld->ndim < 1 || fld->ndim > 3) return RD_ERR_INVALID_ARG;
  if (!(p->eb > 0.0) || !isfinite(p->eb)) return RD_ERR_INVALID_ARG;
  if (p->eb_mode != RD_EB_REL && p->eb_mode != RD_EB_ABS) return RD_ERR_INVALID_ARG;
  if (p->ec_mode != RD_EC_PAPER && p->ec_mode != RD_EC_ALL) return RD_ERR_INVALID_ARG;
  if (!(p->r_sp >= 1e-6 && p->r_sp <= 1.0)) return RD_ERR_INVALID_ARG;
  if (p->quant_radius < 1 || p->quant_radius > 32768) return RD_ERR_INVALID_ARG;
  if (p->sel_rule != RD_SEL_PAPER && p->sel_rule != RD_SEL_HUFFMAN) return RD_ERR_INVALID_ARG;
  if (!isfinite(p->sz_offset)) return RD_ERR_INVALID_ARG;
  return RD_OK;
}

}  // namespace

extern "C" int32_t rd_select_static(const rd_field* fld, const rd_params* prm, rd_result* out,
                                    void* stream) {
  if (!out) return RD_ERR_INVALID_ARG;
  int rc = check(fld, prm);
  if (rc) return rc;
  // the largest field: 2^31 - 1 points (the scratch itself does not grow
  // with the field: fixed alphabet, fixed exponent bins)
  FieldDev f;
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
  f.x = fld->data;
  f.vec_ok = (((uintptr_t)f.x & 15u) == 0) && (f.n[f.d - 1] % 4 == 0);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RD_ERR_CUDA;
  DeviceSlot* slot = nullptr;
  if ((rc = setup_device(dev, &slot))) return rc;
  Workspace* ws = slot->ws;
  cudaStream_t s = (cudaStream_t)stream;

  // block sampling lattice: S = round(1/r_sp) split into primes, each prime
  // (largest first) on the axis with the smallest stride (ties: faster axis)
  long long S = (long long)floor(1.0 / prm->r_sp + 0.5);
  if (S < 1) S = 1;
  long long fac[64];
  int nf = 0;
  for (long long q = 2; q * q <= S; q++)
    while (S % q == 0) {
      fac[nf++] = q;
      S /= q;
    }
  if (S > 1) fac[nf++] = S;
  int st[3] = {1, 1, 1};
  for (int i = nf - 1; i >= 0; i--) {
    int a = f.d - 1;
    for (int k = f.d - 2; k >= 0; k--)
      if (st[k] < st[a]) a = k;
    st[a] = (int)(st[a] * fac[i]);
  }
  f.nblocks = 1;
  f.nsampled = 1;
  unsigned long long npts = 1;
  bool partial = false;
  for (int k = 0; k < f.d; k++) {
    f.B[k] = (f.n[k] + 3) / 4;
    f.s[k] = st[k];
    f.L[k] = (f.B[k] + st[k] - 1) / st[k];
    f.nblocks *= f.B[k];
    f.nsampled *= f.L[k];
    unsigned long long pk = 0;
    for (int b = 0; b < f.B[k]; b += st[k]) pk += (unsigned long long)(f.n[k] - 4 * b < 4 ? f.n[k] - 4 * b : 4);
    npts *= pk;
    partial = partial || (f.n[k] % 4) != 0;
  }
  ParamsDev p;
  p.eb = prm->eb;
  p.eb_mode = prm->eb_mode;
  p.ec_mode = prm->ec_mode;
  p.R = prm->quant_radius;
  p.sel_rule = prm->sel_rule;
  p.sz_offset = prm->sz_offset;
  const int d = f.d;
  const int m = prm->ec_mode == RD_EC_ALL ? (1 << (2 * d)) : (d == 1 ? 3 : d == 2 ? 9 : 16);
  const unsigned long long ncoeff = (unsigned long long)f.nsampled * m;
  const int passes = P_ZFP_EST | P_SZ_EST;
  int zparts = 0;

  // the same launch sequence as rd_select, on the static scratch; the reset
  // kernel clears accumulators, histograms and result records first
  cudaError_t e = launch_reset(ws, s);
  const DeltaArgs da{1, DELTA_FROM_MSE, 0.0, 1, 0, ncoeff, npts};
  if (e == cudaSuccess) e = launch_range(f, p, ws, slot->range_ctas, s);
  if (e == cudaSuccess) e = launch_zfp(f, p, P_ZFP_EST, da, ws, slot->zfp_ctas[d], s, &zparts);
  if (e == cudaSuccess) e = launch_sz_est(f, p, ws, slot->sz_est_ctas[d], s);
  if (e == cudaSuccess) e = launch_code_stats(ws, 1, slot->xlogx, s);
  if (e == cudaSuccess) e = launch_finish(p, ws, passes, zparts, 0, f.N, npts, s);
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
  for (int k = 0; k < 3; k++) r.strides[k] = k < d ? f.s[k] : 0;
  r.n_blocks = (uint64_t)f.nblocks;
  if (!(r.flags & RD_F_CONSTANT)) {
    r.n_sampled_blocks = (uint64_t)f.nsampled;
    r.r_sp_eff = (double)f.nsampled / (double)f.nblocks;
    r.zfp_npoints = npts;
    r.zfp_ncoeff = ncoeff;
  }
  if (partial) r.flags |= RD_F_PARTIAL_BLOCKS;
  *out = r;
  return RD_OK;
}
